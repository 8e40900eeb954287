"""The Viterbi oracle's pins must catch plausible mistakes in it (a planted
error per mutant, compiled on the CPU)."""
import pytest

import oracle
import test_vit_oracle_pins as pins

MUTANTS = {
    "mm_index": ("int best = sat16(Mr[k - 1] + tr(p, T_MM, k));", "int best = sat16(Mr[k] + tr(p, T_MM, k));"),
    "drop_im": ("best = imax(best, sat16(Ir[k - 1] + tr(p, T_IM, k)));", ""),
    "drop_dm": ("best = imax(best, sat16(Dr[k - 1] + tr(p, T_DM, k)));", ""),
    "bm_from_xN": ("best = imax(best, sat16(xB + tr(p, T_BM, k)));", "best = imax(best, sat16(xN + tr(p, T_BM, k)));"),
    "insert_prev_row": ("In[k] = k < M ? imax(sat16(Mr[k] + tr(p, T_MI, k)), sat16(Ir[k] + tr(p, T_II, k))) : -32768;",
                        "In[k] = k < M ? imax(sat16(Mn[k] + tr(p, T_MI, k)), sat16(Ir[k] + tr(p, T_II, k))) : -32768;"),
    "d_from_previous_row": ("Dn[k] = k > 1 ? imax(sat16(Mn[k - 1] + tr(p, T_MD, k)), sat16(Dn[k - 1] + tr(p, T_DD, k))) : -32768;",
                            "Dn[k] = k > 1 ? imax(sat16(Mr[k - 1] + tr(p, T_MD, k)), sat16(Dn[k - 1] + tr(p, T_DD, k))) : -32768;"),
    "no_d_exit": ("xE = imax(xE, imax(Mn[k], Dn[k]));", "xE = imax(xE, Mn[k]);"),
    "j_loop_sign": ("xJ = imax(sat16(xJ + sp[X_JJ]), sat16(xE + sp[X_EJ]));", "xJ = imax(sat16(xJ - sp[X_JJ]), sat16(xE + sp[X_EJ]));"),
    "drop_nn": ("xN = sat16(xN + sp[X_NN]);", ""),
    "c_from_j": ("xC = imax(sat16(xC + sp[X_CC]), sat16(xE + sp[X_EC]));", "xC = imax(sat16(xC + sp[X_CC]), sat16(xJ + sp[X_EC]));"),
    "no_saturation": ("static int sat16(int v) { return v < -32768 ? -32768 : (v > 32767 ? 32767 : v); }",
                      "static int sat16(int v) { return v > 32767 ? 32767 : v; }"),
    "ct_missing": ("const int sc = sat16(xC + sp[X_CT]);", "const int sc = sat16(xC);"),
}

PIN_TESTS = [
    (pins.test_hand_worked_examples, ()),
    (pins.test_equals_unsaturated_integer_dp, (0,)),
    (pins.test_equals_path_enumeration, (0,)),
    (pins.test_single_node_single_residue_closed_form, ()),
]


@pytest.mark.parametrize("name", sorted(MUTANTS))
def test_pins_catch_mutant(name, tmp_path, monkeypatch):
    before, after = MUTANTS[name]
    src = open(oracle._VIT_SRC).read()
    assert src.count(before) == 1, name
    mut = tmp_path / f"{name}.c"
    mut.write_text(src.replace(before, after))
    lib = oracle.load_library(oracle.compile_source([oracle._SRC, str(mut)], str(tmp_path / f"{name}.so")))
    monkeypatch.setattr(oracle, "_lib", lib)
    caught = []
    for fn, args in PIN_TESTS:
        try:
            fn(*args)
        except (AssertionError, RuntimeError):
            caught.append(fn.__name__)
    assert caught, f"no pin notices the mutant {name}"
