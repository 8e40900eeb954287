"""The oracle's pins must catch plausible mistakes in the oracle.

Each mutant below is the oracle source with one small planted error (a
dropped term, a wrong sign, index or comparison, a transposed operand).  The
mutant is compiled on the CPU, swapped in for the real oracle, and the pin
tests of test_oracle_pins.py are run against it: at least one of them must
fail, otherwise the pins would not notice that mistake.
"""
import os

import pytest

import oracle
import test_oracle_pins as pins

MUTANTS = {
    "msv_diag_index": ("int from = prev[k - 1] > xB ? prev[k - 1] : xB;",
                       "int from = prev[k] > xB ? prev[k] : xB;"),
    "msv_drop_bias": ("int v = sat8(from + bias);", "int v = sat8(from);"),
    "msv_drop_inner_cap": ("int v = sat8(from + bias);", "int v = from + bias;"),
    "msv_overflow_strict": ("if (xE >= 255 - bias)", "if (xE > 255 - bias)"),
    "msv_tec_sign": ("int xEj = sat8(xE - (int)p->tec);", "int xEj = sat8(xE + (int)p->tec);"),
    "msv_drop_N_path": ("int bj = (int)p->base > xJ ? (int)p->base : xJ;", "int bj = xJ;"),
    "msv_drop_tbm": ("xB = sat8(bj - (t + (int)p->tbm));", "xB = sat8(bj - t);"),
    "msv_init_xB": ("int xB = sat8((int)p->base - (t + (int)p->tbm));",
                    "int xB = sat8((int)p->base - t);"),
    "msv_nat_sign": ("float num = (float)(xJ - t - (int)p->base);",
                     "float num = (float)(xJ + t - (int)p->base);"),
    "ssv_diag_index": ("int v = prev[k - 1] + bias - cost_of(p, x, k);",
                       "int v = prev[k] + bias - cost_of(p, x, k);"),
    "ssv_drop_floor": ("      v = sat8(v);\n      cur[k] = v;\n      if (v > R) R = v;",
                       "      v = v > 255 ? 255 : v;\n      cur[k] = v;\n      if (v > R) R = v;"),
    "ssv_flag_cmp": ("if (R == 255) {", "if (R >= 254) {"),
    "ssv_nat_tjb_once": ("(int)p->tec - 2 * t);", "(int)p->tec - t);"),
    "invalid_code_cmp": ("if (x >= p->K) return 255;", "if (x > p->K) return 255;"),
    "cost_transposed": ("return p->cost[(size_t)x * (size_t)p->M + (size_t)(k - 1)];",
                        "return p->cost[(size_t)(k - 1) * (size_t)p->K + (size_t)x];"),
    "tjb_lut_last": ("return p->tjb_by_len[L < p->n_tjb ? L : p->n_tjb - 1];",
                     "return p->tjb_by_len[p->n_tjb - 1];"),
}

PIN_TESTS = [
    (pins.test_hand_worked_examples, ()),
    (pins.test_ssv_equals_segment_enumeration, (0,)),
    (pins.test_ssv_equals_segment_enumeration, (1,)),
    (pins.test_msv_equals_unbounded_integer_dp, (0,)),
    (pins.test_msv_int_dp_covers_overflow_and_j_reuse, ()),
    (pins.test_msv_equals_path_enumeration, (0,)),
    (pins.test_empty_sequence, ()),
    (pins.test_single_node_closed_form, ()),
    (pins.test_single_residue_closed_form, ()),
    (pins.test_constant_cost_ssv, (3,)),
    (pins.test_constant_cost_ssv, (127,)),
    (pins.test_codes_at_or_above_K_score_cost_255, ()),
    (pins.test_tjb_lut_selects_by_length, ()),
    (pins.test_nat_against_exact_arithmetic, ()),
]


@pytest.mark.parametrize("name", sorted(MUTANTS))
def test_pins_catch_mutant(name, tmp_path, monkeypatch):
    before, after = MUTANTS[name]
    src = open(oracle._SRC).read()
    assert src.count(before) == 1, f"mutation site for {name} not found exactly once"
    mut_c = tmp_path / f"{name}.c"
    mut_c.write_text(src.replace(before, after))
    lib = oracle.load_library(oracle.compile_source(str(mut_c), str(tmp_path / f"{name}.so")))
    monkeypatch.setattr(oracle, "_lib", lib)
    caught = []
    for fn, args in PIN_TESTS:
        try:
            fn(*args)
        except AssertionError:
            caught.append(fn.__name__)
    assert caught, f"no pin notices the mutant {name}"
