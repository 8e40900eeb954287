"""Pins of the oracle's SSV -> MSV hand-off (Sec. 2.1), and mutants of it.

The stage rule read from Sec. 2.1: SSV scores every sequence; a sequence is
re-scored by MSV when its SSV score overflowed or its SSV nat score is at
least the caller's threshold (inclusive); every other sequence comes out of
the MSV stage as filtered (raw 0, flag 2, nat NaN).  The pins check the rule
on a hand table of (flag, nat, threshold) cases whose answers follow from the
rule alone, and the whole two-stage oracle against the two one-stage oracles
(each pinned in test_oracle_pins.py) on a database with overflowing
sequences and a threshold placed exactly on a sequence's score.

The mutants plant the plausible mistakes of such a rule -- a strict instead
of an inclusive threshold, the overflow clause dropped, filtered entries not
marked, the pass count taken from the wrong array -- in a copy of the oracle's
Python source, and the pins must fail on every one of them.
"""
import os
import types

import numpy as np
import pytest

import oracle
from paper_1707_09683_gb300 import synth


def _pipeline_case():
    """A realistic profile, a database with planted segments of its own
    emissions (some SSV scores overflow)."""
    rng = np.random.default_rng(11)
    prof = synth.make_profile(300, rng)
    db = synth.make_database(400, 200.0, 10, 600, rng)
    synth.plant_segments(db, [prof], 0.15, rng, seg=(150, 300))
    return prof, db


def check_hand_table(orc=oracle):
    """The selection rule on hand cases (flag, nat, threshold) -> passes."""
    thr = np.float32(-2.5)
    below = np.nextafter(thr, np.float32(-np.inf))
    flag = np.array([0, 0, 1, 1, 0, 0, 0, 1, 0], np.uint8)
    nat = np.array([thr, below, -50.0, np.inf, np.nan, np.inf, 7.0, np.nan, -np.inf], np.float32)
    want = np.array([True, False, True, True, False, True, True, True, False])
    got = np.asarray(orc.ssv_passes(flag, nat, float(thr)))
    assert got.dtype == bool and np.array_equal(got, want), got
    # A threshold of -inf passes every sequence with a number for a score.
    got = np.asarray(orc.ssv_passes(flag, nat, -np.inf))
    assert np.array_equal(got, ~np.isnan(nat) | (flag != 0)), got


def check_two_stages(orc=oracle):
    """pipeline() = SSV everywhere, MSV on the passing sequences, the others
    filtered; a sequence whose SSV nat equals the threshold passes, one ulp
    above it does not."""
    prof, db = _pipeline_case()
    sr, sf, sn = oracle.ssv(prof, db.residues, db.offsets, db.lengths)
    mr_all, mf_all, mn_all = oracle.msv(prof, db.residues, db.offsets, db.lengths)
    assert sf.sum() >= 3, "the case needs overflowing SSV scores"
    finite = np.flatnonzero(sf == 0)
    j = int(finite[np.argsort(sn[finite])[len(finite) * 9 // 10]])   # near the top decile
    thr = float(sn[j])
    for t, j_passes in ((thr, True), (float(np.nextafter(np.float32(thr), np.float32(np.inf))), False)):
        (a, b, c), (mr, mf, mn), npass = orc.pipeline(prof, db.residues, db.offsets, db.lengths, t)
        assert np.array_equal(a, sr) and np.array_equal(b, sf)
        assert np.array_equal(c.view(np.uint32), sn.view(np.uint32))
        keep = (sf == 1) | (sn >= np.float32(t))
        assert bool(keep[j]) == j_passes
        assert npass == int(keep.sum())
        assert np.array_equal(mr[keep], mr_all[keep]) and np.array_equal(mf[keep], mf_all[keep])
        assert np.array_equal(mn[keep].view(np.uint32), mn_all[keep].view(np.uint32))
        assert np.all(mr[~keep] == 0) and np.all(mf[~keep] == 2) and np.all(np.isnan(mn[~keep]))
        # Every overflowed SSV score reached MSV, which overflows too (an SSV
        # path is an MSV path).
        assert np.all(mf[sf == 1] == 1)


def test_selection_rule_hand_table():
    check_hand_table()


def test_two_stage_oracle_against_one_stage_oracles():
    check_two_stages()


MUTANTS = {
    "threshold_strict": ("(nat >= np.float32(ssv_min_nat))", "(nat > np.float32(ssv_min_nat))"),
    "overflow_clause_dropped": ("return (flag != 0) | (nat >= np.float32(ssv_min_nat))",
                                "return (nat >= np.float32(ssv_min_nat))"),
    "filtered_flag_not_marked": ("mf = np.full(n, 2, np.uint8)", "mf = np.full(n, 0, np.uint8)"),
    "filtered_nat_zero": ("mn = np.full(n, np.nan, np.float32)", "mn = np.zeros(n, np.float32)"),
    "count_from_mask_size": ("return (sr, sf, sn), (mr, mf, mn), int(idx.size)",
                             "return (sr, sf, sn), (mr, mf, mn), int(keep.size)"),
}


def _mutant_module(before, after):
    path = os.path.join(os.path.dirname(oracle.__file__), "__init__.py")
    src = open(path).read()
    assert src.count(before) == 1, before
    mod = types.ModuleType("oracle_pipeline_mutant")
    mod.__file__ = path
    exec(compile(src.replace(before, after), path, "exec"), mod.__dict__)
    return mod


@pytest.mark.parametrize("name", sorted(MUTANTS))
def test_pins_catch_pipeline_mutant(name):
    mod = _mutant_module(*MUTANTS[name])
    caught = []
    for check in (check_hand_table, check_two_stages):
        try:
            check(mod)
        except AssertionError:
            caught.append(check.__name__)
    assert caught, f"no pin notices the mutant {name}"
