"""Pins of the scalar oracle against things other than itself.

Each test checks the oracle (oracle/mpf_oracle.c) against a fact fixed by the
paper or by the mathematics of the recurrences, computed here by a different
route:

* hand-worked examples (tests/golden/oracle_hand_examples.json);
* SSV (Alg. 7, single segment, J removed as in Sec. 2.1) equals the best
  ungapped diagonal segment found by brute-force enumeration, capped at 255;
* MSV (Alg. 2 with the J/B update, Sec. 2.1) equals an unbounded integer DP
  whenever the two byte preconditions hold (no byte floor or cap can fire
  before the overflow threshold), and equals a path-level enumeration of
  every set of ordered ungapped hits on tiny inputs;
* closed forms (M = 1, L = 0, L = 1, constant-cost profiles);
* invariants between the two filters and under appending residues;
* the nat score against exact rational arithmetic within float32 rounding.

No CUDA code is involved.
"""
import itertools
import json
import math
import os
from fractions import Fraction

import numpy as np
import pytest

import oracle
from paper_1707_09683_gb300 import synth

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "oracle_hand_examples.json")


class P:
    """Plain profile record for the oracle."""

    def __init__(self, cost, bias, tbm, tec, tjb, base, scale=synth.SCALE, lut=None):
        cost = np.asarray(cost, dtype=np.uint8)
        self.K, self.M = cost.shape
        self.cost = cost
        self.bias, self.tbm, self.tec, self.tjb_fixed, self.base = bias, tbm, tec, tjb, base
        self.tjb_by_len = lut
        self.scale = float(np.float32(scale))


def one(filter_, prof, seq):
    seq = np.asarray(seq, dtype=np.uint8)
    raw, flag, nat = oracle.scan(filter_, prof, seq, np.array([0], np.uint64),
                                 np.array([seq.size], np.uint32))
    return int(raw[0]), int(flag[0]), float(nat[0])


def t_of(prof, L):
    if prof.tjb_by_len is None:
        return prof.tjb_fixed
    lut = prof.tjb_by_len
    return int(lut[min(L, lut.size - 1)])


def s_of(prof, x, k):
    """Signed match score bias - cost of node k (0-based), residue x."""
    c = 255 if x >= prof.K else int(prof.cost[x, k])
    return prof.bias - c


# ---------------------------------------------------------------- golden ---

def test_hand_worked_examples():
    cases = json.load(open(GOLDEN))["cases"]
    assert len(cases) >= 5
    for c in cases:
        prof = P(c["cost"], c["bias"], c["tbm"], c["tec"], c["tjb"], c["base"])
        for name, f in (("msv", oracle.MSV), ("ssv", oracle.SSV)):
            raw, flag, nat = one(f, prof, c["seq"])
            exp = c[name]
            assert (raw, flag) == (exp["raw"], exp["flag"]), (c["name"], name)
            if flag:
                assert math.isinf(nat) and nat > 0
            else:
                want = np.float32(exp["nat_numerator"]) / np.float32(prof.scale) - np.float32(3.0)
                assert nat == pytest.approx(float(want), abs=1e-6), (c["name"], name)


# ------------------------------------------------------- SSV brute force ---

def ssv_brute(prof, seq):
    """max(0, best sum over every ungapped diagonal segment), capped at 255."""
    best = 0
    L, M = len(seq), prof.M
    for i0 in range(L):
        for k0 in range(M):
            tot = 0
            for d in range(min(L - i0, M - k0)):
                tot += s_of(prof, seq[i0 + d], k0 + d)
                best = max(best, tot)
    return min(best, 255), int(best >= 255)


@pytest.mark.parametrize("seed", range(6))
def test_ssv_equals_segment_enumeration(seed):
    rng = np.random.default_rng(1000 + seed)
    for _ in range(60):
        M = int(rng.integers(1, 13))
        K = int(rng.integers(1, 6))
        bias = int(rng.choice([0, 5, 20, 60, 128, 200, 255]))
        prof = P(rng.integers(0, 256, size=(K, M)), bias, int(rng.integers(0, 40)),
                 int(rng.integers(0, 6)), int(rng.integers(0, 30)), 190)
        if rng.random() < 0.5:   # low costs: long positive runs, saturation
            prof.cost = rng.integers(0, bias + 8, size=(K, M)).clip(0, 255).astype(np.uint8)
        L = int(rng.integers(0, 13))
        seq = rng.integers(0, K + 2, size=L)       # includes codes >= K
        raw, flag, _ = one(oracle.SSV, prof, seq)
        assert (raw, flag) == ssv_brute(prof, seq), (M, K, bias, L)


# ------------------------------------------------ MSV vs integer DP pin ----

def msv_int_dp(prof, seq):
    """The MSV recurrence with unbounded integers (no byte floor or cap)."""
    M = prof.M
    t = t_of(prof, len(seq))
    NEG = -(1 << 40)
    D = np.full(M, NEG, dtype=np.int64)
    XJ = 0
    XB = prof.base - (t + prof.tbm)
    thr = 255 - prof.bias
    table = np.array([[s_of(prof, x, k) for k in range(M)] for x in range(32)], dtype=np.int64)
    for x in seq:
        prev = np.concatenate(([NEG], D[:-1]))
        D = np.maximum(prev, XB) + table[x]
        XE = int(D.max())
        if XE >= thr:
            return 255, 1
        XJ = max(XJ, XE - prof.tec)
        XB = max(prof.base, XJ) - (t + prof.tbm)
    return XJ, 0


def preconditions_hold(prof, L):
    t = t_of(prof, L)
    return prof.base >= t + prof.tbm and prof.base + prof.bias <= 255 + t + prof.tbm


@pytest.mark.parametrize("seed", range(8))
def test_msv_equals_unbounded_integer_dp(seed):
    rng = np.random.default_rng(2000 + seed)
    done = 0
    while done < 150:
        M = int(rng.integers(1, 20))
        K = int(rng.integers(1, 21))
        bias = int(rng.integers(0, 70))
        prof = P(rng.integers(0, 256, size=(K, M)), bias, int(rng.integers(0, 70)),
                 int(rng.integers(0, 8)), int(rng.integers(0, 45)), int(rng.integers(100, 256)))
        mode = rng.random()
        if mode < 0.3:    # strong profile: hits, J reuse and overflow
            prof.cost = rng.integers(0, bias + 4, size=(K, M)).clip(0, 255).astype(np.uint8)
        L = int(rng.integers(0, 40))
        if not preconditions_hold(prof, L):
            continue
        seq = rng.integers(0, K + 1, size=L)
        assert one(oracle.MSV, prof, seq)[:2] == msv_int_dp(prof, seq)
        done += 1


def test_msv_int_dp_covers_overflow_and_j_reuse():
    """The integer-DP pin must exercise both the overflow exit and hits
    chained through J, or it pins nothing about them."""
    rng = np.random.default_rng(7)
    n_flag = n_j = 0
    for _ in range(400):
        M = int(rng.integers(2, 12))
        prof = P(rng.integers(0, 30, size=(4, M)), 25, 10, 2, 8, 190)
        seq = rng.integers(0, 4, size=int(rng.integers(5, 30)))
        raw, flag = msv_int_dp(prof, seq)
        assert one(oracle.MSV, prof, seq)[:2] == (raw, flag)
        n_flag += flag
        n_j += (not flag) and raw > prof.base
    assert n_flag > 10 and n_j > 10


# ------------------------------------------ MSV path enumeration pin -------

def msv_paths(prof, seq):
    """Enumerate every ordered set of non-overlapping ungapped hits.

    A hit is a diagonal segment (rows i0..i1, nodes k0..k0+i1-i0).  Entering
    a hit costs t + tbm from B, where B is reached from N (score base) or
    from J (the previous hit's end); leaving costs tec.  The final score is
    the best J value (0 if no hit), and the overflow flag is raised if any
    partial hit reaches 255 - bias.
    """
    L, M = len(seq), prof.M
    t = t_of(prof, L)
    thr = 255 - prof.bias
    segs = []   # (i0, i1, partial sums list)
    for i0 in range(L):
        for k0 in range(M):
            tot = 0
            for d in range(min(L - i0, M - k0)):
                tot += s_of(prof, seq[i0 + d], k0 + d)
                segs.append((i0, i0 + d, tot))
    best = 0
    flag = 0

    def rec(next_row, jprev):
        nonlocal best, flag
        entry = max(prof.base, jprev) - (t + prof.tbm)
        for (i0, i1, tot) in segs:
            if i0 < next_row:
                continue
            if entry + tot >= thr:
                flag = 1
            j = entry + tot - prof.tec
            best = max(best, j)
            rec(i1 + 1, j)

    rec(0, -(1 << 30))
    return (255, 1) if flag else (best, 0)


@pytest.mark.parametrize("seed", range(4))
def test_msv_equals_path_enumeration(seed):
    rng = np.random.default_rng(3000 + seed)
    done = 0
    while done < 40:
        M = int(rng.integers(1, 4))
        K = int(rng.integers(1, 4))
        bias = int(rng.integers(10, 40))
        prof = P(rng.integers(0, bias + 20, size=(K, M)).clip(0, 255), bias,
                 int(rng.integers(0, 6)), int(rng.integers(0, 4)), int(rng.integers(0, 6)),
                 int(rng.choice([20, 60, 190, 225])))
        L = int(rng.integers(0, 6))
        if not preconditions_hold(prof, L):
            continue
        seq = rng.integers(0, K, size=L)
        assert one(oracle.MSV, prof, seq)[:2] == msv_paths(prof, seq), (M, K, L)
        done += 1


# ---------------------------------------------------------- closed forms ---

def test_empty_sequence():
    prof = P([[3, 4, 5]], 10, 7, 3, 11, 190)
    for f in (oracle.MSV, oracle.SSV):
        raw, flag, nat = one(f, prof, [])
        assert (raw, flag) == (0, 0)
    _, _, nat = one(oracle.MSV, prof, [])
    exact = Fraction(0 - 11 - 190) / Fraction(prof.scale) - 3
    assert abs(nat - float(exact)) <= 4e-6 * abs(float(exact))
    _, _, nat = one(oracle.SSV, prof, [])
    exact = Fraction(0 - 7 - 3 - 22) / Fraction(prof.scale) - 3
    assert abs(nat - float(exact)) <= 4e-6 * abs(float(exact))


def test_single_node_closed_form():
    """M = 1 and xJ never above base: every row is a fresh one-cell hit, so
    raw = max(0, xB + bias - min_i cost(x_i) - tec)."""
    rng = np.random.default_rng(11)
    for _ in range(200):
        K = int(rng.integers(1, 8))
        bias = int(rng.integers(0, 40))
        prof = P(rng.integers(0, 256, size=(K, 1)), bias, int(rng.integers(0, 40)),
                 int(rng.integers(0, 6)), int(rng.integers(0, 30)), 190)
        L = int(rng.integers(1, 30))
        seq = rng.integers(0, K, size=L)
        xB = max(0, prof.base - (prof.tjb_fixed + prof.tbm))
        cmin = min(int(prof.cost[x, 0]) for x in seq)
        hit = max(0, xB + bias - cmin)
        if hit >= 255 - bias or hit - prof.tec > prof.base:
            continue
        raw, flag, _ = one(oracle.MSV, prof, seq)
        assert (raw, flag) == (max(0, hit - prof.tec), 0)


def test_single_residue_closed_form():
    rng = np.random.default_rng(12)
    for _ in range(200):
        M = int(rng.integers(1, 30))
        K = 3
        bias = int(rng.integers(0, 50))
        prof = P(rng.integers(0, 256, size=(K, M)), bias, int(rng.integers(0, 40)),
                 int(rng.integers(0, 6)), int(rng.integers(0, 30)), 190)
        x = int(rng.integers(0, K))
        best = max(bias - int(c) for c in prof.cost[x])
        raw, flag, _ = one(oracle.SSV, prof, [x])
        assert (raw, flag) == (min(255, max(0, best)), int(best >= 255))
        xB = max(0, prof.base - (prof.tjb_fixed + prof.tbm))
        xE = max(0, xB + best)
        raw, flag, _ = one(oracle.MSV, prof, [x])
        if xE >= 255 - bias:
            assert (raw, flag) == (255, 1)
        else:
            assert (raw, flag) == (max(0, xE - prof.tec), 0)


@pytest.mark.parametrize("d", [-5, 0, 1, 3, 17, 60, 127])
def test_constant_cost_ssv(d):
    """bias - cost = d everywhere: the best segment is the longest diagonal."""
    bias = 200
    for M in (1, 4, 9):
        for L in (0, 1, 2, 5, 12):
            prof = P(np.full((2, M), bias - d), bias, 5, 3, 9, 190)
            raw, flag, _ = one(oracle.SSV, prof, [0] * L)
            exact = max(0, d * min(M, L))
            assert (raw, flag) == (min(255, exact), int(exact >= 255))


# ------------------------------------------------------------ invariants ---

def test_filter_invariants_on_generated_profiles():
    rng = np.random.default_rng(5)
    profs = [synth.make_profile(M, rng) for M in (20, 60, 150)]
    db = synth.make_database(300, 120, 5, 600, rng)
    synth.plant_segments(db, profs, 0.3, rng)
    n_flag = n_ok = 0
    for p in profs:
        mr, mf, mn = oracle.msv(p, db.residues, db.offsets, db.lengths)
        sr, sf, sn = oracle.ssv(p, db.residues, db.offsets, db.lengths)
        assert np.all(mf[sf == 1] == 1), "an SSV overflow implies an MSV overflow"
        ok = (mf == 0) & (sf == 0) & (sr > 0)
        assert np.all(mn[ok] >= sn[ok] - 1e-5), "MSV is at least the single best hit"
        n_flag += int(mf.sum())
        n_ok += int(ok.sum())
    assert n_flag > 0 and n_ok > 0


def test_appending_residues_never_lowers_ssv():
    rng = np.random.default_rng(9)
    p = synth.make_profile(40, rng)
    seq = synth.draw_residues(200, rng)
    prev = -1
    for L in range(0, 201, 10):
        raw, _, _ = one(oracle.SSV, p, seq[:L])
        assert raw >= prev
        prev = raw


def test_codes_at_or_above_K_score_cost_255():
    rng = np.random.default_rng(13)
    base = rng.integers(0, 256, size=(5, 7))
    wide = np.vstack([base, np.full((3, 7), 255)])
    for bias in (10, 200):
        pk = P(base, bias, 4, 2, 6, 190)
        pw = P(wide, bias, 4, 2, 6, 190)
        seq = rng.integers(0, 8, size=40)
        for f in (oracle.MSV, oracle.SSV):
            assert one(f, pk, seq) == one(f, pw, seq)


def test_tjb_lut_selects_by_length():
    lut = np.array([1, 2, 3, 9], dtype=np.uint8)
    p_lut = P([[4, 6, 8]], 12, 5, 3, 0, 190, lut=lut)
    for L, t in ((0, 1), (2, 3), (3, 9), (10, 9)):
        p_fix = P([[4, 6, 8]], 12, 5, 3, t, 190)
        seq = [0] * L
        for f in (oracle.MSV, oracle.SSV):
            assert one(f, p_lut, seq) == one(f, p_fix, seq)


def test_nat_against_exact_arithmetic():
    rng = np.random.default_rng(21)
    p = synth.make_profile(80, rng)
    db = synth.make_database(200, 150, 10, 500, rng)
    t = p.tjb_by_len[np.minimum(db.lengths, p.tjb_by_len.size - 1)].astype(int)
    inv = 1 / Fraction(p.scale)
    for f, num in ((oracle.MSV, lambda r, t: r - t - p.base),
                   (oracle.SSV, lambda r, t: r - p.tbm - p.tec - 2 * t)):
        raw, flag, nat = oracle.scan(f, p, db.residues, db.offsets, db.lengths)
        for r, fl, n, tt in zip(raw, flag, nat, t):
            if fl:
                assert math.isinf(n)
                continue
            exact = float(num(int(r), int(tt)) * inv - 3)
            assert abs(n - exact) <= 3 * np.spacing(np.float32(abs(exact)) + np.float32(1))


def test_index_selects_and_threads_agree():
    rng = np.random.default_rng(31)
    p = synth.make_profile(64, rng)
    db = synth.make_database(500, 100, 1, 400, rng)
    full = oracle.msv(p, db.residues, db.offsets, db.lengths, nthreads=1)
    par = oracle.msv(p, db.residues, db.offsets, db.lengths, nthreads=4)
    for a, b in zip(full, par):
        np.testing.assert_array_equal(a, b)
    idx = np.array([499, 3, 3, 0, 250], np.uint64)
    sub = oracle.msv(p, db.residues, db.offsets, db.lengths, index=idx)
    for a, b in zip(full, sub):
        np.testing.assert_array_equal(a[idx.astype(np.int64)], b)
