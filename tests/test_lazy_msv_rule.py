"""The decision rules of the MSV passes that hold the begin score (the tiled
pass of long models and the striped kernels' held pass), restated in numpy,
against the oracle (CPU).

For models longer than the striped table the MSV kernel sweeps the model
in tiles with the begin score b held at its initial value, where v =
max(0, dp - b) follows the SSV recurrence (Alg. 7's form), and decides each
sequence from the first row whose maximum over the model passes
T = min(base + tec - b, 255 - bias - b - 1): none (raw from the largest
cell, or from the best single-cell score of the residues when no cell rose
above b), an overflow at that row, the last row, or otherwise a row after
which xB would move (the sequence is rescored exactly).  This test checks
that every outcome but the last equals Alg. 2 as the oracle computes it,
on random profiles that satisfy the rule's precondition (the begin path
cannot saturate: sat(base - tjb - tbm) < 255 - bias), with enough strong
profiles and planted hits that every outcome occurs.  The striped held pass
decides from the largest cell of the whole sequence instead of the first row
above T: overflow at or above 255 - bias - b, exact at or below T, rescored
in between.
"""
import numpy as np
import pytest

import oracle
from paper_1707_09683_gb300 import synth


def _sat8(v):
    return min(255, max(0, v))


def _tjb(rec, L):
    if rec.tjb_by_len is not None:
        return int(rec.tjb_by_len[min(L, len(rec.tjb_by_len) - 1)])
    return int(rec.tjb_fixed)


def _holds_b(rec):
    tmin = int(rec.tjb_by_len.min()) if rec.tjb_by_len is not None else int(rec.tjb_fixed)
    return rec.bias < 255 and _sat8(rec.base - (tmin + rec.tbm)) < 255 - rec.bias


def lazy_msv(rec, seq):
    """(raw, flag) by the tiled pass's rule, or None for a rescored sequence."""
    M, L = rec.M, len(seq)
    s = rec.bias - np.vstack([rec.cost.astype(np.int64), np.full((32 - rec.K, M), 255, np.int64)])
    t = _tjb(rec, L)
    cap = 255 - rec.bias
    b = min(_sat8(rec.base - (t + rec.tbm)), cap)
    T = min(rec.base + rec.tec - b, cap - b - 1)
    v = np.zeros(M, np.int64)
    V, first, m_first = 0, None, None
    for i, x in enumerate(seq):
        prev = np.concatenate(([0], v[:-1]))
        v = np.maximum(0, prev + s[x])
        m = int(v.max())
        V = max(V, m)
        if first is None and m > T:
            first, m_first = i, m
    if L == 0:
        return 0, 0
    if first is not None:
        if b + m_first >= cap:
            return 255, 1
        if first + 1 < L:
            return None
        return max(0, b + V - rec.tec), 0
    if V > 0:
        return max(0, b + V - rec.tec), 0
    g = max(int(s[x].max()) for x in seq)
    return max(0, b + g - rec.tec), 0


def held_msv(rec, seq):
    """(raw, flag) by the striped kernels' held pass (MSV_HELD), or None for
    a sequence it lists for exact rescoring: b held for every row, V the
    largest cell of any row; V >= 255 - bias - b is an overflow, V <= T
    leaves the held rows exact, anything between is rescored."""
    M, L = rec.M, len(seq)
    s = rec.bias - np.vstack([rec.cost.astype(np.int64), np.full((32 - rec.K, M), 255, np.int64)])
    t = _tjb(rec, L)
    cap = 255 - rec.bias
    b = min(_sat8(rec.base - (t + rec.tbm)), cap)
    T = min(rec.base + rec.tec - b, cap - b - 1)
    v = np.zeros(M, np.int64)
    V = 0
    for x in seq:
        v = np.maximum(0, np.concatenate(([0], v[:-1])) + s[x])
        V = max(V, int(v.max()))
    if L == 0:
        return 0, 0
    if V >= cap - b:
        return 255, 1
    if V > T:
        return None
    if V > 0:
        return max(0, b + V - rec.tec), 0
    g = max(int(s[x].max()) for x in seq)
    return max(0, b + g - rec.tec), 0


def _cases(rng):
    """Realistic profiles with planted hits, and uniform profiles of several
    strengths, keeping those that hold b."""
    out = []
    for _ in range(6):
        rec = synth.make_profile(int(rng.integers(20, 120)), rng)
        db = synth.make_database(40, 60, 5, 200, rng)
        synth.plant_segments(db, [rec], 0.4, rng, seg=(5, 60))
        out.append((rec, db))
    for cost_hi, bias in ((255, None), (120, 40), (80, 40), (60, 30), (40, 30)):
        for _ in range(4):
            rec = synth.random_profile(int(rng.integers(1, 60)), int(rng.integers(1, 33)), rng, cost_hi=cost_hi,
                                       bias=bias, tbm=int(rng.integers(0, 30)), tec=int(rng.integers(0, 10)),
                                       with_lut=bool(rng.integers(2)))
            out.append((rec, synth.random_database(30, 80, rng, alphabet=32, min_len=0)))
    return [(r, d) for r, d in out if _holds_b(r)]


@pytest.mark.parametrize("rule", [lazy_msv, held_msv], ids=["tiled", "held"])
@pytest.mark.parametrize("seed", range(3))
def test_tiled_msv_rule_matches_alg2(seed, rule):
    oracle.build()
    rng = np.random.default_rng(2024 + seed)
    outcomes = {"none": 0, "overflow": 0, "rescored": 0}
    for rec, db in _cases(rng):
        raw, flag, _ = oracle.msv(rec, db.residues, db.offsets, db.lengths)
        for k in range(db.n_seqs):
            o, L = int(db.offsets[k]), int(db.lengths[k])
            got = rule(rec, db.residues[o:o + L])
            if got is None:
                outcomes["rescored"] += 1
                continue
            assert got == (int(raw[k]), int(flag[k])), (rec.M, k, got, int(raw[k]), int(flag[k]))
            outcomes["overflow" if got[1] else "none"] += 1
    assert all(n > 0 for n in outcomes.values()), outcomes


@pytest.mark.parametrize("rule", [lazy_msv, held_msv], ids=["tiled", "held"])
def test_tiled_msv_rule_threshold_edges(rule):
    """Scores placed on T, T + 1 and the overflow boundary 255 - bias - b
    (and one either side), on one- to three-node models, over every
    sequence of length 1 to 3: the threshold and the overflow test of the
    rule match Alg. 2 exactly at their edges."""
    oracle.build()
    rng = np.random.default_rng(77)
    checked = 0
    # T is base + tec - b in the first three, the overflow bound
    # 255 - bias - b - 1 in the last two.
    for bias, tbm, tec, base in ((20, 5, 3, 190), (60, 10, 2, 190), (40, 0, 0, 150), (60, 10, 6, 190),
                                 (90, 20, 9, 180)):
        b = min(_sat8(base - (0 + tbm)), 255 - bias)
        cap = 255 - bias
        T = min(base + tec - b, cap - b - 1)
        targets = sorted({T - 1, T, T + 1, cap - b - 1, cap - b, cap - b + 1})
        for M in (1, 2, 3):
            for tgt in targets:
                c = bias - tgt
                if not 0 <= c <= 255:
                    continue
                rec = synth.random_profile(M, 2, rng, cost_hi=255, bias=bias, tbm=tbm, tec=tec, base=base)
                rec.tjb_fixed = 0
                rec.cost[:] = 255
                rec.cost[0, :] = c                      # code 0 scores tgt at every node
                rec.cost[1, 0] = min(255, bias + 3)     # code 1: a small loss at node 1
                if not _holds_b(rec):
                    continue
                seqs = [np.array(s, np.uint8) for L in (1, 2, 3)
                        for s in np.ndindex(*(3,) * L)]  # codes 0, 1 and 2 (>= K)
                lengths = np.array([len(s) for s in seqs], np.uint32)
                offsets = np.zeros(len(seqs), np.uint64)
                np.cumsum(lengths[:-1], dtype=np.uint64, out=offsets[1:])
                residues = np.concatenate(seqs)
                raw, flag, _ = oracle.msv(rec, residues, offsets, lengths)
                for k, sq in enumerate(seqs):
                    got = rule(rec, sq)
                    if got is not None:
                        assert got == (int(raw[k]), int(flag[k])), (bias, M, tgt, sq.tolist(), got)
                        checked += 1
    assert checked > 500


def test_packed_threshold_test_equals_the_halfwise_comparison():
    """The striped MSV kernel tests "some 16-bit half of the running maximum
    exceeds the key K" as ((vacc + pack2(0x7fff - K)) & 0x80008000) != 0.
    For halves and keys in [0, 0x7fff] that equals the comparison of each
    half, and no half's sum carries into the other."""
    h = np.arange(0, 0x8000, dtype=np.int64)
    for K in list(range(0, 0x8000, 97)) + [0x7bff, 0x7ffe, 0x7fff]:
        s = h + (0x7fff - K)
        assert np.all(s < 0x10000)
        assert np.array_equal((s & 0x8000) != 0, h > K)
    rng = np.random.default_rng(4)
    lo = rng.integers(0, 0x8000, 200000, dtype=np.int64)
    hi = rng.integers(0, 0x8000, 200000, dtype=np.int64)
    K = rng.integers(0, 0x8000, 200000, dtype=np.int64)
    packed = (lo | (hi << 16)) + ((0x7fff - K) | ((0x7fff - K) << 16))
    got = (packed & 0x80008000) != 0
    assert np.array_equal(got, (lo > K) | (hi > K))


def held_sweep_max(rec, seq):
    """The largest cell V of the held-b sweep (the recurrence both the held
    MSV pass and SSV run: v = max(0, v'[k-1] + s))."""
    M = rec.M
    s = rec.bias - np.vstack([rec.cost.astype(np.int64), np.full((32 - rec.K, M), 255, np.int64)])
    v = np.zeros(M, np.int64)
    V = 0
    for x in seq:
        v = np.maximum(0, np.concatenate(([0], v[:-1])) + s[x])
        V = max(V, int(v.max()))
    return V


@pytest.mark.parametrize("seed", range(3))
def test_one_sweep_gives_both_filters(seed):
    """Both filters from one sweep (MPF_MSV_SSV): the held sweep's largest
    cell V gives SSV as Alg. 7 defines it (raw = min(V, 255), overflow iff
    V >= 255) and the held MSV decision, on the same profiles and planted
    sequences as above and on strong profiles whose segments overflow;
    every SSV score and flag of the oracle is matched."""
    oracle.build()
    rng = np.random.default_rng(4040 + seed)
    checked = flags = 0
    strong = [(synth.random_profile(int(rng.integers(5, 60)), 20, rng, cost_hi=26, bias=20, base=190, tbm=10,
                                    tec=3, tjb=8), synth.random_database(40, 120, rng, alphabet=20, min_len=0))
              for _ in range(4)]
    for rec, db in _cases(rng) + [c for c in strong if _holds_b(c[0])]:
        sraw, sflag, _ = oracle.ssv(rec, db.residues, db.offsets, db.lengths)
        raw, flag, _ = oracle.msv(rec, db.residues, db.offsets, db.lengths)
        for k in range(db.n_seqs):
            o, L = int(db.offsets[k]), int(db.lengths[k])
            sq = db.residues[o:o + L]
            V = held_sweep_max(rec, sq)
            assert (min(V, 255), int(V >= 255)) == (int(sraw[k]), int(sflag[k])), (rec.M, k, V)
            got = held_msv(rec, sq)
            if got is not None:
                assert got == (int(raw[k]), int(flag[k]))
            checked += 1
            flags += int(V >= 255)
    assert checked > 500 and flags > 0
