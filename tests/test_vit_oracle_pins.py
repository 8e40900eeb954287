"""Pins of the P7Viterbi oracle (oracle/mpf_vit_oracle.c) against things other
than itself: hand-worked cases, an unsaturated integer DP written
differently (vectorised rows, explicit -inf), and a brute-force enumeration
of every Plan-7 path (N loop, hits through M/I/D states, J between hits, C
loop) on tiny inputs."""
import functools
import json
import math
import os

import numpy as np
import pytest

import oracle
from paper_1707_09683_gb300 import synth

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "viterbi_hand_examples.json")
NEG = -32768


class VP:
    def __init__(self, msc, trans, special, base, scale=synth.VIT_SCALE):
        self.msc = np.asarray(msc, np.int16)
        self.trans = np.asarray(trans, np.int16)
        self.special = np.asarray(special, np.int16)
        self.K, self.M = self.msc.shape
        self.base = base
        self.scale = float(np.float32(scale))


def one(p, seq):
    seq = np.asarray(seq, np.uint8)
    s, f, n = oracle.viterbi(p, seq, np.zeros(1, np.uint64), np.array([seq.size], np.uint32))
    return int(s[0]), int(f[0]), float(n[0])


def test_hand_worked_examples():
    cases = json.load(open(GOLDEN))["cases"]
    for c in cases:
        tr = np.array(c["trans"], np.int16).T.copy() if np.array(c["trans"]).shape[0] == 8 else None
        p = VP(c["msc"], np.array(c["trans"], np.int16), c["special"], c["base"])
        s, f, nat = one(p, c["seq"])
        assert (s, f) == (c["score"], c["flag"]), c["name"]
        if not f:
            want = np.float32(c["score"] - c["base"]) / np.float32(p.scale) - np.float32(3)
            assert nat == pytest.approx(float(want), abs=1e-6)


# ------------------------------------------------------ unsaturated DP ---

def vit_int(p, seq):
    """Eq. 1 and the special states over unbounded integers, -inf exact."""
    M = p.M
    t = {n: p.trans[i].astype(np.int64) for i, n in enumerate(oracle.VIT_TRANSITIONS)}
    for n in t:
        t[n] = np.where(t[n] == NEG, -10**15, t[n])   # -32768 inputs mean impossible
    sp = dict(zip(oracle.VIT_SPECIALS, p.special.astype(np.int64)))
    NI = -10**15
    Mr = np.full(M, NI); Ir = np.full(M, NI); Dr = np.full(M, NI)
    xN, xJ, xC = p.base, NI, NI
    xB = xN + sp["NB"]
    for x in seq:
        e = p.msc[x].astype(np.int64) if x < p.K else np.full(M, NI)
        shM = np.concatenate(([NI], Mr[:-1])); shI = np.concatenate(([NI], Ir[:-1]))
        shD = np.concatenate(([NI], Dr[:-1]))
        Mn = np.maximum.reduce([shM + t["MM"], shI + t["IM"], shD + t["DM"], xB + t["BM"]]) + e
        In = np.maximum(Mr + t["MI"], Ir + t["II"])
        In[-1] = NI
        Dn = np.full(M, NI)
        for k in range(1, M):
            Dn[k] = max(Mn[k - 1] + t["MD"][k], Dn[k - 1] + t["DD"][k])
        xE = max(Mn.max(), Dn.max())
        xN = xN + sp["NN"]
        xC = max(xC + sp["CC"], xE + sp["EC"])
        xJ = max(xJ + sp["JJ"], xE + sp["EJ"])
        xB = max(xN + sp["NB"], xJ + sp["JB"])
        Mr, Ir, Dr = Mn, In, Dn
    return xC + sp["CT"]


def small_profile(rng, M, K, lo=-300, hi=200):
    tr = rng.integers(lo, hi, size=(8, M)).astype(np.int16)
    tr[1:4, 0] = NEG; tr[6, 0] = NEG; tr[7, :min(2, M)] = NEG; tr[4:6, M - 1] = NEG
    return VP(rng.integers(lo, hi, size=(K, M)), tr, rng.integers(lo, hi, size=8), int(rng.integers(-500, 500)))


@pytest.mark.parametrize("seed", range(4))
def test_equals_unsaturated_integer_dp(seed):
    rng = np.random.default_rng(600 + seed)
    for _ in range(60):
        M = int(rng.integers(1, 9)); K = int(rng.integers(1, 5))
        p = small_profile(rng, M, K)
        seq = rng.integers(0, K, size=int(rng.integers(1, 25)))
        s, f, _ = one(p, seq)
        assert f == 0
        assert s == vit_int(p, seq), (M, K, len(seq))


# ---------------------------------------------------- path enumeration ---

def vit_paths(p, seq):
    """Best score over every Plan-7 path, by explicit enumeration: N emits a
    prefix, then hits (local alignments entered B->M_k, moving through M, I, D
    states, leaving M_j or D_j to E) separated by J regions, then C."""
    M, L = p.M, len(seq)
    tr = {n: [int(v) for v in p.trans[i]] for i, n in enumerate(oracle.VIT_TRANSITIONS)}
    sp = dict(zip(oracle.VIT_SPECIALS, [int(v) for v in p.special]))
    def e(i, k):                      # residue i (0-based) emitted by M_k (0-based)
        return int(p.msc[seq[i], k]) if seq[i] < p.K else None
    def ok(v):
        return v is not None and v > NEG

    @functools.lru_cache(maxsize=None)
    def hit(i, state, k):
        """Best score from state (M/I/D at node k, residue i consumed by it or,
        for D, the last consumed residue is i) to E; returns {end_row: score}."""
        best = {}
        def put(r, v):
            if r not in best or v > best[r]:
                best[r] = v
        if state in ("M", "D"):
            put(i, 0)                                    # exit to E
        if state == "M":
            if k + 1 < M and i + 1 < L and ok(tr["MM"][k + 1]) and ok(e(i + 1, k + 1)):
                for r, v in hit(i + 1, "M", k + 1).items():
                    put(r, v + tr["MM"][k + 1] + e(i + 1, k + 1))
            if k < M - 1 and i + 1 < L and ok(tr["MI"][k]):
                for r, v in hit(i + 1, "I", k).items():
                    put(r, v + tr["MI"][k])
            if k + 1 < M and ok(tr["MD"][k + 1]):
                for r, v in hit(i, "D", k + 1).items():
                    put(r, v + tr["MD"][k + 1])
        elif state == "I":
            if i + 1 < L and ok(tr["II"][k]):
                for r, v in hit(i + 1, "I", k).items():
                    put(r, v + tr["II"][k])
            if k + 1 < M and i + 1 < L and ok(tr["IM"][k + 1]) and ok(e(i + 1, k + 1)):
                for r, v in hit(i + 1, "M", k + 1).items():
                    put(r, v + tr["IM"][k + 1] + e(i + 1, k + 1))
        else:  # D
            if k + 1 < M and i + 1 < L and ok(tr["DM"][k + 1]) and ok(e(i + 1, k + 1)):
                for r, v in hit(i + 1, "M", k + 1).items():
                    put(r, v + tr["DM"][k + 1] + e(i + 1, k + 1))
            if k + 1 < M and ok(tr["DD"][k + 1]):
                for r, v in hit(i, "D", k + 1).items():
                    put(r, v + tr["DD"][k + 1])
        return best

    @functools.lru_cache(maxsize=None)
    def from_b(s, vb):
        """Best final score given B reached before row s (hit starts at row s)
        with score vb."""
        best = None
        for k in range(M):
            if not (ok(tr["BM"][k]) and ok(e(s, k))):
                continue
            for r, v in hit(s, "M", k).items():
                xe = vb + tr["BM"][k] + e(s, k) + v
                c = xe + sp["EC"] + (L - 1 - r) * sp["CC"] + sp["CT"]     # to C, loop to the end
                best = c if best is None else max(best, c)
                for s2 in range(r + 1, L):                                 # through J
                    vj = xe + sp["EJ"] + (s2 - 1 - r) * sp["JJ"] + sp["JB"]
                    b2 = from_b(s2, vj)
                    if b2 is not None:
                        best = max(best, b2)
        return best

    best = None
    for s in range(L):
        vb = p.base + s * sp["NN"] + sp["NB"]
        b = from_b(s, vb)
        if b is not None:
            best = b if best is None else max(best, b)
    return best


@pytest.mark.parametrize("seed", range(3))
def test_equals_path_enumeration(seed):
    rng = np.random.default_rng(700 + seed)
    done = 0
    while done < 40:
        M = int(rng.integers(1, 4)); K = int(rng.integers(1, 3))
        p = small_profile(rng, M, K, lo=-60, hi=40)
        seq = rng.integers(0, K, size=int(rng.integers(1, 5)))
        want = vit_paths(p, seq)
        if want is None:
            continue
        s, f, _ = one(p, seq)
        assert (s, f) == (want, 0), (M, K, list(seq))
        done += 1


def test_single_node_single_residue_closed_form():
    rng = np.random.default_rng(5)
    for _ in range(100):
        p = small_profile(rng, 1, 3)
        x = int(rng.integers(0, 3))
        sp = dict(zip(oracle.VIT_SPECIALS, [int(v) for v in p.special]))
        want = p.base + sp["NB"] + int(p.trans[0, 0]) + int(p.msc[x, 0]) + sp["EC"] + sp["CT"]
        assert one(p, [x])[:2] == (want, 0)


def test_generated_profiles_and_codes_at_or_above_K():
    rng = np.random.default_rng(8)
    p = synth.make_vit_profile(60, rng)
    db = synth.make_database(200, 150, 10, 400, rng)
    s, f, n = oracle.viterbi(p, db.residues, db.offsets, db.lengths, nthreads=4)
    assert f.sum() == 0 and np.all(np.isfinite(n))
    # Codes >= K behave as extra residue rows scoring -32768 at every node.
    wide = np.vstack([p.msc, np.full((32 - p.K, p.M), NEG, np.int16)])
    pk = VP(p.msc, p.trans, p.special, p.base)
    pw = VP(wide, p.trans, p.special, p.base)
    for _ in range(30):
        seq = rng.integers(0, 32, size=int(rng.integers(0, 40)))
        assert one(pk, seq) == one(pw, seq)


def test_stage_selection_rule():
    """MSV -> Viterbi hand-off (Sec. 2.1): overflowed MSV scores pass whatever
    their nat, SSV-filtered entries (flag 2, NaN) never pass, the threshold
    is inclusive, and unselected entries read -32768 / 2 / NaN."""
    rng = np.random.default_rng(5)
    p = synth.make_vit_profile(20, rng)
    db = synth.random_database(6, 30, rng, alphabet=20, min_len=1)
    flag = np.array([0, 0, 1, 2, 0, 1], np.uint8)
    nat = np.array([1.0, 0.999, -50.0, np.nan, 2.0, np.inf], np.float32)
    (s, f, n), npass = oracle.viterbi_stage(p, db.residues, db.offsets, db.lengths, flag, nat, 1.0)
    sel = np.array([True, False, True, False, True, True])
    assert npass == 4
    full = oracle.viterbi(p, db.residues, db.offsets, db.lengths)
    assert np.array_equal(s[sel], full[0][sel]) and np.array_equal(f[sel], full[1][sel])
    assert np.all(s[~sel] == -32768) and np.all(f[~sel] == 2) and np.all(np.isnan(n[~sel]))
