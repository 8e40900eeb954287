"""The lane-segment algorithm of the Viterbi kernels, restated in Python,
against the Viterbi oracle (CPU).

Each kernel splits a row of Eq. 1 into S contiguous node segments (S = 32
lanes for one warp per sequence, 128 for the team kernel's quarter-lanes)
and computes, per row:
  * per segment a delete chain that assumes minus infinity enters it;
  * per segment the map d -> max(A, min(d + B, C)) of the delete score
    entering it to the score at its end, the maps composed in node order to
    give the true delete score entering every segment;
  * from those, the chain carried into the next row (its value at every
    node: max(local chain, carried chain));
  * E as the maximum of M and of the delete scores, the carried chain's
    maximum over a segment being its entry value plus the largest prefix
    sum of D->D there.
This test runs that algorithm with the general kernel's two-sided
saturation and checks score and overflow against the oracle on adversarial
profiles (including positive delete chains that climb from -32768 across
segments), for S = 32 and S = 128, so that a wrong composition, a wrong
entry of the carried chain or a missing D term in E shows up on the CPU.
"""
import numpy as np
import pytest

import oracle
from paper_1707_09683_gb300 import synth

NEG, POS, INF = -32768, 32767, -(1 << 29)


def _sat(v):
    return max(NEG, min(POS, v))


def segment_viterbi(v, seq, S):
    """(score, flag) of one sequence by the segmented row algorithm."""
    M = v.M
    Q = -(-M // S)
    seg = [(s * Q, min(M, (s + 1) * Q)) for s in range(S)]
    tr = [[int(x) for x in row] for row in v.trans]
    BM, MM, IM, DM, MI, II, MD, DD = tr
    tNN, tNB, tEC, tCC, tCT, tEJ, tJJ, tJB = (int(x) for x in v.special)
    # Per segment: Bsuf / Csuf, the composite of x -> min(x + tDD, POS) over
    # its nodes after the first, and maxP, the largest prefix sum of those
    # tDD (0 included).
    consts = []
    for a, b in seg:
        if b <= a:
            consts.append(None)
            continue
        B, C, mp = 0, 1 << 40, 0
        for k in range(a + 1, b):
            B, C = B + DD[k], min(C + DD[k], POS)
            mp = max(mp, B)
        consts.append((B, C, mp))
    Mp = [NEG] * M
    Ip = [NEG] * M
    Dloc = [NEG] * M          # previous row's segment-local chain
    X0 = [INF] * S            # chain carried into each segment's first node
    xN = int(v.base)
    xJ = xC = NEG
    xB = _sat(xN + tNB)
    Dtrue_prev_end = [NEG] * S   # previous row: true D at the node before each segment
    for x in seq:
        Mn = [NEG] * M
        In = [NEG] * M
        Dn = [NEG] * M
        ends = []
        mxM = mxD = NEG
        for s, (a, b) in enumerate(seg):
            if b <= a:
                ends.append(INF)
                continue
            X = X0[s]
            d = INF
            for k in range(a, b):
                if k > a:
                    X = min(X + DD[k], POS)
                Dprev_true = max(Dloc[k], X)          # previous row's true D at node k
                if k == a:
                    dM, dI, dD = (Mp[k - 1], Ip[k - 1], Dtrue_prev_end[s]) if k > 0 else (NEG, NEG, NEG)
                else:
                    dM, dI, dD = Mp[k - 1], Ip[k - 1], prev_true_D
                e = int(v.msc[x, k]) if x < v.K else NEG
                best = max(_sat(dM + MM[k]), _sat(dI + IM[k]), _sat(dD + DM[k]), _sat(xB + BM[k]))
                Mn[k] = _sat(best + e)
                In[k] = max(_sat(Mp[k] + MI[k]), _sat(Ip[k] + II[k]))
                d = INF if k == a else max(_sat(Mn[k - 1] + MD[k]), min(d + DD[k], POS))
                Dn[k] = NEG if k == a else d
                mxM = max(mxM, Mn[k])
                if k > a:
                    mxD = max(mxD, d)
                prev_true_D = Dprev_true
            ends.append(d)
        # Compose the segments' maps in node order: true D at each segment end.
        Dend = []
        carry = NEG            # true D entering segment 0 (D_1 = -inf)
        entry = []
        for s, (a, b) in enumerate(seg):
            if b <= a:
                entry.append(carry)
                Dend.append(carry)
                continue
            Bs, Cs, _ = consts[s]
            a0 = NEG if a == 0 else _sat(Mn[a - 1] + MD[a])
            d_first = NEG if a == 0 else max(min(carry + DD[a], POS), a0)   # true D at the first node
            A = max(ends[s], min(d_first + Bs, Cs)) if b - a > 1 else d_first
            entry.append(carry)
            Dend.append(A)
            carry = A
        # E over M and the true delete scores of this row.
        xE = mxM
        newX0 = []
        for s, (a, b) in enumerate(seg):
            if b <= a:
                newX0.append(INF)
                continue
            d_first = NEG if a == 0 else max(min(entry[s] + DD[a], POS), _sat(Mn[a - 1] + MD[a]))
            newX0.append(d_first)
            xd = max(mxD, d_first + consts[s][2])
            xE = max(xE, min(xd, POS))
        if xE >= POS:
            return POS, 1
        Mp, Ip, Dloc = Mn, In, Dn
        X0 = newX0
        Dtrue_prev_end = [entry[s] for s in range(S)]
        xN = _sat(xN + tNN)
        xC = max(_sat(xC + tCC), _sat(xE + tEC))
        xJ = max(_sat(xJ + tJJ), _sat(xE + tEJ))
        xB = max(_sat(xN + tNB), _sat(xJ + tJB))
    return _sat(xC + tCT), 0


def _profiles(rng):
    out = []
    for lo, hi in ((-32768, 32767), (-3000, 3000), (-300, 300), (-500, 40), (-20, 500)):
        out.append(synth.random_vit_profile(int(rng.integers(1, 200)), int(rng.integers(1, 33)), rng, lo=lo, hi=hi))
    for kind in (0, 1):
        out.append(synth.positive_chain_vit_profile(int(rng.integers(40, 300)), 20, rng, kind))
    out.append(synth.make_vit_profile(int(rng.integers(30, 300)), rng))
    return out


@pytest.mark.parametrize("S", [32, 128])
@pytest.mark.parametrize("seed", range(2))
def test_segment_rule_matches_oracle(S, seed):
    oracle.build()
    rng = np.random.default_rng(31 + seed)
    n = 0
    for v in _profiles(rng):
        db = synth.random_database(6, 14, rng, alphabet=32, min_len=0)
        score, flag, _ = oracle.viterbi(v, db.residues, db.offsets, db.lengths)
        for k in range(db.n_seqs):
            o, L = int(db.offsets[k]), int(db.lengths[k])
            got = segment_viterbi(v, db.residues[o:o + L], S)
            assert got == (int(score[k]), int(flag[k])), (v.M, S, k, got, int(score[k]), int(flag[k]))
            n += 1
    assert n == 48
