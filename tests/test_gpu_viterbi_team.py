"""The Viterbi team kernel (four warps per sequence), on the GPU against the
oracle, bit-exact.

The MSV -> Viterbi stage (rank lists counted on the device) scores profiles
whose scores are all <= 0 and M > 224 with a team of four warps per
sequence, each sweeping a quarter of every lane's segment.  The cases cover
segment lengths whose quarters are ragged or leave the last quarter empty
(Q = 8, 9, 13, 76, 96 nodes per lane), the smallest and largest team
lengths, overflow, pass fractions from a few sequences to all of them,
empty and one-residue sequences, one call that mixes team, one-warp and
general-kernel queries, scans with more sequences than the team kernel
takes (the one-warp kernels), and one launch whose two queries of the same
length fall on either side of the team limit on the device.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle
from paper_1707_09683_gb300 import build, mpf, synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    build.build()
    oracle.build()
    return mpf.Context(0)


def _dev(n, dtype):
    return torch.empty(max(n, 1), dtype=dtype, device=torch.device("cuda", 0))


def _stage(ctx, vprofs, dbh, keep, rng):
    """Rescore vprofs over dbh with synthetic MSV outputs that pass a
    fraction `keep` of the finite scores; compare with the oracle."""
    db = mpf.Database(ctx, dbh.residues, dbh.offsets, dbh.lengths)
    vps = [mpf.VitProfile(ctx, v) for v in vprofs]
    n, q = db.n_seqs, len(vps)
    mf = rng.choice(np.array([0, 1, 2], np.uint8), size=q * n, p=[0.9, 0.04, 0.06])
    mn = rng.normal(0.0, 4.0, q * n).astype(np.float32)
    mn[mf == 2] = np.nan
    mn[mf == 1] = np.inf
    fin = mn[mf == 0]
    thr = float(np.quantile(fin, 1.0 - keep)) if 0 < keep < 1 else (1e30 if keep == 0 else -1e30)
    s, f, x = _dev(q * n, torch.int16), _dev(q * n, torch.uint8), _dev(q * n, torch.float32)
    n_pass = _dev(q, torch.int32)
    mpf.viterbi_rescore(ctx, vps, db, torch.from_numpy(mf).cuda(), torch.from_numpy(mn).cuda(), thr,
                        s, f, x, n_pass)
    ctx.sync()
    gs, gf, gn, gp = s.cpu().numpy(), f.cpu().numpy(), x.cpu().numpy(), n_pass.cpu().numpy()
    n_ovf = 0
    for i, v in enumerate(vprofs):
        sl = slice(i * n, (i + 1) * n)
        (ws, wf, wn), npass = oracle.viterbi_stage(v, dbh.residues, dbh.offsets, dbh.lengths, mf[sl], mn[sl],
                                                   thr, nthreads=16)
        assert int(gp[i]) == npass, (i, v.M)
        assert np.array_equal(gf[sl], wf), (i, v.M, np.flatnonzero(gf[sl] != wf)[:8])
        assert np.array_equal(gs[sl], ws), (i, v.M, np.flatnonzero(gs[sl] != ws)[:8])
        assert np.array_equal(gn[sl].view(np.uint32), wn.view(np.uint32)), (i, v.M)
        n_ovf += int((wf == 1).sum())
    for p in vps:
        p.close()
    db.close()
    return n_ovf


@pytest.mark.parametrize("M", [225, 256, 257, 288, 300, 401, 2405, 3072])
def test_team_lengths(ctx, M):
    """Q = 8 (225-256), 9 (257-288: quarters of 3, 3, 3 and an empty one),
    10, 13 (quarters 4, 4, 4, 1), 76 and 96 nodes per lane."""
    rng = np.random.default_rng(1000 + M)
    wl = synth.make_workload(0, n_seqs=1500)
    _stage(ctx, [synth.make_vit_profile(M, rng)], wl.db, 0.3, rng)


@pytest.mark.parametrize("keep", [0.0, 0.001, 0.05, 1.0])
def test_team_pass_fractions(ctx, keep):
    rng = np.random.default_rng(1100 + int(keep * 1000))
    wl = synth.make_workload(1, n_seqs=4000)
    _stage(ctx, [synth.make_vit_profile(m, rng) for m in (800, 1600, 2405)], wl.db, keep, rng)


@pytest.mark.parametrize("seed", range(4))
def test_team_adversarial_nonpositive_moves(ctx, seed):
    """Moves <= 0 with arbitrary match scores: saturation at -32768 and
    overflow from positive matches."""
    rng = np.random.default_rng(1200 + seed)
    M = int(rng.integers(225, 3073))
    lo, hi = [(-32768, 32767), (-3000, 3000), (-600, 4000), (-20, 32767)][seed]
    v = synth.random_vit_profile(M, int(rng.integers(1, 33)), rng, lo=lo, hi=hi, moves_hi=0)
    db = synth.random_database(600, 150, rng, alphabet=32, min_len=0)
    n_ovf = _stage(ctx, [v], db, 1.0, rng)
    if seed == 3:
        assert n_ovf > 0


def test_team_short_sequences(ctx):
    rng = np.random.default_rng(1300)
    lengths = np.array([0, 1, 0, 2, 3, 5, 0, 1, 4, 7, 1], np.uint32)
    offsets = np.zeros(lengths.size, np.uint64)
    np.cumsum(lengths[:-1], dtype=np.uint64, out=offsets[1:])
    residues = rng.integers(0, 32, int(lengths.sum())).astype(np.uint8)
    db = synth.Database(residues=residues, offsets=offsets, lengths=lengths)
    _stage(ctx, [synth.make_vit_profile(700, rng)], db, 1.0, rng)


def test_team_mixed_with_other_kernels(ctx):
    """Team (fast, M > 224), one-warp (fast, M <= 224) and general-kernel
    queries in one rescore call, concurrently on the fork streams."""
    rng = np.random.default_rng(1400)
    wl = synth.make_workload(1, n_seqs=3000)
    vprofs = [synth.make_vit_profile(2405, rng), synth.make_vit_profile(100, rng),
              synth.random_vit_profile(900, 20, rng, lo=-3000, hi=300),
              synth.make_vit_profile(1000, rng), synth.make_vit_profile(48, rng)]
    _stage(ctx, vprofs, wl.db, 0.5, rng)


def _short_db(n, rng, max_len=16):
    return synth.random_database(n, max_len, rng, alphabet=20, min_len=1)


@pytest.mark.parametrize("M", [300, 1100, 2600])
def test_one_warp_kernel_many_sequences(ctx, M):
    """A scan of 20,000 sequences: more than the team kernel's limit for
    these lengths (about Q/8 sequences per resident one-warp worker), so the
    one-warp kernels score it (plain rows; at M = 2600 the variant without
    the stored D row)."""
    rng = np.random.default_rng(1500 + M)
    db = _short_db(20000, rng)
    dbd = mpf.Database(ctx, db.residues, db.offsets, db.lengths)
    v = synth.make_vit_profile(M, rng)
    vp = mpf.VitProfile(ctx, v)
    n = dbd.n_seqs
    s, f, x = _dev(n, torch.int16), _dev(n, torch.uint8), _dev(n, torch.float32)
    mpf.viterbi_scan(ctx, [vp], dbd, s, f, x)
    ctx.sync()
    ws, wf, wn = oracle.viterbi(v, db.residues, db.offsets, db.lengths, nthreads=16)
    assert np.array_equal(f.cpu().numpy(), wf)
    assert np.array_equal(s.cpu().numpy(), ws)
    assert np.array_equal(x.cpu().numpy().view(np.uint32), wn.view(np.uint32))
    vp.close()
    dbd.close()


def test_dual_launch_splits_queries_by_survivors(ctx):
    """Two queries of one length in one rescore call (one launch group):
    one passes every sequence (one-warp kernel), the other a few (team
    kernel); the choice is taken on the device from the survivor counts."""
    rng = np.random.default_rng(1600)
    db = _short_db(20000, rng)
    dbd = mpf.Database(ctx, db.residues, db.offsets, db.lengths)
    vprofs = [synth.make_vit_profile(1100, rng), synth.make_vit_profile(1100, rng)]
    vps = [mpf.VitProfile(ctx, v) for v in vprofs]
    n = dbd.n_seqs
    mf = np.zeros(2 * n, np.uint8)
    mn = np.zeros(2 * n, np.float32)
    mn[n:] = rng.normal(0.0, 1.0, n).astype(np.float32)
    thr = float(np.quantile(mn[n:], 0.99))          # query 0: all pass; query 1: 1%
    mn[:n] = thr + 1.0
    s, f, x = _dev(2 * n, torch.int16), _dev(2 * n, torch.uint8), _dev(2 * n, torch.float32)
    n_pass = _dev(2, torch.int32)
    mpf.viterbi_rescore(ctx, vps, dbd, torch.from_numpy(mf).cuda(), torch.from_numpy(mn).cuda(), thr,
                        s, f, x, n_pass)
    ctx.sync()
    gs, gf, gn, gp = s.cpu().numpy(), f.cpu().numpy(), x.cpu().numpy(), n_pass.cpu().numpy()
    for i, v in enumerate(vprofs):
        sl = slice(i * n, (i + 1) * n)
        (ws, wf, wn), npass = oracle.viterbi_stage(v, db.residues, db.offsets, db.lengths, mf[sl], mn[sl],
                                                   thr, nthreads=16)
        assert int(gp[i]) == npass
        assert np.array_equal(gf[sl], wf) and np.array_equal(gs[sl], ws)
        assert np.array_equal(gn[sl].view(np.uint32), wn.view(np.uint32))
    assert int(gp[0]) == n and 0 < int(gp[1]) < n // 50
    for p in vps:
        p.close()
    dbd.close()
