"""P7Viterbi filter (Eq. 1) on the GPU against the oracle, bit-exact.

Scores, overflow flags and nat scores of the CUDA kernel must equal the
scalar oracle's for every sequence: realistic profiles at model lengths from
one node to the largest, with every kind of ragged end of the 32 lane
segments; adversarial profiles with uniform int16 scores (saturation at both
ends, overflow, positive transitions) for both kernels; positive delete
chains that start from -32768 and reach the begin state's row; several
queries of different lengths and kernels in one launch; host and device
outputs; the hand-worked golden cases; and the MSV -> Viterbi stage.
"""
import json
import os

import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle
from paper_1707_09683_gb300 import build, mpf, synth

pytestmark = pytest.mark.gpu

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "viterbi_hand_examples.json")


@pytest.fixture(scope="module")
def ctx():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    build.build()
    oracle.build()
    return mpf.Context(0)


def _dev(n, dtype):
    return torch.empty(max(n, 1), dtype=dtype, device=torch.device("cuda", 0))


def _scan_device(ctx, vps, db, n_q):
    n = db.n_seqs
    s, f, x = _dev(n_q * n, torch.int16), _dev(n_q * n, torch.uint8), _dev(n_q * n, torch.float32)
    mpf.viterbi_scan(ctx, vps, db, s, f, x)
    ctx.sync()
    return s.cpu().numpy()[:n_q * n], f.cpu().numpy()[:n_q * n], x.cpu().numpy()[:n_q * n]


def _check(got, want, tag):
    gs, gf, gn = got
    ws, wf, wn = want
    assert np.array_equal(gf, wf), (tag, np.flatnonzero(gf != wf)[:10])
    assert np.array_equal(gs, ws), (tag, np.flatnonzero(gs != ws)[:10])
    assert np.array_equal(gn.view(np.uint32), wn.view(np.uint32)), tag


def _run(ctx, vprofs, dbh, nthreads=16):
    db = mpf.Database(ctx, dbh.residues, dbh.offsets, dbh.lengths)
    vps = [mpf.VitProfile(ctx, v) for v in vprofs]
    got = _scan_device(ctx, vps, db, len(vps))
    n = db.n_seqs
    for i, v in enumerate(vprofs):
        want = oracle.viterbi(v, dbh.residues, dbh.offsets, dbh.lengths, nthreads=nthreads)
        sl = slice(i * n, (i + 1) * n)
        _check((got[0][sl], got[1][sl], got[2][sl]), want, (i, v.M))
    for p in vps:
        p.close()
    db.close()
    return got


@pytest.mark.parametrize("M", [1, 2, 31, 32, 33, 63, 100, 257, 400])
def test_realistic_profiles(ctx, M):
    rng = np.random.default_rng(100 + M)
    wl = synth.make_workload(0, n_seqs=1500)
    v = synth.make_vit_profile(M, rng)
    _run(ctx, [v], wl.db)


def test_long_model(ctx):
    rng = np.random.default_rng(7)
    wl = synth.make_workload(0, n_seqs=300)
    _run(ctx, [synth.make_vit_profile(2405, rng)], wl.db)


def test_largest_model(ctx):
    rng = np.random.default_rng(8)
    db = synth.random_database(40, 300, rng, alphabet=20)
    _run(ctx, [synth.make_vit_profile(mpf.max_striped_length(), rng)], db)


@pytest.mark.parametrize("seed", range(6))
def test_adversarial_profiles(ctx, seed):
    rng = np.random.default_rng(200 + seed)
    M = int(rng.integers(1, 300))
    K = int(rng.integers(1, 33))
    lo, hi = [(-32768, 32767), (-3000, 3000), (-300, 40), (-32768, -20000),
              (-50, 500), (0, 32767)][seed]
    v = synth.random_vit_profile(M, K, rng, lo=lo, hi=hi)
    db = synth.random_database(700, 120, rng, alphabet=32)
    got = _run(ctx, [v], db)
    if seed == 5:
        assert got[1].any()   # positive scores overflow


@pytest.mark.parametrize("seed", range(6))
def test_adversarial_nonpositive_moves(ctx, seed):
    """Transition and special scores <= 0 (the fast kernel) with arbitrary
    match scores: saturation at -32768, overflow from positive matches."""
    rng = np.random.default_rng(300 + seed)
    M = int(rng.integers(1, 700))
    K = int(rng.integers(1, 33))
    lo, hi = [(-32768, 32767), (-3000, 3000), (-300, 300), (-32768, 0),
              (-600, 4000), (-20, 32767)][seed]
    v = synth.random_vit_profile(M, K, rng, lo=lo, hi=hi, moves_hi=0)
    db = synth.random_database(700, 150, rng, alphabet=32)
    got = _run(ctx, [v], db)
    if seed == 5:
        assert got[1].any()


@pytest.mark.parametrize("M", [1100, 2100, 2600, 3000])
def test_long_segment_variants(ctx, M):
    """Long segments (35-94 nodes per lane), realistic and adversarial (moves
    <= 0).  With 160 sequences these scans go to the team kernel; the
    one-warp kernel's long-segment variants (deeper unrolling, no stored D
    row) are checked on 20,000 sequences in test_gpu_viterbi_team."""
    rng = np.random.default_rng(400 + M)
    db = synth.random_database(160, 220, rng, alphabet=32)
    _run(ctx, [synth.make_vit_profile(M, rng),
               synth.random_vit_profile(M - 7, 29, rng, lo=-2500, hi=2500, moves_hi=0)], db)


@pytest.mark.parametrize("M", [1, 2, 33, 95, 300, 1000, 2405, 3072])
@pytest.mark.parametrize("kind", [0, 1])
def test_positive_delete_chains(ctx, M, kind):
    rng = np.random.default_rng(500 + 7 * M + kind)
    db = synth.random_database(200 if M > 1000 else 600, 60, rng, alphabet=32, min_len=0)
    _run(ctx, [synth.positive_chain_vit_profile(M, int(rng.integers(1, 33)), rng, kind)], db)


@pytest.mark.parametrize("M", [700, 1500, 2405, 3072])
def test_general_kernel_long_models(ctx, M):
    """The general kernel at segment lengths where it unrolls deeper, with
    mixed-sign scores of realistic and saturating size."""
    rng = np.random.default_rng(600 + M)
    db = synth.random_database(150, 200, rng, alphabet=32)
    _run(ctx, [synth.random_vit_profile(M, 25, rng, lo=-3000, hi=400),
               synth.random_vit_profile(M - 5, 32, rng, lo=-32768, hi=32767)], db)


def test_multi_query_launch(ctx):
    rng = np.random.default_rng(9)
    wl = synth.make_workload(0, n_seqs=800)
    vprofs = [synth.make_vit_profile(M, rng) for M in (45, 700, 1, 128, 333)]
    vprofs.append(synth.random_vit_profile(90, 20, rng, lo=-400, hi=60))        # general kernel
    vprofs.append(synth.random_vit_profile(1500, 20, rng, lo=-400, hi=60))
    vprofs.append(synth.random_vit_profile(70, 20, rng, lo=-900, hi=400, moves_hi=0))
    _run(ctx, vprofs, wl.db)


def test_empty_and_short_sequences(ctx):
    rng = np.random.default_rng(10)
    lengths = np.array([0, 1, 0, 2, 3, 5, 0, 1], np.uint32)
    offsets = np.zeros(lengths.size, np.uint64)
    np.cumsum(lengths[:-1], dtype=np.uint64, out=offsets[1:])
    residues = rng.integers(0, 32, int(lengths.sum())).astype(np.uint8)
    db = synth.Database(residues=residues, offsets=offsets, lengths=lengths)
    _run(ctx, [synth.make_vit_profile(50, rng),
               synth.random_vit_profile(37, 7, rng, lo=-2000, hi=2000)], db)


def test_golden_cases(ctx):
    with open(GOLDEN) as fh:
        cases = json.load(fh)["cases"]
    for c in cases:
        v = synth.VitProfile(M=c["M"], K=c["K"], msc=np.array(c["msc"], np.int16),
                             trans=np.array(c["trans"], np.int16),
                             special=np.array(c["special"], np.int16), base=c["base"],
                             scale=float(np.float32(c.get("scale", synth.VIT_SCALE))))
        seq = np.array(c["seq"], np.uint8)
        db = mpf.Database(ctx, seq, np.zeros(1, np.uint64), np.array([seq.size], np.uint32))
        vp = mpf.VitProfile(ctx, v)
        s, f, x = _scan_device(ctx, [vp], db, 1)
        assert int(f[0]) == int(c["flag"]), c["name"]
        assert int(s[0]) == int(c["score"]), c["name"]
        vp.close()
        db.close()


def test_host_outputs_match_device_outputs(ctx):
    rng = np.random.default_rng(11)
    wl = synth.make_workload(0, n_seqs=500)
    db = mpf.Database(ctx, wl.db.residues, wl.db.offsets, wl.db.lengths)
    vps = [mpf.VitProfile(ctx, synth.make_vit_profile(M, rng)) for M in (80, 200)]
    n = db.n_seqs
    hs, hf, hn = np.zeros(2 * n, np.int16), np.zeros(2 * n, np.uint8), np.zeros(2 * n, np.float32)
    mpf.viterbi_scan(ctx, vps, db, hs, hf, hn)
    ds, df, dn = _scan_device(ctx, vps, db, 2)
    assert np.array_equal(hs, ds) and np.array_equal(hf, df)
    assert np.array_equal(hn.view(np.uint32), dn.view(np.uint32))


@pytest.mark.parametrize("keep", [0.0, 0.02, 0.3, 1.0])
def test_msv_to_viterbi_stage(ctx, keep):
    rng = np.random.default_rng(12)
    wl = synth.make_workload(2, n_seqs=6000, n_queries=3)
    dbh = wl.db
    db = mpf.Database(ctx, dbh.residues, dbh.offsets, dbh.lengths)
    vprofs = [synth.make_vit_profile(p.M, rng) for p in wl.profiles]
    vps = [mpf.VitProfile(ctx, v) for v in vprofs]
    n, q = db.n_seqs, len(vps)
    # MSV-stage inputs as the pipeline leaves them: flags 0 / 1 / 2 (filtered,
    # NaN), finite nat scores elsewhere.
    mf = rng.choice(np.array([0, 1, 2], np.uint8), size=q * n, p=[0.85, 0.05, 0.10])
    mn = rng.normal(0.0, 4.0, q * n).astype(np.float32)
    mn[mf == 2] = np.nan
    mn[mf == 1] = np.inf
    fin = mn[mf == 0]
    thr = float(np.quantile(fin, 1.0 - keep)) if 0 < keep < 1 else (1e30 if keep == 0 else -1e30)
    d_mf = torch.from_numpy(mf).cuda()
    d_mn = torch.from_numpy(mn).cuda()
    s, f, x = _dev(q * n, torch.int16), _dev(q * n, torch.uint8), _dev(q * n, torch.float32)
    n_pass = _dev(q, torch.int32)
    mpf.viterbi_rescore(ctx, vps, db, d_mf, d_mn, thr, s, f, x, n_pass)
    ctx.sync()
    gs, gf, gn, gp = s.cpu().numpy(), f.cpu().numpy(), x.cpu().numpy(), n_pass.cpu().numpy()
    for i, v in enumerate(vprofs):
        sl = slice(i * n, (i + 1) * n)
        want, npass = oracle.viterbi_stage(v, dbh.residues, dbh.offsets, dbh.lengths, mf[sl], mn[sl],
                                           thr, nthreads=16)
        assert int(gp[i]) == npass
        _check((gs[sl], gf[sl], gn[sl]), want, (keep, i))
    for p in vps:
        p.close()
    db.close()


def test_three_stage_pipeline(ctx):
    """SSV -> MSV -> Viterbi on device buffers end to end."""
    rng = np.random.default_rng(13)
    wl = synth.make_workload(2, n_seqs=5000, n_queries=2)
    dbh = wl.db
    db = mpf.Database(ctx, dbh.residues, dbh.offsets, dbh.lengths)
    profs = [mpf.Profile(ctx, p) for p in wl.profiles]
    vprofs = [synth.make_vit_profile(p.M, rng) for p in wl.profiles]
    vps = [mpf.VitProfile(ctx, v) for v in vprofs]
    n, q = db.n_seqs, len(profs)
    ssv_out = (_dev(q * n, torch.uint8), _dev(q * n, torch.uint8), _dev(q * n, torch.float32))
    msv_out = (_dev(q * n, torch.uint8), _dev(q * n, torch.uint8), _dev(q * n, torch.float32))
    n1 = _dev(q, torch.int32)
    ssv_thr, msv_thr = 0.5, 2.0
    mpf.pipeline_scan(ctx, profs, db, ssv_thr, ssv_out, msv_out, n1)
    s, f, x = _dev(q * n, torch.int16), _dev(q * n, torch.uint8), _dev(q * n, torch.float32)
    n2 = _dev(q, torch.int32)
    mpf.viterbi_rescore(ctx, vps, db, msv_out[1], msv_out[2], msv_thr, s, f, x, n2)
    ctx.sync()
    gs, gf, gn, gp = s.cpu().numpy(), f.cpu().numpy(), x.cpu().numpy(), n2.cpu().numpy()
    for i, p in enumerate(wl.profiles):
        _, (mr, mf, mn), _ = oracle.pipeline(p, dbh.residues, dbh.offsets, dbh.lengths, ssv_thr,
                                             nthreads=16)
        want, npass = oracle.viterbi_stage(vprofs[i], dbh.residues, dbh.offsets, dbh.lengths, mf,
                                           mn, msv_thr, nthreads=16)
        sl = slice(i * n, (i + 1) * n)
        assert int(gp[i]) == npass
        _check((gs[sl], gf[sl], gn[sl]), want, i)


def test_invalid_arguments(ctx):
    rng = np.random.default_rng(14)
    too_long = synth.make_vit_profile(mpf.max_model_length() + 1, rng)
    with pytest.raises(mpf.MpfError) as e:
        mpf.VitProfile(ctx, too_long)
    assert e.value.status == mpf.MPF_EUNSUPPORTED
    bad_scale = synth.make_vit_profile(20, rng)
    bad_scale.scale = 0.0
    with pytest.raises(mpf.MpfError) as e:
        mpf.VitProfile(ctx, bad_scale)
    assert e.value.status == mpf.MPF_EINVAL
    dbh = synth.random_database(20, 30, rng)
    db = mpf.Database(ctx, dbh.residues, dbh.offsets, dbh.lengths)
    vp = mpf.VitProfile(ctx, synth.make_vit_profile(30, rng))
    n = db.n_seqs
    host_flag = np.zeros(n, np.uint8)
    host_nat = np.zeros(n, np.float32)
    s, f, x = _dev(n, torch.int16), _dev(n, torch.uint8), _dev(n, torch.float32)
    with pytest.raises(mpf.MpfError) as e:      # stage inputs must be device buffers
        mpf.viterbi_rescore(ctx, [vp], db, host_flag, host_nat, 0.0, s, f, x, _dev(1, torch.int32))
    assert e.value.status == mpf.MPF_EINVAL
    with pytest.raises(mpf.MpfError) as e:      # NaN threshold
        mpf.viterbi_rescore(ctx, [vp], db, f, x, float("nan"), s, f, x, _dev(1, torch.int32))
    assert e.value.status == mpf.MPF_EINVAL
    vp.close()
    db.close()
