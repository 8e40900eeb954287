"""SSV -> MSV hand-off and P-values on the GPU against the oracle."""
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
    return torch.empty(n, dtype=dtype, device=torch.device("cuda", 0))


@pytest.mark.parametrize("keep", [0.0, 0.03, 0.5, 1.0])
def test_pipeline_matches_oracle(ctx, keep):
    wl = synth.make_workload(2, n_seqs=9000, n_queries=5)   # planted: overflows pass too
    db = mpf.Database(ctx, wl.db.residues, wl.db.offsets, wl.db.lengths)
    profs = [mpf.Profile(ctx, p) for p in wl.profiles]
    n, q = db.n_seqs, len(profs)
    # threshold so that about `keep` of the sequences pass (from the oracle's SSV)
    sn_all = np.concatenate([oracle.ssv(p, wl.db.residues, wl.db.offsets, wl.db.lengths, nthreads=8)[2]
                             for p in wl.profiles])
    fin = sn_all[np.isfinite(sn_all)]
    thr = float(np.quantile(fin, 1.0 - keep)) if 0 < keep < 1 else (1e30 if keep == 0 else -1e30)
    ssv_out = (_dev(q * n, torch.uint8), _dev(q * n, torch.uint8), _dev(q * n, torch.float32))
    msv_out = (_dev(q * n, torch.uint8), _dev(q * n, torch.uint8), _dev(q * n, torch.float32))
    n_pass = _dev(q, torch.int32)
    mpf.pipeline_scan(ctx, profs, db, thr, ssv_out, msv_out, n_pass)
    ctx.sync()
    got_s = [t.cpu().numpy() for t in ssv_out]
    got_m = [t.cpu().numpy() for t in msv_out]
    got_n = n_pass.cpu().numpy()
    for i, p in enumerate(wl.profiles):
        (sr, sf, sn), (mr, mf, mn), npass = oracle.pipeline(p, wl.db.residues, wl.db.offsets,
                                                            wl.db.lengths, thr, nthreads=8)
        sl = slice(i * n, (i + 1) * n)
        assert np.array_equal(got_s[0][sl], sr) and np.array_equal(got_s[1][sl], sf)
        assert np.array_equal(got_s[2][sl].view(np.uint32), sn.view(np.uint32))
        assert int(got_n[i]) == npass
        assert np.array_equal(got_m[0][sl], mr) and np.array_equal(got_m[1][sl], mf)
        assert np.array_equal(got_m[2][sl].view(np.uint32), mn.view(np.uint32))
    if 0 < keep < 1:
        assert 0 < got_n.sum() < q * n


def test_pvalues_within_float32_error(ctx):
    rng = np.random.default_rng(3)
    mu, lam = -3.7, float(np.float32(np.log(2)))
    x = np.concatenate([rng.normal(0, 6, 20000), [np.inf, np.nan, mu, 40.0, -40.0]]).astype(np.float32)
    d = torch.from_numpy(x).cuda()
    out = torch.empty_like(d)
    mpf.pvalues(ctx, d, mu, lam, out)
    ctx.sync()
    got = out.cpu().numpy().astype(np.float64)
    want = oracle.gumbel_pvalue(x.astype(np.float64), float(np.float32(mu)), lam)
    # float32 evaluation: t = lam (x - mu) carries ~2 ulp, exp/expm1 ~2 ulp each,
    # so the relative error is bounded by ~2^-23 (|t| + 6).
    t = np.abs(lam * (x.astype(np.float64) - mu))
    tol = 2.0 ** -23 * (np.where(np.isfinite(t), t, 0) + 6) * np.abs(want) + 1e-37
    ok = np.isfinite(want)
    assert np.all(np.abs(got[ok] - want[ok]) <= tol[ok])
    assert got[-5] == 0.0 and np.isnan(got[-4])


def test_hand_off_rejects_overlapping_buffers(ctx):
    """The hand-offs read one stage's outputs while they write the next
    stage's: buffers that share memory are refused (MPF_EINVAL) before any
    work is queued, and a correct call on the same context still succeeds."""
    wl = synth.make_workload(0, n_seqs=500, n_queries=1)
    db = mpf.Database(ctx, wl.db.residues, wl.db.offsets, wl.db.lengths)
    prof = mpf.Profile(ctx, wl.profiles[0])
    n = db.n_seqs
    lib = mpf.load()
    arr = mpf._handles([prof])
    ssv = (_dev(n, torch.uint8), _dev(n, torch.uint8), _dev(n, torch.float32))
    msv = (_dev(n, torch.uint8), _dev(n, torch.uint8), _dev(n, torch.float32))
    n_pass = _dev(1, torch.int32)
    big = _dev(8 * n, torch.float32)
    p = lambda t: t.data_ptr()
    aliased = [
        (p(ssv[0]), p(ssv[1]), p(ssv[2]), p(msv[0]), p(ssv[1]), p(msv[2])),   # msv_flag = ssv_flag
        (p(ssv[0]), p(ssv[1]), p(ssv[2]), p(msv[0]), p(msv[1]), p(ssv[2])),   # msv_nat = ssv_nat
        (p(ssv[0]), p(ssv[1]), p(big), p(msv[0]), p(msv[1]), p(big) + 4 * n - 4),   # one float shared
    ]
    for a in aliased:
        st = lib.mpf_pipeline_scan(ctx.handle, arr, 1, db.handle, 0.0, *a, p(n_pass))
        assert st == mpf.MPF_EINVAL, mpf.strerror(st)
    # MSV -> Viterbi: the Viterbi outputs may not overlap the MSV inputs.
    vp = mpf.VitProfile(ctx, synth.make_vit_profile(wl.profiles[0].M, np.random.default_rng(2)))
    varr = mpf._handles([vp])
    score = _dev(n, torch.int16)
    st = lib.mpf_viterbi_rescore(ctx.handle, varr, 1, db.handle, p(msv[1]), p(msv[2]), 0.0,
                                 p(score), p(msv[1]), p(big), p(n_pass))
    assert st == mpf.MPF_EINVAL, mpf.strerror(st)
    st = lib.mpf_viterbi_rescore(ctx.handle, varr, 1, db.handle, p(msv[1]), p(msv[2]), 0.0,
                                 p(score), p(ssv[1]), p(msv[2]), p(n_pass))
    assert st == mpf.MPF_EINVAL, mpf.strerror(st)
    ctx.sync()
    mpf.pipeline_scan(ctx, [prof], db, 0.0, ssv, msv, n_pass)
    ctx.sync()
    (sr, sf, sn), (mr, mf, mn), npass = oracle.pipeline(wl.profiles[0], wl.db.residues, wl.db.offsets,
                                                        wl.db.lengths, 0.0, nthreads=4)
    assert int(n_pass.item()) == npass
    assert np.array_equal(msv[1].cpu().numpy(), mf) and np.array_equal(msv[0].cpu().numpy(), mr)
    vp.close()
    prof.close()
    db.close()
