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
