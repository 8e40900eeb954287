"""P7Viterbi filter (Eq. 1) on models longer than the shared-memory rows
hold (3,073 to 100,000 nodes: the kernels' device-memory rows), on the GPU
against the oracle, bit-exact on score, flag and nat.

Realistic profiles (the fast kernel) and adversarial ones (the general
kernel, including positive delete chains) at lengths with every kind of
ragged lane segment, the longest model, one call that mixes shared-memory
and device-memory groups of both kernels, and the MSV -> Viterbi stage on a
long model.
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


def _run(ctx, vprofs, dbh, nthreads=16):
    db = mpf.Database(ctx, dbh.residues, dbh.offsets, dbh.lengths)
    vps = [mpf.VitProfile(ctx, v) for v in vprofs]
    n, q = db.n_seqs, len(vps)
    s, f, x = _dev(q * n, torch.int16), _dev(q * n, torch.uint8), _dev(q * n, torch.float32)
    mpf.viterbi_scan(ctx, vps, db, s, f, x)
    ctx.sync()
    gs, gf, gn = s.cpu().numpy(), f.cpu().numpy(), x.cpu().numpy()
    n_ovf = 0
    for i, v in enumerate(vprofs):
        ws, wf, wn = oracle.viterbi(v, dbh.residues, dbh.offsets, dbh.lengths, nthreads=nthreads)
        sl = slice(i * n, (i + 1) * n)
        assert np.array_equal(gf[sl], wf), (i, v.M, np.flatnonzero(gf[sl] != wf)[:8])
        assert np.array_equal(gs[sl], ws), (i, v.M, np.flatnonzero(gs[sl] != ws)[:8])
        assert np.array_equal(gn[sl].view(np.uint32), wn.view(np.uint32)), (i, v.M)
        n_ovf += int(wf.sum())
    for p in vps:
        p.close()
    db.close()
    return n_ovf


@pytest.mark.parametrize("M", [3073, 3100, 4001, 6000, 12345])
def test_realistic_long_profiles(ctx, M):
    rng = np.random.default_rng(700 + M)
    wl = synth.make_workload(0, n_seqs=400 if M < 10000 else 120)
    _run(ctx, [synth.make_vit_profile(M, rng)], wl.db)


@pytest.mark.parametrize("seed", range(4))
def test_adversarial_long_profiles(ctx, seed):
    rng = np.random.default_rng(800 + seed)
    M = int(rng.integers(3073, 7000))
    K = int(rng.integers(1, 33))
    lo, hi, moves_hi = [(-32768, 32767, None), (-3000, 3000, None), (-3000, 3000, 0), (-600, 4000, 0)][seed]
    v = synth.random_vit_profile(M, K, rng, lo=lo, hi=hi, moves_hi=moves_hi)
    db = synth.random_database(250, 150, rng, alphabet=32)
    _run(ctx, [v], db)


@pytest.mark.parametrize("kind", [0, 1])
def test_positive_delete_chains_long(ctx, kind):
    rng = np.random.default_rng(900 + kind)
    db = synth.random_database(150, 60, rng, alphabet=32, min_len=0)
    _run(ctx, [synth.positive_chain_vit_profile(5000, 20, rng, kind)], db)


def test_overflow_on_long_model(ctx):
    rng = np.random.default_rng(901)
    v = synth.random_vit_profile(4500, 20, rng, lo=-50, hi=600, moves_hi=0)
    db = synth.random_database(120, 200, rng, alphabet=20, min_len=1)
    assert _run(ctx, [v], db) > 0


def test_longest_model(ctx):
    rng = np.random.default_rng(902)
    M = mpf.max_model_length()
    db = synth.random_database(12, 40, rng, alphabet=20)
    _run(ctx, [synth.make_vit_profile(M, rng), synth.random_vit_profile(M - 31, 20, rng, lo=-3000, hi=500)], db)


@pytest.mark.parametrize("M", [2405, 2800])
def test_device_rows_below_striped_length(ctx, M):
    """Lengths where shared-memory rows leave six or fewer warps per SM, on a
    database with enough sequences (8 per resident warp: 19,456 on 152 SMs)
    that the scan keeps the rows in device memory; a fast and a general
    profile."""
    rng = np.random.default_rng(905 + M)
    db = synth.random_database(21000, 24, rng, alphabet=20, min_len=1)
    _run(ctx, [synth.make_vit_profile(M, rng), synth.random_vit_profile(M, 20, rng, lo=-2500, hi=300)], db)


def test_mixed_groups_in_one_call(ctx):
    """Shared-memory and device-memory groups of both kernels, concurrently
    on the context's fork streams, each device-memory group with its own
    scratch."""
    rng = np.random.default_rng(903)
    wl = synth.make_workload(0, n_seqs=500)
    vprofs = [synth.make_vit_profile(3500, rng),
              synth.make_vit_profile(400, rng),
              synth.random_vit_profile(4200, 20, rng, lo=-3000, hi=300),
              synth.random_vit_profile(90, 20, rng, lo=-400, hi=60),
              synth.make_vit_profile(8000, rng)]
    _run(ctx, vprofs, wl.db)


def test_msv_to_viterbi_stage_long_model(ctx):
    rng = np.random.default_rng(904)
    wl = synth.make_workload(2, n_seqs=1500, n_queries=1)
    M = 4200
    rec = synth.make_profile(M, rng)
    vrec = synth.make_vit_profile(M, rng)
    db = mpf.Database(ctx, wl.db.residues, wl.db.offsets, wl.db.lengths)
    prof = mpf.Profile(ctx, rec)
    vp = mpf.VitProfile(ctx, vrec)
    n = db.n_seqs
    ssv_out = (_dev(n, torch.uint8), _dev(n, torch.uint8), _dev(n, torch.float32))
    msv_out = (_dev(n, torch.uint8), _dev(n, torch.uint8), _dev(n, torch.float32))
    n_pass = _dev(1, torch.int32)
    mpf.pipeline_scan(ctx, [prof], db, -1e9, ssv_out, msv_out, n_pass)   # SSV passes all
    s, f, x = _dev(n, torch.int16), _dev(n, torch.uint8), _dev(n, torch.float32)
    vpass = _dev(1, torch.int32)
    ctx.sync()
    mf, mn = msv_out[1].cpu().numpy(), msv_out[2].cpu().numpy()
    msv_thr = float(np.quantile(mn[np.isfinite(mn)], 0.7))   # NaN: filtered by SSV; inf: overflow
    mpf.viterbi_rescore(ctx, [vp], db, msv_out[1], msv_out[2], msv_thr, s, f, x, vpass)
    ctx.sync()
    (ws, wf, wn), npass = oracle.viterbi_stage(vrec, wl.db.residues, wl.db.offsets, wl.db.lengths,
                                               mf, mn, msv_thr, nthreads=16)
    assert int(vpass.cpu().numpy()[0]) == npass and npass > 0
    assert np.array_equal(f.cpu().numpy(), wf)
    assert np.array_equal(s.cpu().numpy(), ws)
    assert np.array_equal(x.cpu().numpy().view(np.uint32), wn.view(np.uint32))
    vp.close()
    prof.close()
    db.close()


def test_more_groups_than_fork_streams(ctx):
    """Twelve launch groups in one call (distinct lengths and kernels: one
    warp per sequence, team, general, rows in device memory), more than the
    context's eight fork streams, each device-row group with its own slice
    of scratch."""
    rng = np.random.default_rng(906)
    wl = synth.make_workload(0, n_seqs=400)
    vprofs = [synth.make_vit_profile(m, rng) for m in (40, 90, 150, 230, 500, 1000, 2405, 3500, 6000)]
    vprofs += [synth.random_vit_profile(m, 20, rng, lo=-3000, hi=300) for m in (120, 1500, 4100)]
    _run(ctx, vprofs, wl.db)
