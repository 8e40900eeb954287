"""Models longer than the striped kernels hold (the long-model kernel), on
the GPU against the oracle, bit-exact on raw, flag and nat.

Realistic and adversarial profiles at lengths that leave every possible
ragged end (M mod 128, the partial last word of a lane, the last tile of
the tiled kernels), planted hits that send some sequences from the tiled
MSV pass to the exact kernel, the largest supported model, single scans,
batches and plans that mix long and striped profiles, rank lists from the
SSV -> MSV hand-off, and the configuration and allocation-free calls that
long profiles do not take.
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


def _check_filter(ctx, gf, of, recs, dbh, nthreads=16, table=None):
    db = mpf.Database(ctx, dbh.residues, dbh.offsets, dbh.lengths)
    profs = [mpf.Profile(ctx, r) for r in recs]
    if table is not None:
        for pr in profs:
            pr.set_table_memory(gf, table)
    n, q = db.n_seqs, len(profs)
    raw, flag, nat = _dev(q * n, torch.uint8), _dev(q * n, torch.uint8), _dev(q * n, torch.float32)
    mpf.scan_batch(ctx, gf, profs, db, raw, flag, nat)
    ctx.sync()
    raw, flag, nat = raw.cpu().numpy(), flag.cpu().numpy(), nat.cpu().numpy()
    n_flag = 0
    for i, r in enumerate(recs):
        er, ef, en = oracle.scan(of, r, dbh.residues, dbh.offsets, dbh.lengths, nthreads=nthreads)
        sl = slice(i * n, (i + 1) * n)
        assert np.array_equal(flag[sl], ef), (gf, r.M, np.flatnonzero(flag[sl] != ef)[:8])
        assert np.array_equal(raw[sl], er), (gf, r.M, np.flatnonzero(raw[sl] != er)[:8])
        assert np.array_equal(nat[sl].view(np.uint32), en.view(np.uint32)), (gf, r.M)
        n_flag += int(ef.sum())
    for p in profs:
        p.close()
    db.close()
    return n_flag


def _both(ctx, recs, dbh):
    return sum(_check_filter(ctx, gf, of, recs, dbh)
               for gf, of in ((mpf.MSV, oracle.MSV), (mpf.SSV, oracle.SSV)))


@pytest.mark.parametrize("M", [3073, 3100, 3201, 4000, 5001, 12345])
def test_realistic_long_profiles(ctx, M):
    rng = np.random.default_rng(M)
    wl = synth.make_workload(0, n_seqs=600)
    _both(ctx, [synth.make_profile(M, rng)], wl.db)


@pytest.mark.parametrize("seed", range(5))
def test_adversarial_long_profiles(ctx, seed):
    rng = np.random.default_rng(40 + seed)
    M = int(rng.integers(3073, 7000))
    K = int(rng.integers(1, 33))
    bias = [0, 17, 128, 250, 255][seed]
    rec = synth.random_profile(M, K, rng, bias=bias, with_lut=bool(seed % 2))
    db = synth.random_database(300, 200, rng, alphabet=32)
    _both(ctx, [rec], db)


@pytest.mark.parametrize("M", [29000, 31000])
def test_byte_row_storage_lengths(ctx, M):
    """Around the length where the exact MSV kernel's DP row switches from
    16-bit pairs to bytes (fewer than four warps per SM with pairs): a
    profile whose begin score cannot be held (bias 250) takes that kernel;
    the others the tiled kernels."""
    rng = np.random.default_rng(M)
    wl = synth.make_workload(0, n_seqs=120)
    _both(ctx, [synth.make_profile(M, rng), synth.random_profile(M + 77, 24, rng, bias=90),
                synth.random_profile(M + 5, 20, rng, bias=250)], wl.db)


def test_strong_long_profile_overflows_and_chains(ctx):
    rng = np.random.default_rng(5)
    rec = synth.random_profile(4100, 20, rng, cost_hi=40, bias=30, tbm=5, tec=2)
    db = synth.random_database(200, 400, rng, alphabet=20, min_len=1)
    assert _both(ctx, [rec], db) > 0


@pytest.mark.parametrize("M", [3500, 5000])
def test_planted_hits_mix_tiled_and_exact_msv(ctx, M):
    """Realistic long profile, 30% of the sequences carrying a segment drawn
    from its own emissions: for about a third of them xJ passes base in
    mid-sequence, so the tiled MSV pass leaves them to the exact
    lane-segment kernel, and the others it scores itself; both filters,
    bit-exact."""
    rng = np.random.default_rng(10 + M)
    rec = synth.make_profile(M, rng)
    db = synth.make_database(400, 355, 10, 2000, rng)
    synth.plant_segments(db, [rec], 0.3, rng)
    _both(ctx, [rec], db)


def test_long_profiles_on_empty_and_zero_length_databases(ctx):
    """No sequences, and only sequences of length 0 or 1: the tiled kernels'
    columns and the MSV fallback list at their smallest."""
    rng = np.random.default_rng(11)
    recs = [synth.make_profile(4000, rng), synth.random_profile(3300, 20, rng, cost_hi=40, bias=30, tbm=5, tec=2)]
    lengths = np.array([0, 1, 0, 1, 1, 0], np.uint32)
    offsets = np.zeros(lengths.size, np.uint64)
    np.cumsum(lengths[:-1], dtype=np.uint64, out=offsets[1:])
    tiny = synth.Database(residues=rng.integers(0, 20, int(lengths.sum())).astype(np.uint8),
                          offsets=offsets, lengths=lengths)
    _both(ctx, recs, tiny)
    empty = synth.Database(residues=np.zeros(0, np.uint8), offsets=np.zeros(0, np.uint64),
                           lengths=np.zeros(0, np.uint32))
    db = mpf.Database(ctx, empty.residues, empty.offsets, empty.lengths)
    profs = [mpf.Profile(ctx, r) for r in recs]
    out = (_dev(0, torch.uint8), _dev(0, torch.uint8), _dev(0, torch.float32))
    for f in (mpf.MSV, mpf.SSV):
        mpf.scan_batch(ctx, f, profs, db, *out)
    ctx.sync()
    for p in profs:
        p.close()
    db.close()


def test_largest_model(ctx):
    rng = np.random.default_rng(6)
    M = mpf.max_model_length()
    rec = synth.make_profile(M, rng)
    db = synth.random_database(12, 60, rng, alphabet=20)
    _both(ctx, [rec], db)
    with pytest.raises(mpf.MpfError) as e:
        mpf.Profile(ctx, synth.random_profile(M + 1, 20, rng))
    assert e.value.status == mpf.MPF_EUNSUPPORTED


def test_batch_and_plan_mix_long_and_striped(ctx):
    rng = np.random.default_rng(7)
    wl = synth.make_workload(0, n_seqs=800)
    recs = [synth.make_profile(m, rng) for m in (300, 3500, 2405, 6000, 48)]
    _both(ctx, recs, wl.db)
    db = mpf.Database(ctx, wl.db.residues, wl.db.offsets, wl.db.lengths)
    profs = [mpf.Profile(ctx, r) for r in recs]
    n, q = db.n_seqs, len(profs)
    outs = [(_dev(q * n, torch.uint8), _dev(q * n, torch.uint8), _dev(q * n, torch.float32))
            for _ in range(2)]
    mpf.scan_batch(ctx, mpf.MSV, profs, db, *outs[0])
    plan = mpf.Plan(ctx, mpf.MSV, profs, db, *outs[1])
    plan.capture_graph()
    plan.launch()
    ctx.sync()
    for a, b in zip(outs[0], outs[1]):
        assert torch.equal(a, b)
    plan.close()


def test_pipeline_with_long_profiles(ctx):
    rng = np.random.default_rng(8)
    wl = synth.make_workload(2, n_seqs=3000, n_queries=2)
    recs = [synth.make_profile(4200, rng), wl.profiles[0]]
    db = mpf.Database(ctx, wl.db.residues, wl.db.offsets, wl.db.lengths)
    profs = [mpf.Profile(ctx, r) for r in recs]
    n, q = db.n_seqs, len(profs)
    ssv_out = (_dev(q * n, torch.uint8), _dev(q * n, torch.uint8), _dev(q * n, torch.float32))
    msv_out = (_dev(q * n, torch.uint8), _dev(q * n, torch.uint8), _dev(q * n, torch.float32))
    n_pass = _dev(q, torch.int32)
    thr = -6.0
    mpf.pipeline_scan(ctx, profs, db, thr, ssv_out, msv_out, n_pass)
    ctx.sync()
    got_m = [t.cpu().numpy() for t in msv_out]
    got_n = n_pass.cpu().numpy()
    for i, r in enumerate(recs):
        _, (mr, mf, mn), npass = oracle.pipeline(r, wl.db.residues, wl.db.offsets, wl.db.lengths,
                                                 thr, nthreads=16)
        sl = slice(i * n, (i + 1) * n)
        assert int(got_n[i]) == npass
        assert np.array_equal(got_m[0][sl], mr) and np.array_equal(got_m[1][sl], mf)
        assert np.array_equal(got_m[2][sl].view(np.uint32), mn.view(np.uint32))


def test_long_profiles_take_one_configuration(ctx):
    rng = np.random.default_rng(9)
    p = mpf.Profile(ctx, synth.make_profile(3500, rng))
    assert p.get_config(mpf.MSV) == (32, 0) and p.get_config(mpf.SSV) == (32, 0)
    with pytest.raises(mpf.MpfError):
        p.set_config(mpf.MSV, 32, 48)
    db = mpf.Database(ctx, *(lambda d: (d.residues, d.offsets, d.lengths))(
        synth.random_database(10, 50, rng)))
    n = db.n_seqs
    with pytest.raises(mpf.MpfError) as e:
        mpf.scan_noalloc(ctx, mpf.MSV, p, db, _dev(n, torch.uint8), _dev(n, torch.uint8))
    assert e.value.status == mpf.MPF_EUNSUPPORTED


@pytest.mark.parametrize("table", [mpf.TABLE_AUTO, mpf.TABLE_SHARED])
def test_tiles_in_tensor_and_shared_memory(ctx, table):
    """The tiled kernels with the tile's scores in tensor memory (the
    automatic choice: one block of 16 warps per SM) and in shared memory:
    ragged last tiles, planted hits that send sequences from the tiled MSV
    pass to the exact kernel, a strong profile that overflows, and the
    both-filter sweep of the same profiles; all against the oracle."""
    rng = np.random.default_rng(91 + table)
    recs = [synth.make_profile(M, rng) for M in (3073, 4100, 5000)]
    recs.append(synth.random_profile(3500, 20, rng, cost_hi=26, bias=20, base=190, tbm=10, tec=3, tjb=8))
    dbh = synth.make_database(700, 400, 0, 3000, rng)
    synth.plant_segments(dbh, recs[:3], 0.1, rng, seg=(30, 300))
    n_flag = 0
    for gf, of in ((mpf.MSV, oracle.MSV), (mpf.SSV, oracle.SSV)):
        n_flag += _check_filter(ctx, gf, of, recs, dbh, table=table)
    assert n_flag > 0
    db = mpf.Database(ctx, dbh.residues, dbh.offsets, dbh.lengths)
    profs = [mpf.Profile(ctx, r) for r in recs]
    for pr in profs:
        for gf in (mpf.MSV, mpf.SSV):
            pr.set_table_memory(gf, table)
            assert pr.get_table_memory(gf) == (mpf.TABLE_TENSOR if table == mpf.TABLE_AUTO else mpf.TABLE_SHARED)
    n, q = db.n_seqs, len(profs)
    outs = [_dev(2 * q * n, dt) for dt in (torch.uint8, torch.uint8, torch.float32)]
    plan = mpf.Plan(ctx, mpf.MSV_SSV, profs, db, *outs)
    assert all(g["filters"] == 3 for g in plan.groups())
    plan.launch()
    ctx.sync()
    got = [t.cpu().numpy() for t in outs]
    plan.close()
    for fb, of in enumerate((oracle.MSV, oracle.SSV)):
        for i, r in enumerate(recs):
            er, ef, en = oracle.scan(of, r, dbh.residues, dbh.offsets, dbh.lengths, nthreads=16)
            sl = slice((fb * q + i) * n, (fb * q + i + 1) * n)
            assert np.array_equal(got[1][sl], ef) and np.array_equal(got[0][sl], er), (fb, r.M)
            assert np.array_equal(got[2][sl].view(np.uint32), en.view(np.uint32)), (fb, r.M)
    for pr in profs:
        pr.close()
    db.close()
