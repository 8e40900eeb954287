"""GPU parity: the CUDA scans through the C ABI against the scalar oracle.

Scores, overflow flags and nat scores must be bit-identical (integer work,
and a nat score computed by the same IEEE float operations).  Inputs are the
seeded synthetic workloads plus adversarial profiles and databases.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle
from paper_1707_09683_gb300 import build, mpf, synth

pytestmark = pytest.mark.gpu

FILTERS = ((mpf.MSV, oracle.MSV), (mpf.SSV, oracle.SSV))


@pytest.fixture(scope="module")
def ctx():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    build.build()
    oracle.build()
    c = mpf.Context(0)
    yield c
    c.sync()


def run_gpu(ctx, filt, prof, db, on_device=True):
    n = db.n_seqs
    if on_device:
        dev = torch.device("cuda", 0)
        raw = torch.empty(n, dtype=torch.uint8, device=dev)
        flag = torch.empty(n, dtype=torch.uint8, device=dev)
        nat = torch.empty(n, dtype=torch.float32, device=dev)
    else:
        raw = np.empty(n, np.uint8)
        flag = np.empty(n, np.uint8)
        nat = np.empty(n, np.float32)
    (mpf.msv_scan if filt == mpf.MSV else mpf.ssv_scan)(ctx, prof, db, raw, flag, nat)
    ctx.sync()
    if on_device:
        return raw.cpu().numpy(), flag.cpu().numpy(), nat.cpu().numpy()
    return raw, flag, nat


def assert_same(got, exp, what=""):
    graw, gflag, gnat = got
    eraw, eflag, enat = exp
    bad = np.flatnonzero((graw != eraw) | (gflag != eflag))
    assert bad.size == 0, f"{what}: {bad.size} raw/flag mismatches, first at {bad[:5]}: " \
        f"gpu {graw[bad[:5]]}/{gflag[bad[:5]]} oracle {eraw[bad[:5]]}/{eflag[bad[:5]]}"
    badn = np.flatnonzero(gnat.view(np.uint32) != enat.view(np.uint32))
    assert badn.size == 0, f"{what}: nat mismatch at {badn[:5]}: {gnat[badn[:5]]} vs {enat[badn[:5]]}"


def check_profile(ctx, p, db, ddb=None, filters=FILTERS, index=None, configs=None, arith=None):
    prof = mpf.Profile(ctx, p)
    if arith is not None:
        for gf, _ in filters:
            prof.set_arith(gf, arith)
    ddb = ddb or mpf.Database(ctx, db.residues, db.offsets, db.lengths)
    for gf, of in filters:
        exp = oracle.scan(of, p, db.residues, db.offsets, db.lengths, index=index, nthreads=8)
        for cfg in (configs or [None]):
            if cfg is not None:
                prof.set_config(gf, *cfg)
            got = run_gpu(ctx, gf, prof, ddb)
            if index is not None:
                got = tuple(a[index.astype(np.int64)] for a in got)
            assert_same(got, exp, f"filter {gf} M={p.M} cfg={cfg}")
    prof.close()


# ------------------------------------------------------------- workloads ---

def test_plain_workload_m100_full(ctx):
    """The M = 100, 10,000-sequence workload, every sequence."""
    wl = synth.make_workload(0)
    check_profile(ctx, wl.profiles[0], wl.db)


def test_model_length_sweep_small_db(ctx):
    """Every model length of the sweep workload on its first 3,000 sequences
    (tiles of every lane-group size, ragged model tails)."""
    wl = synth.make_workload(1, n_seqs=3000)
    ddb = mpf.Database(ctx, wl.db.residues, wl.db.offsets, wl.db.lengths)
    for p in wl.profiles:
        check_profile(ctx, p, wl.db, ddb)


def test_planted_overflow_batch_sample(ctx):
    """Uneven-batch workload shape with planted segments: overflow flags."""
    wl = synth.make_workload(2, n_seqs=4000, n_queries=6)
    ddb = mpf.Database(ctx, wl.db.residues, wl.db.offsets, wl.db.lengths)
    n_flag = 0
    for p in wl.profiles:
        prof = mpf.Profile(ctx, p)
        for gf, of in FILTERS:
            exp = oracle.scan(of, p, wl.db.residues, wl.db.offsets, wl.db.lengths, nthreads=8)
            got = run_gpu(ctx, gf, prof, ddb)
            assert_same(got, exp, f"planted M={p.M} filter {gf}")
            n_flag += int(exp[1].sum())
    assert n_flag > 0, "the planted workload must exercise overflow"


# ----------------------------------------------------------- adversarial ---

@pytest.mark.parametrize("seed", range(4))
def test_adversarial_profiles(ctx, seed):
    """Uniform random cost bytes, free special bytes (including begin scores
    that hit the 255 cap), residue codes 0..31, lengths 0..300."""
    rng = np.random.default_rng(500 + seed)
    db = synth.random_database(700, 300, rng, alphabet=32)
    ddb = mpf.Database(ctx, db.residues, db.offsets, db.lengths)
    for M in (1, 2, 3, 7, 33, 64, 65, 130, 257, 600, 1111):
        K = int(rng.integers(1, 33))
        p = synth.random_profile(M, K, rng, cost_hi=int(rng.choice([40, 255])),
                                 bias=int(rng.choice([0, 12, 60, 130, 254, 255])),
                                 base=int(rng.choice([60, 190, 250])),
                                 with_lut=bool(rng.integers(2)))
        check_profile(ctx, p, db, ddb)


@pytest.mark.parametrize("arith", [mpf.ARITH_I16, mpf.ARITH_F16])
def test_both_cell_arithmetics(ctx, arith):
    """Integer (DPX) and half-precision (HFMA2) cells give the same scores:
    adversarial bytes, strong profiles (J reuse, overflow far past 255) and
    long sequences whose cells would leave the exact half range after
    saturation."""
    rng = np.random.default_rng(900 + arith)
    db = synth.random_database(400, 600, rng, alphabet=32)
    long_db = synth.make_database(40, 8000, 4000, 12000, rng)
    ddb = mpf.Database(ctx, db.residues, db.offsets, db.lengths)
    lddb = mpf.Database(ctx, long_db.residues, long_db.offsets, long_db.lengths)
    for M in (1, 9, 64, 250, 700, 2405):
        p = synth.random_profile(M, int(rng.integers(1, 33)), rng,
                                 cost_hi=int(rng.choice([30, 255])),
                                 bias=int(rng.choice([5, 40, 130, 255])),
                                 base=int(rng.choice([120, 190, 250])), with_lut=True)
        check_profile(ctx, p, db, ddb, arith=arith)
        strong = synth.random_profile(M, 20, rng, cost_hi=24, bias=20, base=190, tbm=10, tec=3, tjb=8)
        check_profile(ctx, strong, long_db, lddb, arith=arith)
    for M in (100, 800):
        check_profile(ctx, synth.make_profile(M, rng), long_db, lddb, arith=arith)


@pytest.mark.parametrize("arith", [mpf.ARITH_I16, mpf.ARITH_F16])
def test_tensor_memory_table(ctx, arith):
    """One-sequence-per-warp kernels with the score rows in tensor memory
    equal the shared-memory kernels and the oracle at every word count: all
    words in TMEM (8-24 words per lane, with and without a two-word tail) or
    24 in TMEM and the rest in shared memory (26-48); on a database of the 20
    amino-acid codes (every row in TMEM) and one of all 32 codes (with 24 TMEM
    words only 21 codes get a TMEM row: the rest read shared memory);
    adversarial bytes, realistic profiles, strong profiles with J chaining
    and overflow."""
    rng = np.random.default_rng(1300 + arith)
    db20 = synth.make_database(500, 300, 1, 3000, rng)
    db32 = synth.random_database(400, 700, rng, alphabet=32)
    strong_db = synth.random_database(200, 900, rng, alphabet=20, min_len=1)
    dbs = [(db, mpf.Database(ctx, db.residues, db.offsets, db.lengths)) for db in (db20, db32, strong_db)]
    for words in (8, 10, 14, 22, 24, 26, 30, 38, 48):
        M = 64 * words - int(rng.integers(0, 64))
        profiles = [
            (synth.make_profile(M, rng), dbs[:2]),
            (synth.random_profile(M, int(rng.integers(1, 33)), rng, cost_hi=255,
                                  bias=int(rng.choice([0, 20, 130, 255])),
                                  base=int(rng.choice([120, 190, 250])), with_lut=True), dbs[1:2]),
            (synth.random_profile(M, 20, rng, cost_hi=26, bias=20, base=190, tbm=10, tec=3, tjb=8),
             dbs[2:]),
        ]
        for p, targets in profiles:
            prof = mpf.Profile(ctx, p)
            for gf, of in FILTERS:
                prof.set_arith(gf, arith)
                prof.set_config(gf, 32, words)
            for db, ddb in targets:
                for gf, of in FILTERS:
                    exp = oracle.scan(of, p, db.residues, db.offsets, db.lengths, nthreads=8)
                    for where in (mpf.TABLE_AUTO, mpf.TABLE_SHARED):
                        prof.set_table_memory(gf, where)
                        want = mpf.TABLE_TENSOR if where == mpf.TABLE_AUTO else mpf.TABLE_SHARED
                        if gf == mpf.MSV and prof.get_table_memory(gf) == mpf.TABLE_SHARED and \
                                where == mpf.TABLE_AUTO:
                            want = mpf.TABLE_SHARED   # MSV_DIRECT profiles have no TMEM kernel
                        assert prof.get_table_memory(gf) == want
                        got = run_gpu(ctx, gf, prof, ddb)
                        assert_same(got, exp, f"tmem={where} arith={arith} words={words} M={M} filter {gf}")
            prof.close()


def test_strong_profiles_hit_j_and_overflow(ctx):
    """Low costs: long hits, chained J transitions, MSV and SSV overflow."""
    rng = np.random.default_rng(77)
    db = synth.random_database(500, 400, rng, alphabet=20, min_len=1)
    ddb = mpf.Database(ctx, db.residues, db.offsets, db.lengths)
    seen_flag = seen_j = 0
    for M in (5, 40, 150, 500):
        for bias in (8, 20, 40):
            p = synth.random_profile(M, 20, rng, cost_hi=bias + 6, bias=bias, base=190,
                                     tbm=20, tec=3, tjb=10)
            check_profile(ctx, p, db, ddb)
            r, f, _ = oracle.msv(p, db.residues, db.offsets, db.lengths, nthreads=8)
            seen_flag += int(f.sum())
            seen_j += int(((f == 0) & (r > 190)).sum())
    assert seen_flag > 0 and seen_j > 0


def test_every_kernel_configuration(ctx):
    """Each (lanes, words) pair that covers M scores identically."""
    rng = np.random.default_rng(3)
    db = synth.random_database(300, 200, rng, alphabet=21)
    ddb = mpf.Database(ctx, db.residues, db.offsets, db.lengths)
    for M in (24, 90, 300):
        p = synth.make_profile(M, rng)
        cfgs = [(lg, w) for lg in (1, 2, 4, 8, 16, 32) for w in range(4, 49, 2)
                if 2 * lg * w >= M and 2 * lg * w < M + 2 * lg * 16]
        check_profile(ctx, p, db, ddb, configs=cfgs)


def test_edge_databases(ctx):
    rng = np.random.default_rng(5)
    p = synth.make_profile(50, rng)
    # all empty, single residue, one long sequence, many tiny ones
    cases = [
        synth.Database(np.zeros(0, np.uint8), np.zeros(3, np.uint64), np.zeros(3, np.uint32)),
        synth.Database(np.array([4], np.uint8), np.zeros(1, np.uint64), np.ones(1, np.uint32)),
        synth.make_database(1, 20000, 20000, 20000, rng),
        synth.make_database(5000, 3, 1, 8, rng),
    ]
    for db in cases:
        check_profile(ctx, p, db)


def test_tensor_memory_table_edge_databases(ctx):
    """The TMEM kernels (whole-warp configurations, both filters, the held MSV
    pass with its rescoring launch) on the edge databases: all sequences
    empty, a single residue, one 20,000-residue sequence, many 1-8 residue
    ones, and a mix of empty and long sequences; profiles with all words in
    TMEM (8 and 14 words) and with part in shared memory (38 words)."""
    rng = np.random.default_rng(55)
    cases = [
        synth.Database(np.zeros(0, np.uint8), np.zeros(3, np.uint64), np.zeros(3, np.uint32)),
        synth.Database(np.array([4], np.uint8), np.zeros(1, np.uint64), np.ones(1, np.uint32)),
        synth.make_database(1, 20000, 20000, 20000, rng),
        synth.make_database(3000, 3, 1, 8, rng),
    ]
    mix = synth.make_database(400, 300, 0, 4000, rng)
    mix.lengths[::3] = 0
    cases.append(synth.Database(mix.residues, mix.offsets, mix.lengths))
    for words in (8, 14, 38):
        p = synth.make_profile(64 * words - 9, rng)
        for db in cases:
            check_profile(ctx, p, db, configs=[(32, words)])


def test_saturated_bias_and_empty_sequences(ctx):
    """bias = 255 puts the MSV overflow threshold at 0: every non-empty
    sequence overflows at its first row, an empty one never does; padding
    rows after a sequence's end must not count as rows."""
    rng = np.random.default_rng(9)
    lengths = np.array([0, 1, 2, 3, 0, 5, 0, 40, 0, 1], np.uint32)
    offsets = np.zeros(lengths.size, np.uint64)
    offsets[1:] = np.cumsum(lengths[:-1])
    db = synth.Database(rng.integers(0, 20, int(lengths.sum())).astype(np.uint8), offsets, lengths)
    for bias in (255, 254, 200):
        for M in (3, 70):
            p = synth.random_profile(M, 20, rng, bias=bias, base=190)
            check_profile(ctx, p, db)


def test_host_and_device_outputs_agree(ctx):
    wl = synth.make_workload(0, n_seqs=2000)
    p = wl.profiles[0]
    prof = mpf.Profile(ctx, p)
    ddb = mpf.Database(ctx, wl.db.residues, wl.db.offsets, wl.db.lengths)
    for gf, _ in FILTERS:
        a = run_gpu(ctx, gf, prof, ddb, on_device=True)
        b = run_gpu(ctx, gf, prof, ddb, on_device=False)
        assert_same(a, b, "host vs device outputs")


# ------------------------------------------------------- batch and plans ---

def test_batch_and_graph_equal_single_scans(ctx):
    wl = synth.make_workload(2, n_seqs=3000, n_queries=10)
    ddb = mpf.Database(ctx, wl.db.residues, wl.db.offsets, wl.db.lengths)
    profs = [mpf.Profile(ctx, p) for p in wl.profiles]
    n, q = ddb.n_seqs, len(profs)
    dev = torch.device("cuda", 0)
    for gf, of in FILTERS:
        single = [run_gpu(ctx, gf, pr, ddb) for pr in profs]
        raw = np.empty(q * n, np.uint8)
        flag = np.empty(q * n, np.uint8)
        nat = np.empty(q * n, np.float32)
        mpf.scan_batch(ctx, gf, profs, ddb, raw, flag, nat)
        draw = torch.empty(q * n, dtype=torch.uint8, device=dev)
        dflag = torch.empty(q * n, dtype=torch.uint8, device=dev)
        dnat = torch.empty(q * n, dtype=torch.float32, device=dev)
        plan = mpf.Plan(ctx, gf, profs, ddb, draw, dflag, dnat)
        assert plan.kernel_launches >= 1
        plan.launch()
        ctx.sync()
        eager = (draw.cpu().numpy(), dflag.cpu().numpy(), dnat.cpu().numpy())
        draw.zero_(), dflag.zero_(), dnat.zero_()
        torch.cuda.synchronize()
        plan.capture_graph()
        for _ in range(2):
            plan.launch()
        ctx.sync()
        graph = (draw.cpu().numpy(), dflag.cpu().numpy(), dnat.cpu().numpy())
        plan.close()
        for i in range(q):
            sl = slice(i * n, (i + 1) * n)
            exp = oracle.scan(of, wl.profiles[i], wl.db.residues, wl.db.offsets, wl.db.lengths,
                              nthreads=8)
            assert_same(single[i], exp, f"single q{i}")
            assert_same((raw[sl], flag[sl], nat[sl]), exp, f"batch q{i}")
            assert_same(tuple(a[sl] for a in eager), exp, f"plan q{i}")
            assert_same(tuple(a[sl] for a in graph), exp, f"graph q{i}")


def _plan_outputs(ctx, gf, profs, ddb, graph=False):
    """Run one plan of profs; returns (its launch groups, per-query outputs)."""
    n, q = ddb.n_seqs, len(profs)
    dev = torch.device("cuda", 0)
    outs = [torch.full((q * n,), 7, dtype=dt, device=dev) for dt in (torch.uint8, torch.uint8, torch.float32)]
    plan = mpf.Plan(ctx, gf, profs, ddb, *outs)
    groups = plan.groups()
    if graph:
        plan.capture_graph()
    for _ in range(2 if graph else 1):
        plan.launch()
    ctx.sync()
    res = [t.cpu().numpy() for t in outs]
    plan.close()
    return groups, [tuple(a[i * n:(i + 1) * n] for a in res) for i in range(q)]


def _packed_batch(ctx, rng, configs, make):
    """Profiles with explicit (lanes, words) for both filters."""
    recs, profs = [], []
    for lanes, words in configs:
        rec = make(2 * lanes * words - int(rng.integers(0, 2 * lanes)))
        prof = mpf.Profile(ctx, rec)
        for gf, _ in FILTERS:
            prof.set_config(gf, lanes, words)
        recs.append(rec)
        profs.append(prof)
    return recs, profs


def test_packed_queries_per_warp(ctx):
    """Plans whose queries of 1 to 16 lanes share one sequence per warp
    (32 / lanes queries, score rows in tensor memory) equal the oracle and
    the one-query scans: full sets and a set with an empty slot, sets with
    every word in TMEM (12-14 words) and with the rest in shared memory, with
    and without a two-word tail, queries padded to their set's word count,
    queries left to the one-query kernels, strong profiles that overflow and
    chain J (the held MSV pass with its rescoring launch), a graph-captured
    replay, and the same batch with every table set to shared memory
    (nothing packed)."""
    rng = np.random.default_rng(808)
    db = synth.make_database(800, 330, 0, 4000, rng)
    strong_db = synth.random_database(300, 500, rng, alphabet=20, min_len=0)
    real = ([(16, 18), (16, 30), (16, 46), (16, 18), (16, 30)] + [(8, 12)] * 4 + [(8, 22)] * 4 + [(8, 38)]
            + [(4, 26)] * 7 + [(2, 20)] * 7 + [(2, 22)] * 7 + [(1, 14)] * 27)
    strong = [(8, 22)] * 4 + [(16, 18)] * 2 + [(4, 12)] * 8 + [(16, 26)]
    batches = [
        (db, _packed_batch(ctx, rng, real, lambda M: synth.make_profile(M, rng))),
        (strong_db, _packed_batch(ctx, rng, strong, lambda M: synth.random_profile(
            M, 20, rng, cost_hi=26, bias=20, base=190, tbm=10, tec=3, tjb=8))),
    ]
    # Sets (lanes, words, table, queries per warp, queries): a set costs
    # (32 / lanes) x its words, a query alone 5/4 of its own words.
    want_real = sorted([(16, 18, mpf.TABLE_TENSOR, 2, 2), (16, 30, mpf.TABLE_TENSOR, 2, 2),
                        (16, 46, mpf.TABLE_SHARED, 1, 1), (8, 12, mpf.TABLE_TENSOR, 4, 4),
                        (8, 22, mpf.TABLE_TENSOR, 4, 4), (8, 38, mpf.TABLE_SHARED, 1, 1),
                        (4, 26, mpf.TABLE_TENSOR, 8, 7), (2, 22, mpf.TABLE_TENSOR, 16, 14),
                        (1, 14, mpf.TABLE_TENSOR, 32, 27)])
    seen_flag = 0
    for bi, (sdb, (recs, profs)) in enumerate(batches):
        ddb = mpf.Database(ctx, sdb.residues, sdb.offsets, sdb.lengths)
        for gf, of in FILTERS:
            groups, got = _plan_outputs(ctx, gf, profs, ddb, graph=(bi == 0))
            key = sorted((g["lanes"], g["words"], g["table"], g["queries_per_warp"], g["n_queries"])
                         for g in groups)
            if bi == 0 and gf == mpf.SSV:
                assert key == want_real, key
            assert sum(g["n_queries"] for g in groups) == len(profs)
            for lanes in sorted({c[0] for c in (real if bi == 0 else strong)} - {32}):
                assert any(g["lanes"] == lanes and g["queries_per_warp"] == 32 // lanes for g in groups), \
                    (lanes, key)
            for pr in profs:
                pr.set_table_memory(gf, mpf.TABLE_SHARED)
            groups_s, got_s = _plan_outputs(ctx, gf, profs, ddb)
            assert all(g["queries_per_warp"] == 1 for g in groups_s)
            for pr in profs:
                pr.set_table_memory(gf, mpf.TABLE_AUTO)
            for i, (rec, pr) in enumerate(zip(recs, profs)):
                exp = oracle.scan(of, rec, sdb.residues, sdb.offsets, sdb.lengths, nthreads=8)
                what = f"batch {bi} filter {gf} q{i} cfg={pr.get_config(gf)} M={rec.M}"
                assert_same(got[i], exp, "packed " + what)
                assert_same(got_s[i], exp, "shared " + what)
                assert_same(run_gpu(ctx, gf, pr, ddb), exp, "single " + what)
                seen_flag += int(exp[1].sum()) if bi == 1 else 0
        for pr in profs:
            pr.close()
        ddb.close()
    assert seen_flag > 0


def test_msv_and_ssv_in_one_sweep(ctx):
    """MPF_MSV_SSV plans and batches (one sweep for both filters where the
    profile allows it) equal the oracle for both filters and the two
    one-filter plans: whole-warp queries with the table in TMEM and in
    shared memory, packed sets of narrow queries, a long model (the tiled
    sweep, with the lane-segment kernel rescoring what it lists), strong
    profiles that overflow and chain J (held-pass rescoring), and queries
    that cannot be fused and run each filter's kernels instead: table
    memories that differ, fp16 SSV cells, different configurations per
    filter, an MSV that needs the per-row J/B update.  Graph replay and host
    outputs too."""
    rng = np.random.default_rng(4242)
    db = synth.make_database(900, 330, 0, 4000, rng)
    strong_db = synth.random_database(300, 500, rng, alphabet=20, min_len=0)
    recs = [synth.make_profile(M, rng) for M in (60, 250, 500, 700, 1300, 2405)]
    recs += [synth.make_profile(2 * 8 * 22 - 3, rng) for _ in range(4)]       # a packed set
    recs += [synth.make_profile(400, rng), synth.make_profile(900, rng), synth.make_profile(3500, rng)]
    recs.append(synth.random_profile(300, 20, rng, bias=250, base=250, tbm=0))   # MSV without held b
    strong = [synth.random_profile(M, 20, rng, cost_hi=26, bias=20, base=190, tbm=10, tec=3, tjb=8)
              for M in (150, 352, 352, 352, 352, 1500, 2405, 3300)]
    for bi, (sdb, rlist) in enumerate(((db, recs), (strong_db, strong))):
        ddb = mpf.Database(ctx, sdb.residues, sdb.offsets, sdb.lengths)
        profs = [mpf.Profile(ctx, r) for r in rlist]
        if bi == 0:
            for pr in profs[6:10]:
                for gf, _ in FILTERS:
                    pr.set_config(gf, 8, 22)
            profs[1].set_table_memory(mpf.MSV, mpf.TABLE_SHARED)     # table memories differ: not fused
            profs[5].set_table_memory(mpf.MSV, mpf.TABLE_SHARED)
            profs[5].set_table_memory(mpf.SSV, mpf.TABLE_SHARED)     # fused, shared-memory table
            profs[10].set_arith(mpf.SSV, mpf.ARITH_F16)              # fp16 SSV: not fused
            profs[11].set_config(mpf.SSV, 32, 16)                    # configurations differ: not fused
        else:
            for pr in profs[1:5]:
                for gf, _ in FILTERS:
                    pr.set_config(gf, 8, 22)
        n, q = ddb.n_seqs, len(profs)
        dev = torch.device("cuda", 0)
        outs = [torch.full((2 * q * n,), 7, dtype=dt, device=dev) for dt in (torch.uint8, torch.uint8, torch.float32)]
        plan = mpf.Plan(ctx, mpf.MSV_SSV, profs, ddb, *outs)
        groups = plan.groups()
        # Fused: every query but the four that cannot be (bi == 0) or all.
        n_fused = sum(g["n_queries"] for g in groups if g["filters"] == 3)
        assert n_fused == (q - 4 if bi == 0 else q), groups
        if bi == 0:   # the long model's tiled sweep
            assert any(g["filters"] == 3 and g["words"] == 0 for g in groups), groups
        assert sum(g["n_queries"] for g in groups if g["filters"] == 1) == q - n_fused
        assert sum(g["n_queries"] for g in groups if g["filters"] == 2) == q - n_fused
        assert any(g["filters"] == 3 and g["queries_per_warp"] == 4 for g in groups)
        assert any(g["filters"] == 3 and g["table"] == mpf.TABLE_TENSOR and g["lanes"] == 32 for g in groups)
        if bi == 0:
            plan.capture_graph()
        for _ in range(2):
            plan.launch()
        ctx.sync()
        fused = [t.cpu().numpy() for t in outs]
        plan.close()
        host = (np.empty(2 * q * n, np.uint8), np.empty(2 * q * n, np.uint8), np.empty(2 * q * n, np.float32))
        mpf.scan_batch(ctx, mpf.MSV_SSV, profs, ddb, *host)
        for fb, (gf, of) in enumerate(FILTERS):
            _, sep = _plan_outputs(ctx, gf, profs, ddb)
            for i, rec in enumerate(rlist):
                exp = oracle.scan(of, rec, sdb.residues, sdb.offsets, sdb.lengths, nthreads=8)
                sl = slice((fb * q + i) * n, (fb * q + i + 1) * n)
                what = f"batch {bi} filter {gf} q{i} M={rec.M}"
                assert_same(tuple(a[sl] for a in fused), exp, "fused plan " + what)
                assert_same(tuple(a[sl] for a in host), exp, "fused batch " + what)
                assert_same(sep[i], exp, "one-filter plan " + what)
        for pr in profs:
            pr.close()
        ddb.close()


# ------------------------------------------------------------ arguments ---

def test_invalid_arguments(ctx):
    rng = np.random.default_rng(1)
    bad = synth.Database(np.array([1, 2, 40], np.uint8), np.zeros(1, np.uint64),
                         np.full(1, 3, np.uint32))
    with pytest.raises(mpf.MpfError) as e:
        mpf.Database(ctx, bad.residues, bad.offsets, bad.lengths)
    assert e.value.status == mpf.MPF_EINVAL
    out_of_range = synth.Database(np.array([1, 2], np.uint8), np.array([1], np.uint64),
                                  np.full(1, 5, np.uint32))
    with pytest.raises(mpf.MpfError):
        mpf.Database(ctx, out_of_range.residues, out_of_range.offsets, out_of_range.lengths)
    big = synth.random_profile(mpf.max_model_length() + 1, 20, rng)
    with pytest.raises(mpf.MpfError) as e:
        mpf.Profile(ctx, big)
    assert e.value.status == mpf.MPF_EUNSUPPORTED
    p = mpf.Profile(ctx, synth.make_profile(100, rng))
    with pytest.raises(mpf.MpfError):
        p.set_config(mpf.MSV, 1, 8)        # 16 cells < M
    with pytest.raises(mpf.MpfError):
        p.set_config(mpf.MSV, 3, 8)        # not a built lane count
    p.set_config(mpf.MSV, 4, 16)
    assert p.get_config(mpf.MSV) == (4, 16)
    p.set_config(mpf.MSV, 0, 0)
    assert p.get_config(mpf.MSV) != (4, 16)
