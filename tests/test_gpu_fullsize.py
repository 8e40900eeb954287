"""Full-size workloads through the launch configuration the bench times.

Each database is generated at its full size and scored by graph-captured
batched plans (one per filter); the oracle then checks, one sequence at a
time, a sample of the outputs: the longest and shortest sequences, planted
ones where the workload has them, and random ones.  Bit-exact.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle
from paper_1707_09683_gb300 import build, mpf, synth

pytestmark = pytest.mark.gpu


def sample_index(db, rng, planted=None, n_random=600, n_edge=60):
    order = np.argsort(db.lengths, kind="stable")
    pick = [order[:n_edge], order[-n_edge:], rng.choice(db.n_seqs, n_random, replace=False)]
    if planted is not None and planted.size:
        pick.append(rng.choice(planted, min(planted.size, 300), replace=False))
    return np.unique(np.concatenate(pick)).astype(np.uint64)


def run_and_check(wl, queries, rng, planted=None):
    ctx = mpf.Context(0)
    db = mpf.Database(ctx, wl.db.residues, wl.db.offsets, wl.db.lengths)
    profs = [mpf.Profile(ctx, wl.profiles[i]) for i in queries]
    n, q = db.n_seqs, len(profs)
    dev = torch.device("cuda", 0)
    idx = sample_index(wl.db, rng, planted)
    n_flag = 0
    for gf, of in ((mpf.MSV, oracle.MSV), (mpf.SSV, oracle.SSV)):
        raw = torch.empty(q * n, dtype=torch.uint8, device=dev)
        flag = torch.empty(q * n, dtype=torch.uint8, device=dev)
        nat = torch.empty(q * n, dtype=torch.float32, device=dev)
        plan = mpf.Plan(ctx, gf, profs, db, raw, flag, nat)
        plan.capture_graph()
        plan.launch()
        ctx.sync()
        raw_h, flag_h, nat_h = raw.cpu().numpy(), flag.cpu().numpy(), nat.cpu().numpy()
        plan.close()
        for j, i in enumerate(queries):
            exp = oracle.scan(of, wl.profiles[i], wl.db.residues, wl.db.offsets, wl.db.lengths,
                              index=idx, nthreads=16)
            sel = j * n + idx.astype(np.int64)
            assert np.array_equal(raw_h[sel], exp[0]), (wl.name, gf, i)
            assert np.array_equal(flag_h[sel], exp[1]), (wl.name, gf, i)
            assert np.array_equal(nat_h[sel].view(np.uint32), exp[2].view(np.uint32)), (wl.name, gf, i)
            n_flag += int(exp[1].sum())
    for p in profs:
        p.close()
    db.close()
    ctx.close()
    return n_flag


@pytest.fixture(scope="module", autouse=True)
def built():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    build.build()
    oracle.build()


def test_model_length_sweep_full_database():
    wl = synth.make_workload(1)
    run_and_check(wl, list(range(len(wl.profiles))), np.random.default_rng(11))


def test_overflow_batch_full_database():
    wl = synth.make_workload(2)
    rng = np.random.default_rng(12)
    queries = sorted(rng.choice(len(wl.profiles), 8, replace=False).tolist())
    assert run_and_check(wl, queries, rng, planted=wl.planted) > 0


def test_throughput_workload_full_database():
    wl = synth.make_workload(4, n_queries=12)
    run_and_check(wl, list(range(12)), np.random.default_rng(13))


def test_pipeline_and_viterbi_stage_full_database():
    """The three stages as the bench times them (workload 1 in full, SSV
    threshold at the 98th percentile of the SSV nat scores, the same value
    for MSV -> Viterbi); sampled sequences checked one by one."""
    wl = synth.make_workload(1)
    rng = np.random.default_rng(14)
    ctx = mpf.Context(0)
    db = mpf.Database(ctx, wl.db.residues, wl.db.offsets, wl.db.lengths)
    profs = [mpf.Profile(ctx, p) for p in wl.profiles]
    vrecs = [synth.make_vit_profile(p.M, np.random.default_rng(500 + i)) for i, p in enumerate(wl.profiles)]
    vps = [mpf.VitProfile(ctx, v) for v in vrecs]
    n, q = db.n_seqs, len(profs)
    dev = torch.device("cuda", 0)
    mk = lambda t: torch.empty(q * n, dtype=t, device=dev)
    ssv_out = (mk(torch.uint8), mk(torch.uint8), mk(torch.float32))
    msv_out = (mk(torch.uint8), mk(torch.uint8), mk(torch.float32))
    n1 = torch.empty(q, dtype=torch.int32, device=dev)
    # threshold from a first SSV pass, as the bench does
    plan = mpf.Plan(ctx, mpf.SSV, profs, db, *ssv_out)
    plan.launch()
    ctx.sync()
    plan.close()
    sn = ssv_out[2]
    fin = sn[torch.isfinite(sn)]
    thr = float(torch.quantile(fin[:: max(1, fin.numel() // 4_000_000)], 0.98))
    mpf.pipeline_scan(ctx, profs, db, thr, ssv_out, msv_out, n1)
    vs, vf, vn = mk(torch.int16), mk(torch.uint8), mk(torch.float32)
    n2 = torch.empty(q, dtype=torch.int32, device=dev)
    mpf.viterbi_rescore(ctx, vps, db, msv_out[1], msv_out[2], thr, vs, vf, vn, n2)
    ctx.sync()
    sr, sf, snat = (t.cpu().numpy() for t in ssv_out)
    mr, mf, mnat = (t.cpu().numpy() for t in msv_out)
    gvs, gvf, gvn = vs.cpu().numpy(), vf.cpu().numpy(), vn.cpu().numpy()
    got1, got2 = n1.cpu().numpy(), n2.cpu().numpy()
    for i, p in enumerate(wl.profiles):
        sl = slice(i * n, (i + 1) * n)
        pass1 = (sf[sl] != 0) | (snat[sl] >= np.float32(thr))
        pass2 = (mf[sl] == 1) | (mnat[sl] >= np.float32(thr))
        assert int(got1[i]) == int(pass1.sum()) and int(got2[i]) == int(pass2.sum())
        assert np.all(mf[sl][~pass1] == 2) and np.all(gvf[sl][~pass2] == 2)
        idx = sample_index(wl.db, rng, n_random=150, n_edge=20)
        er, ef, en = oracle.ssv(p, wl.db.residues, wl.db.offsets, wl.db.lengths, index=idx, nthreads=16)
        j = idx.astype(np.int64)
        assert np.array_equal(sr[sl][j], er) and np.array_equal(sf[sl][j], ef)
        assert np.array_equal(snat[sl][j].view(np.uint32), en.view(np.uint32))
        passing = np.flatnonzero(pass1)
        take = rng.choice(passing, min(120, passing.size), replace=False).astype(np.uint64)
        er, ef, en = oracle.msv(p, wl.db.residues, wl.db.offsets, wl.db.lengths, index=take, nthreads=16)
        k = take.astype(np.int64)
        assert np.array_equal(mr[sl][k], er) and np.array_equal(mf[sl][k], ef)
        assert np.array_equal(mnat[sl][k].view(np.uint32), en.view(np.uint32))
        passing = np.flatnonzero(pass2)
        take = rng.choice(passing, min(60, passing.size), replace=False).astype(np.uint64)
        es, ef, en = oracle.viterbi(vrecs[i], wl.db.residues, wl.db.offsets, wl.db.lengths, index=take,
                                    nthreads=16)
        k = take.astype(np.int64)
        assert np.array_equal(gvs[sl][k], es) and np.array_equal(gvf[sl][k], ef)
        assert np.array_equal(gvn[sl][k].view(np.uint32), en.view(np.uint32))
    for v in vps:
        v.close()
    for p in profs:
        p.close()
    db.close()
    ctx.close()


def test_long_model_full_database():
    """A 5,000-node model (the long-model kernel) against workload 1 in full,
    as the bench measures it; sampled sequences checked one by one."""
    wl = synth.make_workload(1)
    rec = synth.make_profile(5000, np.random.default_rng(900))
    ctx = mpf.Context(0)
    db = mpf.Database(ctx, wl.db.residues, wl.db.offsets, wl.db.lengths)
    prof = mpf.Profile(ctx, rec)
    n = db.n_seqs
    dev = torch.device("cuda", 0)
    rng = np.random.default_rng(15)
    idx = sample_index(wl.db, rng, n_random=300, n_edge=20)
    for gf, of in ((mpf.MSV, oracle.MSV), (mpf.SSV, oracle.SSV)):
        out = [torch.empty(n, dtype=t, device=dev) for t in (torch.uint8, torch.uint8, torch.float32)]
        plan = mpf.Plan(ctx, gf, [prof], db, *out)
        plan.launch()
        ctx.sync()
        plan.close()
        got = [t.cpu().numpy() for t in out]
        want = oracle.scan(of, rec, wl.db.residues, wl.db.offsets, wl.db.lengths, index=idx, nthreads=16)
        j = idx.astype(np.int64)
        assert np.array_equal(got[0][j], want[0]) and np.array_equal(got[1][j], want[1])
        assert np.array_equal(got[2][j].view(np.uint32), want[2].view(np.uint32))
    prof.close()
    db.close()
    ctx.close()


def test_serving_workload_full_database_through_the_server():
    """The serving workload at its stated size: 5,000,000 sequences (1.78 G
    residues) resident on the device, ten queries of log-uniform M served
    through the continuous-batching server with overlapping batches; a sample
    of every query's SSV and MSV outputs (the longest and shortest sequences
    and random ones) equals the oracle one sequence at a time."""
    from paper_1707_09683_gb300.serve import Request, ScanServer
    wl = synth.make_workload(3, n_queries=10)
    assert wl.db.n_seqs == 5_000_000
    rng = np.random.default_rng(13)
    idx = sample_index(wl.db, rng, n_random=500, n_edge=40)
    server = ScanServer(wl.db, n_streams=3, max_batch=2, max_queue=32, keep_results=True)
    reqs = [Request(i, p, arrival=0.002 * i) for i, p in enumerate(wl.profiles)]
    stats = server.run(reqs, offered_rate=500.0)
    assert stats.served == len(reqs) and stats.rejected == 0
    assert stats.max_inflight_batches >= 2
    sel = idx.astype(np.int64)
    for r in reqs:
        for gf, of in ((mpf.SSV, oracle.SSV), (mpf.MSV, oracle.MSV)):
            exp = oracle.scan(of, r.profile, wl.db.residues, wl.db.offsets, wl.db.lengths,
                              index=idx, nthreads=16)
            got = r.result[gf]
            assert np.array_equal(got[0][sel], exp[0]), (r.rid, gf)
            assert np.array_equal(got[1][sel], exp[1]), (r.rid, gf)
            assert np.array_equal(got[2][sel].view(np.uint32), exp[2].view(np.uint32)), (r.rid, gf)
        r.result = None
    server.close()
