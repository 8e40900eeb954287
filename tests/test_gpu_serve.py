"""Serving: continuous batching gives every request the result it gets alone.

Requests of different model lengths arrive while earlier batches are still
on the GPU; they are launched on other streams and overlap.  Each request's
SSV and MSV outputs must equal a standalone scan of its profile (bit-exact,
the stated tolerance is zero) and, on a subset, the oracle.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle
from paper_1707_09683_gb300 import build, mpf, synth
from paper_1707_09683_gb300.serve import Request, ScanServer

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def setup():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    build.build()
    oracle.build()
    wl = synth.make_workload(3, n_seqs=6000, n_queries=14)
    return wl


def standalone(ctx, db, rec):
    prof = mpf.Profile(ctx, rec)
    n = db.n_seqs
    out = {}
    for filt in (mpf.SSV, mpf.MSV):
        raw = np.empty(n, np.uint8)
        flag = np.empty(n, np.uint8)
        nat = np.empty(n, np.float32)
        (mpf.ssv_scan if filt == mpf.SSV else mpf.msv_scan)(ctx, prof, db, raw, flag, nat)
        out[filt] = (raw, flag, nat)
    prof.close()
    return out


def test_results_same_alone_and_in_the_mix(setup):
    wl = setup
    server = ScanServer(wl.db, n_streams=3, max_batch=3, max_queue=64, keep_results=True)
    reqs = [Request(i, p, arrival=0.0005 * i) for i, p in enumerate(wl.profiles)]
    stats = server.run(reqs, offered_rate=2000.0)
    assert stats.served == len(reqs) and stats.rejected == 0
    assert stats.max_inflight_batches >= 2, "batches must overlap on the device"
    ctx = server.ctxs[1]
    for r in reqs:
        alone = standalone(ctx, server.db, r.profile)
        for filt in (mpf.SSV, mpf.MSV):
            got, exp = r.result[filt], alone[filt]
            assert np.array_equal(got[0], exp[0]) and np.array_equal(got[1], exp[1]), (r.rid, filt)
            assert np.array_equal(got[2].view(np.uint32), exp[2].view(np.uint32)), (r.rid, filt)
    for r in reqs[:3]:
        for filt, of in ((mpf.SSV, oracle.SSV), (mpf.MSV, oracle.MSV)):
            exp = oracle.scan(of, r.profile, wl.db.residues, wl.db.offsets, wl.db.lengths, nthreads=8)
            assert np.array_equal(r.result[filt][0], exp[0]) and np.array_equal(r.result[filt][1], exp[1])
    server.close()


def test_bounded_queue_rejects_overload(setup):
    wl = setup
    server = ScanServer(wl.db, n_streams=1, max_batch=2, max_queue=3)
    reqs = [Request(i, p, arrival=0.0) for i, p in enumerate(wl.profiles[:10])]
    stats = server.run(reqs, offered_rate=1e6)
    assert stats.rejected > 0 and stats.served + stats.rejected == 10
    assert all(r.completed >= r.arrival for r in reqs if not r.rejected)
    server.close()


def test_long_model_waits_while_short_ones_are_admitted_past_it(setup):
    """Admission by footprint: with a work budget that holds one long model
    and a few short ones, a second long model that arrives while the first
    is on the GPU waits, the short models queued behind it are admitted past
    it, and it runs once the first has retired.  Every result still equals
    the standalone scan."""
    wl = setup
    rng = np.random.default_rng(21)
    long1, long2 = synth.make_profile(2000, rng), synth.make_profile(1800, rng)
    shorts = [synth.make_profile(m, rng) for m in (50, 64, 72, 80)]
    res = int(wl.db.lengths.sum())
    budget = 2 * res * (long1.M + 4 * 80)
    server = ScanServer(wl.db, n_streams=4, max_batch=1, max_queue=16, keep_results=True,
                        work_budget=budget)
    recs = [long1, long2] + shorts
    reqs = [Request(i, p, arrival=0.0) for i, p in enumerate(recs)]
    fp = [server.footprint(r) for r in reqs]
    assert fp[0].smem_bytes > fp[2].smem_bytes and fp[0].cells > fp[2].cells
    assert all(f.hbm_bytes >= server.slot_bytes for f in fp)
    stats = server.run(reqs, offered_rate=0.0)
    assert stats.served == len(reqs) and stats.rejected == 0
    order = server.admit_order
    assert order[0] == 0, order
    assert order.index(1) > order.index(2), order          # a short model passed the long one
    assert reqs[1].bypassed >= 1 and stats.waited_for_budget >= 1
    assert reqs[1].admitted >= reqs[0].completed - 1e-6   # it ran after the first long model
    ctx = server.ctxs[1]
    for r in reqs:
        alone = standalone(ctx, server.db, r.profile)
        for filt in (mpf.SSV, mpf.MSV):
            got, exp = r.result[filt], alone[filt]
            assert np.array_equal(got[0], exp[0]) and np.array_equal(got[1], exp[1]), (r.rid, filt)
            assert np.array_equal(got[2].view(np.uint32), exp[2].view(np.uint32)), (r.rid, filt)
    server.close()


def test_starving_request_blocks_further_bypass(setup):
    """After a waiting request has been passed over max_bypass times, no later
    request is admitted before it."""
    wl = setup
    rng = np.random.default_rng(22)
    long1, long2 = synth.make_profile(2000, rng), synth.make_profile(1900, rng)
    shorts = [synth.make_profile(60, rng) for _ in range(6)]
    res = int(wl.db.lengths.sum())
    server = ScanServer(wl.db, n_streams=2, max_batch=1, max_queue=16,
                        work_budget=2 * res * (long1.M + 60), max_bypass=1)
    reqs = [Request(i, p, arrival=0.0) for i, p in enumerate([long1, long2] + shorts)]
    stats = server.run(reqs)
    assert stats.served == len(reqs)
    order = server.admit_order
    # long2 is passed at most once; every short model after the first waits for it.
    assert reqs[1].bypassed <= 1
    assert all(order.index(1) < order.index(i) for i in range(3, len(reqs))), order
    server.close()
