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
