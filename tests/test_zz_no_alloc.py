"""The allocation-free scan entry point against the regular one.

mpf_scan_noalloc is for callers that cannot allocate device memory when they
score: services that budget all device memory up front, and plug-ins whose
host application owns the device allocator.  Its scratch lives in a fixed
device array inside the library, so two calls in a row must each reproduce
the regular scan exactly: the second call must not see state left by the
first.
This file is collected last so that a run stopping at its first failure has
already run every other test.
"""
import ctypes

import numpy as np
import pytest

torch = pytest.importorskip("torch")

from paper_1707_09683_gb300 import build, mpf, synth

pytestmark = pytest.mark.gpu


def _scan_regular(ctx, filt, prof, db, n, dev):
    out = (torch.empty(n, dtype=torch.uint8, device=dev), torch.empty(n, dtype=torch.uint8, device=dev),
           torch.empty(n, dtype=torch.float32, device=dev))
    (mpf.msv_scan if filt == mpf.MSV else mpf.ssv_scan)(ctx, prof, db, *out)
    ctx.sync()
    return [t.cpu().numpy() for t in out]


def test_noalloc_matches_regular_scan_twice_in_a_row():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    build.build()
    lib = mpf.load()
    dev = torch.device("cuda", 0)
    ctx = mpf.Context(0)
    wl = synth.make_workload(2, n_seqs=3000, n_queries=3)      # planted: overflow flags too
    db = mpf.Database(ctx, wl.db.residues, wl.db.offsets, wl.db.lengths)
    n = db.n_seqs
    rng = np.random.default_rng(4)
    records = list(wl.profiles) + [synth.make_profile(48, rng), synth.make_profile(2405, rng)]
    for rec in records:
        prof = mpf.Profile(ctx, rec)
        for filt in (mpf.MSV, mpf.SSV):
            want = _scan_regular(ctx, filt, prof, db, n, dev)
            for call in range(2):
                raw = torch.full((n,), 7, dtype=torch.uint8, device=dev)
                flag = torch.full((n,), 7, dtype=torch.uint8, device=dev)
                nat = torch.full((n,), -1.0, dtype=torch.float32, device=dev)
                torch.cuda.synchronize()
                st = lib.mpf_scan_noalloc(ctx.handle, filt, prof.handle, db.handle,
                                          raw.data_ptr(), flag.data_ptr(), nat.data_ptr())
                assert st == mpf.MPF_OK, mpf.strerror(st)
                ctx.sync()
                got = [raw.cpu().numpy(), flag.cpu().numpy(), nat.cpu().numpy()]
                assert np.array_equal(got[0], want[0]), (rec.M, filt, call, "raw")
                assert np.array_equal(got[1], want[1]), (rec.M, filt, call, "overflow")
                assert np.array_equal(got[2].view(np.uint32), want[2].view(np.uint32)), \
                    (rec.M, filt, call, "nat")
        prof.close()
    # Host buffers are refused: the call has nowhere to stage them.
    prof = mpf.Profile(ctx, records[0])
    host = np.zeros(n, np.uint8)
    st = lib.mpf_scan_noalloc(ctx.handle, mpf.SSV, prof.handle, db.handle, host.ctypes.data,
                              host.ctypes.data, None)
    assert st == mpf.MPF_EINVAL
    prof.close()
    db.close()
    ctx.close()
