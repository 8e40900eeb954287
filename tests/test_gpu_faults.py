"""Failures made on the host, reported as status codes, with the context
still usable afterwards.

Device memory is exhausted by holding almost all of it in a torch tensor
(allocation failures are ordinary CUDA errors, not GPU faults): a database
upload and a scan that needs output scratch must fail with MPF_ENOMEM, and
once the memory is released the same context must score correctly.  The
kernels themselves have no device-side waits (work is taken with atomics and
no block waits on another), so there is no timeout path to exercise.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle
from paper_1707_09683_gb300 import build, mpf, synth

pytestmark = pytest.mark.gpu

HEADROOM = 96 << 20     # bytes left free while memory is held


@pytest.fixture(scope="module")
def ctx():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    build.build()
    oracle.build()
    return mpf.Context(0)


def _hold_memory():
    torch.cuda.empty_cache()
    free, _ = torch.cuda.mem_get_info(0)
    if free <= HEADROOM + (64 << 20):
        pytest.skip("not enough free device memory to exhaust safely")
    return torch.empty(free - HEADROOM, dtype=torch.uint8, device=torch.device("cuda", 0))


def test_database_upload_out_of_memory_then_recovers(ctx):
    rng = np.random.default_rng(21)
    n = 2000
    lengths = np.full(n, 100_000, np.uint32)          # 200 MB of residues
    offsets = np.arange(n, dtype=np.uint64) * np.uint64(100_000)
    residues = rng.integers(0, 20, int(lengths.sum()), dtype=np.uint8)
    hold = _hold_memory()
    try:
        with pytest.raises(mpf.MpfError) as e:
            mpf.Database(ctx, residues, offsets, lengths)
        assert e.value.status == mpf.MPF_ENOMEM
    finally:
        del hold
        torch.cuda.empty_cache()
    # Recovered: a small database and scan on the same context match the oracle.
    wl = synth.make_workload(0, n_seqs=300)
    db = mpf.Database(ctx, wl.db.residues, wl.db.offsets, wl.db.lengths)
    prof = mpf.Profile(ctx, wl.profiles[0])
    raw, flag = np.zeros(300, np.uint8), np.zeros(300, np.uint8)
    nat = np.zeros(300, np.float32)
    mpf.msv_scan(ctx, prof, db, raw, flag, nat)
    er, ef, en = oracle.msv(wl.profiles[0], wl.db.residues, wl.db.offsets, wl.db.lengths, nthreads=8)
    assert np.array_equal(raw, er) and np.array_equal(flag, ef)
    assert np.array_equal(nat.view(np.uint32), en.view(np.uint32))
    prof.close()
    db.close()


def test_scan_scratch_out_of_memory_then_recovers(ctx):
    rng = np.random.default_rng(22)
    n = 500_000                                        # one-residue sequences
    dbh = synth.Database(residues=rng.integers(0, 20, n, dtype=np.uint8),
                         offsets=np.arange(n, dtype=np.uint64), lengths=np.ones(n, np.uint32))
    db = mpf.Database(ctx, dbh.residues, dbh.offsets, dbh.lengths)
    recs = [synth.make_profile(50, rng) for _ in range(40)]
    profs = [mpf.Profile(ctx, r) for r in recs]
    q = len(profs)
    raw, flag = np.zeros(q * n, np.uint8), np.zeros(q * n, np.uint8)
    nat = np.zeros(q * n, np.float32)
    mpf.scan_batch(ctx, mpf.SSV, profs[:1], db, raw[:n], flag[:n], nat[:n])   # tables built
    hold = _hold_memory()
    try:
        with pytest.raises(mpf.MpfError) as e:        # host outputs need 6 B x 20 M of scratch
            mpf.scan_batch(ctx, mpf.SSV, profs, db, raw, flag, nat)
        assert e.value.status == mpf.MPF_ENOMEM
    finally:
        del hold
        torch.cuda.empty_cache()
    mpf.scan_batch(ctx, mpf.SSV, profs, db, raw, flag, nat)
    for i in (0, q - 1):
        er, ef, en = oracle.ssv(recs[i], dbh.residues, dbh.offsets, dbh.lengths, nthreads=8)
        sl = slice(i * n, (i + 1) * n)
        assert np.array_equal(raw[sl], er) and np.array_equal(flag[sl], ef)
        assert np.array_equal(nat[sl].view(np.uint32), en.view(np.uint32))
    for p in profs:
        p.close()
    db.close()
