"""The N > 1 path on CPU: two gloo ranks shard a database, score their
shards (with the oracle standing in for the GPU scan), gather the outputs,
and must reproduce the single-process result exactly; the bench's
max-over-ranks timing reduction is checked the same way."""
import os
import socket

import numpy as np
import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

from paper_1707_09683_gb300 import shard, synth


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, result_q):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        import oracle
        import bench
        wl = synth.make_workload(0, n_seqs=900)
        p = wl.profiles[0]
        res, off, ln, (lo, hi) = shard.local_database(wl.db, rank, world)
        outs = []
        for f in (oracle.MSV, oracle.SSV):
            r, fl, nat = oracle.scan(f, p, res, off, ln)
            outs += [torch.from_numpy(r), torch.from_numpy(fl), torch.from_numpy(nat)]
        bounds = shard.shard_bounds(wl.db.lengths, world)
        full = shard.gather_outputs(outs, bounds, rank, world)
        slowest = bench.max_over_ranks(1.5 + rank, world)
        result_q.put((rank, [t.numpy() for t in full], slowest, (lo, hi)))
    finally:
        dist.destroy_process_group()


def test_sharded_scan_gathers_to_the_single_process_result():
    import oracle
    oracle.build()
    world = 2
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, world, port, q)) for r in range(world)]
    for pr in procs:
        pr.start()
    got = [q.get(timeout=120) for _ in range(world)]
    for pr in procs:
        pr.join(timeout=60)
        assert pr.exitcode == 0
    wl = synth.make_workload(0, n_seqs=900)
    p = wl.profiles[0]
    ref = []
    for f in (oracle.MSV, oracle.SSV):
        ref += list(oracle.scan(f, p, wl.db.residues, wl.db.offsets, wl.db.lengths))
    for rank, full, slowest, (lo, hi) in got:
        assert slowest == 2.5                      # max over ranks of 1.5 + rank
        for a, b in zip(full, ref):
            assert np.array_equal(a.view(np.uint8), b.view(np.uint8))
    spans = sorted(b for _, _, _, b in got)
    assert spans[0][0] == 0 and spans[-1][1] == 900 and spans[0][1] == spans[1][0]


def _sharded_worker(rank, world, port, result_q):
    """The bench's N > 1 path (shard.ShardedScan) with the oracle as the
    scorer: several queries, outputs [query][sequence] gathered in database
    order."""
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        import oracle
        wl = synth.make_workload(1, n_seqs=700, n_queries=3)
        job = shard.ShardedScan(wl.db, rank, world, len(wl.profiles))

        def scorer(res, off, ln):
            outs = []
            for f in (oracle.MSV, oracle.SSV):
                per = [oracle.scan(f, p, res, off, ln) for p in wl.profiles]
                for k in range(3):
                    outs.append(torch.from_numpy(np.concatenate([o[k] for o in per])))
            return outs

        full = job.gather(job.run(scorer))
        result_q.put((rank, [t.numpy() for t in full], job.n_local))
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("world", [2, 3])
def test_sharded_scan_class_gathers_query_major_outputs(world):
    import oracle
    oracle.build()
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_sharded_worker, args=(r, world, port, q)) for r in range(world)]
    for pr in procs:
        pr.start()
    got = [q.get(timeout=180) for _ in range(world)]
    for pr in procs:
        pr.join(timeout=60)
        assert pr.exitcode == 0
    wl = synth.make_workload(1, n_seqs=700, n_queries=3)
    ref = []
    for f in (oracle.MSV, oracle.SSV):
        per = [oracle.scan(f, p, wl.db.residues, wl.db.offsets, wl.db.lengths) for p in wl.profiles]
        for k in range(3):
            ref.append(np.concatenate([o[k] for o in per]))
    assert sum(n for _, _, n in got) == 700
    for rank, full, _ in got:
        for a, b in zip(full, ref):
            assert np.array_equal(a.view(np.uint8), b.view(np.uint8)), rank


def test_shard_bounds_balance_and_cover():
    rng = np.random.default_rng(2)
    lengths = rng.integers(0, 5000, size=10_001).astype(np.uint32)
    for world in (1, 2, 3, 8):
        b = shard.shard_bounds(lengths, world)
        assert b[0][0] == 0 and b[-1][1] == lengths.size
        assert all(b[i][1] == b[i + 1][0] for i in range(world - 1))
        tot = [int(lengths[lo:hi].sum()) for lo, hi in b]
        assert max(tot) - min(tot) <= 2 * int(lengths.max())
    assert shard.shard_bounds(np.zeros(0, np.uint32), 4) == [(0, 0)] * 4


def _failing_worker(rank, world, port, result_q):
    """Rank 1 fails before the gather (an exception between steps, none of
    its work in flight); rank 0 must get an error from its collective within
    the process group's timeout instead of waiting forever."""
    import datetime
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world,
                            timeout=datetime.timedelta(seconds=5))
    try:
        wl = synth.make_workload(0, n_seqs=200)
        bounds = shard.shard_bounds(wl.db.lengths, world)
        lo, hi = bounds[rank]
        local = [torch.zeros(hi - lo, dtype=torch.uint8)]
        if rank == 1:
            result_q.put((rank, "raised"))
            raise RuntimeError("injected rank failure")
        try:
            shard.gather_outputs(local, bounds, rank, world)
            result_q.put((rank, "gathered"))
        except Exception as e:   # the collective reports the lost peer
            result_q.put((rank, "error: " + type(e).__name__))
    finally:
        try:
            dist.destroy_process_group()
        except Exception:
            pass


def test_failed_rank_surfaces_as_a_collective_error():
    world = 2
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_failing_worker, args=(r, world, port, q)) for r in range(world)]
    for pr in procs:
        pr.start()
    got = dict(q.get(timeout=120) for _ in range(world))
    for pr in procs:
        pr.join(timeout=60)
    assert got[1] == "raised"
    assert got[0].startswith("error:")
    assert procs[1].exitcode != 0
