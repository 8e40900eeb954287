"""Database sharding across GPUs (one process per GPU).

Sequences are independent (Sec. 3.1, tier 1; Sec. 6 on spreading sequences
over GPUs), so a database splits into contiguous, residue-balanced shards,
every query is scored against every shard, and the only exchange is a gather
of per-sequence outputs -- there is no reduction and no collective inside
the scan.  ``shard_bounds`` is the split, ``local_database`` the rank's part,
``gather_outputs`` / ``gather_query_outputs`` the exchange (any
torch.distributed backend; CPU tensors with gloo, device tensors with NCCL),
and ``ShardedScan`` ties them together around a caller's scorer: the bench
runs it with the GPU scans, the multi-process CPU test with the oracle.
"""
from __future__ import annotations

from typing import List, Sequence, Tuple

import numpy as np


def shard_bounds(lengths: np.ndarray, world: int) -> List[Tuple[int, int]]:
    """Contiguous sequence ranges [lo, hi) with near-equal residue totals."""
    n = int(lengths.size)
    if world < 1:
        raise ValueError("world must be >= 1")
    csum = np.concatenate(([0], np.cumsum(lengths, dtype=np.uint64))).astype(np.float64)
    total = csum[-1]
    cuts = [0]
    for r in range(1, world):
        cuts.append(int(np.searchsorted(csum, total * r / world, side="left")))
    cuts.append(n)
    cuts = np.maximum.accumulate(np.clip(cuts, 0, n))
    return [(int(cuts[r]), int(cuts[r + 1])) for r in range(world)]


def local_database(db, rank: int, world: int):
    """The rank's shard as (residues, offsets, lengths, (lo, hi))."""
    lo, hi = shard_bounds(db.lengths, world)[rank]
    lengths = np.ascontiguousarray(db.lengths[lo:hi])
    if hi > lo:
        start = int(db.offsets[lo])
        end = int(db.offsets[hi - 1]) + int(db.lengths[hi - 1])
        residues = db.residues[start:end]
        offsets = (db.offsets[lo:hi] - np.uint64(start)).astype(np.uint64)
    else:
        residues = np.zeros(0, np.uint8)
        offsets = np.zeros(0, np.uint64)
    return residues, offsets, lengths, (lo, hi)


def gather_outputs(local: Sequence, bounds: List[Tuple[int, int]], rank: int, world: int):
    """Gather per-sequence outputs of every rank, in database order, on all
    ranks.  ``local`` is a list of 1-D torch tensors (one per output array,
    length hi - lo of this rank)."""
    import torch
    import torch.distributed as dist
    width = max(hi - lo for lo, hi in bounds)
    out = []
    for t in local:
        pad = torch.zeros(width, dtype=t.dtype, device=t.device)
        pad[: t.numel()] = t
        parts = [torch.zeros_like(pad) for _ in range(world)]
        dist.all_gather(parts, pad)
        out.append(torch.cat([parts[r][: hi - lo] for r, (lo, hi) in enumerate(bounds)]))
    return out


def gather_query_outputs(local: Sequence, bounds: List[Tuple[int, int]], rank: int, world: int,
                         n_q: int):
    """Like ``gather_outputs`` for outputs of n_q queries: each local tensor
    is [n_q][hi - lo] (query-major, as a batched scan writes them); the
    result is [n_q][n] in database order, on every rank."""
    import torch
    import torch.distributed as dist
    width = max(hi - lo for lo, hi in bounds)
    out = []
    for t in local:
        nloc = t.numel() // max(n_q, 1)
        pad = torch.zeros((n_q, width), dtype=t.dtype, device=t.device)
        pad[:, :nloc] = t.view(n_q, nloc)
        parts = [torch.empty_like(pad) for _ in range(world)]
        dist.all_gather(parts, pad)
        full = torch.cat([parts[r][:, : hi - lo] for r, (lo, hi) in enumerate(bounds)], dim=1)
        out.append(full.reshape(-1))
    return out


class ShardedScan:
    """One database scored by the ranks of a process group, each rank its
    residue-balanced shard.

    ``scorer(residues, offsets, lengths)`` scores the rank's shard and
    returns a list of 1-D tensors, each [n_q][n_local] (raw, flag and nat
    per filter, say); ``run()`` calls it and ``gather()`` assembles the
    tensors of every rank into [n_q][n] in database order."""

    def __init__(self, db, rank: int, world: int, n_q: int):
        self.rank, self.world, self.n_q = rank, world, n_q
        self.bounds = shard_bounds(db.lengths, world)
        self.residues, self.offsets, self.lengths, (self.lo, self.hi) = local_database(db, rank, world)
        self.n_local = self.hi - self.lo
        self.n_residues_local = int(self.lengths.sum(dtype=np.uint64))

    def run(self, scorer):
        return scorer(self.residues, self.offsets, self.lengths)

    def gather(self, local):
        return gather_query_outputs(local, self.bounds, self.rank, self.world, self.n_q)
