"""Database sharding across GPUs (one process per GPU).

Sequences are independent (Sec. 3.1, tier 1), so a database splits into
contiguous, residue-balanced shards, every query is scored against every
shard, and the only exchange is a gather of per-sequence outputs -- there is
no reduction and no collective inside the scan.  ``shard_bounds`` is the
split, ``local_database`` the rank's part, ``gather_outputs`` the exchange
(any torch.distributed backend; CPU tensors with gloo, device tensors with
NCCL).
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
