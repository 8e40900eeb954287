"""Continuous-batching scan server over one resident database.

Requests carry a query profile; each is scored against the whole database
with both filters (SSV and MSV, the two heuristic stages of Sec. 2.1).  The
loop keeps the database, the per-stream output arenas and the in-flight
profiles on the device and does three things until the work is drained:

* retire: a batch whose completion event has fired hands its results (copied
  to pinned host memory on the batch's stream) to its requests, releases its
  profiles and plans, and frees its stream;
* admit: arrivals enter a bounded queue (a full queue rejects);
* launch: while a stream is free, queued requests are admitted into its
  arena -- up to ``max_batch`` queries, the HBM footprint of one arena -- and
  launched as one plan per filter (queries of different model length M run
  as concurrent kernels of their shared-memory configurations).

Requests that arrive while other batches are on the GPU are launched on the
next free stream, so their kernels overlap the running ones on the device.
All scoring happens in libmpf.so; this module is host-side orchestration.
"""
from __future__ import annotations

import collections
import statistics
import time
from dataclasses import dataclass, field
from typing import Deque, List, Optional

import numpy as np

from . import mpf


@dataclass
class Request:
    rid: int
    profile: object            # synth.Profile-like record
    arrival: float = 0.0       # seconds from the start of the run
    admitted: float = -1.0
    completed: float = -1.0
    rejected: bool = False
    result: Optional[dict] = None

    @property
    def latency(self) -> float:
        return self.completed - self.arrival


@dataclass
class _Batch:
    stream_idx: int
    requests: List[Request]
    profiles: list
    plans: list
    event: object
    launched: float


@dataclass
class ServerStats:
    offered_rate: float
    served: int
    rejected: int
    wall_s: float
    cells: int
    p50_ms: float
    p99_ms: float
    mean_batch: float
    max_inflight_batches: int
    gcups: float = field(init=False)

    def __post_init__(self):
        self.gcups = self.cells / self.wall_s / 1e9 if self.wall_s > 0 else 0.0

    def as_dict(self):
        return {"offered_qps": self.offered_rate, "served": self.served,
                "rejected": self.rejected, "wall_s": self.wall_s, "gcups": self.gcups,
                "p50_ms": self.p50_ms, "p99_ms": self.p99_ms, "mean_batch": self.mean_batch,
                "max_inflight_batches": self.max_inflight_batches}


class ScanServer:
    """Continuous batching over ``n_streams`` contexts sharing one database."""

    FILTERS = (mpf.SSV, mpf.MSV)

    def __init__(self, db_record, device: int = 0, n_streams: int = 4, max_batch: int = 8,
                 max_queue: int = 64, keep_results: bool = False, nat: bool = True):
        import torch
        self.torch = torch
        self.device = device
        self.ctxs = [mpf.Context(device) for _ in range(n_streams)]
        self.db = mpf.Database(self.ctxs[0], db_record.residues, db_record.offsets,
                               db_record.lengths)
        self.ctxs[0].sync()
        self.n = self.db.n_seqs
        self.residues = self.db.n_residues
        self.max_batch = max_batch
        self.max_queue = max_queue
        self.keep = keep_results
        self.want_nat = nat
        dev = torch.device("cuda", device)
        nf = len(self.FILTERS)
        cap = max_batch * self.n
        # Per-stream arenas: device outputs [filter][query][sequence] and their
        # pinned host mirrors.  The arena is the HBM footprint of one batch.
        self.d_raw = [torch.empty(nf * cap, dtype=torch.uint8, device=dev) for _ in self.ctxs]
        self.d_flag = [torch.empty(nf * cap, dtype=torch.uint8, device=dev) for _ in self.ctxs]
        self.d_nat = [torch.empty(nf * cap, dtype=torch.float32, device=dev) if nat else None
                      for _ in self.ctxs]
        self.h_raw = [torch.empty(nf * cap, dtype=torch.uint8, pin_memory=True) for _ in self.ctxs]
        self.h_flag = [torch.empty(nf * cap, dtype=torch.uint8, pin_memory=True) for _ in self.ctxs]
        self.h_nat = [torch.empty(nf * cap, dtype=torch.float32, pin_memory=True) if nat else None
                      for _ in self.ctxs]
        self.busy = [False] * len(self.ctxs)
        self.queue: Deque[Request] = collections.deque()
        self.inflight: List[_Batch] = []
        self.max_inflight = 0
        self.batch_sizes: List[int] = []

    @property
    def footprint_bytes(self) -> int:
        per = 2 * self.max_batch * self.n * (2 + (4 if self.want_nat else 0))
        return per * len(self.ctxs)

    # -------------------------------------------------------------- phases --
    def _launch(self, si: int, reqs: List[Request], now: float):
        torch = self.torch
        ctx = self.ctxs[si]
        profs = [mpf.Profile(ctx, r.profile) for r in reqs]
        q = len(reqs)
        plans = []
        for fi, filt in enumerate(self.FILTERS):
            off = fi * self.max_batch * self.n
            sl = slice(off, off + q * self.n)
            nat = self.d_nat[si][sl] if self.want_nat else None
            plans.append(mpf.Plan(ctx, filt, profs, self.db, self.d_raw[si][sl],
                                  self.d_flag[si][sl], nat))
        stream = ctx.torch_stream()
        with torch.cuda.stream(stream):
            for pl in plans:
                pl.launch()
            for fi in range(len(self.FILTERS)):
                off = fi * self.max_batch * self.n
                sl = slice(off, off + q * self.n)
                self.h_raw[si][sl].copy_(self.d_raw[si][sl], non_blocking=True)
                self.h_flag[si][sl].copy_(self.d_flag[si][sl], non_blocking=True)
                if self.want_nat:
                    self.h_nat[si][sl].copy_(self.d_nat[si][sl], non_blocking=True)
            ev = torch.cuda.Event()
            ev.record(stream)
        for r in reqs:
            r.admitted = now
        self.busy[si] = True
        self.inflight.append(_Batch(si, reqs, profs, plans, ev, now))
        self.max_inflight = max(self.max_inflight, len(self.inflight))
        self.batch_sizes.append(q)

    def _retire(self, now_fn):
        done = [b for b in self.inflight if b.event.query()]
        for b in done:
            t = now_fn()
            si = b.stream_idx
            for i, r in enumerate(b.requests):
                r.completed = t
                if self.keep:
                    res = {}
                    for fi, filt in enumerate(self.FILTERS):
                        off = fi * self.max_batch * self.n + i * self.n
                        sl = slice(off, off + self.n)
                        res[filt] = (self.h_raw[si][sl].numpy().copy(),
                                     self.h_flag[si][sl].numpy().copy(),
                                     self.h_nat[si][sl].numpy().copy() if self.want_nat else None)
                    r.result = res
            for pl in b.plans:
                pl.close()
            for p in b.profiles:
                p.close()
            self.busy[si] = False
            self.inflight.remove(b)
        return len(done)

    def _admit_and_launch(self, now: float):
        while self.queue:
            free = [i for i, bz in enumerate(self.busy) if not bz]
            if not free:
                return
            reqs = [self.queue.popleft() for _ in range(min(self.max_batch, len(self.queue)))]
            self._launch(free[0], reqs, now)

    # ----------------------------------------------------------------- run --
    def run(self, requests: List[Request], offered_rate: float = 0.0,
            timeout_s: float = 600.0) -> ServerStats:
        """Replay requests at their arrival times (seconds from now)."""
        pending = collections.deque(sorted(requests, key=lambda r: r.arrival))
        t0 = time.perf_counter()

        def now():
            return time.perf_counter() - t0

        while pending or self.queue or self.inflight:
            t = now()
            if t > timeout_s:
                raise TimeoutError("server run exceeded its time limit")
            while pending and pending[0].arrival <= t:
                r = pending.popleft()
                if len(self.queue) >= self.max_queue:
                    r.rejected = True
                else:
                    self.queue.append(r)
            self._retire(now)
            self._admit_and_launch(now())
            if not self.queue and self.inflight and (not pending or pending[0].arrival > now()):
                time.sleep(0.0002)
        served = [r for r in requests if not r.rejected]
        lat = sorted(r.latency * 1e3 for r in served)
        cells = sum(r.profile.M for r in served) * self.residues * len(self.FILTERS)
        first = min((r.arrival for r in requests), default=0.0)
        last = max((r.completed for r in served), default=0.0)
        return ServerStats(
            offered_rate=offered_rate, served=len(served),
            rejected=sum(r.rejected for r in requests), wall_s=max(1e-9, last - first),
            cells=cells,
            p50_ms=float(np.percentile(lat, 50)) if lat else float("nan"),
            p99_ms=float(np.percentile(lat, 99)) if lat else float("nan"),
            mean_batch=statistics.mean(self.batch_sizes) if self.batch_sizes else 0.0,
            max_inflight_batches=self.max_inflight)

    def close(self):
        for b in list(self.inflight):
            b.event.synchronize()
        self._retire(lambda: 0.0)
        for c in self.ctxs:
            c.sync()
        # Tensors first (torch tracks the streams they were copied on), then
        # the database and the contexts.
        self.d_raw = self.d_flag = self.d_nat = None
        self.h_raw = self.h_flag = self.h_nat = None
        self.db.close()
        for c in self.ctxs:
            c.close()
