"""Continuous-batching scan server over one resident database.

Requests carry a query profile; each is scored against the whole database
with both filters (SSV and MSV, the two heuristic stages of Sec. 2.1).  The
loop keeps the database, the per-stream output arenas and a cache of query
profiles (with their score tables) on the device and does three things until
the work is drained:

* retire: a batch whose completion event has fired hands its results (copied
  to pinned host memory on the batch's stream) to its requests and frees its
  stream and its share of the budgets;
* admit: arrivals enter a bounded queue (a full queue rejects);
* launch: while a stream is free, queued requests are admitted into its
  arena by footprint and launched as one plan for both filters
  (``MPF_MSV_SSV``: a query whose MSV holds its begin score is swept once
  for the two; queries of different model length M run as concurrent
  kernels of their configurations, narrow ones packed several to a warp).

Footprint of a request (``Footprint``): the HBM it holds while in flight --
its output slot (6 bytes per sequence and filter) and the device memory of
its profile's score tables -- the shared memory one block of its kernels
takes (from the profile's kernel configuration), and its work, M x residues
x 2 cells.  A request is admitted when its HBM bytes fit what the in-flight
requests leave of ``hbm_budget`` and its work fits what they leave of
``work_budget``.  The queue is scanned in arrival order, so a request that
does not fit (a long model while others run) waits while later requests that
do fit are admitted past it; after it has been passed over ``max_bypass``
times nothing more may pass it until it fits, so it cannot starve.  A request
larger than a whole budget is admitted alone once nothing else is in flight.

Requests that arrive while other batches are on the GPU are launched on the
next free stream, so their kernels overlap the running ones on the device.
All scoring happens in libmpf.so; this module is host-side orchestration.
"""
from __future__ import annotations

import collections
import statistics
import time
from dataclasses import dataclass, field
from typing import Deque, Dict, List, Optional

import numpy as np

from . import mpf


@dataclass
class Footprint:
    hbm_bytes: int        # output slot + score tables while in flight
    smem_bytes: int       # shared memory of one block of its kernels (largest filter)
    cells: int            # M x residues x filters


@dataclass
class Request:
    rid: int
    profile: object            # synth.Profile-like record
    arrival: float = 0.0       # seconds from the start of the run
    admitted: float = -1.0
    completed: float = -1.0
    rejected: bool = False
    bypassed: int = 0          # batches admitted past it while it waited
    footprint: Optional[Footprint] = None
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
    hbm: int
    cells: int


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
    mean_wait_ms: float = 0.0          # arrival -> admission
    max_queue: int = 0                 # deepest queue seen
    bypass_events: int = 0             # (request, batch) pairs where a batch passed a waiting request
    waited_for_budget: int = 0         # requests passed over at least once
    gcups: float = field(init=False)

    def __post_init__(self):
        self.gcups = self.cells / self.wall_s / 1e9 if self.wall_s > 0 else 0.0

    def as_dict(self):
        return {"offered_qps": self.offered_rate, "served": self.served,
                "rejected": self.rejected, "wall_s": self.wall_s, "gcups": self.gcups,
                "p50_ms": self.p50_ms, "p99_ms": self.p99_ms, "mean_batch": self.mean_batch,
                "max_inflight_batches": self.max_inflight_batches,
                "mean_wait_ms": self.mean_wait_ms, "max_queue": self.max_queue,
                "bypass_events": self.bypass_events, "waited_for_budget": self.waited_for_budget}


class ScanServer:
    """Continuous batching over ``n_streams`` contexts sharing one database.

    hbm_budget:  bytes of output slots + score tables the in-flight requests
                 may hold (default: every arena full, plus 64 MB of tables).
    work_budget: cells the in-flight requests may carry (default: no limit).
    """

    FILTERS = (mpf.SSV, mpf.MSV)

    def __init__(self, db_record, device: int = 0, n_streams: int = 4, max_batch: int = 8,
                 max_queue: int = 64, keep_results: bool = False, nat: bool = True,
                 hbm_budget: Optional[int] = None, work_budget: Optional[int] = None,
                 max_bypass: int = 8, profile_cache: int = 256, arith: int = mpf.ARITH_AUTO):
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
        self.arith = arith
        dev = torch.device("cuda", device)
        nf = len(self.FILTERS)
        cap = max_batch * self.n
        # Per-stream arenas: device outputs of a batch of q requests as the
        # both-filter plan writes them ([MSV: q x n][SSV: q x n]) and their
        # pinned host mirrors; one request holds n sequences per filter.
        self.d_raw = [torch.empty(nf * cap, dtype=torch.uint8, device=dev) for _ in self.ctxs]
        self.d_flag = [torch.empty(nf * cap, dtype=torch.uint8, device=dev) for _ in self.ctxs]
        self.d_nat = [torch.empty(nf * cap, dtype=torch.float32, device=dev) if nat else None
                      for _ in self.ctxs]
        self.h_raw = [torch.empty(nf * cap, dtype=torch.uint8, pin_memory=True) for _ in self.ctxs]
        self.h_flag = [torch.empty(nf * cap, dtype=torch.uint8, pin_memory=True) for _ in self.ctxs]
        self.h_nat = [torch.empty(nf * cap, dtype=torch.float32, pin_memory=True) if nat else None
                      for _ in self.ctxs]
        self.slot_bytes = nf * self.n * (2 + (4 if nat else 0))
        self.hbm_budget = (hbm_budget if hbm_budget is not None
                           else n_streams * max_batch * self.slot_bytes + (64 << 20))
        self.work_budget = work_budget
        self.max_bypass = max_bypass
        self.busy = [False] * len(self.ctxs)
        self.queue: Deque[Request] = collections.deque()
        self.inflight: List[_Batch] = []
        self.inflight_hbm = 0
        self.inflight_cells = 0
        self.max_inflight = 0
        self.batch_sizes: List[int] = []
        self.admit_order: List[int] = []
        # Resident query profiles (keyed by the record object), least recently
        # used first; a profile in flight is never released.
        self.profile_cache = profile_cache
        self._profiles: "collections.OrderedDict[int, tuple]" = collections.OrderedDict()
        self._in_use: Dict[int, int] = collections.defaultdict(int)

    @property
    def footprint_bytes(self) -> int:
        """Device bytes of the output arenas."""
        return self.slot_bytes * self.max_batch * len(self.ctxs)

    # ---------------------------------------------------------- profiles --
    def _profile(self, rec):
        key = id(rec)
        hit = self._profiles.get(key)
        if hit is not None:
            self._profiles.move_to_end(key)
            return hit[0]
        prof = mpf.Profile(self.ctxs[0], rec)
        for f in self.FILTERS:
            prof.set_arith(f, self.arith)
        self._profiles[key] = (prof, rec)
        while len(self._profiles) > self.profile_cache:
            old = next((k for k in self._profiles if self._in_use[k] == 0), None)
            if old is None:
                break
            p, _ = self._profiles.pop(old)
            p.close()
        return prof

    def footprint(self, req: Request) -> Footprint:
        if req.footprint is None:
            prof = self._profile(req.profile)
            fps = [prof.footprint(f) for f in self.FILTERS]
            req.footprint = Footprint(
                hbm_bytes=self.slot_bytes + sum(t for _, t in fps),
                smem_bytes=max(s for s, _ in fps),
                cells=int(req.profile.M) * int(self.residues) * len(self.FILTERS))
        return req.footprint

    def prepare(self, records):
        """Make these query profiles resident with their score tables built
        (creating a plan builds them; nothing is launched), so the requests
        that use them pay no set-up on the latency path."""
        sl = slice(0, 2 * self.n)
        for rec in records:
            prof = self._profile(rec)
            pl = mpf.Plan(self.ctxs[0], mpf.MSV_SSV, [prof], self.db, self.d_raw[0][sl], self.d_flag[0][sl],
                          self.d_nat[0][sl] if self.want_nat else None)
            pl.close()

    # -------------------------------------------------------------- phases --
    def _launch(self, si: int, reqs: List[Request], now: float):
        torch = self.torch
        ctx = self.ctxs[si]
        profs = [self._profile(r.profile) for r in reqs]
        for r in reqs:
            self._in_use[id(r.profile)] += 1
        q = len(reqs)
        # One plan for both filters: a query whose MSV holds its begin score
        # is swept once for the two (MPF_MSV_SSV), others run each filter.
        sl = slice(0, 2 * q * self.n)
        nat = self.d_nat[si][sl] if self.want_nat else None
        plans = [mpf.Plan(ctx, mpf.MSV_SSV, profs, self.db, self.d_raw[si][sl], self.d_flag[si][sl], nat)]
        stream = ctx.torch_stream()
        with torch.cuda.stream(stream):
            for pl in plans:
                pl.launch()
            self.h_raw[si][sl].copy_(self.d_raw[si][sl], non_blocking=True)
            self.h_flag[si][sl].copy_(self.d_flag[si][sl], non_blocking=True)
            if self.want_nat:
                self.h_nat[si][sl].copy_(self.d_nat[si][sl], non_blocking=True)
            ev = torch.cuda.Event()
            ev.record(stream)
        hbm = sum(r.footprint.hbm_bytes for r in reqs)
        cells = sum(r.footprint.cells for r in reqs)
        for r in reqs:
            r.admitted = now
            self.admit_order.append(r.rid)
        self.busy[si] = True
        self.inflight_hbm += hbm
        self.inflight_cells += cells
        self.inflight.append(_Batch(si, reqs, profs, plans, ev, now, hbm, cells))
        self.max_inflight = max(self.max_inflight, len(self.inflight))
        self.batch_sizes.append(q)

    def _retire(self, now_fn):
        done = [b for b in self.inflight if b.event.query()]
        for b in done:
            t = now_fn()
            si = b.stream_idx
            q = len(b.requests)
            for i, r in enumerate(b.requests):
                r.completed = t
                if self.keep:
                    res = {}
                    for filt in self.FILTERS:
                        off = ((0 if filt == mpf.MSV else q) + i) * self.n
                        sl = slice(off, off + self.n)
                        res[filt] = (self.h_raw[si][sl].numpy().copy(),
                                     self.h_flag[si][sl].numpy().copy(),
                                     self.h_nat[si][sl].numpy().copy() if self.want_nat else None)
                    r.result = res
                self._in_use[id(r.profile)] -= 1
            for pl in b.plans:
                pl.close()
            self.busy[si] = False
            self.inflight_hbm -= b.hbm
            self.inflight_cells -= b.cells
            self.inflight.remove(b)
        return len(done)

    def _fits(self, fp: Footprint, hbm: int, cells: int, alone: bool) -> bool:
        if alone:    # nothing else in flight or chosen: even an oversized request may run
            return True
        if hbm + fp.hbm_bytes > self.hbm_budget:
            return False
        return self.work_budget is None or cells + fp.cells <= self.work_budget

    def _admit_and_launch(self, now: float):
        while self.queue:
            free = [i for i, bz in enumerate(self.busy) if not bz]
            if not free:
                return
            batch: List[Request] = []
            passed: List[Request] = []
            hbm, cells = self.inflight_hbm, self.inflight_cells
            for r in self.queue:
                if len(batch) == self.max_batch:
                    break
                fp = self.footprint(r)
                if self._fits(fp, hbm, cells, alone=not self.inflight and not batch):
                    batch.append(r)
                    hbm += fp.hbm_bytes
                    cells += fp.cells
                else:
                    passed.append(r)
                    if r.bypassed >= self.max_bypass:
                        break      # it has waited long enough: nothing more passes it
            if not batch:
                return
            # Requests passed over by this batch (they stay queued, in order).
            for r in passed:
                if any(b.arrival >= r.arrival for b in batch):
                    r.bypassed += 1
            chosen = set(id(r) for r in batch)
            self.queue = collections.deque(r for r in self.queue if id(r) not in chosen)
            self._launch(free[0], batch, now)

    # ----------------------------------------------------------------- run --
    def run(self, requests: List[Request], offered_rate: float = 0.0,
            timeout_s: float = 600.0) -> ServerStats:
        """Replay requests at their arrival times (seconds from now)."""
        pending = collections.deque(sorted(requests, key=lambda r: r.arrival))
        self.batch_sizes = []
        self.max_inflight = 0
        max_queue = 0
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
            max_queue = max(max_queue, len(self.queue))
            self._retire(now)
            self._admit_and_launch(now())
            if not self.queue and self.inflight and (not pending or pending[0].arrival > now()):
                time.sleep(0.0002)
            elif self.queue and self.inflight:
                time.sleep(0.0001)
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
            max_inflight_batches=self.max_inflight,
            mean_wait_ms=statistics.mean((r.admitted - r.arrival) * 1e3 for r in served) if served else 0.0,
            max_queue=max_queue,
            bypass_events=sum(r.bypassed for r in served),
            waited_for_budget=sum(1 for r in served if r.bypassed > 0))

    def close(self):
        for b in list(self.inflight):
            b.event.synchronize()
        self._retire(lambda: 0.0)
        for c in self.ctxs:
            c.sync()
        for p, _ in self._profiles.values():
            p.close()
        self._profiles.clear()
        # Tensors first (torch tracks the streams they were copied on), then
        # the database and the contexts.
        self.d_raw = self.d_flag = self.d_nat = None
        self.h_raw = self.h_flag = self.h_nat = None
        self.db.close()
        for c in self.ctxs:
            c.close()
