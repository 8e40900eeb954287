"""Kernel-configuration selection for the scan kernels.

Two selectors:

* ``paper_policy`` restates the paper's rule (Sec. 3.1 Eq. 2-3 and Sec. 3.4
  Eq. 4-5): with warp size s, register width w_r and value width w_v, a warp
  aligns S = 2^i sequences (1 <= i <= log2(s w_r / w_v)), each with
  L = ceil(s / S) threads holding W = s w_r / (w_v S) cells per loop step, and
  H = max(2, ceil(m / W)) steps.  Eq. 4 takes the largest S whose W_S H_max
  covers the model (H_max = 45 for MSV, 50 for SSV, the unrolling limits of
  Table 1); models beyond W_2 H_max use the single-sequence kernel (S = 1).
  The switch of Sec. 3.4.2 additionally sends models up to m_min = 20 to the
  32-sequence kernel and models above m_max (2450 MSV, 1000 SSV) to S = 1.
* ``Autotuner`` times every built (lanes, words) configuration that covers a
  model on the caller's database and keeps the fastest; the paper's point,
  mapped onto this library's kernels, is one of the candidates.  It then
  times the shard factor of the winner (work items per query = factor x
  resident blocks: the granularity of the dynamic load balance that replaces
  the paper's static block assignment and Alg. 1) and keeps the best.  For
  whole-warp configurations it also times the table in shared memory only
  against the table in tensor memory.

In this library a lane group of ``lanes`` threads holds one sequence (the
paper's L, so S = 32 / lanes) and each thread holds ``words`` registers of
two 16-bit cells (the paper's H counts registers of four 8-bit cells).
"""
from __future__ import annotations

import json
import math
import os
from dataclasses import dataclass
from typing import Dict, List, Optional, Tuple

WARP = 32          # s: threads per warp
REG_BITS = 32      # w_r
VALUE_BITS = 8     # w_v
H_MAX = {"msv": 45, "ssv": 50}
M_MIN = 20
M_MAX = {"msv": 2450, "ssv": 1000}

LANES = (1, 2, 4, 8, 16, 32)
SHARD_FACTORS = (1, 2, 4)
WORDS = tuple(sorted(set(range(4, 49, 4)) | set(range(6, 48, 4))))   # %4 == 2: two-word tail


@dataclass(frozen=True)
class PaperChoice:
    S: int      # sequences per warp (1 = single-sequence kernel)
    W: int      # cells per loop step per thread group
    L: int      # threads per thread group
    H: int      # loop steps


def _w(S: int) -> int:
    return WARP * REG_BITS // (VALUE_BITS * S)


def paper_policy(m: int, filt: str, switch: bool = True) -> PaperChoice:
    """Eq. 4/5 kernel choice for a model of length m (filt 'msv' or 'ssv')."""
    if m < 1:
        raise ValueError("model length must be positive")
    hmax = H_MAX[filt]
    s_values = [2 ** i for i in range(1, int(math.log2(WARP * REG_BITS // VALUE_BITS)) + 1)]
    if switch and m <= M_MIN:
        S = 32
    elif switch and m > M_MAX[filt]:
        S = 1
    elif m > _w(2) * hmax:
        S = 1
    else:
        S = max(S for S in s_values if _w(S) * hmax >= m)
    W = _w(S)
    return PaperChoice(S=S, W=W, L=max(1, -(-WARP // S)), H=max(2, -(-m // W)))


def covering_words(m: int, lanes: int) -> int:
    w = -(-m // (2 * lanes))
    return max(4, -(-w // 2) * 2)


def paper_point(m: int, filt: str) -> Optional[Tuple[int, int]]:
    """The paper's choice mapped onto (lanes, words) of this library: lanes =
    threads per group; words = registers needed for the model, or the next
    wider group if they exceed the largest built word count."""
    ch = paper_policy(m, filt)
    lanes = min(32, ch.L)
    while lanes <= 32:
        w = covering_words(m, lanes)
        if w <= WORDS[-1]:
            return lanes, w
        lanes *= 2
    return None


def candidates(m: int, max_waste: float = 0.3, min_words: int = 8) -> List[Tuple[int, int]]:
    """Built configurations that cover m with at most max_waste padding and
    at least min_words registers per lane (fewer leaves the per-row work of
    a lane dominated by the shift and residue handling)."""
    out = []
    for lanes in LANES:
        for w in WORDS:
            cells = 2 * lanes * w
            if cells >= m and (cells - m) / cells <= max_waste and w >= min_words:
                out.append((lanes, w))
    if not out:      # tiny models: the smallest covering configuration
        out.append((1, covering_words(m, 1)))
    pp = paper_point(m, "msv")
    if pp and pp not in out:
        out.append(pp)
    return out


class Autotuner:
    """Times candidate configurations on a database and remembers the best
    per (filter, model length).  Results can be saved to / loaded from JSON."""

    def __init__(self, ctx, db, cache_path: Optional[str] = None, reps: int = 3,
                 tensor_memory: bool = True):
        self.ctx = ctx
        self.tensor_memory = tensor_memory   # False: every candidate keeps its table in shared memory
        self.db = db
        self.reps = reps
        self.cache_path = cache_path
        self.table: Dict[str, Tuple[int, int]] = {}
        self.timings: Dict[str, Dict[str, float]] = {}
        if cache_path and os.path.exists(cache_path):
            with open(cache_path) as f:
                self.table = {k: tuple(v) for k, v in json.load(f).items()}

    @staticmethod
    def key(filt: int, m: int) -> str:
        return f"{'msv' if filt == 0 else 'ssv'}:{m}"

    def _time(self, prof, filt, lanes, words, outs, factor: int = 1) -> float:
        import torch
        from . import mpf
        try:
            prof.set_config(filt, lanes, words)
            prof.set_shard_factor(filt, factor)
        except mpf.MpfError:      # no kernel built for this pair in this arithmetic
            return float("inf")
        plan = mpf.Plan(self.ctx, filt, [prof], self.db, *outs)
        stream = self.ctx.torch_stream()
        plan.launch()
        self.ctx.sync()
        best = float("inf")
        for _ in range(self.reps):
            a = torch.cuda.Event(enable_timing=True)
            b = torch.cuda.Event(enable_timing=True)
            a.record(stream)
            plan.launch()
            b.record(stream)
            b.synchronize()
            best = min(best, a.elapsed_time(b))
        plan.close()
        return best

    def tune(self, prof, filt: int, force: bool = False, shards: bool = True) -> Tuple[int, int]:
        """Pick and set the fastest configuration (lanes, words) for this
        profile, then its shard factor; returns (lanes, words)."""
        import torch
        k = self.key(filt, prof.M)
        from . import mpf
        if not force and k in self.table:
            cfg = self.table[k]
            prof.set_config(filt, cfg[0], cfg[1])
            prof.set_shard_factor(filt, cfg[2] if len(cfg) > 2 else 1)
            prof.set_table_memory(filt, cfg[3] if len(cfg) > 3 else mpf.TABLE_AUTO)
            return cfg[0], cfg[1]
        n = self.db.n_seqs
        dev = torch.device("cuda", self.ctx.device)
        outs = (torch.empty(n, dtype=torch.uint8, device=dev),
                torch.empty(n, dtype=torch.uint8, device=dev), None)
        times = {}
        for lanes, words in candidates(prof.M):
            prof.set_table_memory(filt, mpf.TABLE_AUTO if self.tensor_memory else mpf.TABLE_SHARED)
            times[f"{lanes}x{words}"] = self._time(prof, filt, lanes, words, outs)
            if lanes == 32 and prof.get_table_memory(filt) == mpf.TABLE_TENSOR:
                # the same configuration with the table in shared memory only
                prof.set_table_memory(filt, mpf.TABLE_SHARED)
                times[f"{lanes}x{words}s"] = self._time(prof, filt, lanes, words, outs)
        best = min(times, key=times.get)
        table = mpf.TABLE_SHARED if best.endswith("s") or not self.tensor_memory else mpf.TABLE_AUTO
        lanes, words = (int(x) for x in best.rstrip("s").split("x"))
        prof.set_table_memory(filt, table)
        factor = 1
        if shards:
            ft = {1: times[best]}
            for f in SHARD_FACTORS[1:]:
                ft[f] = self._time(prof, filt, lanes, words, outs, f)
                times[f"{best}/{f}"] = ft[f]
            factor = min(ft, key=ft.get)
        prof.set_config(filt, lanes, words)
        prof.set_shard_factor(filt, factor)
        self.table[k] = (lanes, words, factor, table)
        self.timings[k] = times
        return lanes, words

    def save(self, path: Optional[str] = None):
        path = path or self.cache_path
        if path:
            with open(path, "w") as f:
                json.dump({k: list(v) for k, v in self.table.items()}, f, indent=1)
