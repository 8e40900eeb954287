"""MSV + SSV scan throughput on one GB300 (or N, one process per GPU).

A step is one pass of the whole hot path over the model-length sweep
workload: every query profile (M = 48, 100, 200, 400, 800, 1600, 2405)
scored against every sequence of the 500,000-sequence database with both
filters.  The timed form is the batched one (one graph-captured plan per
filter: persistent kernels pulling (query, shard) work items); the plain
one-kernel-per-query form is timed beside it.

GCUPS = sum over queries of M x database residues (padding excluded) per
second, both filters counted (Sec. 4: residues x model length / kernel time).

  python bench.py [--gpus N] [--steps K] [--warmup W] [--workload 0..4]
  python bench.py --impl reference      # the scalar oracle on host cores
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "MSV and SSV GCUPS (batched/served vs plain per-query) on 1 GB300; p50/p99 query latency"
PEAKS = os.path.join(ROOT, "MEASURED_PEAKS.json")
# Integer-SIMD roofline: per SM and clock, 64 lanes of the 32-bit integer /
# 16x2 DPX pipe (measured), 4 byte cells per 32-bit op, and the paper's op
# count per cell (Alg. 2: 4 for MSV; Alg. 7: 2 for SSV).
INT_LANES_PER_SM_CLK = 64
CELLS_PER_LANE_OP = 4
OPS_PER_CELL = {"msv": 4, "ssv": 2}


# DRAM bytes per launch (dram__bytes_read.sum + dram__bytes_write.sum) from the
# ncu captures summarised in profiles/, keyed by kernel, workload and model
# length; only used while the kernel is the one that was captured.
NCU_TRAFFIC = {
    # held MSV pass + its exact rescoring launch (profiles/scan_kernel_tmem_m2405_msweep500k.md)
    ("scan_kernel<32,38,MSV_HELD,TMEM>", "msweep_500k", 2405): 187.900928e6 + 3.704576e6 + 0.258816e6,
    ("scan_kernel<32,38,SSV,TMEM>", "msweep_500k", 2405): 187.970560e6 + 3.762432e6,
}
KERNEL_SOURCE = os.path.join(ROOT, "paper_1707_09683_gb300", "csrc", "mpf_scan_kernel.cuh")
KERNEL_SOURCE_SHA256 = "0e77766bf6a845c614e6a1de6f039389f88f67e468cac41aad9192c93c827c93"


def log(*a):
    print(*a, file=sys.stderr, flush=True)


class ClockSampler:
    """nvidia-smi clocks and throttle reasons during the timed region."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.lines = []

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.Q}",
                 "--format=csv,noheader,nounits", "-lms", "100"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except OSError:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def __exit__(self, *a):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx.append(float(f[2]))
            except ValueError:
                continue
            for n, v in zip(names, f[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(n)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"], "samples": 0}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm)}


def dist_init(args):
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        import torch.distributed as dist
        backend = "nccl" if args.impl == "mpf" else "gloo"
        dist.init_process_group(backend=backend)
    return world, rank, local


def barrier(world):
    if world > 1:
        import torch
        import torch.distributed as dist
        if dist.get_backend() == "nccl":
            dist.barrier(device_ids=[torch.cuda.current_device()])
        else:
            dist.barrier()


def max_over_ranks(x: float, world: int) -> float:
    if world == 1:
        return x
    import torch
    import torch.distributed as dist
    dev = torch.device("cuda", torch.cuda.current_device()) if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([x], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def r_int(filt: str, nsm: int, sm_mhz: float) -> float:
    """Integer-SIMD roofline of a filter in GCUPS."""
    return nsm * INT_LANES_PER_SM_CLK * CELLS_PER_LANE_OP / OPS_PER_CELL[filt] * sm_mhz * 1e6 / 1e9


# Per-SM-clock rates from profiles/ubench_issue_rates_gb300.md.
SMEM_B_PER_CLK = 128.0
TMEM_B_PER_CLK = 385.7
ALU_LANES_PER_CLK = 64.0
FMA_LANES_PER_CLK = 64.0
TM_WORDS_ALL, TM_WORDS_PART = 14, 12   # words per lane from TMEM (all up to 14, else 12)


def design_ceiling(filt, lanes, words, tm, f16, m, nsm, sm_mhz):
    """Ceiling of a striped kernel configuration in GCUPS (model cells): the
    lowest of its table-read and cell-update limits per SM clock, times the
    model's share of the padded cells.  Per 32-bit word (two cells) and DP
    row: 4 B of table (from TMEM for the first 12 or 14 words of a lane
    with tm, else from shared memory), one cell update (DPX on the ALU pipe, or
    HFMA2 on the FMA pipe) and half a 3-input max (ALU)."""
    ht = (words if words <= TM_WORDS_ALL else TM_WORDS_PART) if tm else 0
    lim = {}
    smem_b = 4.0 * (words - ht) / words
    if smem_b > 0:
        lim["shared-memory table reads"] = SMEM_B_PER_CLK / smem_b * 2
    if ht:
        lim["TMEM table reads"] = TMEM_B_PER_CLK / (4.0 * ht / words) * 2
    alu_ops = 0.5 + (0.0 if f16 else 1.0)
    lim["ALU pipe (cell update + running max)" if not f16 else "ALU pipe (running max)"] = \
        ALU_LANES_PER_CLK / alu_ops * 2
    if f16:
        lim["FMA pipe (cell update)"] = FMA_LANES_PER_CLK / 1.0 * 2
    name = min(lim, key=lim.get)
    cells_clk = lim[name]
    g = nsm * cells_clk * sm_mhz * 1e6 / 1e9 * m / (2 * lanes * words)
    basis = ("per SM clock: " + ", ".join(f"{k} {v:.1f}" for k, v in lim.items()) +
             f" cells; x {nsm} SMs x {sm_mhz:.0f} MHz x M / padded cells ({m}/{2 * lanes * words})")
    return g, name, basis


def cpu_baseline(wl, n_sample: int, seed: int = 7):
    """The oracle as it stands, on a bounded sample of the workload."""
    import oracle
    cores = os.cpu_count() or 1
    rng = np.random.default_rng(seed)
    n = wl.db.n_seqs
    idx = np.sort(rng.choice(n, size=min(n_sample, n), replace=False)).astype(np.uint64)
    res = int(wl.db.lengths[idx.astype(np.int64)].sum())
    cells = 0
    t0 = time.perf_counter()
    for p in wl.profiles:
        for f in (oracle.MSV, oracle.SSV):
            oracle.scan(f, p, wl.db.residues, wl.db.offsets, wl.db.lengths, index=idx, nthreads=cores)
            cells += p.M * res
    dt = time.perf_counter() - t0
    return {"value": cells / dt / 1e9, "unit": "GCUPS", "cores": cores, "kind": "oracle",
            "sample": f"{idx.size} random sequences ({res} residues) x {len(wl.profiles)} queries "
                      f"x MSV+SSV = {cells:.3e} cells in {dt:.1f} s"}, dt


def run_reference(args):
    world, rank, local = dist_init(args)
    if rank != 0:
        return
    from paper_1707_09683_gb300 import synth
    import oracle
    oracle.build()
    wl = synth.make_workload(args.workload)
    for _ in range(args.warmup):
        cpu_baseline(wl, 200)
    vals = []
    base = None
    for k in range(args.steps):
        base, dt = cpu_baseline(wl, args.ref_sample, seed=100 + k)
        vals.append(base["value"])
    v = statistics.median(vals)
    base["value"] = v
    line = {"metric": METRIC, "value": v, "unit": "GCUPS", "n_gpus": args.gpus, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": None, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "u8", "data": "synthetic",
            "config": {"workload": wl.name, "queries": [p.M for p in wl.profiles],
                       "n_seqs": wl.db.n_seqs},
            "impl": "reference", "cpu_baseline": base,
            "e2e": {"value": v, "unit": "GCUPS", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def run_mpf(args):
    import torch
    world, rank, local = dist_init(args)
    torch.cuda.set_device(local)
    from paper_1707_09683_gb300 import build, mpf, synth
    build.build()
    dev = torch.device("cuda", local)

    t0 = time.time()
    # N > 1: one database of N times the workload's sequences (the same seeded
    # draws on every rank), sharded by residues; rank r scores shard r and
    # the outputs are gathered (weak scaling: a rank's share stays the size of
    # the one-GPU workload).
    base_n = args.n_seqs or synth.WORKLOADS[args.workload]["n_seqs"]
    wl = synth.make_workload(args.workload, n_seqs=base_n * world, n_queries=args.n_queries)
    job = None
    if world > 1:
        from paper_1707_09683_gb300 import shard
        job = shard.ShardedScan(wl.db, rank, world, len(wl.profiles))
        db_arrays = (job.residues, job.offsets, job.lengths)
    else:
        db_arrays = (wl.db.residues, wl.db.offsets, wl.db.lengths)
    total_res = int(wl.db.lengths.sum(dtype=np.uint64))
    log(f"[rank {rank}] workload {wl.name}: {wl.db.n_seqs} seqs, {total_res} residues, "
        f"{len(wl.profiles)} queries ({time.time() - t0:.1f} s)")
    ctx = mpf.Context(local)
    stream = ctx.torch_stream()
    db = mpf.Database(ctx, *db_arrays)
    profs = [mpf.Profile(ctx, p) for p in wl.profiles]
    arith = {"auto": mpf.ARITH_AUTO, "i16": mpf.ARITH_I16, "f16": mpf.ARITH_F16}[args.arith]
    table = {"auto": mpf.TABLE_AUTO, "shared": mpf.TABLE_SHARED}[args.table]
    for pr in profs:
        for code in (mpf.MSV, mpf.SSV):
            pr.set_arith(code, arith)
            pr.set_table_memory(code, table)
    # Kernel configurations (lanes per sequence, words per lane) from the
    # autotuner, each candidate timed on the whole database.
    tuned = {}
    if args.tune and len({p.M for p in wl.profiles}) <= 16:
        from paper_1707_09683_gb300 import autotune
        t_tune = time.time()
        tuner = autotune.Autotuner(ctx, db, reps=1, tensor_memory=args.table == "auto")
        for pr in profs:
            for name, code in (("msv", mpf.MSV), ("ssv", mpf.SSV)):
                tuner.tune(pr, code)
                tuned.setdefault(name, {})[pr.M] = list(tuner.table[tuner.key(code, pr.M)])
        log(f"[rank {rank}] autotuned {len(profs)} queries in {time.time() - t_tune:.1f} s: {tuned}")
    n, q = db.n_seqs, len(profs)
    res = db.n_residues
    cells_per_filter = sum(p.M for p in wl.profiles) * res
    filters = (("msv", mpf.MSV), ("ssv", mpf.SSV))
    outs = {f: (torch.empty(q * n, dtype=torch.uint8, device=dev),
                torch.empty(q * n, dtype=torch.uint8, device=dev),
                torch.empty(q * n, dtype=torch.float32, device=dev)) for f, _ in filters}

    # Batched: one plan per filter, captured as CUDA graphs.
    plans = {f: mpf.Plan(ctx, code, profs, db, *outs[f]) for f, code in filters}
    for pl in plans.values():
        pl.capture_graph()
    launches_per_step = sum(pl.kernel_launches for pl in plans.values())
    # Plain: one kernel launch per query and filter.
    plain = {f: [mpf.Plan(ctx, code, [pr], db, *(t[i * n:(i + 1) * n] for t in outs[f]))
                 for i, pr in enumerate(profs)] for f, code in filters}

    def step_batched():
        for f, _ in filters:
            plans[f].launch()

    def time_steps(fn, k, name="timed"):
        # NVTX range around the timed launches: a profiler can keep to them
        # (ncu --nvtx --nvtx-include "timed_batched/").
        ev0 = torch.cuda.Event(enable_timing=True)
        ev1 = torch.cuda.Event(enable_timing=True)
        ctx.sync()
        barrier(world)
        torch.cuda.nvtx.range_push(name)
        with torch.cuda.stream(stream):
            ev0.record(stream)
            for _ in range(k):
                fn()
            ev1.record(stream)
        torch.cuda.nvtx.range_pop()
        ev1.synchronize()
        ctx.sync()
        barrier(world)
        return ev0.elapsed_time(ev1) / k   # ms per step

    for _ in range(args.warmup):
        step_batched()
    ctx.sync()
    with ClockSampler(local) as clk:
        ms_batched = time_steps(step_batched, args.steps, "timed_batched")
    clocks = clk.summary()
    ms_batched = max_over_ranks(ms_batched, world)

    # Plain per-query launches, each bracketed by events (per-kernel durations).
    per_kernel = {f: [] for f, _ in filters}

    def step_plain(record=False):
        evs = []
        with torch.cuda.stream(stream):
            for f, _ in filters:
                for i, pl in enumerate(plain[f]):
                    if record:
                        a = torch.cuda.Event(enable_timing=True)
                        b = torch.cuda.Event(enable_timing=True)
                        a.record(stream)
                        pl.launch()
                        b.record(stream)
                        evs.append((f, i, a, b))
                    else:
                        pl.launch()
        return evs

    for _ in range(args.warmup):
        step_plain()
    ctx.sync()
    ms_plain = time_steps(step_plain, args.steps, "timed_plain")
    ms_plain = max_over_ranks(ms_plain, world)
    for _ in range(max(1, args.steps // 2)):
        for f, i, a, b in step_plain(record=True):
            b.synchronize()
            per_kernel[f].append((i, a.elapsed_time(b)))

    # Both filters in one sweep (MPF_MSV_SSV): a query's two filters share a
    # sweep when MSV holds its begin score and both use the same kernel
    # configuration, so the SSV settings take MSV's tuned ones for this plan.
    fused = None
    if args.fused:
        for pr in profs:
            m = tuned.get("msv", {}).get(pr.M)
            if m:
                pr.set_config(mpf.SSV, m[0], m[1])
                pr.set_shard_factor(mpf.SSV, m[2])
                pr.set_table_memory(mpf.SSV, m[3])
        f_outs = tuple(torch.empty(2 * q * n, dtype=dt, device=dev)
                       for dt in (torch.uint8, torch.uint8, torch.float32))
        fplan = mpf.Plan(ctx, mpf.MSV_SSV, profs, db, *f_outs)
        fplan.capture_graph()
        f_groups = fplan.groups()
        for pr in profs:
            m = tuned.get("ssv", {}).get(pr.M)
            if m:
                pr.set_config(mpf.SSV, m[0], m[1])
                pr.set_shard_factor(mpf.SSV, m[2])
                pr.set_table_memory(mpf.SSV, m[3])
        for _ in range(args.warmup):
            fplan.launch()
        ctx.sync()
        ms_fused = max_over_ranks(time_steps(fplan.launch, args.steps, "timed_fused"), world)
        step_batched()
        ctx.sync()
        same = all(bool(torch.equal(f_outs[k][:q * n], outs["msv"][k]) and
                        torch.equal(f_outs[k][q * n:], outs["ssv"][k])) for k in range(3))
        n_fused = sum(g["n_queries"] for g in f_groups if g["filters"] == 3)
        log(f"[rank {rank}] MSV+SSV in one sweep: {ms_fused:.2f} ms per step against batched "
            f"{ms_batched:.2f}; {n_fused} of {q} queries in one sweep; outputs equal: {same}")
        fused = {"ms_per_step": ms_fused, "kernel_launches_per_step": fplan.kernel_launches,
                 "queries_in_one_sweep": n_fused, "queries": q,
                 "sweeps_per_step": sum(g["n_queries"] for g in f_groups),
                 "equals_one_filter_plans": same,
                 "form": "one graph-captured MPF_MSV_SSV plan: both filters' outputs from one sweep per query "
                         "(MSV cells less the held begin score are the SSV cells)"}
        fplan.close()

    # Roofline of the dominant kernel: the (filter, query) launch with the
    # largest total device time in the plain form.
    tot = {f: sum(ms for _, ms in per_kernel[f]) for f, _ in filters}
    by_launch = {}
    for f, _ in filters:
        for i, ms in per_kernel[f]:
            by_launch.setdefault((f, i), []).append(ms)
    dom_f, dom_i = max(by_launch, key=lambda k: sum(by_launch[k]))
    durs = by_launch[(dom_f, dom_i)]
    avg_ms = sum(durs) / len(durs)
    dom_m = wl.profiles[dom_i].M
    achieved = dom_m * res / (avg_ms * 1e-3) / 1e9      # GCUPS of one launch
    dom_code = mpf.MSV if dom_f == "msv" else mpf.SSV
    lanes, words = profs[dom_i].get_config(dom_code)
    dom_tm = profs[dom_i].get_table_memory(dom_code) == mpf.TABLE_TENSOR
    sm_mhz = clocks.get("sm_mhz") or 2070.0
    nsm = torch.cuda.get_device_properties(dev).multi_processor_count
    peak = r_int(dom_f, nsm, sm_mhz)
    f16 = args.arith == "f16"
    mode_name = ("MSV_HELD" if dom_f == "msv" else "SSV") + ("_F16" if f16 else "") + (",TMEM" if dom_tm else "")
    import hashlib
    src_ok = hashlib.sha256(open(KERNEL_SOURCE, "rb").read()).hexdigest() == KERNEL_SOURCE_SHA256
    kname = f"scan_kernel<{lanes},{words},{mode_name}>"
    traffic = NCU_TRAFFIC.get((kname, wl.name, dom_m)) if src_ok else None
    ceiling = design_ceiling(dom_f, lanes, words, dom_tm, f16, dom_m, nsm, sm_mhz)
    roofline = {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "GCUPS",
                "frac": achieved / peak, "traffic": traffic,
                "traffic_note": "ncu dram__bytes_read.sum + dram__bytes_write.sum of this kernel on this "
                                "workload (profiles/); null when the kernel source changed since the "
                                "capture; algorithmic bytes per launch: %.0f" % (res + 6 * n),
                "kernel": f"{kname} M={dom_m}",
                "launches_averaged": len(durs), "avg_launch_ms": avg_ms,
                "design_ceiling": {"peak": ceiling[0], "frac": achieved / ceiling[0], "limiter": ceiling[1],
                                   "basis": ceiling[2]},
                "algorithmic_cells_per_launch": dom_m * res,
                "peak_basis": f"{nsm} SMs x {INT_LANES_PER_SM_CLK} packed-integer lane-ops/clk/SM "
                              f"(DPX/PRMT/LOP3, profiles/ubench_issue_rates_gb300.md) x "
                              f"{CELLS_PER_LANE_OP} byte cells/op / {OPS_PER_CELL[dom_f]} ops/cell "
                              f"(Alg. {'2' if dom_f == 'msv' else '7'}) x {sm_mhz:.0f} MHz "
                              f"(median SM clock in the timed region)"}

    # Whole-job throughput: every rank's cells (the full database when sharded).
    job_cells_per_filter = sum(p.M for p in wl.profiles) * total_res
    gcups_batched = 2 * job_cells_per_filter / (ms_batched * 1e-3) / 1e9
    gcups_plain = 2 * job_cells_per_filter / (ms_plain * 1e-3) / 1e9
    per_filter_plain = {f: sum(wl.profiles[i].M * res for i, _ in per_kernel[f]) /
                        (tot[f] * 1e-3) / 1e9 for f, _ in filters}
    # The same over the queries with M >= 400, against R_int of the filter.
    ge400 = {}
    for f, _ in filters:
        sel = [(i, ms) for i, ms in per_kernel[f] if wl.profiles[i].M >= 400]
        if sel:
            g = sum(wl.profiles[i].M * res for i, _ in sel) / (sum(ms for _, ms in sel) * 1e-3) / 1e9
            ge400[f] = {"gcups": g, "r_int": r_int(f, nsm, sm_mhz), "frac": g / r_int(f, nsm, sm_mhz)}

    # Extra line, not the headline: the same batched step with the cells held
    # as fp16 integers (cell update on the FMA pipe).
    f16_line = None
    if args.f16_line and args.arith != "f16":
        for pr in profs:
            for _, code in filters:
                pr.set_arith(code, mpf.ARITH_F16)
        plans16 = {f: mpf.Plan(ctx, code, profs, db, *outs[f]) for f, code in filters}
        for pl in plans16.values():
            pl.capture_graph()

        def step16():
            for f, _ in filters:
                plans16[f].launch()

        for _ in range(args.warmup):
            step16()
        ms16 = max_over_ranks(time_steps(step16, args.steps), world)
        for pl in plans16.values():
            pl.close()
        for pr in profs:
            for _, code in filters:
                pr.set_arith(code, arith)
        f16_line = {"value": 2 * job_cells_per_filter / (ms16 * 1e-3) / 1e9, "unit": "GCUPS",
                    "ms_per_step": ms16, "dtype": "f16",
                    "note": "extra line, not the headline: the batched step with fp16 cells "
                            "(HFMA2.RELU on the FMA pipe, exact integers below 2048)"}
        log(f"fp16-cell line: {f16_line['value']:.0f} GCUPS ({ms16:.1f} ms per step)")

    # End to end through the public API with host buffers: profiles built from
    # host bytes, both filters batched into host outputs, profiles released.
    raw_h = np.empty(q * n, np.uint8)
    flag_h = np.empty(q * n, np.uint8)
    nat_h = np.empty(q * n, np.float32)
    h2d = sum(p.cost.nbytes + (p.tjb_by_len.nbytes if p.tjb_by_len is not None else 0)
              for p in wl.profiles)
    d2h = 2 * (raw_h.nbytes + flag_h.nbytes + nat_h.nbytes)

    def step_e2e():
        ps = [mpf.Profile(ctx, p) for p in wl.profiles]
        for pr in ps:
            for name, code in filters:
                pr.set_arith(code, arith)
                pr.set_table_memory(code, table)
                if tuned:
                    lanes_w = tuned[name][pr.M]   # lanes, words, shard factor, table memory
                    pr.set_config(code, lanes_w[0], lanes_w[1])
                    pr.set_shard_factor(code, lanes_w[2])
                    pr.set_table_memory(code, lanes_w[3])
        for _, code in filters:
            mpf.scan_batch(ctx, code, ps, db, raw_h, flag_h, nat_h)
        for p in ps:
            p.close()

    step_e2e()
    barrier(world)
    t1 = time.perf_counter()
    e2e_steps = max(1, min(args.steps, 3))
    for _ in range(e2e_steps):
        step_e2e()
    e2e_s = (time.perf_counter() - t1) / e2e_steps
    e2e_s = max_over_ranks(e2e_s, world)
    e2e_gcups = 2 * job_cells_per_filter / e2e_s / 1e9

    # N > 1: the exchange -- every rank's outputs gathered into database
    # order on every rank (NCCL all-gather of device tensors), after one step.
    sharding = None
    if job is not None:
        step_batched()
        ctx.sync()
        barrier(world)
        t_g = time.perf_counter()
        full = job.gather([t for f, _ in filters for t in outs[f]])
        torch.cuda.synchronize()
        gather_s = max_over_ranks(time.perf_counter() - t_g, world)
        sharding = {"world": world, "shard": [job.lo, job.hi], "bounds": job.bounds,
                    "local_residues": job.n_residues_local, "gather_s": gather_s,
                    "gathered_bytes_per_rank": int(sum(t.numel() * t.element_size() for t in full)),
                    "path": "shard.ShardedScan: residue-balanced shards of one database, "
                            "shard.gather_query_outputs (NCCL all_gather) after the scans"}
        del full

    # Two-stage filter (SSV over everything, MSV over the sequences whose SSV
    # score passes): threshold at the 98th percentile of this step's SSV nat
    # scores, so about 2% pass, the fraction Sec. 2.1 reports for the stage.
    pipe = None
    if args.pipeline:
        sn = outs["ssv"][2].float()
        fin = sn[torch.isfinite(sn)]
        thr = float(torch.quantile(fin[:: max(1, fin.numel() // 4_000_000)], 0.98))
        p_ssv = tuple(torch.empty_like(t) for t in outs["ssv"])
        p_msv = tuple(torch.empty_like(t) for t in outs["msv"])
        n_pass = torch.empty(q, dtype=torch.int32, device=dev)
        run_pipe = lambda: mpf.pipeline_scan(ctx, profs, db, thr, p_ssv, p_msv, n_pass)
        for _ in range(args.warmup):
            run_pipe()
        ms_pipe = time_steps(run_pipe, args.steps)
        passed = int(n_pass.sum().item())
        pipe = {"ms_per_step": ms_pipe, "ssv_min_nat": thr, "pass_fraction": passed / (q * n),
                "queries_x_db_gcups": cells_per_filter / (ms_pipe * 1e-3) / 1e9,
                "vs_both_filters_on_all_ms": ms_batched}
        log(f"pipeline: {ms_pipe:.1f} ms per step, {100 * passed / (q * n):.2f}% pass SSV "
            f"(both filters on everything: {ms_batched:.1f} ms)")

    # Third stage: the P7Viterbi filter (Eq. 1) over the sequences whose MSV
    # score passed (one Viterbi profile per query, same model lengths).
    vit = None
    if args.pipeline and args.viterbi:
        vit = run_viterbi_stage(args, ctx, db, wl, profs, p_msv, thr, run_pipe, time_steps, clocks, dev)

    # Models longer than the striped kernels hold (§8(f)-3): one query of
    # args.long_m nodes against the whole database, both filters.
    long_model = None
    if args.long_m and world == 1:
        long_model = run_long_model(args, ctx, db, wl, time_steps, clocks, dev)

    # Many-query workloads: the 64-query overflow batch (2 M sequences) and
    # the first queries of the 1,000-query throughput workload (10 M
    # sequences), batched against plain.
    batch_workloads = None
    if world == 1 and args.batch_workloads:
        batch_workloads = [run_small_workload(args, ctx, dev),
                           run_batch_workload(args, ctx, 2, None, time_steps, dev),
                           run_batch_workload(args, ctx, 4, args.w4_queries, time_steps, dev)]

    # Serving: continuous batching of arriving queries (model lengths drawn as
    # in the serving workload) against the resident database, per offered load.
    serving = None
    if world == 1 and not args.no_serve:
        t_s = time.time()
        wl_serv = synth.make_workload(args.serve_workload, n_seqs=args.serve_seqs)
        log(f"serving workload {wl_serv.name}: {wl_serv.db.n_seqs} seqs ({time.time() - t_s:.1f} s)")
        serving = run_serving(wl_serv, args.serve_rates, args.serve_requests, local,
                              work_budget_queries=args.serve_work_budget)
        del wl_serv

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu:
        cpu, _ = cpu_baseline(wl, args.cpu_sample)

    if rank == 0:
        line = {
            "metric": METRIC, "value": gcups_batched, "unit": "GCUPS", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_batched,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f16" if args.arith == "f16" else "i16",
            "sharding": sharding,
            "data": "synthetic",
            "config": {"workload": wl.name, "queries": [p.M for p in wl.profiles],
                       "n_seqs": int(wl.db.n_seqs), "residues": total_res, "filters": ["msv", "ssv"],
                       "per_rank": {"n_seqs": n, "residues": res},
                       "form": "batched persistent plan per filter, CUDA-graph replay",
                       "cell_arith": ("fp16 cells holding exact integers, HFMA2.RELU on the FMA pipe"
                                      if args.arith == "f16" else
                                      "16-bit integer cells, two per register, DPX on the integer pipe; "
                                      "exact byte semantics of Alg. 2 / Alg. 7; no floating point"),
                       "table_memory": args.table,
                       "kernel_configs": tuned or "default",
                       "l2": "database (%.0f MB) larger than L2; no flush" % (res / 1e6),
                       "cells_per_step": 2 * job_cells_per_filter},
            "plain": {"value": gcups_plain, "unit": "GCUPS", "ms_per_step": ms_plain,
                      "per_filter_gcups": per_filter_plain, "m_ge_400": ge400},
            "batched_over_plain": gcups_batched / gcups_plain,
            "msv_ssv_one_sweep": fused and dict(
                fused, value=2 * job_cells_per_filter / (fused["ms_per_step"] * 1e-3) / 1e9, unit="GCUPS",
                over_plain=ms_plain / fused["ms_per_step"], over_batched=ms_batched / fused["ms_per_step"],
                cells_note="GCUPS counts both filters' cells (2 x M x residues per query) as the headline "
                           "does; one sweep updates M x residues cells for the two"),
            "f16_cells_extra_line": f16_line,
            "roofline": roofline,
            "cpu_baseline": cpu,
            "e2e": {"value": e2e_gcups, "unit": "GCUPS", "h2d_bytes_per_step": int(h2d),
                    "d2h_bytes_per_step": int(d2h), "s_per_step": e2e_s,
                    "path": "mpf_profile_create from host bytes + mpf_scan_batch (MSV, SSV) into "
                            "host buffers + mpf_profile_destroy; database resident"},
            "pipeline": pipe,
            "viterbi": vit,
            "long_model": long_model,
            "serving": serving,
            "batch_workloads": batch_workloads,
            "gpu_launches": launches_per_step * args.steps,
            "clocks": clocks,
        }
        print(json.dumps(line), flush=True)
    for pl in list(plans.values()) + [p for f in plain for p in plain[f]]:
        pl.close()
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


# DPX operations per cell of the saturating Viterbi recurrence once every
# sat() is a single add-then-max (moves <= 0): 4 for the best predecessor of
# M, 1 for the emission, 2 for I, 2 for D, 1 for the E maximum.
VIT_OPS_PER_CELL = 10


def run_viterbi_stage(args, ctx, db, wl, profs, p_msv, thr, run_pipe, time_steps, clocks, dev):
    import torch
    from paper_1707_09683_gb300 import mpf, synth
    n, q = db.n_seqs, len(profs)
    vrecs = [synth.make_vit_profile(p.M, np.random.default_rng(500 + i))
             for i, p in enumerate(wl.profiles)]
    vps = [mpf.VitProfile(ctx, v) for v in vrecs]
    v_out = (torch.empty(q * n, dtype=torch.int16, device=dev),
             torch.empty(q * n, dtype=torch.uint8, device=dev),
             torch.empty(q * n, dtype=torch.float32, device=dev))
    n_v = torch.empty(q, dtype=torch.int32, device=dev)
    run_vit = lambda: mpf.viterbi_rescore(ctx, vps, db, p_msv[1], p_msv[2], thr, *v_out, n_v)
    for _ in range(args.warmup):
        run_vit()
    ms_vit = time_steps(run_vit, args.steps)
    ms_three = time_steps(lambda: (run_pipe(), run_vit()), args.steps)
    lens = torch.from_numpy(wl.db.lengths.astype(np.int64)).to(dev)
    sel = (v_out[1].view(q, n) != 2)
    cells = float(sum(int(lens[sel[i]].sum().item()) * wl.profiles[i].M for i in range(q)))
    passed = int(n_v.sum().item())
    gcups = cells / (ms_vit * 1e-3) / 1e9
    nsm = torch.cuda.get_device_properties(dev).multi_processor_count
    sm_mhz = clocks.get("sm_mhz") or 2070.0
    peak = nsm * INT_LANES_PER_SM_CLK / VIT_OPS_PER_CELL * sm_mhz * 1e6 / 1e9
    for v in vps:
        v.close()
    log(f"viterbi: {ms_vit:.2f} ms per step over {passed} (query, sequence) pairs, "
        f"{gcups:.1f} GCUPS; three stages {ms_three:.1f} ms")
    return {"metric": "Viterbi GCUPS over the MSV survivors", "value": gcups, "unit": "GCUPS",
            "ms_per_step": ms_vit, "msv_min_nat": thr, "pairs_scored": passed,
            "pass_fraction": passed / (q * n), "cells_per_step": cells,
            "three_stage_ms_per_step": ms_three,
            "kernel": "viterbi_fast_kernel (all moves <= 0)",
            "roofline": {"bound": "alu", "achieved": gcups, "peak": peak, "unit": "GCUPS",
                         "frac": gcups / peak, "traffic": None,
                         "timed": "mpf_viterbi_rescore per step (3 selection kernels + 1 Viterbi kernel)",
                         "peak_basis": f"{nsm} SMs x {INT_LANES_PER_SM_CLK} DPX lanes/clk / "
                                       f"{VIT_OPS_PER_CELL} ops per cell x {sm_mhz:.0f} MHz"}}


def run_long_model(args, ctx, db, wl, time_steps, clocks, dev):
    import torch
    from paper_1707_09683_gb300 import mpf, synth
    rec = synth.make_profile(args.long_m, np.random.default_rng(900))
    prof = mpf.Profile(ctx, rec)
    n, res = db.n_seqs, db.n_residues
    outs = (torch.empty(n, dtype=torch.uint8, device=dev), torch.empty(n, dtype=torch.uint8, device=dev),
            torch.empty(n, dtype=torch.float32, device=dev))
    nsm = torch.cuda.get_device_properties(dev).multi_processor_count
    sm_mhz = clocks.get("sm_mhz") or 2070.0
    out = {"M": args.long_m, "config": list(prof.get_config(mpf.MSV)), "n_seqs": n,
           "cells_per_launch": args.long_m * res,
           "kernel": ("MSV: " + ("tile_kernel_tm<MSV> (1,024-node tiles in TMEM, b held) + long_kernel over the "
                                 "sequences it lists" if prof.get_table_memory(mpf.MSV) == mpf.TABLE_TENSOR else
                                 "long_kernel (lane segments, DP row in shared memory)") +
                      "; SSV: tile_kernel_tm<SSV> (1,024-node tiles in TMEM, DP row in registers)")}
    steps = max(1, min(args.steps, 3))
    for name, code in (("msv", mpf.MSV), ("ssv", mpf.SSV)):
        pl = mpf.Plan(ctx, code, [prof], db, *outs)
        pl.launch()
        ms = time_steps(pl.launch, steps)
        pl.close()
        g = args.long_m * res / (ms * 1e-3) / 1e9
        peak = nsm * INT_LANES_PER_SM_CLK * CELLS_PER_LANE_OP / OPS_PER_CELL[name] * sm_mhz * 1e6 / 1e9
        out[name] = {"gcups": g, "ms_per_launch": ms, "roofline_frac": g / peak, "peak": peak,
                     "kernel": ("tile_kernel_tm<MSV>" if prof.get_table_memory(mpf.MSV) == mpf.TABLE_TENSOR
                                else "long_kernel") if name == "msv" else "tile_kernel_tm<SSV>"}
        log(f"long model M={args.long_m}: {name} {g:.1f} GCUPS ({ms:.1f} ms per launch)")
    prof.close()
    out["roofline_basis"] = "integer-SIMD roofline of the striped kernels (same formula as roofline.peak)"
    # P7Viterbi on the same model length (DP rows in device memory), one
    # query against the first sequences of the database.
    k = min(args.long_vit_seqs, wl.db.n_seqs)
    vdb = mpf.Database(ctx, wl.db.residues, wl.db.offsets[:k], wl.db.lengths[:k])
    vp = mpf.VitProfile(ctx, synth.make_vit_profile(args.long_m, np.random.default_rng(901)))
    vouts = (torch.empty(k, dtype=torch.int16, device=dev), torch.empty(k, dtype=torch.uint8, device=dev),
             torch.empty(k, dtype=torch.float32, device=dev))
    run = lambda: mpf.viterbi_scan(ctx, [vp], vdb, *vouts)
    run()
    ms = time_steps(run, steps)
    cells = float(args.long_m) * vdb.n_residues
    g = cells / (ms * 1e-3) / 1e9
    peak = nsm * INT_LANES_PER_SM_CLK / VIT_OPS_PER_CELL * sm_mhz * 1e6 / 1e9
    out["viterbi"] = {"gcups": g, "ms_per_launch": ms, "n_seqs": k, "cells_per_launch": cells,
                      "roofline_frac": g / peak, "peak": peak,
                      "kernel": "viterbi_fast_kernel, DP rows in device memory"}
    log(f"long model M={args.long_m}: viterbi {g:.1f} GCUPS on {k} sequences ({ms:.1f} ms per launch)")
    vp.close()
    vdb.close()
    return out


def run_serving(wl_serv, rates, n_requests, device, seed=3, work_budget_queries=None):
    """p50/p99 latency and GCUPS of the continuous-batching server per offered
    load (Poisson arrivals) on the serving workload's database: each query's
    M is log-uniform in [50, 2000] (the workload's own query draws, reused
    across rates), both filters over every sequence.  Profiles are made
    resident before the first rate (the server's profile cache)."""
    from paper_1707_09683_gb300 import synth
    from paper_1707_09683_gb300.serve import Request, ScanServer
    import math
    recs = [wl_serv.profiles[i % len(wl_serv.profiles)] for i in range(n_requests)]
    res = int(wl_serv.db.lengths.sum(dtype=np.uint64))
    mean_m = sum(p.M for p in recs) / len(recs)
    budget = None
    if work_budget_queries:
        budget = int(work_budget_queries * 2 * res * mean_m)
    server = ScanServer(wl_serv.db, device=device, n_streams=4, max_batch=8,
                        max_queue=max(256, 2 * n_requests), work_budget=budget)
    t0 = time.time()
    server.prepare(list({id(p): p for p in recs}.values()))
    log(f"serving: {len(set(map(id, recs)))} profiles resident in {time.time() - t0:.1f} s")
    server.run([Request(-1 - i, recs[i], arrival=0.0) for i in range(min(8, n_requests))])
    out = []
    for rate in rates:
        arr = synth.poisson_arrivals(rate, n_requests, seed)
        reqs = [Request(i, recs[i], arrival=float(arr[i] - arr[0])) for i in range(n_requests)]
        st = server.run(reqs, offered_rate=rate, timeout_s=900.0)
        out.append(st.as_dict())
        log(f"serving {rate:6.1f} q/s: p50 {st.p50_ms:8.1f} ms p99 {st.p99_ms:8.1f} ms "
            f"{st.gcups:9.1f} GCUPS batch {st.mean_batch:.1f} wait {st.mean_wait_ms:.1f} ms")
    fp = server.footprint_bytes
    server.close()
    # Capacity: the served rate at the highest offered load (queries per
    # second); the knee: the first offered load whose p99 latency is more than
    # three times that of the lightest load.
    top = out[-1]
    capacity = top["served"] / top["wall_s"] if top["wall_s"] > 0 else None
    knee = next((r["offered_qps"] for r in out if r["p99_ms"] > 3 * out[0]["p99_ms"]), None)
    return {"unit": "ms / GCUPS", "workload": wl_serv.name, "n_seqs": int(wl_serv.db.n_seqs),
            "residues": res, "requests_per_rate": n_requests, "filters": ["ssv", "msv"],
            "query_M": "log-uniform [50, 2000] (mean %.0f)" % mean_m, "streams": 4, "max_batch": 8,
            "admission": "by footprint: output slot + score tables (HBM), shared memory per block, "
                         "work budget %s" % ("none" if budget is None else f"{budget:.3e} cells"),
            "output_arena_bytes": fp, "capacity_qps": capacity, "knee_offered_qps": knee,
            "by_rate": out}


def run_batch_workload(args, ctx, idx, n_queries, time_steps, dev, steps=3):
    """Batched vs plain on a many-query workload: every query against the
    whole database with both filters; kernel configurations from the
    autotuner timed on a random 200,000-sequence sample of the database
    (args.batch_tune), else the default ones.
    Batched: one graph-captured plan per filter, queries of fewer than 32
    lanes packed 32 / lanes to a warp where that pays; plain: one launch per
    query and filter; batched_unpacked: the same plans with packing turned
    off (the tables of the queries of fewer than 32 lanes set to shared
    memory, which their plain scans use anyway).  Padding: the padded cells the kernels compute (model padded
    to whole lane stripes, packed queries to their set's words, empty slots
    of a set counted) per model cell."""
    import torch
    from paper_1707_09683_gb300 import mpf, synth
    t0 = time.time()
    wl = synth.make_workload(idx, n_queries=n_queries)
    gen_s = time.time() - t0
    db = mpf.Database(ctx, wl.db.residues, wl.db.offsets, wl.db.lengths)
    n, res, q = db.n_seqs, db.n_residues, len(wl.profiles)
    profs = [mpf.Profile(ctx, p) for p in wl.profiles]
    filters = (("msv", mpf.MSV), ("ssv", mpf.SSV))
    tune_s, tuned = None, {}
    if args.batch_tune:
        from paper_1707_09683_gb300 import autotune
        t_t = time.time()
        sel = np.sort(np.random.default_rng(7).choice(wl.db.n_seqs, size=min(200000, wl.db.n_seqs),
                                                     replace=False))
        sdb = mpf.Database(ctx, wl.db.residues, wl.db.offsets[sel], wl.db.lengths[sel])
        tuner = autotune.Autotuner(ctx, sdb, reps=1)
        for pr in profs:
            for name, code in filters:
                tuner.tune(pr, code, shards=False)   # shard factor 1: the sample is a tenth of the database
                tuned.setdefault(name, {})[pr.M] = list(tuner.table[tuner.key(code, pr.M)])
        sdb.close()
        tune_s = time.time() - t_t
        log(f"{wl.name}: autotuned {q} queries on {sel.size} sequences in {tune_s:.1f} s")
    outs = {f: tuple(torch.empty(q * n, dtype=dt, device=dev)
                     for dt in (torch.uint8, torch.uint8, torch.float32)) for f, _ in filters}
    plans = {f: mpf.Plan(ctx, code, profs, db, *outs[f]) for f, code in filters}
    for pl in plans.values():
        pl.capture_graph()
    narrow = [(pr, code) for pr in profs for _, code in filters if pr.get_config(code)[0] < 32]
    for pr, code in narrow:
        pr.set_table_memory(code, mpf.TABLE_SHARED)
    unpacked = {f: mpf.Plan(ctx, code, profs, db, *outs[f]) for f, code in filters}
    for pr, code in narrow:
        pr.set_table_memory(code, mpf.TABLE_AUTO)
    for pl in unpacked.values():
        pl.capture_graph()
    plain = {f: [mpf.Plan(ctx, code, [pr], db, *(t[i * n:(i + 1) * n] for t in outs[f]))
                 for i, pr in enumerate(profs)] for f, code in filters}
    f_outs = tuple(torch.empty(2 * q * n, dtype=dt, device=dev) for dt in (torch.uint8, torch.uint8, torch.float32))
    # The one-sweep plan takes each query's MSV configuration for both filters.
    for pr in profs:
        m = tuned.get("msv", {}).get(pr.M)
        if m:
            pr.set_config(mpf.SSV, m[0], m[1])
            pr.set_table_memory(mpf.SSV, m[3])
    fplan = mpf.Plan(ctx, mpf.MSV_SSV, profs, db, *f_outs)
    for pr in profs:
        m = tuned.get("ssv", {}).get(pr.M)
        if m:
            pr.set_config(mpf.SSV, m[0], m[1])
            pr.set_table_memory(mpf.SSV, m[3])
    fplan.capture_graph()
    n_fused = sum(g["n_queries"] for g in fplan.groups() if g["filters"] == 3)

    def step_b():
        for f, _ in filters:
            plans[f].launch()

    def step_f():
        fplan.launch()

    def step_u():
        for f, _ in filters:
            unpacked[f].launch()

    def step_p():
        for f, _ in filters:
            for pl in plain[f]:
                pl.launch()

    for _ in range(2):
        step_b()
        step_u()
        step_p()
        step_f()
    ms_b, ms_u, ms_p, ms_f = [], [], [], []
    for _ in range(steps):            # interleaved, so drift hits every form alike
        ms_b.append(time_steps(step_b, 1))
        ms_u.append(time_steps(step_u, 1))
        ms_p.append(time_steps(step_p, 1))
        ms_f.append(time_steps(step_f, 1))
    step_b()
    ctx.sync()
    f_same = all(bool(torch.equal(f_outs[k][:q * n], outs["msv"][k]) and
                      torch.equal(f_outs[k][q * n:], outs["ssv"][k])) for k in range(3))
    f_launches = fplan.kernel_launches
    fplan.close()
    del f_outs
    cells = 2 * sum(p.M for p in wl.profiles) * res
    padded = 0                        # plain scans: each query in its own layout
    for pr, rec in zip(profs, wl.profiles):
        for f, code in filters:
            lanes, words = pr.get_config(code)
            padded += (2 * lanes * words if words else rec.M) * res
    padded_b = 0                      # batched plans: as their launch groups run
    groups = {}
    for (f, code), pl in zip(filters, plans.values()):
        m_other = sum(rec.M for pr, rec in zip(profs, wl.profiles) if not pr.get_config(code)[1])
        for g in pl.groups():
            if g["words"]:
                slots = -(-g["n_queries"] // g["queries_per_warp"]) * g["queries_per_warp"]
                padded_b += slots * 2 * g["lanes"] * g["words"] * res
            key = (g["lanes"], g["words"], g["table"], g["queries_per_warp"])
            groups[key] = groups.get(key, 0) + g["n_queries"]
        padded_b += m_other * res
    packed = sum(v for k, v in groups.items() if k[3] > 1)
    launches = sum(pl.kernel_launches for pl in plans.values())
    for pl in list(plans.values()) + list(unpacked.values()) + [p for f in plain for p in plain[f]]:
        pl.close()
    for pr in profs:
        pr.close()
    db.close()
    gb = cells / (statistics.median(ms_b) * 1e-3) / 1e9
    gu = cells / (statistics.median(ms_u) * 1e-3) / 1e9
    gf = cells / (statistics.median(ms_f) * 1e-3) / 1e9
    gp = cells / (statistics.median(ms_p) * 1e-3) / 1e9
    # The oracle on a bounded sample of the same workload (two queries).
    cpu = None
    if not args.no_cpu:
        import oracle
        rng = np.random.default_rng(31)
        idx = np.sort(rng.choice(wl.db.n_seqs, size=min(3000, wl.db.n_seqs), replace=False)).astype(np.uint64)
        sres = int(wl.db.lengths[idx.astype(np.int64)].sum())
        picks = [wl.profiles[0], wl.profiles[len(wl.profiles) // 2]]
        t_c = time.perf_counter()
        for p in picks:
            for f in (oracle.MSV, oracle.SSV):
                oracle.scan(f, p, wl.db.residues, wl.db.offsets, wl.db.lengths, index=idx,
                            nthreads=os.cpu_count() or 1)
        dt = time.perf_counter() - t_c
        ccells = 2 * sum(p.M for p in picks) * sres
        cpu = {"value": ccells / dt / 1e9, "unit": "GCUPS", "cores": os.cpu_count() or 1, "kind": "oracle",
               "sample": f"{idx.size} random sequences ({sres} residues) x queries M = "
                         f"{[p.M for p in picks]} x MSV+SSV in {dt:.1f} s"}
    out = {"workload": wl.name, "queries": q, "n_seqs": n, "residues": res,
           "query_M": [p.M for p in wl.profiles] if q <= 16 else f"{min(p.M for p in wl.profiles)}-"
                                                                  f"{max(p.M for p in wl.profiles)}",
           "batched": {"gcups": gb, "ms_per_step": ms_b, "kernel_launches_per_step": launches,
                       "form": "one graph-captured plan per filter",
                       "packed_query_filters": packed, "padding_ratio": padded_b / cells},
           "batched_unpacked": {"gcups": gu, "ms_per_step": ms_u,
                                "form": "the same plans, queries of fewer than 32 lanes unpacked"},
           "plain": {"gcups": gp, "ms_per_step": ms_p, "kernel_launches_per_step": 2 * q,
                     "padding_ratio": padded / cells},
           "msv_ssv_one_sweep": {"gcups": gf, "ms_per_step": ms_f, "kernel_launches_per_step": f_launches,
                                 "queries_in_one_sweep": n_fused, "equals_one_filter_plans": f_same,
                                 "form": "one graph-captured MPF_MSV_SSV plan (packed sets included); GCUPS "
                                         "counts both filters' cells"},
           "batched_over_plain": gb / gp,
           "batched_unpacked_over_plain": gu / gp,
           "one_sweep_over_plain": gf / gp,
           "spread": {"batched": (max(ms_b) - min(ms_b)) / statistics.median(ms_b),
                      "batched_unpacked": (max(ms_u) - min(ms_u)) / statistics.median(ms_u),
                      "plain": (max(ms_p) - min(ms_p)) / statistics.median(ms_p)},
           "padding_ratio": padded / cells, "cells_per_step": cells,
           "configs": {f"{k[0]}x{k[1]}{'+tmem' if k[2] == mpf.TABLE_TENSOR else ''}"
                       f"{f'/{k[3]}q' if k[3] > 1 else ''}": v for k, v in sorted(groups.items())},
           "kernel_configs": ("autotuned on a random 200,000-sequence sample (%.1f s)" % tune_s
                              if tune_s is not None else "default"),
           "generate_s": gen_s, "cpu_baseline": cpu}
    log(f"{wl.name}: one sweep MSV+SSV {gf:.0f} GCUPS ({n_fused}/{q} queries, equal outputs {f_same})")
    log(f"{wl.name}: batched {gb:.0f} GCUPS (unpacked {gu:.0f}), plain {gp:.0f}, ratio {gb / gp:.4f}, "
        f"{launches} launches per batched step, {packed} packed query-filters, "
        f"padding batched {padded_b / cells:.3f} plain {padded / cells:.3f}")
    return out


def run_small_workload(args, ctx, dev, reps=5):
    """The one-query workload (M = 100, 10,000 sequences, 3.5 M residues):
    both filters, plain scans, each timed after writing a 512 MB buffer (the
    database fits in L2, so the cache is flushed before every launch); the
    oracle scores the whole database."""
    import torch
    import oracle
    from paper_1707_09683_gb300 import mpf, synth
    wl = synth.make_workload(0)
    db = mpf.Database(ctx, wl.db.residues, wl.db.offsets, wl.db.lengths)
    n, res = db.n_seqs, db.n_residues
    prof = mpf.Profile(ctx, wl.profiles[0])
    outs = [torch.empty(n, dtype=dt, device=dev) for dt in (torch.uint8, torch.uint8, torch.float32)]
    flush = torch.empty(512 << 20, dtype=torch.uint8, device=dev)
    stream = ctx.torch_stream()
    out = {"workload": wl.name, "M": wl.profiles[0].M, "n_seqs": n, "residues": res,
           "l2": "512 MB written before every timed launch"}
    for name, code in (("msv", mpf.MSV), ("ssv", mpf.SSV)):
        pl = mpf.Plan(ctx, code, [prof], db, *outs)
        pl.launch()
        ctx.sync()
        ms = []
        for _ in range(reps):
            with torch.cuda.stream(stream):
                flush.fill_(1)
                a = torch.cuda.Event(enable_timing=True)
                b = torch.cuda.Event(enable_timing=True)
                a.record(stream)
                pl.launch()
                b.record(stream)
            b.synchronize()
            ms.append(a.elapsed_time(b))
        pl.close()
        out[name] = {"gcups": wl.profiles[0].M * res / (statistics.median(ms) * 1e-3) / 1e9,
                     "ms": statistics.median(ms), "config": list(prof.get_config(code))}
    if not args.no_cpu:
        t_c = time.perf_counter()
        for f in (oracle.MSV, oracle.SSV):
            oracle.scan(f, wl.profiles[0], wl.db.residues, wl.db.offsets, wl.db.lengths,
                        nthreads=os.cpu_count() or 1)
        dt = time.perf_counter() - t_c
        out["cpu_baseline"] = {"value": 2 * wl.profiles[0].M * res / dt / 1e9, "unit": "GCUPS",
                               "cores": os.cpu_count() or 1, "kind": "oracle",
                               "sample": f"the whole database, both filters, in {dt:.2f} s"}
    prof.close()
    db.close()
    log(f"{wl.name}: MSV {out['msv']['gcups']:.0f} SSV {out['ssv']['gcups']:.0f} GCUPS")
    return out


def run_profile_case(args):
    """Small case for ncu: the 500,000-sequence database (larger than L2) and
    one query of M = args.profile_m; one warm-up and one measured run.
    Forms (args.profile_form): plain -- one plan per filter (per run: the
    held MSV pass, its rescoring launch, SSV); fused -- one MPF_MSV_SSV plan
    (the one-sweep kernel, its rescoring launch); packed -- 32 /
    args.profile_lanes queries of M = args.profile_m at that lane count in
    one plan per filter, so they run as one packed set (per run: held MSV
    set, rescoring, SSV set)."""
    if args.profile_form != "plain":
        return run_profile_case_batch(args)
    import torch
    from paper_1707_09683_gb300 import build, mpf, synth
    build.build()
    wl = synth.make_workload(1)
    rng = np.random.default_rng(0)
    prof_rec = next((p for p in wl.profiles if p.M == args.profile_m), None) or \
        synth.make_profile(args.profile_m, rng)
    ctx = mpf.Context(0)
    k = min(args.profile_seqs or wl.db.n_seqs, wl.db.n_seqs)
    db = mpf.Database(ctx, wl.db.residues, wl.db.offsets[:k], wl.db.lengths[:k])
    prof = mpf.Profile(ctx, prof_rec)
    n = db.n_seqs
    dev = torch.device("cuda", 0)
    outs = [torch.empty(n, dtype=torch.uint8, device=dev), torch.empty(n, dtype=torch.uint8, device=dev),
            torch.empty(n, dtype=torch.float32, device=dev)]
    plans = [mpf.Plan(ctx, f, [prof], db, *outs) for f in (mpf.MSV, mpf.SSV)]
    for rep in range(2):
        for pl in plans:
            pl.launch()
        ctx.sync()
    for pl in plans:
        pl.close()
    print(json.dumps({"profile_case": wl.name, "M": prof_rec.M, "n_seqs": n,
                      "residues": db.n_residues, "config_msv": prof.get_config(mpf.MSV),
                      "config_ssv": prof.get_config(mpf.SSV)}))


def run_profile_case_batch(args):
    import torch
    from paper_1707_09683_gb300 import build, mpf, synth
    build.build()
    wl = synth.make_workload(1)
    rng = np.random.default_rng(0)
    ctx = mpf.Context(0)
    k = min(args.profile_seqs or wl.db.n_seqs, wl.db.n_seqs)
    db = mpf.Database(ctx, wl.db.residues, wl.db.offsets[:k], wl.db.lengths[:k])
    n = db.n_seqs
    dev = torch.device("cuda", 0)
    if args.profile_form == "fused":
        recs = [next((p for p in wl.profiles if p.M == args.profile_m), None) or
                synth.make_profile(args.profile_m, rng)]
    else:
        recs = [synth.make_profile(args.profile_m, rng) for _ in range(32 // args.profile_lanes)]
    profs = [mpf.Profile(ctx, r) for r in recs]
    if args.profile_form == "packed":
        words = -(-args.profile_m // (2 * args.profile_lanes))
        words += words % 2
        for pr in profs:
            for f in (mpf.MSV, mpf.SSV):
                pr.set_config(f, args.profile_lanes, words)
    q = len(profs)
    if args.profile_form == "fused":
        outs = [torch.empty(2 * q * n, dtype=dt, device=dev) for dt in (torch.uint8, torch.uint8, torch.float32)]
        plans = [mpf.Plan(ctx, mpf.MSV_SSV, profs, db, *outs)]
    else:
        outs = [torch.empty(q * n, dtype=dt, device=dev) for dt in (torch.uint8, torch.uint8, torch.float32)]
        plans = [mpf.Plan(ctx, f, profs, db, *outs) for f in (mpf.MSV, mpf.SSV)]
    groups = [g for pl in plans for g in pl.groups()]
    for rep in range(2):
        for pl in plans:
            pl.launch()
        ctx.sync()
    launches = sum(pl.kernel_launches for pl in plans)
    for pl in plans:
        pl.close()
    print(json.dumps({"profile_case": wl.name, "form": args.profile_form, "M": args.profile_m, "queries": q,
                      "n_seqs": n, "residues": db.n_residues, "groups": groups,
                      "kernel_launches_per_run": launches}))


def run_throughput_all_queries(args):
    """The 1,000-query throughput workload end to end: every query against
    the whole 10 M-sequence database (3.5 G residues), both filters, as one
    plan per query and filter (plain), one plan per filter (batched) and one
    both-filter plan (one sweep), each timed over one run with CUDA events
    (minutes each, so no repetition; raw and flag outputs, no nat).  The two forms' outputs are
    compared in full; three queries (shortest, median and longest M) are
    checked against the oracle on 2,000 random sequences."""
    import torch
    import oracle
    from paper_1707_09683_gb300 import build, mpf, synth
    build.build()
    oracle.build()
    t0 = time.time()
    wl = synth.make_workload(4)
    gen_s = time.time() - t0
    ctx = mpf.Context(0)
    db = mpf.Database(ctx, wl.db.residues, wl.db.offsets, wl.db.lengths)
    n, res, q = db.n_seqs, db.n_residues, len(wl.profiles)
    profs = [mpf.Profile(ctx, p) for p in wl.profiles]
    dev = torch.device("cuda", 0)
    cells = 2 * sum(p.M for p in wl.profiles) * res
    stream = ctx.torch_stream()

    def timed(fn):
        a = torch.cuda.Event(enable_timing=True)
        b = torch.cuda.Event(enable_timing=True)
        ctx.sync()
        with torch.cuda.stream(stream):
            a.record(stream)
            fn()
            b.record(stream)
        b.synchronize()
        ctx.sync()
        return a.elapsed_time(b)

    filters = (("msv", mpf.MSV), ("ssv", mpf.SSV))
    outs = {f: (torch.empty(q * n, dtype=torch.uint8, device=dev), torch.empty(q * n, dtype=torch.uint8, device=dev))
            for f, _ in filters}
    t_p = time.time()
    plans = {f: mpf.Plan(ctx, code, profs, db, *outs[f], None) for f, code in filters}
    f_outs = (torch.empty(2 * q * n, dtype=torch.uint8, device=dev),
              torch.empty(2 * q * n, dtype=torch.uint8, device=dev))
    fplan = mpf.Plan(ctx, mpf.MSV_SSV, profs, db, *f_outs, None)
    plan_s = time.time() - t_p
    groups = {f: pl.groups() for f, pl in plans.items()}
    # Plain: one plan per query and filter, writing into the same outputs.
    plain = [mpf.Plan(ctx, code, [pr], db, outs[f][0][i * n:(i + 1) * n], outs[f][1][i * n:(i + 1) * n], None)
             for f, code in filters for i, pr in enumerate(profs)]
    with ClockSampler(0) as clk:
        ms_p = timed(lambda: [pl.launch() for pl in plain])
        ms_b = timed(lambda: [pl.launch() for pl in plans.values()])
        ms_f = timed(fplan.launch)
    for pl in plain:
        pl.close()
    same = all(bool(torch.equal(f_outs[k][:q * n], outs["msv"][k]) and torch.equal(f_outs[k][q * n:], outs["ssv"][k]))
               for k in range(2))
    rng = np.random.default_rng(5)
    idx = np.sort(rng.choice(n, size=2000, replace=False)).astype(np.uint64)
    order = np.argsort([p.M for p in wl.profiles])
    picks = [int(order[0]), int(order[len(order) // 2]), int(order[-1])]
    ok = True
    for i in picks:
        for f, of in (("msv", oracle.MSV), ("ssv", oracle.SSV)):
            er, ef, _ = oracle.scan(of, wl.profiles[i], wl.db.residues, wl.db.offsets, wl.db.lengths, index=idx,
                                    nthreads=os.cpu_count() or 1)
            sl = slice(i * n, (i + 1) * n)
            ok = ok and np.array_equal(outs[f][0][sl].cpu().numpy()[idx.astype(np.int64)], er) and \
                np.array_equal(outs[f][1][sl].cpu().numpy()[idx.astype(np.int64)], ef)
    print(json.dumps({
        "workload": wl.name, "queries": q, "n_seqs": n, "residues": res, "cells_both_filters": cells,
        "generate_s": gen_s, "plan_create_s": plan_s,
        "batched": {"ms": ms_b, "gcups": cells / (ms_b * 1e-3) / 1e9,
                    "kernel_launches": sum(pl.kernel_launches for pl in plans.values()),
                    "launch_groups_per_filter": len(groups["msv"]),
                    "packed_query_filters": sum(g["n_queries"] for f in groups for g in groups[f]
                                                if g["queries_per_warp"] > 1)},
        "plain": {"ms": ms_p, "gcups": cells / (ms_p * 1e-3) / 1e9, "kernel_launches": 2 * q},
        "batched_over_plain": ms_p / ms_b, "one_sweep_over_plain": ms_p / ms_f,
        "one_sweep": {"ms": ms_f, "gcups": cells / (ms_f * 1e-3) / 1e9, "kernel_launches": fplan.kernel_launches,
                      "queries_in_one_sweep": sum(g["n_queries"] for g in fplan.groups() if g["filters"] == 3),
                      "equals_batched": same,
                      "cells_note": "GCUPS count both filters' cells"},
        "oracle_sample": {"ok": ok, "queries_M": [wl.profiles[i].M for i in picks], "sequences": int(idx.size)},
        "clocks": clk.summary()}), flush=True)
    for pl in list(plans.values()) + [fplan]:
        pl.close()


def run_profile_viterbi(args):
    """Small case for ncu: the first args.profile_vit_seqs sequences of the
    500,000-sequence database against one Viterbi profile of M =
    args.profile_m; one warm-up and one measured scan (kernel launches 0, 1)."""
    import torch
    from paper_1707_09683_gb300 import build, mpf, synth
    build.build()
    wl = synth.make_workload(1)
    k = min(args.profile_vit_seqs, wl.db.n_seqs)
    ctx = mpf.Context(0)
    db = mpf.Database(ctx, wl.db.residues, wl.db.offsets[:k], wl.db.lengths[:k])
    vp = mpf.VitProfile(ctx, synth.make_vit_profile(args.profile_m, np.random.default_rng(0)))
    dev = torch.device("cuda", 0)
    outs = (torch.empty(k, dtype=torch.int16, device=dev), torch.empty(k, dtype=torch.uint8, device=dev),
            torch.empty(k, dtype=torch.float32, device=dev))
    for rep in range(2):
        mpf.viterbi_scan(ctx, [vp], db, *outs)
        ctx.sync()
    print(json.dumps({"profile_case": "viterbi", "M": args.profile_m, "n_seqs": k,
                      "residues": db.n_residues}))


UBENCH_OPS = [  # (code, name, unit) of the microbenchmarks in ubench/mpf_ubench.cu
    (0, "iadd (add.u32)", "lane-ops/clk/SM"), (1, "lop3", "lane-ops/clk/SM"),
    (2, "prmt", "lane-ops/clk/SM"), (3, "imad (mad.lo.u32)", "lane-ops/clk/SM"),
    (4, "dpx viaddmax.s16x2", "lane-ops/clk/SM"), (5, "dpx vimax3.s16x2", "lane-ops/clk/SM"),
    (6, "hfma2.relu", "lane-ops/clk/SM"), (7, "vaddus4 (4x8-bit SIMD)", "lane-ops/clk/SM"),
    (8, "vsubus4 (4x8-bit SIMD)", "lane-ops/clk/SM"), (9, "vmaxu4 (4x8-bit SIMD)", "lane-ops/clk/SM"),
    (10, "viaddmax.s16x2 + hfma2.relu pairs", "lane-ops/clk/SM"),
    (11, "viaddmax.s16x2 + prmt pairs", "lane-ops/clk/SM"),
    (12, "dpx viaddmax.s32", "lane-ops/clk/SM"), (13, "dpx vimax3.s32", "lane-ops/clk/SM"),
    (20, "lds.128 conflict-free", "B/clk/SM"), (21, "tcgen05.ld 32x32b.x16 (TMEM)", "B/clk/SM"),
    (22, "lds.128 + tcgen05.ld together", "B/clk/SM"), (23, "shfl.bfly", "lane-ops/clk/SM"),
]


def run_ubench(args):
    """Issue rates and on-chip bandwidths per SM and SM clock cycle (clock64
    between block barriers, so independent of the clock frequency): the
    denominators of the integer-SIMD roofline and of the shared-memory /
    tensor-memory table ceilings."""
    import ctypes
    from paper_1707_09683_gb300 import build
    lib = ctypes.CDLL(build.build_ubench())
    lib.mpf_ubench_run.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                   ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_double)]
    lib.mpf_ubench_run.restype = ctypes.c_int
    out = []
    for code, name, unit in UBENCH_OPS:
        iters = 1500 if code < 20 else 3000
        best, cyc = 0.0, 0.0
        for _ in range(3):
            r, c = ctypes.c_double(), ctypes.c_double()
            rc = lib.mpf_ubench_run(0, code, iters, ctypes.byref(r), ctypes.byref(c))
            if rc != 0:
                raise RuntimeError(f"ubench {name}: status {rc}")
            if r.value > best:
                best, cyc = r.value, c.value
        out.append({"op": name, "rate": best, "unit": unit, "cycles": cyc})
        log(f"ubench {name:38s} {best:8.2f} {unit}")
    print(json.dumps({"ubench": out}), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="mpf", choices=["mpf", "reference"])
    ap.add_argument("--workload", type=int, default=1)
    ap.add_argument("--n-seqs", type=int, default=None)
    ap.add_argument("--n-queries", type=int, default=None)
    ap.add_argument("--no-tune", dest="tune", action="store_false")
    ap.add_argument("--cpu-sample", type=int, default=40000)
    ap.add_argument("--ref-sample", type=int, default=12000)
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--arith", default="auto", choices=["auto", "i16", "f16"])
    ap.add_argument("--table", default="auto", choices=["auto", "shared"],
                    help="score-table memory of the striped kernels (auto: TMEM where it applies)")
    ap.add_argument("--no-serve", action="store_true")
    ap.add_argument("--no-batch-workloads", dest="batch_workloads", action="store_false",
                    help="skip the 64-query and 10 M-sequence batched-vs-plain measurements")
    ap.add_argument("--batch-tune", action="store_true",
                    help="many-query workloads: kernel configurations autotuned on a 200,000-sequence sample "
                         "(default: the default configurations, which measured faster batched)")
    ap.add_argument("--w4-queries", type=int, default=16,
                    help="queries of the 10 M-sequence workload in its batched-vs-plain measurement")
    ap.add_argument("--no-f16-line", dest="f16_line", action="store_false",
                    help="skip the extra fp16-cell measurement")
    ap.add_argument("--no-pipeline", dest="pipeline", action="store_false")
    ap.add_argument("--no-fused", dest="fused", action="store_false",
                    help="skip the one-sweep MSV+SSV plan (MPF_MSV_SSV)")
    ap.add_argument("--no-viterbi", dest="viterbi", action="store_false")
    ap.add_argument("--long-m", type=int, default=5000,
                    help="model length of the long-model measurement (0: skip)")
    ap.add_argument("--long-vit-seqs", type=int, default=40000,
                    help="sequences of the long-model Viterbi measurement")
    ap.add_argument("--serve-rates", type=float, nargs="+", default=[5, 10, 15, 20, 25, 500])
    ap.add_argument("--serve-requests", type=int, default=200)
    ap.add_argument("--serve-workload", type=int, default=3,
                    help="workload whose database the serving measurement uses (3: 5 M sequences)")
    ap.add_argument("--serve-seqs", type=int, default=None, help="serving: first N sequences only")
    ap.add_argument("--serve-work-budget", type=float, default=None,
                    help="serving: work budget in mean-query units (default: none)")
    ap.add_argument("--profile-case", action="store_true")
    ap.add_argument("--profile-m", type=int, default=2405)
    ap.add_argument("--profile-form", default="plain", choices=["plain", "fused", "packed"])
    ap.add_argument("--profile-lanes", type=int, default=8, help="packed profile case: lanes per sequence")
    ap.add_argument("--profile-seqs", type=int, default=0,
                    help="profile case: first N sequences of the database (0: all)")
    ap.add_argument("--profile-viterbi", action="store_true")
    ap.add_argument("--profile-vit-seqs", type=int, default=20000)
    ap.add_argument("--ubench", action="store_true",
                    help="run the issue-rate / on-chip bandwidth microbenchmarks and exit")
    ap.add_argument("--throughput-all-queries", action="store_true",
                    help="the 1,000-query, 10 M-sequence workload end to end (one run per form, about 9 "
                         "minutes) and exit")
    args = ap.parse_args()
    if args.ubench:
        run_ubench(args)
    elif args.throughput_all_queries:
        run_throughput_all_queries(args)
    elif args.profile_viterbi:
        run_profile_viterbi(args)
    elif args.profile_case:
        run_profile_case(args)
    elif args.impl == "reference":
        run_reference(args)
    else:
        run_mpf(args)


if __name__ == "__main__":
    main()
