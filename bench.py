#!/usr/bin/env python
"""SymmSpMV benchmark on GB300 (one JSON line on stdout).

Headline workload (default): the periodic Heisenberg XXZ chain L=26, Sz=0
sector (10,400,600 rows, 80,708,656 stored upper nonzeros, 151,016,712 full
nonzeros), FP64 values, x ~ U[-1,1) (seed 3) -- a synthetic stand-in for the
paper's Spin-26 matrix.  One step = one b = A x through the library's
SymmSpMV path (schedule built before timing, as the paper excludes
preprocessing).  Beside it, on the same permuted matrix: the full-CRS SpMV
(the traffic baseline), the all-FP64 executor (the plain FP64 form), the
conflict-free RACE executors, the input order, FP32-stored values, and the
reductions alone.  The default run also measures the other workloads of the
paper's classes, each in its own block of the line: the 27-point stencil
200^3 (SymmSpMV, FP32-stored values with their error against the FP64
oracle, SymmSpMM k = 4, 8, 16 in FP64 and FP32 values), the Anderson model
32^3 (L2-resident: time only), and the batch of 64 matrices in one CUDA
graph.

Roofline: algorithmic bytes (v+4) nnz_u + 4 N + 24 k N (x read, b read and
written: the count of Eq. "SymmSpMV_intensity" at the optimal alpha, which
the reduction-based executors also move: b is zeroed, accumulated in L2 and
written back) over the launch's CUDA-event time, against the measured copy
bandwidth and, as the paper's range, the load-only bandwidth measured here;
SymmSpMM also against min(HBM * I, FP64 roof), the FP64 roof being the
FP64 FMA rate measured here over the row sums' multiply-adds, the FP64 work
that stays on the FP64 pipe (the all-FP64 roof is given beside it).

Timing: W warm-up steps, then K steps bracketed by a barrier and
torch.cuda.synchronize(), CUDA events on the stream the kernels run on;
vectors rotate through ring buffers of 4 x and 4 b (each 83 MB) and the
matrix is 1.05 GB, so every step's inputs exceed the 129 MB L2.  Several
GPUs (torchrun) run independent replicas (no data exchange); value is the
sum over ranks of the flops divided by the slowest rank's time.

--impl reference times the oracle's CPU RACE execution (the paper's own
method: the oracle's schedule for N_t = host threads, phases in order with a
barrier, the leaves of a phase on the host cores) on bounded repetitions of
the same matrix.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

WORKLOAD_DESC = {
    "xxz26": "Heisenberg XXZ chain L=26 periodic, Sz=0 (10,400,600 rows), J=1, Delta=1, FP64 upper CRS, "
             "x~U[-1,1) seed 3, RACE-permuted",
    "st27_200": "3D 27-point stencil 200^3 nonperiodic SPD, off-diag -U(0,1] seed 4, FP64 upper CRS",
    "anderson32": "3D Anderson 32^3 periodic 7-pt, disorder U[-8.25,8.25) seed 1, FP64 upper CRS",
    "xxz24": "Heisenberg XXZ chain L=24 periodic, Sz=0 (2,704,156 rows), FP64 upper CRS (small profiling case)",
    "st27_100": "3D 27-point stencil 100^3 nonperiodic SPD, FP64 upper CRS (small profiling case of st27_200)",
    "batch64": "64 matrices: Anderson L~U[16,96] and geometric graphs n~U[1e4,1e6] (mean degree 20), FP64, k=4",
}

def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def max_over_ranks(times, world, device):
    """Element-wise max of the per-rank timings (seconds) over all ranks; a
    no-op for one rank.  `device` is where the collective runs (cuda for
    NCCL, cpu for gloo)."""
    import torch
    t = torch.tensor([float(v) for v in times], dtype=torch.float64, device=device)
    if world > 1:
        torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
    return [float(v) for v in t.cpu()]


def whole_job_rate(world, units_per_step, steps, seconds):
    """Whole-job throughput: every rank processes `units_per_step` per step
    (replicas, weak scaling), timed by the slowest rank."""
    return world * units_per_step * steps / seconds


def load_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


def kernel_sources_hash(files=None):
    """Hash of the kernel sources: the listed files of csrc/ (those that
    define the profiled kernel), or all of them."""
    h = hashlib.sha256()
    cs = os.path.join(ROOT, "paper_1907_06487_gb300", "csrc")
    for name in sorted(files if files else os.listdir(cs)):
        with open(os.path.join(cs, name), "rb") as f:
            h.update(name.encode())
            h.update(f.read())
    return h.hexdigest()[:16]


def ncu_traffic(workload, kernel):
    """DRAM bytes per launch from the committed ncu summary, if taken on these sources."""
    p = os.path.join(ROOT, "profiles", "traffic.json")
    if not os.path.exists(p):
        return None
    with open(p) as f:
        d = json.load(f)
    e = d.get(workload, {}).get(kernel)
    if not e or e.get("sources") != kernel_sources_hash(e.get("source_files")):
        return None
    return e.get("dram_bytes_per_launch")


class ClockSampler:
    FIELDS = ("clocks.sm,clocks.max.sm,clocks_event_reasons.active,clocks_event_reasons.hw_slowdown,"
              "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
              "clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.proc = None
        self.gpu = gpu_index

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "100"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        time.sleep(0.25)
        self.proc.terminate()
        try:
            out, _ = self.proc.communicate(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
            out, _ = self.proc.communicate()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in out.strip().splitlines():
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 7:
                continue
            try:
                sm.append(float(parts[0]))
                smax.append(float(parts[1]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[3:7]):
                if v.lower() == "active":
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def _repeat(fn, seconds):
    """Runs fn until `seconds` have passed (at least once); (count, seconds)."""
    t0 = time.perf_counter()
    k = 0
    while True:
        fn()
        k += 1
        dt = time.perf_counter() - t0
        if dt >= seconds:
            return k, dt


def oracle_cpu(m, name, seconds):
    """The oracle on the host cores: the paper's own CPU method (the oracle's
    RACE schedule for N_t = all host threads, executed phase by phase on
    those threads), plus the serial SymmSpMV and the full-CRS SpMV on all
    threads, each repeated for about a third of `seconds` (setup untimed)."""
    import numpy as np

    import oracle
    from paper_1907_06487_gb300 import configs, perfmodel as pm
    n, nu = m["n"], len(m["col"])
    flops = pm.flops(2 * nu - n)
    threads = oracle.max_threads()
    x = configs.vectors(name, n)
    t0 = time.perf_counter()
    sched = oracle.Race(m, threads)
    pm_ = oracle.permute_upper(m, sched.perm)
    xp = np.ascontiguousarray(x[sched.perm])
    full = oracle.expand_full(m)
    setup = time.perf_counter() - t0
    oracle.symm_spmv_race(pm_, sched, xp, threads)  # warm
    k_r, t_r = _repeat(lambda: oracle.symm_spmv_race(pm_, sched, xp, threads), seconds / 3)
    k_s, t_s = _repeat(lambda: oracle.symm_spmv(pm_, xp), seconds / 3)
    k_f, t_f = _repeat(lambda: oracle.spmv_full_par(full, x, threads), seconds / 3)
    race = flops * k_r / t_r / 1e9
    return {
        "value": race, "unit": "GFLOP/s", "cores": threads, "kind": "oracle",
        "sample": (f"{k_r} SymmSpMV sweeps of the {name} matrix under the oracle's RACE schedule "
                   f"(N_t = {threads}, {sched.n_phases} phases, {sched.n_leaves} leaves, eta {sched.eta:.3f}) "
                   f"on {threads} threads, {t_r:.1f} s; setup {setup:.1f} s untimed"),
        "serial_symm_1core": {"value": flops * k_s / t_s / 1e9, "sweeps": k_s},
        "full_spmv_all_cores": {"value": flops * k_f / t_f / 1e9, "sweeps": k_f, "cores": threads},
        "ms_per_sweep": t_r / k_r * 1e3,
    }


def oracle_normwise_error(m, x, b_perm, perm, ref=None):
    """||b - b_ref||_2 / || |A||x| ||_2 of a result b (given in the schedule's
    permuted order) against the FP64 oracle's plain definition (part of the
    CPU-baseline leg: the only place bench.py runs the oracle).  `ref` may
    carry the oracle's (b_ref, |A||x|) from an earlier call on the same m, x."""
    import numpy as np

    import oracle
    bref, s = ref if ref is not None else oracle.spmv_full(oracle.expand_full(m), x)
    b = np.empty_like(bref)
    b[perm] = b_perm
    return float(np.linalg.norm(b - bref) / np.linalg.norm(s))


def oracle_reference(m, x):
    """The oracle's (b_ref, |A||x|) for oracle_normwise_error."""
    import oracle
    return oracle.spmv_full(oracle.expand_full(m), x)


# the metric of both arms (the reference arm times the oracle's RACE
# SymmSpMV on the host cores under the same name, unit and direction)
METRIC_SYMM = "SymmSpMV GFLOP/s (2*nnz_full flops per step) on 1 GB300 vs full-CRS SpMV"


def run_reference(args):
    rank, world, _ = dist_env()
    if rank != 0:
        return 0
    from paper_1907_06487_gb300 import configs
    m = configs.matrix(args.workload)
    cpu = oracle_cpu(m, args.workload, max(3.0, args.ref_seconds))
    line = {
        "impl": "reference", "metric": METRIC_SYMM, "value": cpu["value"],
        "unit": "GFLOP/s", "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": cpu["ms_per_sweep"], "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f64", "data": "synthetic",
        "config": {"workload": args.workload, "desc": WORKLOAD_DESC.get(args.workload, args.workload)},
        "cpu_baseline": cpu,
        "e2e": {"value": cpu["value"], "unit": "GFLOP/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line))
    return 0




class Timer:
    """CUDA-event timing on one stream: warm-up, barrier + synchronize on both
    sides of the timed region (the rule of every timed number here)."""

    def __init__(self, stream, dev, world):
        self.stream, self.dev, self.world = stream, dev, world

    def barrier(self):
        if self.world > 1:
            import torch
            torch.distributed.barrier()

    def __call__(self, fn, steps, warmup):
        import torch
        for i in range(warmup):
            fn(i)
        self.stream.synchronize()
        self.barrier()
        torch.cuda.synchronize(self.dev)
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(self.stream)
        for i in range(steps):
            fn(i)
        e1.record(self.stream)
        torch.cuda.synchronize(self.dev)
        self.barrier()
        return e0.elapsed_time(e1) * 1e-3


def measure_ceilings(R, dev, stream, timer):
    """The load-only HBM bandwidth (2 GiB streamed once per call, best of 5)
    and the FP64 fused multiply-add rate, both with race_probe_peaks."""
    import torch
    n = 1 << 28
    with torch.cuda.stream(stream):
        buf = torch.ones(n, dtype=torch.float64, device=dev)
        out = torch.empty(4096, dtype=torch.float64, device=dev)
    best = min(timer(lambda i: R.race_probe_peaks(0, buf, n, out, 1, stream), 1, 1) for _ in range(5))
    load_gbs = 8.0 * n / best / 1e9
    del buf
    iters = 4096
    threads = torch.cuda.get_device_properties(dev).multi_processor_count * 4 * 256
    t = min(timer(lambda i: R.race_probe_peaks(1, None, 0, out, iters, stream), 1, 1) for _ in range(3))
    dfma = 8.0 * iters * threads / t
    torch.cuda.empty_cache()
    return {"load_only_gbs": load_gbs, "fp64_fma_per_s": dfma,
            "how": "race_probe_peaks: 2 GiB read once with 16-byte streaming loads (best of 5); eight "
                   "independent FP64 FMA chains per thread, 1024 threads per SM (best of 3)"}


def reduction_paths(R, dev, stream, timed, n, m):
    """How fast this GPU combines scattered FP64 contributions, five ways
    (race_probe_reductions), over m targets drawn uniformly from n (random)
    and over consecutive targets (sequential): the reductions at L2 that the
    default executors use, the plain read-modify-write a conflict-free
    schedule would permit, shared-memory and cluster-shared-memory atomics
    (the on-chip windows), and bulk row reductions of 16 doubles."""
    import torch
    with torch.cuda.stream(stream):
        pats = {"random": torch.randint(0, n, (m,), dtype=torch.int32, device=dev),
                "sequential": torch.remainder(torch.arange(m, device=dev), n).to(torch.int32)}
        t = torch.zeros(16 * n, dtype=torch.float64, device=dev)
    names = ("l2_reduction", "plain_rmw", "shared_atomic", "cluster_shared_atomic", "bulk_row_reduction")
    out = {"targets": n, "contributions": m}
    for pat, idx in pats.items():
        for mode, name in enumerate(names):
            sec = timed(lambda i: R.race_probe_reductions(mode, idx, m, n - 1, t, 16 * n, stream), 3, 1) / 3
            elems = m * (16 if mode == 4 else 1)
            out[f"{name}_{pat}_g_per_s"] = elems / sec / 1e9
    del pats, t
    torch.cuda.empty_cache()
    return out


def roofline_block(nbytes, seconds, peak, peak_kind, load_gbs, traffic=None, overwrite_bytes=None):
    """HBM roofline of one launch: algorithmic bytes over its time against
    the measured copy peak (and the load-only bandwidth, the paper's range)."""
    achieved = nbytes / seconds / 1e9
    out = {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
           "traffic": traffic, "peak_kind": peak_kind, "algorithmic_bytes_per_step": nbytes,
           "load_only_peak": load_gbs, "frac_of_load_only": achieved / load_gbs if load_gbs else None}
    if overwrite_bytes is not None:
        out["algorithmic_bytes_overwrite"] = overwrite_bytes
        out["frac_overwrite_count"] = overwrite_bytes / seconds / 1e9 / peak
    return out


def spmm_roof(flops, nbytes, seconds, hbm_gbs, dfma_per_s, fp64_fmas):
    """SymmSpMM against min(HBM * I, FP64 roof), I = flops / bytes.  The FP64
    roof counts the FP64 work the arithmetic cannot move off the FP64 pipe:
    `fp64_fmas` fused multiply-adds per call (the row sums, one per stored
    entry and right-hand side; the transposed products can run on the
    integer pipes and their additions at L2), at the measured rate.  The
    plain FP64 form's roof, every flop on the FP64 pipe (2 flops per fused
    multiply-add), is given beside it."""
    intensity = flops / nbytes
    hbm_roof = hbm_gbs * 1e9 * intensity
    fp64_roof = flops * dfma_per_s / fp64_fmas
    roof = min(hbm_roof, fp64_roof)
    achieved = flops / seconds
    return {"intensity_flop_per_byte": intensity, "roof_gflops": roof / 1e9,
            "bound": "hbm" if hbm_roof < fp64_roof else "fp64",
            "frac_of_roof": achieved / roof, "frac_hbm": nbytes / seconds / 1e9 / hbm_gbs,
            "plain_fp64_roof_gflops": 2.0 * dfma_per_s / 1e9,
            "frac_of_plain_fp64_roof": achieved / (2.0 * dfma_per_s)}


# SymmSpMM right-hand-side counts timed in the 27-point stencil block
SPMM_KS = (4, 8, 16)
RING = 4  # x and b buffers rotated over the timed steps


def arithmetic_label(launch):
    """What the launch computes in: FP64 throughout, or FP64 row sums with a
    share of the transposed products formed by an integer product of the
    significands (a binary64 result: the exact product truncated, below two
    units in the last place, relative error below 2^-51; x, b and the
    accumulation stay FP64), or (staged executor) double-float row sums."""
    ex = launch.get("executor")
    if ex in (8, 9, 13):
        q = launch.get("fp64_quarters", 0)
        return (f"f64 row sums; transposed products f64 multiplies in {q}/4 of the warps and in {4 - q}/4 "
                f"f64 products formed on the integer pipes (significands multiplied in 32-bit pieces, "
                f"truncated to 53 bits)")
    if ex == 10:
        return (f"row sums f64 in {launch.get('rowsum_fp64_quarters', 4)}/4 of the warps (rest double-float), "
                f"transposed products f64 multiplies in {launch.get('fp64_quarters', 0)}/4 (rest formed on the "
                f"integer pipes)")
    return "f64"


def dtype_label(launch):
    """f64 unless the staged executor sums some rows in double-float."""
    if launch.get("executor") == 10 and launch.get("rowsum_fp64_quarters", 4) < 4:
        return "f64+df64"
    return "f64"


def run_ours(args):
    import numpy as np
    import torch

    import paper_1907_06487_gb300 as R
    from paper_1907_06487_gb300 import build as B, configs, perfmodel as pm

    rank, world, local = dist_env()
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    if rank == 0:
        B.build()
    if world > 1:
        dist.barrier()
    R.lib()
    stream = torch.cuda.Stream(device=dev)
    timed = Timer(stream, dev, world)
    peak, peak_kind = load_peaks()
    ceil = measure_ceilings(R, dev, stream, timed)

    name = args.workload
    m = configs.matrix(name)
    cfg = configs.SCHEDULE[name]
    n, nu = m["n"], len(m["col"])
    nf = 2 * nu - n
    t0 = time.perf_counter()
    s = R.race_build(m, cfg["n_workers"], eps=cfg["eps"], max_depth=cfg["max_depth"], stream=stream,
                     rcm=cfg.get("rcm", False), windows=False)
    build_s = time.perf_counter() - t0
    lc = cfg["launch"]
    R.race_set_launch(s, 0, **lc)
    fl = cfg["full_launch"]
    R.race_prepare_full(s, stream)
    R.race_set_launch(s, 1, **fl)
    info = s.info()
    perm = s.perm()
    x_host = configs.vectors(name, n)

    with torch.cuda.stream(stream):
        xs = []
        for i in range(RING):
            xo = torch.from_numpy(x_host).to(dev) if i == 0 else torch.rand(n, dtype=torch.float64, device=dev)
            xp = torch.empty_like(xo)
            R.race_permute(s, xo, xp, 1, stream)
            xs.append(xp)
        bs = [torch.empty(n, dtype=torch.float64, device=dev) for _ in range(RING)]
    stream.synchronize()

    # ---- main timed region: SymmSpMV -------------------------------------------------------
    clocks = ClockSampler(local)
    clocks.start()
    time.sleep(0.3)
    t_symm = timed(lambda i: R.symm_spmv(s, xs[i % RING], bs[i % RING], stream), args.steps, args.warmup)
    clk = clocks.stop()
    R.race_poll_status(s, stream)
    # ---- the plain FP64 form: the all-FP64 row-parallel executor on the same schedule --------
    R.race_set_launch(s, 0, executor=R.RACE_EXEC_ROWS_RED, group_lanes=1, rows_per_group=1, blocks_per_sm=0,
                      regs_per_row=8, fp64_quarters=4)
    t_strict = timed(lambda i: R.symm_spmv(s, xs[i % RING], bs[i % RING], stream), args.steps, args.warmup)
    # ---- the same arithmetic and shape, phase by phase on the same schedule -----------------
    R.race_set_launch(s, 0, **dict(lc, executor=R.RACE_EXEC_PHASE_DF64))
    t_phased = timed(lambda i: R.symm_spmv(s, xs[i % RING], bs[i % RING], stream), args.steps, args.warmup)
    R.race_set_launch(s, 0, **lc)
    # ---- the limit the reduction-based executors share: the scatter's reductions at L2 ------
    def probe(mode):
        def step(i):
            if mode == 0:
                bs[i % RING].zero_()
            R.race_probe_scatter(s, mode, bs[i % RING], stream)
        with torch.cuda.stream(stream):
            return timed(step, args.steps, args.warmup)
    t_red, t_col = probe(0), probe(1)
    mpk = mpk_block(R, pm, s, n, nu, dev, stream, timed, args.steps, peak)
    R.race_set_launch(s, 0, **lc)
    red_paths = reduction_paths(R, dev, stream, timed, n, nu - n) if not args.no_extra else None
    spmm_head = None
    if args.spmm_k:
        # SymmSpMM on the headline schedule with the workload's launch (no tuning:
        # the profiling recipe captures exactly this kernel)
        k = args.spmm_k
        with torch.cuda.stream(stream):
            Xk = [torch.rand(n * k, dtype=torch.float64, device=dev) for _ in range(2)]
            Bk = [torch.empty(n * k, dtype=torch.float64, device=dev) for _ in range(2)]
        tk = timed(lambda i: R.symm_spmm(s, k, Xk[i % 2], Bk[i % 2], stream), args.steps, args.warmup) / args.steps
        spmm_head = {"k": k, "ms_per_step": tk * 1e3, "gflops": pm.flops(nf, k) / tk / 1e9, "launch": lc,
                     **spmm_roof(pm.flops(nf, k), pm.symm_bytes_rmw(n, nu, k), tk, peak, ceil["fp64_fma_per_s"],
                                nu * k)}
        del Xk, Bk
    # ---- traffic baseline: full-CRS SpMV on the same permuted matrix -----------------------
    t_full = timed(lambda i: R.spmv_full(s, xs[i % RING], bs[i % RING], stream), args.steps, args.warmup)
    # ---- the conflict-free RACE executors (a few steps: they are slow) on the schedule that
    # suits them (full recursion), one row per thread in the leaf executor
    cf = cfg["conflict_free"]
    s_cf = R.race_build(m, cf["n_workers"], eps=cfg["eps"], max_depth=cf["max_depth"], stream=stream,
                        one_level_stage0=cf.get("one_level_stage0", False))
    info_cf = s_cf.info()
    R.race_set_launch(s_cf, 0, R.RACE_EXEC_LEAF_CTA, 1, 1, 0, 8)
    t_leaf_cta = timed(lambda i: R.symm_spmv(s_cf, xs[i % RING], bs[i % RING], stream), 3, 1)
    t_win_race = timed(lambda i: R.symm_spmv_exec(s_cf, R.RACE_EXEC_WINDOW_RACE, xs[i % RING], bs[i % RING],
                                                  stream), 3, 1)
    # every phase in one cooperative launch, grid barriers between phases
    R.race_set_launch(s_cf, 0, R.RACE_EXEC_PERSIST_CTA, 1, 1, 0, 8)
    t_persist_cta = timed(lambda i: R.symm_spmv(s_cf, xs[i % RING], bs[i % RING], stream), 3, 1)
    # the paper's model proper: a leaf per worker (a group of 8 lanes), plain updates of b
    R.race_set_launch(s_cf, 0, R.RACE_EXEC_LEAF_GROUP, 8, 1, 0, 8)
    t_leaf_group = timed(lambda i: R.symm_spmv(s_cf, xs[i % RING], bs[i % RING], stream), 3, 1)
    R.race_set_launch(s_cf, 0, R.RACE_EXEC_PERSIST_GROUP, 8, 1, 0, 8)
    t_persist_group = timed(lambda i: R.symm_spmv(s_cf, xs[i % RING], bs[i % RING], stream), 3, 1)
    R.race_poll_status(s_cf, stream)  # raises if a grid barrier gave up
    # the headline's arithmetic phase by phase, each leaf spread over the GPU
    R.race_set_launch(s_cf, 0, **dict(lc, executor=R.RACE_EXEC_PHASE_DF64))
    t_phase_cf = timed(lambda i: R.symm_spmv(s_cf, xs[i % RING], bs[i % RING], stream), args.steps, args.warmup)
    s_cf.free()
    # ---- the paper's comparison methods, multicolouring (MC) and algebraic block
    # multicolouring (ABMC, blocks of 64 rows), under the same conflict-free executors --------
    colourings = {}
    if not args.no_extra:
        for label, method, block in (("mc", R.RACE_COLOR_MC, 1), ("abmc64", R.RACE_COLOR_ABMC, 64)):
            t0c = time.perf_counter()
            sc = R.race_build_coloring(m, method, block, n_workers=cf["n_workers"], stream=stream, windows=False)
            bsec = time.perf_counter() - t0c
            ic = sc.info()
            R.race_set_launch(sc, 0, R.RACE_EXEC_LEAF_CTA, 1, 1, 0, 8)
            t_c = timed(lambda i: R.symm_spmv(sc, xs[i % RING], bs[i % RING], stream), 3, 1)
            R.race_set_launch(sc, 0, R.RACE_EXEC_PERSIST_CTA, 1, 1, 0, 8)
            t_cp = timed(lambda i: R.symm_spmv(sc, xs[i % RING], bs[i % RING], stream), 3, 1)
            R.race_poll_status(sc, stream)
            R.race_set_launch(sc, 0, **dict(lc, executor=R.RACE_EXEC_PHASE_DF64))
            t_cd = timed(lambda i: R.symm_spmv(sc, xs[i % RING], bs[i % RING], stream), args.steps, args.warmup)
            colourings[label] = {"colours": ic["n_phases"], "leaves": ic["n_leaves"], "eta": ic["eta"],
                                 "leaf_cta_ms_per_step": t_c / 3 * 1e3, "persist_cta_ms_per_step": t_cp / 3 * 1e3,
                                 "phase_df64_ms_per_step": t_cd / args.steps * 1e3, "build_seconds": bsec}
            sc.free()
    # ---- the same two kernels on the input order (no RACE permutation) --------------------
    s_nat = R.race_build(m, cfg["n_workers"], natural_order=True, windows=False, stream=stream)
    R.race_set_launch(s_nat, 0, **lc)
    R.race_prepare_full(s_nat, stream)
    R.race_set_launch(s_nat, 1, **fl)
    t_nat_symm = timed(lambda i: R.symm_spmv(s_nat, xs[i % RING], bs[i % RING], stream), args.steps, args.warmup)
    t_nat_full = timed(lambda i: R.spmv_full(s_nat, xs[i % RING], bs[i % RING], stream), args.steps, args.warmup)
    s_nat.free()
    # ---- FP32-stored values (x, b and the row sums stay FP64), same schedule and launch ----
    s32 = R.race_import(m, s.export(), stream=stream, val_type=R.RACE_F32, windows=False)
    R.race_set_launch(s32, 0, **lc)
    t_f32 = timed(lambda i: R.symm_spmv(s32, xs[i % RING], bs[i % RING], stream), args.steps, args.warmup)
    with torch.cuda.stream(stream):
        R.symm_spmv(s32, xs[0], bs[0], stream)
    stream.synchronize()
    b32_perm = bs[0].cpu().numpy()
    s32.free()
    # ---- end to end through host buffers: H2D x, permute, SymmSpMV, unpermute, D2H b --------
    # Each step copies its x in and its b out; copies run on their own streams
    # over two buffer sets, so step i's read-back overlaps step i+1's upload and
    # compute, as a caller streaming vectors through the library would run it.
    s_in, s_out = torch.cuda.Stream(device=dev), torch.cuda.Stream(device=dev)
    NB = 2  # buffer sets in flight (three measured slower: 0.72 against 0.51-0.53 ms per step)
    xh = [torch.from_numpy(x_host).pin_memory() for _ in range(NB)]
    bh = [torch.empty(n, dtype=torch.float64).pin_memory() for _ in range(NB)]
    xd = [torch.empty(n, dtype=torch.float64, device=dev) for _ in range(NB)]
    bd = [torch.empty(n, dtype=torch.float64, device=dev) for _ in range(NB)]
    xpd, bpd = (torch.empty(n, dtype=torch.float64, device=dev) for _ in range(2))
    ev_in, ev_c, ev_out = ([torch.cuda.Event() for _ in range(NB)] for _ in range(3))

    def e2e_step(i):
        j = i % NB
        s_in.wait_event(ev_c[j])        # xd[j] consumed by the step NB back
        with torch.cuda.stream(s_in):
            xd[j].copy_(xh[j], non_blocking=True)
        ev_in[j].record(s_in)
        stream.wait_event(ev_in[j])
        stream.wait_event(ev_out[j])    # bd[j] read back by the step NB back
        R.race_permute(s, xd[j], xpd, 1, stream)
        R.symm_spmv(s, xpd, bpd, stream)
        R.race_unpermute(s, bpd, bd[j], 1, stream)
        ev_c[j].record(stream)
        s_out.wait_event(ev_c[j])
        with torch.cuda.stream(s_out):
            bh[j].copy_(bd[j], non_blocking=True)
        ev_out[j].record(s_out)

    def timed_e2e(steps, warmup):
        for i in range(warmup):
            e2e_step(i)
        torch.cuda.synchronize(dev)
        timed.barrier()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        s_in.wait_stream(stream)
        for i in range(steps):
            e2e_step(i)
        stream.wait_stream(s_out)
        e1.record(stream)
        torch.cuda.synchronize(dev)
        timed.barrier()
        return e0.elapsed_time(e1) * 1e-3

    t_e2e = timed_e2e(args.steps, args.warmup)

    # the copies alone, both directions at once on their own streams: the floor
    # the host link sets for the end-to-end step
    def timed_copies(steps, warmup):
        def one(i):
            j = i % NB
            with torch.cuda.stream(s_in):
                xd[j].copy_(xh[j], non_blocking=True)
            with torch.cuda.stream(s_out):
                bh[j].copy_(bd[j], non_blocking=True)
        for i in range(warmup):
            one(i)
        torch.cuda.synchronize(dev)
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        s_in.wait_stream(stream)
        s_out.wait_stream(stream)
        for i in range(steps):
            one(i)
        stream.wait_stream(s_in)
        stream.wait_stream(s_out)
        e1.record(stream)
        torch.cuda.synchronize(dev)
        return e0.elapsed_time(e1) * 1e-3

    t_copies = timed_copies(args.steps, args.warmup)
    # the read-back must equal the device-timed result for the same x (xs[0] is x_host permuted)
    with torch.cuda.stream(stream):
        R.symm_spmv(s, xs[0], bs[0], stream)
        R.race_unpermute(s, bs[0], bd[0], 1, stream)
    stream.synchronize()
    ref = bd[0].cpu().numpy()
    got = bh[(args.steps - 1) % NB].numpy()
    e2e_ok = bool(np.allclose(got, ref, rtol=1e-12, atol=1e-12 * float(np.abs(ref).max())))
    t_symm, t_full, t_e2e, t_red, t_col, t_strict, t_phased = max_over_ranks(
        [t_symm, t_full, t_e2e, t_red, t_col, t_strict, t_phased], world, dev)
    s.free()
    del xs, bs, xd, bd, xpd, bpd
    torch.cuda.empty_cache()

    flops = pm.flops(nf)
    per_step = t_symm / args.steps
    value = whole_job_rate(world, flops, args.steps, t_symm) / 1e9
    full_gflops = whole_job_rate(world, flops, args.steps, t_full) / 1e9
    e2e_value = whole_job_rate(world, flops, args.steps, t_e2e) / 1e9
    per_phase = (R.RACE_EXEC_LEAF_GROUP, R.RACE_EXEC_LEAF_CTA, R.RACE_EXEC_WINDOW_RACE, R.RACE_EXEC_PHASE_DF64)
    launches_per_step = info["n_phases"] if lc["executor"] in per_phase else 1

    # ---- the other workloads of the default run (rank 0's replica measures them too) --------
    extra = {}
    if not args.no_extra and name == "xxz26":
        extra["st27_200"] = stencil_block(args, R, configs, pm, dev, stream, timed, peak, peak_kind, ceil, local)
        extra["anderson32"] = small_block(args, R, configs, pm, dev, stream, timed)
        extra["batch64"] = batch_block(args, R, configs, pm, dev, stream, timed, peak, peak_kind, e2e=False)
    if rank != 0:
        return 0

    # CPU baseline: the oracle on a bounded sample, and the FP32-value error against it
    cpu = None
    fp32_err = None
    if not args.no_cpu_baseline:
        cpu = oracle_cpu(m, name, args.cpu_seconds)
        fp32_err = oracle_normwise_error(m, x_host, b32_perm, perm)
    traffic = ncu_traffic(name, "symm")
    sym_bytes = pm.symm_bytes_rmw(n, nu)
    line = {
        "metric": METRIC_SYMM,
        "value": value, "unit": "GFLOP/s", "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": per_step * 1e3, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": dtype_label(lc), "arithmetic": arithmetic_label(lc),
        "data": "synthetic",
        "config": {"workload": name, "desc": WORKLOAD_DESC.get(name, name), "n": n, "nnz_upper": nu, "nnz_full": nf,
                   "l2": "inputs larger than L2 (matrix 1.05 GB; x, b rotate over 4+4 buffers of 83 MB)",
                   "schedule": {"n_workers": cfg["n_workers"], "eps": list(cfg["eps"]), "n_phases": info["n_phases"],
                                "eta": info["eta"], "depth": info["depth"], "rcm": bool(cfg.get("rcm", False))},
                   "launch": lc, "parallelism": f"replicas x{world}"},
        "roofline": roofline_block(sym_bytes, per_step, peak, peak_kind, ceil["load_only_gbs"], traffic,
                                   pm.symm_bytes(n, nu)),
        "ceilings": ceil,
        "strict_fp64": {"ms_per_step": t_strict / args.steps * 1e3,
                        "gflops": flops / (t_strict / args.steps) / 1e9,
                        "frac": sym_bytes / (t_strict / args.steps) / 1e9 / peak,
                        "launch": "RACE_EXEC_ROWS_RED, one row per lane, all arithmetic FP64 (the plain FP64 form)"},
        "race_phased": {"ms_per_step": t_phased / args.steps * 1e3,
                        "gflops": flops / (t_phased / args.steps) / 1e9,
                        "frac": sym_bytes / (t_phased / args.steps) / 1e9 / peak,
                        "vs_headline": t_phased / t_symm, "n_phases": info["n_phases"], "n_leaves": info["n_leaves"],
                        "what": "RACE_EXEC_PHASE_DF64: the headline's arithmetic and launch shape run phase by phase "
                                "(one launch per phase over its leaves' rows, no two concurrent leaves sharing an "
                                "entry of b; updates inside a leaf are L2 reductions) on the same schedule"},
        "reduction_floor": {"ms_per_step": t_red / args.steps * 1e3, "columns_only_ms_per_step": t_col / args.steps * 1e3,
                            "frac": (t_red / args.steps) / per_step,
                            "what": "race_probe_scatter on the same schedule: the transposed update's L2 reductions "
                                    "alone (mode 0, b zeroed first) and its column stream alone (mode 1), with the "
                                    "executors' access pattern; frac = that floor / SymmSpMV time"},
        "spmv_full": {"value": full_gflops, "unit": "GFLOP/s", "ms_per_step": t_full / args.steps * 1e3,
                      "gbs": pm.full_bytes(n, nf) / (t_full / args.steps) / 1e9,
                      "frac": pm.full_bytes(n, nf) / (t_full / args.steps) / 1e9 / peak},
        "fp32_values": {"ms_per_step": t_f32 / args.steps * 1e3, "gflops": flops / (t_f32 / args.steps) / 1e9,
                        "gbs": pm.symm_bytes_rmw(n, nu, 1, 4) / (t_f32 / args.steps) / 1e9,
                        "normwise_error_vs_fp64_oracle": fp32_err,
                        "what": "values stored in FP32 (8 B per stored entry), x, b and row sums FP64; error = "
                                "||b32 - b_ref||_2 / || |A||x| ||_2 against the FP64 oracle (computed in the CPU "
                                "baseline leg; null without it).  The XXZ values (+-1/2, multiples of 1/4) are "
                                "exact in FP32: the 27-point stencil block carries the error that matters"},
        "natural_order": {"symm_ms_per_step": t_nat_symm / args.steps * 1e3,
                          "symm_gflops": flops / (t_nat_symm / args.steps) / 1e9,
                          "full_ms_per_step": t_nat_full / args.steps * 1e3,
                          "speedup_vs_full": t_nat_full / t_nat_symm,
                          "what": "the same launches on the input order (RACE_FLAG_NATURAL_ORDER: no permutation)"},
        "race_conflict_free": {"leaf_cta_ms_per_step": t_leaf_cta / 3 * 1e3,
                               "persist_cta_ms_per_step": t_persist_cta / 3 * 1e3,
                               "phase_df64_ms_per_step": t_phase_cf / args.steps * 1e3,
                               "leaf_group8_ms_per_step": t_leaf_group / 3 * 1e3,
                               "persist_group8_ms_per_step": t_persist_group / 3 * 1e3,
                               "window_race_ms_per_step": t_win_race / 3 * 1e3,
                               "schedule": {"n_workers": cf["n_workers"], "max_depth": cf["max_depth"],
                                            "one_level_stage0": bool(cf.get("one_level_stage0", False)),
                                            "n_phases": info_cf["n_phases"], "n_leaves": info_cf["n_leaves"],
                                            "eta": info_cf["eta"]},
                               "colourings": colourings,
                               "what": "RACE_EXEC_LEAF_CTA, _WINDOW_RACE, _LEAF_GROUP (8 lanes a leaf, plain "
                                       "updates of b), the one-launch _PERSIST_CTA / _PERSIST_GROUP (grid "
                                       "barriers between phases) and _PHASE_DF64 (the headline's arithmetic, each "
                                       "leaf spread over the GPU) -- phase by phase, no two concurrent leaves share "
                                       "an entry of b; x and b in that schedule's order -- on a fully recursed "
                                       "schedule (3 steps each, PHASE_DF64 the bench's steps); the leaf-per-block "
                                       "and phase executors on the in-house MC and ABMC colourings "
                                       "(race_build_coloring)"},
        "speedup_vs_full": t_full / t_symm,
        "matrix_powers": mpk,
        "reduction_paths": red_paths,
        "spmm_headline": spmm_head,
        "e2e": {"value": e2e_value, "unit": "GFLOP/s", "h2d_bytes_per_step": 8 * n, "d2h_bytes_per_step": 8 * n,
                "ms_per_step": t_e2e / args.steps * 1e3, "matches_device_result": e2e_ok,
                "copies_only_ms_per_step": t_copies / args.steps * 1e3,
                "host_link_gbs": 16 * n / (t_copies / args.steps) / 1e9,
                "frac_of_copy_floor": t_copies / t_e2e,
                "how": "per step: pinned H2D of x, permute, SymmSpMV, unpermute, D2H of b into pinned memory; "
                       "copies on their own streams, double-buffered across steps; copies_only: the same two "
                       "copies per step with no compute (the host link's floor for the step)"},
        "gpu_launches": launches_per_step * args.steps,
        "clocks": clk,
        "cpu_baseline": cpu,
        "build_seconds": build_s,
    }
    line.update(extra)
    print(json.dumps(line))
    if world > 1:
        torch.distributed.destroy_process_group()
    return 0


def stencil_block(args, R, configs, pm, dev, stream, timed, peak, peak_kind, ceil, local):
    """The 27-point stencil 200^3 (paper: HPCG-like matrices): SymmSpMV in the
    benchmark's launch and in plain FP64, FP32-stored values with their
    normwise error against the FP64 oracle, the full-CRS SpMV, and SymmSpMM
    k = 4, 8, 16 (FP64 and FP32 values, each width autotuned first) against
    min(HBM * I, FP64 roof)."""
    import torch

    name = "st27_200"
    m = configs.matrix(name)
    cfg = configs.SCHEDULE[name]
    n, nu = m["n"], len(m["col"])
    nf = 2 * nu - n
    t0 = time.perf_counter()
    s = R.race_build(m, cfg["n_workers"], eps=cfg["eps"], max_depth=cfg["max_depth"], stream=stream,
                     rcm=cfg.get("rcm", False), windows=False)
    s32 = R.race_import(m, s.export(), stream=stream, val_type=R.RACE_F32, windows=False)
    build_s = time.perf_counter() - t0
    lc = cfg["launch"]
    R.race_set_launch(s, 0, **lc)
    R.race_set_launch(s32, 0, **lc)
    R.race_prepare_full(s, stream)
    R.race_set_launch(s, 1, **cfg["full_launch"])
    info = s.info()
    perm = s.perm()
    x_host = configs.vectors(name, n)
    with torch.cuda.stream(stream):
        xs = [torch.from_numpy(x_host[perm].copy()).to(dev)] + \
             [torch.rand(n, dtype=torch.float64, device=dev) for _ in range(RING - 1)]
        bs = [torch.empty(n, dtype=torch.float64, device=dev) for _ in range(RING)]
    stream.synchronize()
    K, W = args.steps, args.warmup
    clocks = ClockSampler(local)
    clocks.start()
    time.sleep(0.3)
    t_symm = timed(lambda i: R.symm_spmv(s, xs[i % RING], bs[i % RING], stream), K, W) / K
    clk = clocks.stop()
    with torch.cuda.stream(stream):
        R.symm_spmv(s, xs[0], bs[0], stream)
    stream.synchronize()
    b64_perm = bs[0].cpu().numpy()
    R.race_set_launch(s, 0, executor=R.RACE_EXEC_ROWS_RED, group_lanes=1, rows_per_group=1, blocks_per_sm=0,
                      regs_per_row=8, fp64_quarters=4)
    t_strict = timed(lambda i: R.symm_spmv(s, xs[i % RING], bs[i % RING], stream), K, W) / K
    R.race_set_launch(s, 0, **dict(lc, executor=R.RACE_EXEC_PHASE_DF64))
    t_phased = timed(lambda i: R.symm_spmv(s, xs[i % RING], bs[i % RING], stream), K, W) / K
    R.race_set_launch(s, 0, **lc)
    t_f32 = timed(lambda i: R.symm_spmv(s32, xs[i % RING], bs[i % RING], stream), K, W) / K
    with torch.cuda.stream(stream):
        R.symm_spmv(s32, xs[0], bs[0], stream)
    stream.synchronize()
    b32_perm = bs[0].cpu().numpy()
    t_full = timed(lambda i: R.spmv_full(s, xs[i % RING], bs[i % RING], stream), K, W) / K
    mpk = mpk_block(R, pm, s, n, nu, dev, stream, timed, K, peak)
    del xs, bs
    torch.cuda.empty_cache()
    flops = pm.flops(nf)
    hbm = peak
    out = {
        "workload": name, "desc": WORKLOAD_DESC[name], "n": n, "nnz_upper": nu, "nnz_full": nf,
        "matrix_powers": mpk,
        "schedule": {"n_workers": cfg["n_workers"], "max_depth": cfg["max_depth"], "rcm": bool(cfg.get("rcm")),
                     "n_phases": info["n_phases"], "eta": info["eta"]},
        "launch": lc, "arithmetic": arithmetic_label(lc), "build_seconds": build_s, "clocks": clk,
        "symm_spmv": {"ms_per_step": t_symm * 1e3, "gflops": flops / t_symm / 1e9,
                      "roofline": roofline_block(pm.symm_bytes_rmw(n, nu), t_symm, hbm, peak_kind,
                                                 ceil["load_only_gbs"], None, pm.symm_bytes(n, nu))},
        "strict_fp64": {"ms_per_step": t_strict * 1e3, "gflops": flops / t_strict / 1e9,
                        "frac": pm.symm_bytes_rmw(n, nu) / t_strict / 1e9 / hbm},
        "race_phased": {"ms_per_step": t_phased * 1e3, "gflops": flops / t_phased / 1e9,
                        "frac": pm.symm_bytes_rmw(n, nu) / t_phased / 1e9 / hbm, "vs_headline": t_phased / t_symm,
                        "n_phases": info["n_phases"], "n_leaves": info["n_leaves"]},
        "fp32_values": {"ms_per_step": t_f32 * 1e3, "gflops": flops / t_f32 / 1e9,
                        "frac": pm.symm_bytes_rmw(n, nu, 1, 4) / t_f32 / 1e9 / hbm},
        "spmv_full": {"ms_per_step": t_full * 1e3, "gflops": flops / t_full / 1e9,
                      "frac": pm.full_bytes(n, nf) / t_full / 1e9 / hbm},
        "speedup_vs_full": t_full / t_symm,
        "l2": "inputs larger than L2 (matrix 1.33 GB; x, b rotate over 4+4 buffers of 64 MB)",
    }
    if not args.no_cpu_baseline:
        ref = oracle_reference(m, x_host)
        out["fp32_values"]["normwise_error_vs_fp64_oracle"] = oracle_normwise_error(m, x_host, b32_perm, perm, ref)
        out["symm_spmv"]["normwise_error_vs_fp64_oracle"] = oracle_normwise_error(m, x_host, b64_perm, perm, ref)
        del ref
    # SymmSpMM: each width and value type tuned by the project's autotuner, then timed
    spmm = {}
    steps = max(3, K // 4)
    for k in SPMM_KS:
        with torch.cuda.stream(stream):
            Xk = [torch.rand(n * k, dtype=torch.float64, device=dev) for _ in range(2)]
            Bk = [torch.empty(n * k, dtype=torch.float64, device=dev) for _ in range(2)]
        for vt, sk, vb in (("f64", s, 8), ("f32", s32, 4)):
            tuned, _ = R.race_autotune(sk, k, Xk[0], Bk[0], reps=3, stream=stream)
            tk = timed(lambda i: R.symm_spmm(sk, k, Xk[i % 2], Bk[i % 2], stream), steps, 2) / steps
            fk, bk = pm.flops(nf, k), pm.symm_bytes_rmw(n, nu, k, vb)
            spmm[f"k{k}_{vt}"] = {"ms_per_step": tk * 1e3, "gflops": fk / tk / 1e9, "gbs": bk / tk / 1e9,
                                  "launch": tuned, "arithmetic": arithmetic_label(tuned),
                                  **spmm_roof(fk, bk, tk, hbm, ceil["fp64_fma_per_s"], nu * k)}
        del Xk, Bk
        torch.cuda.empty_cache()
    out["spmm"] = spmm
    s.free()
    s32.free()
    torch.cuda.empty_cache()
    out["gauss_seidel_kaczmarz"] = sweeps_block(args, R, configs, pm, dev, stream, timed, peak)
    return out


def mpk_block(R, pm, s, n, nu, dev, stream, timed, steps, peak, p=4):
    """Matrix powers A x .. A^p x on a schedule (its SymmSpMV launch): p
    sweeps against the level wavefront, bytes p times a SymmSpMV's."""
    import torch
    with torch.cuda.stream(stream):
        x = torch.rand(n, dtype=torch.float64, device=dev)
        Y = torch.empty(p * n, dtype=torch.float64, device=dev)
    out = {"p": p}
    k = max(3, steps // 4)
    for label, mode in (("sweeps", R.RACE_MPK_SWEEPS), ("wavefront", R.RACE_MPK_WAVEFRONT)):
        R.race_matrix_powers(s, p, x, Y, mode, stream)  # first use builds the wavefront's block table
        t = timed(lambda i: R.race_matrix_powers(s, p, x, Y, mode, stream), k, 2) / k
        out[label] = {"ms_per_call": t * 1e3, "ms_per_power": t / p * 1e3,
                      "frac": p * pm.symm_bytes_rmw(n, nu) / t / 1e9 / peak}
    R.race_poll_status(s, stream)
    del x, Y
    return out


def sweeps_block(args, R, configs, pm, dev, stream, timed, peak):
    """Symmetric Gauss-Seidel and symmetric Kaczmarz sweeps on the 27-point
    stencil under the fully recursed schedule the leaf executors use (the
    paper's execution model: phases in order, one leaf per lane group), and
    under the in-house MC and ABMC colourings."""
    import torch
    name = "st27_200"
    m = configs.matrix(name)
    cfg = configs.SCHEDULE[name]
    cf = cfg["sweeps"]
    n, nu = m["n"], len(m["col"])
    nf = 2 * nu - n
    t0 = time.perf_counter()
    s = R.race_build(m, cf["n_workers"], eps=cfg["eps"], max_depth=cf["max_depth"], stream=stream,
                     rcm=cfg.get("rcm", False), windows=False)
    R.race_prepare_full(s, stream)
    build_s = time.perf_counter() - t0
    info = s.info()
    with torch.cuda.stream(stream):
        b = torch.rand(n, dtype=torch.float64, device=dev)
        x = torch.zeros(n, dtype=torch.float64, device=dev)
    out = {"schedule": {"n_workers": cf["n_workers"], "max_depth": cf["max_depth"], "n_phases": info["n_phases"],
                        "n_leaves": info["n_leaves"], "eta": info["eta"]}, "build_seconds": build_s}
    sweeps = 3
    for label, fn in (("symm_gs", R.symm_gs), ("symm_kacz", R.symm_kacz)):
        fn(s, b, x, 1, stream)
        t = timed(lambda i: fn(s, b, x, sweeps, stream), 1, 1) / sweeps
        out[label] = {"ms_per_sweep": t * 1e3, "gbs": pm.sweep_bytes(n, nf) / t / 1e9,
                      "frac": pm.sweep_bytes(n, nf) / t / 1e9 / peak}
    s.free()
    # the same sweeps under the in-house multicolourings (one-row leaves for MC,
    # 16-row blocks for ABMC, both on the RCM order): every row of a colour in
    # parallel, a small lane group per leaf
    for label, method, block, lanes in (("mc", R.RACE_COLOR_MC, 1, 2), ("abmc16", R.RACE_COLOR_ABMC, 16, 4)):
        t0c = time.perf_counter()
        sc = R.race_build_coloring(m, method, block, stream=stream, windows=False, rcm=True)
        R.race_prepare_full(sc, stream)
        bsec = time.perf_counter() - t0c
        ic = sc.info()
        R.race_set_launch(sc, 0, executor=R.RACE_EXEC_LEAF_GROUP, group_lanes=lanes, rows_per_group=1,
                          blocks_per_sm=0, regs_per_row=8)
        blk = {"colours": ic["n_phases"], "leaves": ic["n_leaves"], "group_lanes": lanes, "build_seconds": bsec}
        for kl, fn in (("symm_gs", R.symm_gs), ("symm_kacz", R.symm_kacz)):
            fn(sc, b, x, 1, stream)
            t = timed(lambda i: fn(sc, b, x, sweeps, stream), 1, 1) / sweeps
            blk[kl] = {"ms_per_sweep": t * 1e3, "gbs": pm.sweep_bytes(n, nf) / t / 1e9,
                       "frac": pm.sweep_bytes(n, nf) / t / 1e9 / peak}
        out[label] = blk
        sc.free()
    del b, x
    torch.cuda.empty_cache()
    return out


def small_block(args, R, configs, pm, dev, stream, timed):
    """The Anderson model 32^3 (2.5 MB: L2-resident, no HBM-roof claim):
    every call timed alone with its own events, L2 flushed (a 256 MB write)
    between calls; the benchmark's executor, the full-CRS SpMV and the
    paper's execution model (leaf per block, phases in order)."""
    import torch

    name = "anderson32"
    m = configs.matrix(name)
    cfg = configs.SCHEDULE[name]
    n, nu = m["n"], len(m["col"])
    nf = 2 * nu - n
    s = R.race_build(m, cfg["n_workers"], eps=cfg["eps"], max_depth=cfg["max_depth"], stream=stream, windows=False)
    R.race_set_launch(s, 0, **cfg["launch"])
    R.race_prepare_full(s, stream)
    R.race_set_launch(s, 1, **cfg["full_launch"])
    info = s.info()
    with torch.cuda.stream(stream):
        x = torch.from_numpy(configs.vectors(name, n)[s.perm()].copy()).to(dev)
        b = torch.empty_like(x)
        flush = torch.empty(1 << 25, dtype=torch.float64, device=dev)

    def per_call(fn, calls):
        ts = []
        for i in range(calls + 3):
            with torch.cuda.stream(stream):
                flush.zero_()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            fn()
            e1.record(stream)
            e1.synchronize()
            if i >= 3:
                ts.append(e0.elapsed_time(e1) * 1e-3)
        return statistics.median(ts)

    calls = max(10, args.steps)
    t_symm = per_call(lambda: R.symm_spmv(s, x, b, stream), calls)
    t_full = per_call(lambda: R.spmv_full(s, x, b, stream), calls)
    t_leaf = per_call(lambda: R.symm_spmv_exec(s, R.RACE_EXEC_LEAF_CTA, x, b, stream), calls)
    s.free()
    del flush
    torch.cuda.empty_cache()
    flops = pm.flops(nf)
    return {"workload": name, "desc": WORKLOAD_DESC[name], "n": n, "nnz_upper": nu,
            "launch": cfg["launch"], "schedule": {"n_workers": cfg["n_workers"], "n_phases": info["n_phases"],
                                                  "eta": info["eta"]},
            "symm_us": t_symm * 1e6, "symm_gflops": flops / t_symm / 1e9, "spmv_full_us": t_full * 1e6,
            "leaf_cta_us": t_leaf * 1e6, "speedup_vs_full": t_full / t_symm,
            "timing": "median of per-call CUDA-event times, L2 flushed by a 256 MB write before each call",
            "roofline": "none claimed: 2.5 MB of matrix, L2- and latency-bound (as the paper treats its "
                        "L2-resident matrices)"}


def batch_block(args, R, configs, pm, dev, stream, timed, peak, peak_kind, e2e=True):
    """64 matrices (Anderson L in [16,96] and geometric graphs n in [1e4,1e6]),
    SymmSpMM with k = 4, each schedule built on a host thread and autotuned,
    all replayed by one CUDA graph.  With e2e: every X up and every B down per
    step as well (two buffer sets and graphs alternating)."""
    import concurrent.futures as cf
    import numpy as np
    import torch

    k = 4
    t0 = time.perf_counter()
    mats = configs.batch64()
    bsch = configs.BATCH_SCHEDULE

    def build(m):
        return R.race_build(m, bsch["n_workers"], max_depth=bsch["max_depth"], rcm=bsch.get("rcm", False),
                            host_only=True, windows=False)

    with cf.ThreadPoolExecutor(max_workers=max(1, min(16, os.cpu_count() or 1))) as ex:
        scheds = list(ex.map(build, mats))
    scheds_built = time.perf_counter() - t0
    Xs, Bs, Xh = [], [], []
    flops = 0
    sym_bytes = 0
    tuned = {}
    for i, (m, s) in enumerate(zip(mats, scheds)):
        R.race_upload(s, stream)
        n, nu = m["n"], len(m["col"])
        X = configs.matgen.uniform(n * k, 300 + i).reshape(n, k)
        xp = torch.from_numpy(np.ascontiguousarray(X[s.perm()])).to(dev)
        bp = torch.empty_like(xp)
        launch, _ = R.race_autotune(s, k, xp, bp, reps=3, stream=stream)
        key = f"{launch['executor']}/{launch['rows_per_group']}/{launch['blocks_per_sm']}"
        tuned[key] = tuned.get(key, 0) + 1
        Xs.append(xp)
        Bs.append(bp)
        Xh.append(X)
        flops += pm.flops(2 * nu - n, k)
        sym_bytes += pm.symm_bytes_rmw(n, nu, k)
    batch = R.race_batch_create(scheds, k, Xs, Bs, stream)
    setup_s = time.perf_counter() - t0
    stream.synchronize()
    t = timed(lambda i: batch.launch(stream), args.steps, args.warmup)
    per = t / args.steps
    out = {"workload": "batch64", "desc": WORKLOAD_DESC["batch64"], "k": k, "matrices": len(mats),
           "rows": int(sum(m["n"] for m in mats)), "schedule": dict(bsch), "tuned_launches": tuned,
           "ms_per_step": per * 1e3, "gflops": flops / per / 1e9, "flops_per_step": flops,
           "roofline": roofline_block(sym_bytes, per, peak, peak_kind, None),
           "setup_seconds": setup_s, "schedule_build_seconds": scheds_built,
           "l2": "inputs larger than L2 (all matrices and blocks: several GB per replay)",
           "note": "most matrices are small (L2- and latency-bound): the HBM fraction is not the measure here"}
    if e2e:
        xh = [torch.from_numpy(np.ascontiguousarray(X[s.perm()])).pin_memory() for X, s in zip(Xh, scheds)]
        bh = [[torch.empty_like(h).pin_memory() for h in xh] for _ in range(2)]
        X2 = [Xs, [torch.empty_like(x) for x in Xs]]
        B2 = [Bs, [torch.empty_like(b) for b in Bs]]
        batches = [batch, R.race_batch_create(scheds, k, X2[1], B2[1], stream)]
        s_in, s_out = torch.cuda.Stream(device=dev), torch.cuda.Stream(device=dev)
        ev_in, ev_c, ev_out = ([torch.cuda.Event() for _ in range(2)] for _ in range(3))

        def e2e_step(i):
            j = i % 2
            s_in.wait_event(ev_c[j])
            with torch.cuda.stream(s_in):
                for h, d in zip(xh, X2[j]):
                    d.copy_(h, non_blocking=True)
            ev_in[j].record(s_in)
            stream.wait_event(ev_in[j])
            stream.wait_event(ev_out[j])
            batches[j].launch(stream)
            ev_c[j].record(stream)
            s_out.wait_event(ev_c[j])
            with torch.cuda.stream(s_out):
                for h, d in zip(bh[j], B2[j]):
                    h.copy_(d, non_blocking=True)
            ev_out[j].record(s_out)

        for i in range(args.warmup):
            e2e_step(i)
        torch.cuda.synchronize(dev)
        timed.barrier()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        s_in.wait_stream(stream)
        for i in range(args.steps):
            e2e_step(i)
        stream.wait_stream(s_out)
        e1.record(stream)
        torch.cuda.synchronize(dev)
        timed.barrier()
        t_e2e = e0.elapsed_time(e1) * 1e-3
        last = (args.steps - 1) % 2
        ok = all(bool(np.allclose(h.numpy(), d.cpu().numpy(), rtol=1e-12, atol=1e-300))
                 for h, d in zip(bh[last], B2[last]))
        batches[1].free()
        nbytes = sum(x.numel() * 8 for x in xh)
        out["e2e"] = {"seconds": t_e2e, "steps": args.steps, "h2d_bytes_per_step": nbytes,
                      "d2h_bytes_per_step": nbytes, "ms_per_step": t_e2e / args.steps * 1e3,
                      "matches_device_result": ok,
                      "how": "per step: pinned H2D of every X, one graph replay, D2H of every B; two buffer sets "
                             "and graphs alternate, copies on their own streams"}
    batch.free()
    for s in scheds:
        s.free()
    del Xs, Bs
    torch.cuda.empty_cache()
    return out


def run_batch(args):
    """The batch workload on its own line (the metric of that config)."""
    import torch

    import paper_1907_06487_gb300 as R
    from paper_1907_06487_gb300 import build as B, configs, perfmodel as pm

    rank, world, local = dist_env()
    if world > 1:
        torch.distributed.init_process_group("nccl")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    if rank == 0:
        B.build()
    if world > 1:
        torch.distributed.barrier()
    stream = torch.cuda.Stream(device=dev)
    timed = Timer(stream, dev, world)
    peak, peak_kind = load_peaks()
    clocks = ClockSampler(local)
    clocks.start()
    blk = batch_block(args, R, configs, pm, dev, stream, timed, peak, peak_kind, e2e=True)
    clk = clocks.stop()
    t, t_e2e = max_over_ranks([blk["ms_per_step"] * 1e-3 * args.steps, blk["e2e"]["seconds"]], world, dev)
    if rank == 0:
        flops = blk["flops_per_step"]
        e2e = dict(blk.pop("e2e"))
        e2e_line = {"value": whole_job_rate(world, flops, args.steps, t_e2e) / 1e9, "unit": "GFLOP/s",
                    **{k: e2e[k] for k in ("h2d_bytes_per_step", "d2h_bytes_per_step", "ms_per_step",
                                           "matches_device_result", "how")}}
        print(json.dumps({
            "metric": "SymmSpMM GFLOP/s (2*nnz_full*k flops) of a 64-matrix batch in one CUDA graph",
            "value": whole_job_rate(world, flops, args.steps, t) / 1e9, "unit": "GFLOP/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": t / args.steps * 1e3,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": {"workload": "batch64", **{k: blk[k] for k in
                                                                      ("k", "matrices", "rows", "schedule",
                                                                       "tuned_launches", "l2")}},
            "roofline": blk["roofline"], "e2e": e2e_line, "gpu_launches": None, "clocks": clk,
            "cpu_baseline": None, "setup_seconds": blk["setup_seconds"],
            "note": "gpu_launches: one CUDA graph replay per step holding the 64 matrices' kernels"}))
    if world > 1:
        torch.distributed.destroy_process_group()
    return 0


def build_parser():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=50)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="xxz26", choices=sorted(WORKLOAD_DESC))
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-extra", action="store_true",
                    help="measure the headline workload only (no stencil, Anderson and batch blocks)")
    ap.add_argument("--spmm-k", type=int, default=0,
                    help="also time SymmSpMM with this many right-hand sides on the headline schedule")
    ap.add_argument("--cpu-seconds", type=float, default=10.0)
    ap.add_argument("--ref-seconds", type=float, default=60.0)
    return ap


def main():
    args = build_parser().parse_args()
    if args.impl == "reference":
        return run_reference(args)
    if args.workload == "batch64":
        return run_batch(args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
