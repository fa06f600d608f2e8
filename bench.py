#!/usr/bin/env python
"""SymmSpMV benchmark on GB300 (one JSON line on stdout).

Workload (default): the periodic Heisenberg XXZ chain L=26, Sz=0 sector
(10,400,600 rows, 80,708,656 stored upper nonzeros, 151,016,712 full
nonzeros), FP64 values, x ~ U[-1,1) (seed 3) -- a synthetic stand-in for the
paper's Spin-26 matrix.  One step = one b = A x through the library's
SymmSpMV path (schedule built before timing, as the paper excludes
preprocessing).  The full-CRS SpMV of the same permuted matrix is timed
beside it as the traffic baseline.

Timing: W warm-up steps, then K steps bracketed by a barrier and
torch.cuda.synchronize(), CUDA events on the stream the kernels run on;
vectors rotate through ring buffers of 4 x and 4 b (each 83 MB) and the
matrix is 1.05 GB, so every step's inputs exceed the 129 MB L2.  Several
GPUs (torchrun) run independent replicas (no data exchange); value is the
sum over ranks of the flops divided by the slowest rank's time.

--impl reference times the CPU oracle (serial FP64 Alg. "SymmSpMV") on a
bounded number of sweeps of the same matrix on the host cores.
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


# SymmSpMM right-hand-side counts timed per workload (the 27-point stencil: k = 4, 8, 16)
SPMM_KS = {"st27_200": (4, 8, 16), "st27_100": (16,)}


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


def oracle_normwise_error(m, x, b_perm, perm):
    """||b - b_ref||_2 / || |A||x| ||_2 of a result b (given in the schedule's
    permuted order) against the FP64 oracle's plain definition (part of the
    CPU-baseline leg: the only place bench.py runs the oracle)."""
    import numpy as np

    import oracle
    bref, s = oracle.spmv_full(oracle.expand_full(m), x)
    b = np.empty_like(bref)
    b[perm] = b_perm
    return float(np.linalg.norm(b - bref) / np.linalg.norm(s))


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

    name = args.workload
    m = configs.matrix(name)
    cfg = configs.SCHEDULE[name]
    n, nu = m["n"], len(m["col"])
    nf = 2 * nu - n
    t0 = time.perf_counter()
    stream = torch.cuda.Stream(device=dev)
    s = R.race_build(m, cfg["n_workers"], eps=cfg["eps"], max_depth=cfg["max_depth"], stream=stream,
                     rcm=cfg.get("rcm", False))
    build_s = time.perf_counter() - t0
    lc = cfg["launch"]
    R.race_set_launch(s, 0, **lc)
    fl = cfg["full_launch"]
    R.race_prepare_full(s, stream)
    R.race_set_launch(s, 1, **fl)
    info = s.info()
    perm = s.perm()
    x_host = configs.vectors(name, n)

    ring = 4
    with torch.cuda.stream(stream):
        xs = []
        for i in range(ring):
            xo = torch.from_numpy(x_host).to(dev) if i == 0 else torch.rand(n, dtype=torch.float64, device=dev)
            xp = torch.empty_like(xo)
            R.race_permute(s, xo, xp, 1, stream)
            xs.append(xp)
        bs = [torch.empty(n, dtype=torch.float64, device=dev) for _ in range(ring)]
    stream.synchronize()

    def barrier():
        if world > 1:
            torch.distributed.barrier()

    def timed(fn, steps, warmup):
        for i in range(warmup):
            fn(i)
        stream.synchronize()
        barrier()
        torch.cuda.synchronize(dev)
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for i in range(steps):
            fn(i)
        e1.record(stream)
        torch.cuda.synchronize(dev)
        barrier()
        return e0.elapsed_time(e1) * 1e-3

    # ---- main timed region: SymmSpMV -------------------------------------------------------
    clocks = ClockSampler(local)
    clocks.start()
    time.sleep(0.3)
    t_symm = timed(lambda i: R.symm_spmv(s, xs[i % ring], bs[i % ring], stream), args.steps, args.warmup)
    clk = clocks.stop()
    R.race_poll_status(s, stream)
    # ---- the limit the reduction-based executors share: the scatter's reductions at L2 ------
    def probe(mode):
        def step(i):
            if mode == 0:
                bs[i % ring].zero_()
            R.race_probe_scatter(s, mode, bs[i % ring], stream)
        with torch.cuda.stream(stream):
            return timed(step, args.steps, args.warmup)
    t_red, t_col = probe(0), probe(1)
    # ---- traffic baseline: full-CRS SpMV on the same permuted matrix -----------------------
    t_full = timed(lambda i: R.spmv_full(s, xs[i % ring], bs[i % ring], stream), args.steps, args.warmup)
    # ---- the conflict-free RACE executors (a few steps: they are slow) on the schedule that
    # suits them (full recursion), one row per thread in the leaf executor
    cf = cfg["conflict_free"]
    s_cf = R.race_build(m, cf["n_workers"], eps=cfg["eps"], max_depth=cf["max_depth"], stream=stream,
                        one_level_stage0=cf.get("one_level_stage0", False))
    info_cf = s_cf.info()
    R.race_set_launch(s_cf, 0, R.RACE_EXEC_LEAF_CTA, 1, 1, 0, 8)
    t_leaf_cta = timed(lambda i: R.symm_spmv(s_cf, xs[i % ring], bs[i % ring], stream), 3, 1)
    t_win_race = timed(lambda i: R.symm_spmv_exec(s_cf, R.RACE_EXEC_WINDOW_RACE, xs[i % ring], bs[i % ring],
                                                  stream), 3, 1)
    s_cf.free()
    # ---- the same two kernels on the input order (no RACE permutation) --------------------
    s_nat = R.race_build(m, cfg["n_workers"], natural_order=True, windows=False, stream=stream)
    R.race_set_launch(s_nat, 0, **lc)
    R.race_prepare_full(s_nat, stream)
    R.race_set_launch(s_nat, 1, **fl)
    t_nat_symm = timed(lambda i: R.symm_spmv(s_nat, xs[i % ring], bs[i % ring], stream), args.steps, args.warmup)
    t_nat_full = timed(lambda i: R.spmv_full(s_nat, xs[i % ring], bs[i % ring], stream), args.steps, args.warmup)
    s_nat.free()
    # ---- FP32-stored values (x, b and the row sums stay FP64), same launch -----------------
    s32 = R.race_build(m, cfg["n_workers"], eps=cfg["eps"], max_depth=cfg["max_depth"], stream=stream,
                       val_type=R.RACE_F32, windows=False, rcm=cfg.get("rcm", False))
    R.race_set_launch(s32, 0, **lc)
    t_f32 = timed(lambda i: R.symm_spmv(s32, xs[i % ring], bs[i % ring], stream), args.steps, args.warmup)
    # the FP32-valued result for x_host, kept for the normwise error against the FP64 oracle
    with torch.cuda.stream(stream):
        R.symm_spmv(s32, xs[0], bs[0], stream)
    stream.synchronize()
    b32_perm = bs[0].cpu().numpy()
    s32.free()
    # ---- SymmSpMM with several right-hand sides (workloads that name them) ------------------
    spmm = {}
    for k in SPMM_KS.get(name, ()):
        with torch.cuda.stream(stream):
            Xk = [torch.rand(n * k, dtype=torch.float64, device=dev) for _ in range(2)]
            Bk = [torch.empty(n * k, dtype=torch.float64, device=dev) for _ in range(2)]
        # the project's autotuner picks this k's launch shape, then the timed steps run it
        tuned, _ = R.race_autotune(s, k, Xk[0], Bk[0], reps=3, stream=stream)
        tk = timed(lambda i: R.symm_spmm(s, k, Xk[i % 2], Bk[i % 2], stream), max(3, args.steps // 4), 2)
        per_k = tk / max(3, args.steps // 4)
        spmm[str(k)] = {"ms_per_step": per_k * 1e3, "gflops": pm.flops(nf, k) / per_k / 1e9,
                        "gbs": pm.symm_bytes(n, nu, k) / per_k / 1e9, "launch": tuned}
        del Xk, Bk
    if spmm:
        R.race_set_launch(s, 0, **lc)  # the SymmSpMV launch again
    # ---- end to end through host buffers: H2D x, permute, SymmSpMV, unpermute, D2H b --------
    # Each step copies its x in and its b out; copies run on their own streams
    # (double-buffered), so step i's read-back overlaps step i+1's upload and
    # compute, as a caller streaming vectors through the library would run it.
    s_in, s_out = torch.cuda.Stream(device=dev), torch.cuda.Stream(device=dev)
    xh = [torch.from_numpy(x_host).pin_memory() for _ in range(2)]
    bh = [torch.empty(n, dtype=torch.float64).pin_memory() for _ in range(2)]
    xd = [torch.empty(n, dtype=torch.float64, device=dev) for _ in range(2)]
    bd = [torch.empty(n, dtype=torch.float64, device=dev) for _ in range(2)]
    xpd, bpd = (torch.empty(n, dtype=torch.float64, device=dev) for _ in range(2))
    ev_in, ev_c, ev_out = ([torch.cuda.Event() for _ in range(2)] for _ in range(3))

    def e2e_step(i):
        j = i % 2
        s_in.wait_event(ev_c[j])        # xd[j] consumed by the step two back
        with torch.cuda.stream(s_in):
            xd[j].copy_(xh[j], non_blocking=True)
        ev_in[j].record(s_in)
        stream.wait_event(ev_in[j])
        stream.wait_event(ev_out[j])    # bd[j] read back by the step two back
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
        barrier()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        s_in.wait_stream(stream)
        for i in range(steps):
            e2e_step(i)
        stream.wait_stream(s_out)
        e1.record(stream)
        torch.cuda.synchronize(dev)
        barrier()
        return e0.elapsed_time(e1) * 1e-3

    t_e2e = timed_e2e(args.steps, args.warmup)
    # the read-back must equal the device-timed result for the same x (xs[0] is x_host permuted)
    with torch.cuda.stream(stream):
        R.symm_spmv(s, xs[0], bs[0], stream)
        R.race_unpermute(s, bs[0], bd[0], 1, stream)
    stream.synchronize()
    ref = bd[0].cpu().numpy()
    got = bh[(args.steps - 1) % 2].numpy()
    e2e_ok = bool(np.allclose(got, ref, rtol=1e-12, atol=1e-12 * float(np.abs(ref).max())))
    t_symm, t_full, t_e2e, t_red, t_col = max_over_ranks([t_symm, t_full, t_e2e, t_red, t_col], world, dev)

    flops = pm.flops(nf)
    per_step = t_symm / args.steps
    value = whole_job_rate(world, flops, args.steps, t_symm) / 1e9
    full_gflops = whole_job_rate(world, flops, args.steps, t_full) / 1e9
    e2e_value = whole_job_rate(world, flops, args.steps, t_e2e) / 1e9
    sym_bytes = pm.symm_bytes(n, nu)
    achieved = sym_bytes / per_step / 1e9
    peak, peak_kind = load_peaks()
    launches_per_step = 1 if lc["executor"] >= R.RACE_EXEC_ATOMIC else info["n_phases"]
    if rank != 0:
        return 0

    # CPU baseline: the oracle on a bounded sample (a few serial sweeps)
    cpu = None
    fp32_err = None
    if not args.no_cpu_baseline:
        cpu = oracle_cpu(m, name, args.cpu_seconds)
        fp32_err = oracle_normwise_error(m, x_host, b32_perm, perm)
    traffic = ncu_traffic(name, "symm")
    line = {
        "metric": METRIC_SYMM,
        "value": value, "unit": "GFLOP/s", "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": per_step * 1e3, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f64", "data": "synthetic",
        "config": {"workload": name, "desc": WORKLOAD_DESC.get(name, name), "n": n, "nnz_upper": nu, "nnz_full": nf,
                   "l2": "inputs larger than L2 (matrix 1.05 GB; x, b rotate over 4+4 buffers of 83 MB)",
                   "schedule": {"n_workers": cfg["n_workers"], "eps": list(cfg["eps"]), "n_phases": info["n_phases"],
                                "eta": info["eta"], "depth": info["depth"], "rcm": bool(cfg.get("rcm", False))},
                   "launch": lc, "parallelism": f"replicas x{world}"},
        "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
                     "traffic": traffic, "peak_kind": peak_kind,
                     "algorithmic_bytes_per_step": sym_bytes},
        "symm_gbs": achieved,
        "reduction_floor": {"ms_per_step": t_red / args.steps * 1e3, "columns_only_ms_per_step": t_col / args.steps * 1e3,
                            "frac": (t_red / args.steps) / per_step,
                            "what": "race_probe_scatter on the same schedule: the transposed update's L2 reductions "
                                    "alone (mode 0, b zeroed first) and its column stream alone (mode 1), with the "
                                    "executors' access pattern; frac = that floor / SymmSpMV time"},
        "spmv_full": {"value": full_gflops, "unit": "GFLOP/s", "ms_per_step": t_full / args.steps * 1e3,
                      "gbs": pm.full_bytes(n, nf) / (t_full / args.steps) / 1e9},
        "fp32_values": {"ms_per_step": t_f32 / args.steps * 1e3, "gflops": flops / (t_f32 / args.steps) / 1e9,
                        "gbs": pm.symm_bytes(n, nu, 1, 4) / (t_f32 / args.steps) / 1e9,
                        "normwise_error_vs_fp64_oracle": fp32_err,
                        "what": "values stored in FP32 (8 B per stored entry), x, b and row sums FP64; error = "
                                "||b32 - b_ref||_2 / || |A||x| ||_2 against the FP64 oracle (computed in the CPU "
                                "baseline leg; null without it)"},
        "spmm": spmm,
        "natural_order": {"symm_ms_per_step": t_nat_symm / args.steps * 1e3,
                          "symm_gflops": flops / (t_nat_symm / args.steps) / 1e9,
                          "full_ms_per_step": t_nat_full / args.steps * 1e3,
                          "speedup_vs_full": t_nat_full / t_nat_symm,
                          "what": "the same launches on the input order (RACE_FLAG_NATURAL_ORDER: no permutation)"},
        "race_conflict_free": {"leaf_cta_ms_per_step": t_leaf_cta / 3 * 1e3,
                               "window_race_ms_per_step": t_win_race / 3 * 1e3,
                               "schedule": {"n_workers": cf["n_workers"], "max_depth": cf["max_depth"],
                                            "one_level_stage0": bool(cf.get("one_level_stage0", False)),
                                            "n_phases": info_cf["n_phases"], "n_leaves": info_cf["n_leaves"],
                                            "eta": info_cf["eta"]},
                               "what": "RACE_EXEC_LEAF_CTA and RACE_EXEC_WINDOW_RACE (phase by phase, no two concurrent "
                                       "leaves share an entry of b; x and b in that schedule's order) on a fully "
                                       "recursed schedule, 3 steps each"},
        "speedup_vs_full": t_full / t_symm,
        "e2e": {"value": e2e_value, "unit": "GFLOP/s", "h2d_bytes_per_step": 8 * n, "d2h_bytes_per_step": 8 * n,
                "ms_per_step": t_e2e / args.steps * 1e3, "matches_device_result": e2e_ok,
                "how": "per step: pinned H2D of x, permute, SymmSpMV, unpermute, D2H of b into pinned memory; "
                       "copies on their own streams, double-buffered across steps"},
        "gpu_launches": launches_per_step * args.steps,
        "clocks": clk,
        "cpu_baseline": cpu,
        "build_seconds": build_s,
    }
    print(json.dumps(line))
    s.free()
    if world > 1:
        torch.distributed.destroy_process_group()
    return 0


def run_batch(args):
    """64 matrices (Anderson L in [16,96] and geometric graphs n in [1e4,1e6]),
    SymmSpMM with k = 4, each schedule autotuned, all replayed by one CUDA graph."""
    import numpy as np
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
    k = 4
    mats = configs.batch64()
    stream = torch.cuda.Stream(device=dev)
    t0 = time.perf_counter()
    scheds, Xs, Bs, Xh = [], [], [], []
    flops = 0
    sym_bytes = 0
    tuned = {}
    for i, m in enumerate(mats):
        s = R.race_build(m, configs.BATCH_SCHEDULE["n_workers"], max_depth=configs.BATCH_SCHEDULE["max_depth"],
                         stream=stream, rcm=configs.BATCH_SCHEDULE.get("rcm", False))
        n, nu = m["n"], len(m["col"])
        X = configs.matgen.uniform(n * k, 300 + i).reshape(n, k)
        xp = torch.from_numpy(np.ascontiguousarray(X[s.perm()])).to(dev)
        bp = torch.empty_like(xp)
        launch, _ = R.race_autotune(s, k, xp, bp, reps=3, stream=stream)
        key = f"{launch['executor']}/{launch['rows_per_group']}/{launch['blocks_per_sm']}"
        tuned[key] = tuned.get(key, 0) + 1
        scheds.append(s); Xs.append(xp); Bs.append(bp); Xh.append(X)
        flops += pm.flops(2 * nu - n, k)
        sym_bytes += pm.symm_bytes(n, nu, k)
    batch = R.race_batch_create(scheds, k, Xs, Bs, stream)
    setup_s = time.perf_counter() - t0
    stream.synchronize()

    def timed(fn, steps, warmup):
        for i in range(warmup):
            fn(i)
        stream.synchronize()
        if world > 1:
            torch.distributed.barrier()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for i in range(steps):
            fn(i)
        e1.record(stream)
        torch.cuda.synchronize(dev)
        if world > 1:
            torch.distributed.barrier()
        return e0.elapsed_time(e1) * 1e-3

    clocks = ClockSampler(local)
    clocks.start()
    time.sleep(0.3)
    t = timed(lambda i: batch.launch(stream), args.steps, args.warmup)
    clk = clocks.stop()
    # end to end: H2D of every X from pinned host memory, graph, D2H of every B.  Two buffer
    # sets with a graph each, alternating, copies on their own streams: step i's read-back
    # overlaps step i+1's upload and replay.
    xh = [torch.from_numpy(np.ascontiguousarray(X[s.perm()])).pin_memory() for X, s in zip(Xh, scheds)]
    bh = [[torch.empty_like(h).pin_memory() for h in xh] for _ in range(2)]
    X2 = [Xs, [torch.empty_like(x) for x in Xs]]
    B2 = [Bs, [torch.empty_like(b) for b in Bs]]
    batches = [batch, R.race_batch_create(scheds, k, X2[1], B2[1], stream)]
    s_in, s_out = torch.cuda.Stream(device=dev), torch.cuda.Stream(device=dev)
    ev_in, ev_c, ev_out = ([torch.cuda.Event() for _ in range(2)] for _ in range(3))

    def e2e(i):
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

    def timed_e2e(steps, warmup):
        for i in range(warmup):
            e2e(i)
        torch.cuda.synchronize(dev)
        if world > 1:
            torch.distributed.barrier()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        s_in.wait_stream(stream)
        for i in range(steps):
            e2e(i)
        stream.wait_stream(s_out)
        e1.record(stream)
        torch.cuda.synchronize(dev)
        if world > 1:
            torch.distributed.barrier()
        return e0.elapsed_time(e1) * 1e-3

    t_e2e = timed_e2e(args.steps, args.warmup)
    # the read-back of the last step equals the graph's result on the same X
    last = (args.steps - 1) % 2
    e2e_ok = all(bool(np.allclose(h.numpy(), d.cpu().numpy(), rtol=1e-12, atol=1e-300))
                 for h, d in zip(bh[last], B2[last]))
    batches[1].free()
    t, t_e2e = max_over_ranks([t, t_e2e], world, dev)
    per = t / args.steps
    achieved = sym_bytes / per / 1e9
    peak, peak_kind = load_peaks()
    if rank == 0:
        nbytes = sum(x.numel() * 8 for x in xh)
        print(json.dumps({
            "metric": "SymmSpMM GFLOP/s (2*nnz_full*k flops) of a 64-matrix batch in one CUDA graph",
            "value": whole_job_rate(world, flops, args.steps, t) / 1e9, "unit": "GFLOP/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": per * 1e3, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": "batch64", "k": k, "matrices": len(mats),
                       "rows": int(sum(m["n"] for m in mats)), "schedule": dict(configs.BATCH_SCHEDULE),
                       "tuned_launches": tuned,
                       "l2": "inputs larger than L2 (all matrices and blocks: several GB per replay)"},
            "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
                         "traffic": None, "peak_kind": peak_kind, "algorithmic_bytes_per_step": sym_bytes},
            "e2e": {"value": whole_job_rate(world, flops, args.steps, t_e2e) / 1e9, "unit": "GFLOP/s",
                    "h2d_bytes_per_step": nbytes, "d2h_bytes_per_step": nbytes,
                    "ms_per_step": t_e2e / args.steps * 1e3, "matches_device_result": e2e_ok,
                    "how": "per step: pinned H2D of every X, one graph replay, D2H of every B; two buffer sets "
                           "and graphs alternate, copies on their own streams"},
            "gpu_launches": len(mats) * args.steps, "clocks": clk, "cpu_baseline": None,
            "setup_seconds": setup_s}))
    batch.free()
    return 0


def build_parser():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=50)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="xxz26", choices=sorted(WORKLOAD_DESC))
    ap.add_argument("--no-cpu-baseline", action="store_true")
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
