#!/usr/bin/env python3
"""Benchmark: Newton-Raphson iterations per second of the multinomial-logit fit.

Default workload (the largest single-GPU configuration): N=500000 observations,
K=100 alternatives, p=100 individual-specific columns (70 N(0,1), 30
Bernoulli(0.1) indicators, no intercept), f=10 alternative-specific columns
with a generic coefficient, d=0; 9910 coefficients; seeded synthetic data
(paper_1404_3177_gb300.datagen).  One step = one full Newton iteration from
theta = 0 (utility/softmax/log-likelihood/gradient pass, structured Hessian,
Newton solve, step-halving line search, coefficient update), so every step
does the same work.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--precision bf16|tf32|fp64]
                    [--workload c3|c2] [--extras all|none] [--rows N]
    python bench.py --impl reference ...     # the FP64 CPU oracle on the host cores

Timing: CUDA events on the stream the library uses, W untimed warm-up steps,
then K steps bracketed by a barrier and torch.cuda.synchronize(); the inputs
(2.2 GB) are larger than L2, so no flush is needed between steps.  The same
JSON line carries, measured after the timed region (rank 0, one GPU):
the plain float64 mode on the same workload (one step), the batched workload
(2048 uneven fits, BF16 and FP64) and the serving workload (Poisson arrivals;
p50/p99 latency to convergence, fits/s).  With N > 1 GPUs (torchrun) the
observations are sharded: every rank holds a config-3-sized shard of its own
rows of one large fit, the partial l, g and -H are added by one NCCL
all-reduce per iteration and the line-search log-likelihoods by one all-reduce
of two doubles per trial (paper_1404_3177_gb300.sharded); `value` counts each
rank's shard as one unit (weak scaling) at the slowest rank's time.
"""
from __future__ import annotations

import argparse
import hashlib
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

METRIC = "newton_iters_per_s"
UNIT = "iter/s"
CONFIG_NOTE = "inputs larger than L2 (no flush)"

# DRAM traffic of one launch (dram__bytes_read.sum + dram__bytes_write.sum) from ncu captures, keyed by
# workload and kernel, with the SHA-256 (first 16 hex digits) of the kernel's source files when it was
# taken: a figure whose sources have changed since is reported as null.  Where the capture was taken on a
# smaller N of the same shape, the figure is scaled to the full N (the traffic grows in proportion).
MEASURED_TRAFFIC: dict = {
    # ncu --metrics dram__bytes_read.sum,dram__bytes_write.sum (one pass) on
    # `python bench.py --extras none --steps 1 --warmup 1 --no-cpu-baseline`: 68.13 GB read + 7.08 GB written
    ("c3_N500000_K100_p100_d0_f10", "syrk_AtA"): {"bytes": 75.21e9, "sources": "dfc565d9cd2d8e19"},
}
KERNEL_SOURCES = {
    "syrk_AtA": ["paper_1404_3177_gb300/csrc/syrk_tc.cu", "paper_1404_3177_gb300/csrc/hessian.cu"],
    "pass": ["paper_1404_3177_gb300/csrc/pass_tile.cu"],
    "cholesky": ["paper_1404_3177_gb300/csrc/solve_coop.cu", "paper_1404_3177_gb300/csrc/syrk_tc.cu"],
}


def source_hash(files) -> str:
    h = hashlib.sha256()
    for f in files:
        with open(os.path.join(ROOT, f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def measured_traffic(workload: str, kernel: str):
    rec = MEASURED_TRAFFIC.get((workload, kernel))
    if not rec or rec["sources"] != source_hash(KERNEL_SOURCES[kernel]):
        return None
    return rec["bytes"]


def peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        with open(path) as fh:
            return json.load(fh), "measured"
    return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0}, "fallback"


def measure_alu_peaks(dev) -> dict:
    """float32 (TF32 off) and float64 GEMM rates of this GPU, measured here with cuBLAS (torch.matmul), outside
    the timed region: the denominators of the CUDA-core kernels' rooflines."""
    import torch

    out = {}
    prev = torch.backends.cuda.matmul.allow_tf32
    torch.backends.cuda.matmul.allow_tf32 = False
    try:
        for name, dt, n, reps in (("fp32", torch.float32, 8192, 6), ("fp64", torch.float64, 4096, 3)):
            a = torch.randn(n, n, dtype=dt, device=dev)
            b = torch.randn(n, n, dtype=dt, device=dev)
            torch.matmul(a, b)
            torch.cuda.synchronize()
            best = float("inf")
            for _ in range(reps):
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record()
                torch.matmul(a, b)
                e1.record()
                torch.cuda.synchronize()
                best = min(best, e0.elapsed_time(e1) / 1e3)
            out[name + "_tflops"] = 2.0 * n ** 3 / best / 1e12
            del a, b
    finally:
        torch.backends.cuda.matmul.allow_tf32 = prev
    out["how"] = "torch.matmul float32 8192^3 with TF32 off and float64 4096^3 (cuBLAS), best of 6 / 3, CUDA events"
    return out


# ---------------------------------------------------------------------------
# clocks sampled during the timed region
# ---------------------------------------------------------------------------

class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "100"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except (OSError, FileNotFoundError):
            self.proc = None

    def _read(self):
        for ln in self.proc.stdout:
            self.lines.append(ln.strip())

    def stop(self):
        if not self.proc:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        sm, smax, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [x.strip() for x in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax = float(parts[2])
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": smax, "reasons": sorted(reasons),
                "samples": len(sm)}


# ---------------------------------------------------------------------------
# CPU baseline: the FP64 oracle on a bounded sample of the workload
# ---------------------------------------------------------------------------

def _sub(prob, rows):
    from paper_1404_3177_gb300 import datagen
    return datagen.Problem(rows, prob.K, prob.p, prob.d, prob.f, 0, prob.X[:rows], prob.Y[:rows], prob.Z[:rows],
                           prob.choice[:rows], prob.theta_true)


def oracle_iteration_seconds(prob, rows_lg: int, rows_h: int, n_chol: int):
    """Seconds of one oracle Newton iteration on the full workload, EXTRAPOLATED from bounded samples:
    l and g plus one line-search l on `rows_lg` observations and -H on `rows_h` observations (both scaled
    linearly to N), and the Cholesky solve timed at min(n_theta, n_chol) and scaled by (n_theta / n)^3."""
    import oracle

    n = prob.n_theta
    th = np.zeros(n)
    rows_lg = min(rows_lg, prob.N)
    rows_h = min(rows_h, prob.N)
    sub = _sub(prob, rows_lg)
    t0 = time.perf_counter()
    oracle.loglik_grad(sub, th)
    oracle.loglik(sub, th)
    t_lg = (time.perf_counter() - t0) / rows_lg * prob.N
    sub_h = _sub(prob, rows_h)
    t0 = time.perf_counter()
    F = oracle.neg_hessian(sub_h, th)
    t_h = (time.perf_counter() - t0) / rows_h * prob.N
    m = min(n, n_chol)
    Fm = F[:m, :m] * (prob.N / rows_h) + np.eye(m)  # a positive definite block of the sample's -H
    g = np.ones(m)
    t0 = time.perf_counter()
    L = oracle.cholesky(Fm)
    oracle.cholesky_solve(L, g)
    t_c = (time.perf_counter() - t0) * (n / m) ** 3
    del F, Fm
    desc = (f"extrapolated: l, g and one line-search l on {rows_lg} of {prob.N} observations and -H on {rows_h} "
            f"(each scaled to N), plus the Cholesky solve timed at n={m} and scaled by (n_theta/n)^3 to "
            f"n_theta={n}")
    return t_lg + t_h + t_c, desc


def host_cores() -> dict:
    cores = len(os.sched_getaffinity(0)) if hasattr(os, "sched_getaffinity") else (os.cpu_count() or 1)
    return {"cores": cores, "cpu_count_of_host": os.cpu_count()}


def cpu_baseline(prob, args):
    t_iter, desc = oracle_iteration_seconds(prob, args.ref_rows, args.ref_hess_rows, args.ref_chol_n)
    hc = host_cores()
    return {"value": 1.0 / t_iter, "unit": UNIT, "cores": hc["cores"], "kind": "oracle", "sample": desc,
            "extrapolated": True, "host_cpus_visible": hc["cpu_count_of_host"]}


# ---------------------------------------------------------------------------
# distributed helpers
# ---------------------------------------------------------------------------

def dist_init():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl" if _cuda() else "gloo")
    return world, rank, local


def _cuda():
    import torch
    return torch.cuda.is_available()


def barrier(world):
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


def allmax(world, v):
    if world == 1:
        return v
    import torch
    import torch.distributed as dist
    t = torch.tensor([v], dtype=torch.float64, device="cuda" if _cuda() else "cpu")
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def workload_problem(name, rows=None):
    """The workload's problem; rows (optional) replaces its number of observations (same shape and seed)."""
    from paper_1404_3177_gb300 import datagen
    if name == "c3":
        prob = datagen.config3(rows) if rows else datagen.config3()
    else:
        prob = datagen.config2(rows) if rows else datagen.config2()
    return prob, prob.name


# ---------------------------------------------------------------------------
# reference arm: the FP64 CPU oracle as it stands
# ---------------------------------------------------------------------------

def run_reference(args, world, rank):
    """The FP64 CPU oracle as it stands, one bounded (extrapolated) sample per step, rank 0 only."""
    if rank != 0:
        return
    prob, wname = workload_problem(args.workload, args.rows)
    for _ in range(args.warmup):
        oracle_iteration_seconds(prob, args.ref_rows, args.ref_hess_rows, args.ref_chol_n)
    times, desc = [], ""
    for _ in range(args.steps):
        t_iter, desc = oracle_iteration_seconds(prob, args.ref_rows, args.ref_hess_rows, args.ref_chol_n)
        times.append(t_iter)
    t = statistics.mean(times)
    v = 1.0 / t
    hc = host_cores()
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1000 * t, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": wname, "note": CONFIG_NOTE},
            "cpu_baseline": {"value": v, "unit": UNIT, "cores": hc["cores"], "kind": "oracle",
                             "sample": "each step " + desc, "extrapolated": True},
            "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# ---------------------------------------------------------------------------
# our arm: one large fit
# ---------------------------------------------------------------------------

def _host(prob):
    import torch
    t = lambda a: torch.from_numpy(np.ascontiguousarray(a)).pin_memory() if a.size else None  # noqa: E731
    return t(prob.X), t(prob.Y), t(prob.Z), torch.from_numpy(prob.choice).pin_memory()


def _median(infos, k):
    return statistics.median(i[k] for i in infos)


def kernel_times(infos):
    return {"pass": _median(infos, "t_pass_ms"), "build_operands": _median(infos, "t_build_ms"),
            "syrk_AtA": _median(infos, "t_syrk_ms"), "syrk_diag_blocks": _median(infos, "t_band_ms"),
            "z_blocks": _median(infos, "t_zblk_ms"), "assemble": _median(infos, "t_asm_ms"),
            "cholesky": _median(infos, "t_factor_ms"), "solve": _median(infos, "t_solve_ms"),
            "line_search": _median(infos, "t_ls_ms")}


def rooflines_of(prob, precision, kern, infos, pk, alu, wname):
    """Algorithmic work per launch of the main kernels over their CUDA-event times, against the measured peaks."""
    N, K, p, d, f = prob.N, prob.K, prob.p, prob.d, prob.f
    n = prob.n_theta
    mc = (K - 1) * (p + d)
    syrk_flops = float(N) * mc * (mc + 1)
    in_bytes = 4.0 * N * (p + K * (d + f) + 1)
    pass_bytes = in_bytes + 4.0 * N * K + 4.0 * N * f
    tf32_peak = pk["bf16_tflops"] * (1.1 / 2.25)  # nominal TF32 / BF16 dense ratio
    if precision == "fp64":
        syrk = {"bound": "alu", "peak": alu["fp64_tflops"], "peak_of": "measured float64 GEMM (cuBLAS)"}
    elif precision == "tf32":
        syrk = {"bound": "tensor", "peak": tf32_peak, "peak_of": "measured BF16 burst x nominal TF32/BF16 ratio"}
    else:
        syrk = {"bound": "tensor", "peak": pk["bf16_tflops"], "peak_of": "measured BF16 burst"}
    syrk.update(achieved=syrk_flops / (kern["syrk_AtA"] * 1e-3) / 1e12, unit="TFLOP/s",
                traffic=measured_traffic(wname, "syrk_AtA"), work_per_launch=syrk_flops)
    if precision != "fp64" and pk.get("bf16_tflops_sustained"):
        syrk["frac_of_sustained"] = syrk["achieved"] / pk["bf16_tflops_sustained"]
    out = {"syrk_AtA": syrk,
           "pass": {"bound": "hbm", "achieved": pass_bytes / (kern["pass"] * 1e-3) / 1e9, "peak": pk["hbm_gbs"],
                    "peak_of": "measured copy bandwidth", "unit": "GB/s", "traffic": measured_traffic(wname, "pass"),
                    "work_per_launch": pass_bytes},
           "line_search": {"bound": "hbm", "achieved": in_bytes / (kern["line_search"] * 1e-3) / 1e9,
                           "peak": pk["hbm_gbs"], "peak_of": "measured copy bandwidth", "unit": "GB/s",
                           "traffic": None, "work_per_launch": in_bytes}}
    fk = infos[-1].get("factor_kind", 1)
    mixed = infos[-1]["solve_mode"] == 2
    chol_flops = (2.0 if mixed else 1.0) * n ** 3 / 3.0  # L (and L^-1 in the mixed solve)
    if mixed and fk == 2:
        chol = {"bound": "tensor", "peak": tf32_peak, "peak_of": "measured BF16 burst x nominal TF32/BF16 ratio",
                "arith": "float32 factor and inverse, trailing updates 3xTF32 tcgen05, float64 refinement"}
    elif mixed:
        chol = {"bound": "alu", "peak": alu["fp32_tflops"], "peak_of": "measured float32 GEMM (cuBLAS, TF32 off)",
                "arith": "float32 factor and inverse on CUDA cores, float64 refinement"}
    else:
        chol = {"bound": "alu", "peak": alu["fp64_tflops"], "peak_of": "measured float64 GEMM (cuBLAS)",
                "arith": "float64"}
    chol.update(achieved=chol_flops / (kern["cholesky"] * 1e-3) / 1e12, unit="TFLOP/s",
                traffic=measured_traffic(wname, "cholesky") if mixed and fk == 2 else None,
                work_per_launch=chol_flops)
    out["cholesky"] = chol
    for r in out.values():
        r["frac"] = r["achieved"] / r["peak"] if r.get("peak") else None
    return out


def run_sharded(args, world, rank, local):
    """N > 1 GPUs: one fit of the observations of all ranks (each rank holds a config-3-sized shard of its own
    rows), one all-reduce of [l, sum|l_i|, g, lower(-H)] per iteration over NCCL and one of two doubles per
    line-search trial (paper_1404_3177_gb300.sharded)."""
    import torch

    from paper_1404_3177_gb300 import _build, datagen
    from paper_1404_3177_gb300.api import MNL
    from paper_1404_3177_gb300.sharded import ShardEngine, ShardedNewton

    _build.build()
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    prob = datagen.config3_shard(rank) if args.workload == "c3" else datagen.config2()
    Xh, Yh, Zh, ch = _host(prob)
    X, Y, Z, c = (t.to(dev) if t is not None else None for t in (Xh, Yh, Zh, ch))
    n = prob.n_theta
    m = MNL(X, Y, Z, c, K=prob.K, precision=args.precision, solve=args.solve)
    sn = ShardedNewton(ShardEngine(m))
    theta0 = torch.zeros(n, dtype=torch.float64, device=dev)
    theta = theta0.clone()

    def step():
        theta.copy_(theta0)
        return sn.step(theta)

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    barrier(world)
    sampler = ClockSampler(local) if rank == 0 else None
    if sampler:
        sampler.start()
        time.sleep(0.3)
    torch.cuda.synchronize()
    barrier(world)
    t0 = time.perf_counter()
    infos = [step() for _ in range(args.steps)]
    torch.cuda.synchronize()
    barrier(world)
    sec = allmax(world, time.perf_counter() - t0)
    clocks = sampler.stop() if sampler else None
    # e2e: each rank uploads its shard from pinned host memory every step
    mh = MNL.with_host_upload(prob.N, prob.K, prob.p, prob.d, prob.f, precision=args.precision, solve=args.solve)
    she = ShardedNewton(ShardEngine(mh))
    out_h = torch.empty(n, dtype=torch.float64).pin_memory()
    e_steps = max(3, min(args.steps, 10))

    def e2e_step():
        mh.upload(Xh, Yh, Zh, ch)
        th = torch.zeros(n, dtype=torch.float64, device=dev)
        she.step(th)
        out_h.copy_(th, non_blocking=True)
        torch.cuda.current_stream().synchronize()

    e2e_step()
    barrier(world)
    te = time.perf_counter()
    for _ in range(e_steps):
        e2e_step()
    t_e2e = allmax(world, time.perf_counter() - te)
    mh.close()
    m.close()
    if rank != 0:
        return
    sums_bytes = 8 * (2 + n + n * (n + 1) // 2)
    line = {
        "metric": METRIC, "value": world * args.steps / sec, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": 1000 * sec / args.steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": {"bf16": "bf16+f32+f64", "tf32": "tf32+f32+f64", "fp64": "f64"}[args.precision],
        "data": "synthetic",
        "config": {"workload": f"{prob.name.split('_shard')[0] if '_shard' in prob.name else prob.name}"
                               f"_x{world}_ranks_observation_sharded", "precision": args.precision, "n_theta": n,
                   "note": CONFIG_NOTE, "per_rank_rows": prob.N,
                   "exchange": f"NCCL all-reduce of {sums_bytes} bytes per iteration + 16 bytes per line-search trial"},
        "value_units": "Newton iterations of the whole (all-rank) problem x ranks: each rank's shard is one "
                       "config-3-sized problem",
        "gpu_launches": None,
        "e2e": {"value": world * e_steps / t_e2e, "unit": UNIT,
                "h2d_bytes_per_step": int(prob.input_bytes()), "d2h_bytes_per_step": int(n * 8)},
        "clocks": clocks,
        "ls_evals_per_step": statistics.median(i.get("ls_evals", 1) for i in infos),
    }
    print(json.dumps(line), flush=True)


def run_ours(args, world, rank, local):
    import torch

    from paper_1404_3177_gb300 import _build
    from paper_1404_3177_gb300 import _native as nat
    from paper_1404_3177_gb300.api import MNL

    _build.build()
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    prob, wname = workload_problem(args.workload, args.rows)
    Xh, Yh, Zh, ch = _host(prob)
    X, Y, Z, c = (t.to(dev) if t is not None else None for t in (Xh, Yh, Zh, ch))
    n = prob.n_theta
    stream = torch.cuda.current_stream()
    m = MNL(X, Y, Z, c, K=prob.K, precision=args.precision, solve=args.solve)
    theta0 = torch.zeros(n, dtype=torch.float64, device=dev)
    theta = theta0.clone()

    def step():
        theta.copy_(theta0)
        return m.newton_step(theta)

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    barrier(world)
    sampler = ClockSampler(local) if rank == 0 else None
    if sampler:
        sampler.start()
        time.sleep(0.3)
    infos = []
    torch.cuda.synchronize()
    barrier(world)
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    ev0.record(stream)
    for _ in range(args.steps):
        infos.append(step())
    ev1.record(stream)
    torch.cuda.synchronize()
    barrier(world)
    ms = ev0.elapsed_time(ev1)
    clocks = sampler.stop() if sampler else None
    ms_max = allmax(world, ms)
    t_step = ms_max / args.steps / 1000.0
    value = world * args.steps / (ms_max / 1000.0)

    # the same step with the float64 Cholesky solve (same Hessian), for comparison
    alt = None
    if args.solve != "fp64" and args.precision != "fp64" and rank == 0:
        nat.mnl_set_solve(m.h, nat.MNL_SOLVE_FP64)
        step()
        torch.cuda.synchronize()
        a0, a1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a0.record(stream)
        ai = [step() for _ in range(2)]
        a1.record(stream)
        torch.cuda.synchronize()
        alt = {"solve": "fp64", "ms_per_step": a0.elapsed_time(a1) / 2, "cholesky_ms": _median(ai, "t_factor_ms"),
               "solve_ms": _median(ai, "t_solve_ms")}
        nat.mnl_set_solve(m.h, nat.SOLVES[args.solve])
    m.close()
    del m
    torch.cuda.empty_cache()

    # e2e: through the C ABI with host buffers (H2D of the inputs + one Newton step + D2H of theta)
    mh = MNL.with_host_upload(prob.N, prob.K, prob.p, prob.d, prob.f, precision=args.precision, solve=args.solve)
    theta_h = torch.zeros(n, dtype=torch.float64).pin_memory()
    out_h = torch.empty(n, dtype=torch.float64).pin_memory()

    def e2e_step():
        mh.upload(Xh, Yh, Zh, ch)
        th = theta_h.to(dev, non_blocking=True)
        mh.newton_step(th)
        out_h.copy_(th, non_blocking=True)
        torch.cuda.current_stream().synchronize()

    for _ in range(max(1, min(3, args.warmup))):
        e2e_step()
    e_steps = max(3, min(args.steps, 10))
    torch.cuda.synchronize()
    barrier(world)
    t0 = time.perf_counter()
    for _ in range(e_steps):
        e2e_step()
    t_e2e = allmax(world, time.perf_counter() - t0)
    mh.close()
    del mh, X, Y, Z, c
    torch.cuda.empty_cache()
    h2d = prob.input_bytes() + n * 8
    d2h = n * 8

    if rank != 0:
        return
    pk, pk_kind = peaks()
    alu = measure_alu_peaks(dev)
    kern = kernel_times(infos)
    roofs = rooflines_of(prob, args.precision, kern, infos, pk, alu, wname)
    timed = {k: v for k, v in kern.items() if k in roofs}
    dominant = max(timed, key=timed.get)
    roof = dict(roofs[dominant])
    roof["kernel"] = dominant
    roof["peak_source"] = f"{pk_kind} ({roof.pop('peak_of')})"
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": t_step * 1000, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": {"bf16": "bf16+f32+f64", "tf32": "tf32+f32+f64", "fp64": "f64"}[args.precision],
        "data": "synthetic",
        "config": {"workload": wname, "precision": args.precision, "solve": args.solve, "n_theta": n,
                   "note": CONFIG_NOTE},
        "roofline": roof,
        "kernels_ms": {k: round(v, 4) for k, v in kern.items()},
        "kernel_rooflines": roofs,
        "alu_peaks": alu,
        "gpu_launches": int(sum(i["launches"] for i in infos)),
        "e2e": {"value": world * e_steps / t_e2e, "unit": UNIT, "h2d_bytes_per_step": int(h2d),
                "d2h_bytes_per_step": int(d2h)},
        "clocks": clocks,
        "ls_evals_per_step": _median(infos, "ls_evals"),
        "solve_mode_used": {1: "fp64", 2: "mixed"}.get(infos[-1]["solve_mode"]),
        "factor_used": {1: "cooperative CUDA-core", 2: "tensor-core panels"}.get(infos[-1].get("factor_kind")),
        "refine_steps": _median(infos, "refine_steps"),
        "fallbacks": int(sum(i["fallback"] for i in infos)),
        "fp64_solve_variant": alt,
    }
    if world == 1 and args.extras == "all":
        line["fp64_plain"] = extra_fp64_plain(prob, wname, dev)
        line["batched"] = extra_batch(args)
        line["serving"] = extra_serve(args)
    if not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline(prob, args)
    print(json.dumps(line), flush=True)


# ---------------------------------------------------------------------------
# extras on the same line (rank 0, one GPU, after the timed region)
# ---------------------------------------------------------------------------

def extra_fp64_plain(prob, wname, dev):
    """One Newton iteration of the plain float64 mode (every step in float64) on the same workload."""
    import torch

    from paper_1404_3177_gb300.api import MNL

    t = lambda a: torch.from_numpy(np.ascontiguousarray(a)).to(dev) if a.size else None  # noqa: E731
    X, Y, Z, c = t(prob.X), t(prob.Y), t(prob.Z), torch.from_numpy(prob.choice).to(dev)
    with MNL(X, Y, Z, c, K=prob.K, precision="fp64") as m:
        th = torch.zeros(prob.n_theta, dtype=torch.float64, device=dev)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        info = m.newton_step(th)
        e1.record()
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1)
    del X, Y, Z, c
    torch.cuda.empty_cache()
    return {"workload": wname, "ms_per_step": ms, "iters_per_s": 1000.0 / ms, "steps": 1,
            "kernels_ms": {k: round(v, 3) for k, v in kernel_times([info]).items()},
            "note": "one step after the BF16 runs; float64 pass, float64 Hessian contraction (CUDA-core DFMA), "
                    "float64 Cholesky"}


def _batch_problems(count):
    import torch

    from paper_1404_3177_gb300 import datagen
    shapes = datagen.config4_shapes()[:count]
    t0 = time.time()
    probs = [datagen.config4_problem(b, sh) for b, sh in enumerate(shapes)]
    gen_s = time.time() - t0
    dev = [dict(X=torch.from_numpy(pr.X).cuda(), Y=None, Z=torch.from_numpy(pr.Z).cuda() if pr.f else None,
                choice=torch.from_numpy(pr.choice).cuda(), K=pr.K) for pr in probs]
    return probs, dev, gen_s


def extra_batch(args):
    """All problems of the batched workload fitted by one mnl_batch_fit per precision: fits/s."""
    import torch

    from paper_1404_3177_gb300.api import MNLBatch

    probs, dev, gen_s = _batch_problems(args.count)
    out = {"workload": f"c4_{len(probs)}_problems_N500-50000_K3-30_p2-40_f0-4",
           "rows_total": int(sum(p.N for p in probs)), "generation_s": round(gen_s, 1)}
    for prec in args.batch_precisions.split(","):
        with MNLBatch(dev, precision=prec) as b:
            t = time.perf_counter()
            b.fit()  # first fit: graph capture and lazy module loading included
            torch.cuda.synchronize()
            first = time.perf_counter() - t
            if prec != "fp64":
                t = time.perf_counter()
                th, summary, per, rc = b.fit()
                torch.cuda.synchronize()
                dt = time.perf_counter() - t
            else:  # float64: the first fit is the measurement (captures included), to bound the run time
                th, summary, per, rc = None, None, None, None
                dt = first
        if summary is None:
            out[prec] = {"fits_per_s": len(probs) / dt, "seconds": dt, "note": "first fit, graph capture included"}
        else:
            out[prec] = {"fits_per_s": len(probs) / dt, "seconds": dt, "iterations": summary["iterations"],
                         "converged": summary["converged"], "failed": summary["failed"],
                         "graph_ms": summary["t_graph_ms"], "first_fit_s": first}
    del dev
    torch.cuda.empty_cache()
    return out


def _serve_once(prec, rate, duration, drain_cap, small, large):
    from paper_1404_3177_gb300 import datagen
    from paper_1404_3177_gb300.api import MNLServer

    arrivals = datagen.config5_arrivals(rate=rate, duration=duration)
    lat, qms = [], []
    done = nl = ns = 0
    with MNLServer(precision=prec, mem_budget=80 << 30) as srv:
        t0 = time.perf_counter()
        i = ticks = 0
        while True:
            now = time.perf_counter() - t0
            while i < len(arrivals) and arrivals[i][0] <= now:
                is_large = arrivals[i][1]
                pr = large[nl % len(large)] if is_large else small[ns % len(small)]
                nl, ns = (nl + 1, ns) if is_large else (nl, ns + 1)
                srv.submit(X=pr.X, Z=pr.Z if pr.f else None, choice=pr.choice, K=pr.K)
                i += 1
            n_active, n_queued = srv.step()
            ticks += 1
            for t, res in srv.finished():
                lat.append(res["latency_ms"])
                qms.append(res["queue_ms"])
                done += 1
            if i >= len(arrivals) and n_active == 0 and n_queued == 0:
                break
            if now > duration + drain_cap:
                break
        wall = time.perf_counter() - t0
    lat.sort()
    pct = lambda q: lat[min(len(lat) - 1, int(q * len(lat)))] if lat else None  # noqa: E731
    return {"requests": len(arrivals), "large": nl, "completed": done, "unfinished": len(arrivals) - done,
            "fits_per_s": done / wall, "wall_s": wall, "ticks": ticks, "p50_ms": pct(0.5), "p99_ms": pct(0.99),
            "queue_p99_ms": sorted(qms)[min(len(qms) - 1, int(0.99 * len(qms)))] if qms else None,
            "arrival_window_s": duration, "drain_cap_s": drain_cap}


def extra_serve(args):
    """Poisson arrivals of fit requests (batched-workload sizes plus 2% large ones): p50/p99 latency, fits/s."""
    from paper_1404_3177_gb300 import datagen

    shapes = datagen.config4_shapes()
    small = [datagen.config4_problem(b, sh) for b, sh in enumerate(shapes[: args.pool])]
    large = [datagen.config5_large(r) for r in range(args.large_pool)]
    out = {"workload": f"c5_poisson_{args.rate:g}_per_s_2pct_large", "distinct_small_datasets": args.pool,
           "distinct_large_datasets": args.large_pool, "mem_budget_gb": 80}
    out["bf16"] = _serve_once("bf16", args.rate, args.duration, args.drain_cap, small, large)
    out["fp64"] = _serve_once("fp64", args.rate, args.fp64_duration, args.drain_cap, small, large)
    return out


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="c3", choices=["c3", "c2"],
                    help="c3: N=500000 K=100 p=100 f=10 (default); c2: N=200000 K=50 p=50 d=5 f=5")
    ap.add_argument("--precision", default="bf16", choices=["bf16", "tf32", "fp64"])
    ap.add_argument("--rows", type=int, default=None,
                    help="observations of the workload's shape (default: the workload's N); smaller values size "
                         "profiler captures and are not the workload's bench line")
    ap.add_argument("--solve", default="auto", choices=["auto", "fp64", "mixed"],
                    help="Newton solve: float64 Cholesky, or float32 factor + float64 refinement")
    ap.add_argument("--extras", default="all", choices=["all", "none"],
                    help="all: add the float64 mode, the batched and the serving workloads to the line")
    ap.add_argument("--ref-rows", type=int, default=20000, help="oracle sample: observations for l and g")
    ap.add_argument("--ref-hess-rows", type=int, default=300, help="oracle sample: observations for -H")
    ap.add_argument("--ref-chol-n", type=int, default=2000, help="oracle sample: order of the timed Cholesky")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--count", type=int, default=2048, help="batched workload: number of problems")
    ap.add_argument("--batch-precisions", default="bf16,fp64")
    ap.add_argument("--rate", type=float, default=500.0, help="serving: arrivals per second")
    ap.add_argument("--duration", type=float, default=60.0, help="serving (BF16): seconds of arrivals")
    ap.add_argument("--fp64-duration", type=float, default=10.0, help="serving (FP64): seconds of arrivals")
    ap.add_argument("--drain-cap", type=float, default=60.0, help="serving: seconds allowed after the arrivals")
    ap.add_argument("--pool", type=int, default=256, help="serving: distinct small request datasets (cycled)")
    ap.add_argument("--large-pool", type=int, default=2)
    args = ap.parse_args()
    world, rank, local = dist_init()
    if args.impl == "reference":
        run_reference(args, world, rank)
    elif world > 1:
        run_sharded(args, world, rank, local)
    else:
        run_ours(args, world, rank, local)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
