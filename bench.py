#!/usr/bin/env python3
"""Benchmark: Newton-Raphson iterations per second of the multinomial-logit fit.

Workload (default): N=200000 observations, K=50 alternatives, p=50 individual-
specific columns (intercept + 49 N(0,1)), d=5 and f=5 alternative-specific
columns, 2700 coefficients; seeded synthetic data (paper_1404_3177_gb300.datagen).
One step = one full Newton iteration (utilities/softmax/log-likelihood/gradient
pass, structured Hessian, FP64 Cholesky solve, step-halving line search,
coefficient update) from theta = 0, so every step does the same work.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--precision bf16|tf32|fp64]
    python bench.py --impl reference ...     # the FP64 CPU oracle on the host cores

Timing: CUDA events on the stream the library uses, W untimed warm-up steps,
then K steps bracketed by a barrier and torch.cuda.synchronize(); the inputs
(441 MB) are larger than L2, so no flush is needed between steps.  With N > 1
GPUs (torchrun) every rank runs an independent replica of the same fit (the
single-fit path has no multi-GPU exchange yet) and `value` is the sum over
ranks at the slowest rank's time.
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

METRIC = "newton_iters_per_s"
# CUDA-core peaks measured on this machine's GB300 (152 SMs at 2070 MHz) with a
# dependent-chain-free FMA microbenchmark: float64 DFMA 1.06, float64 DMMA 1.10,
# float32 FFMA 71.0 TFLOP/s (cuBLAS DGEMM 1.10, SGEMM 69.8).
# DRAM bytes of one launch (dram__bytes_read.sum + dram__bytes_write.sum) from one ncu capture of each kernel on
# the default workload: the 128 x 256 tcgen05 contraction of the class operands (reads the 1.08 GB operand 1.7
# times, writes its partial tiles), the tiled float32 pass (the 441 MB of inputs once, P and zbar written) and the
# cooperative float32 factor + inverse of the mixed solve (the 29 MB lower triangle; the rest stays in L2).
MEASURED_TRAFFIC = {"bf16": {"syrk_AtA": 1854754304 + 250199296, "pass": 444282112 + 41421056,
                             "cholesky_mixed": 30338816 + 3851520}}
FP64_TFLOPS = 1.06
FP32_TFLOPS = 71.0
UNIT = "iter/s"
WORKLOAD = "c2_N200000_K50_p50_d5_f5"
CONFIG_NOTE = "inputs larger than L2 (no flush)"


def peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        with open(path) as fh:
            return json.load(fh), "measured"
    return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0}, "fallback"


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

def oracle_iteration_seconds(prob, n_sample: int, repeats: int = 1):
    """Seconds of one oracle Newton iteration at the full workload, extrapolated from
    a sample of the observations (terms proportional to N) plus the Cholesky solve
    measured at the full coefficient count (independent of N)."""
    import oracle
    from paper_1404_3177_gb300 import datagen

    sub = datagen.Problem(n_sample, prob.K, prob.p, prob.d, prob.f, 0, prob.X[:n_sample], prob.Y[:n_sample],
                          prob.Z[:n_sample], prob.choice[:n_sample], prob.theta_true)
    th = np.zeros(prob.n_theta)
    per_row = []
    for _ in range(repeats):
        t0 = time.perf_counter()
        _, g = oracle.loglik_grad(sub, th)
        F = oracle.neg_hessian(sub, th)
        oracle.loglik(sub, th)  # one line-search evaluation
        per_row.append((time.perf_counter() - t0) / n_sample)
    # Cholesky + solve of an n x n SPD matrix (the sample's -H scaled to full N)
    t0 = time.perf_counter()
    L = oracle.cholesky(F * (prob.N / n_sample))
    oracle.cholesky_solve(L, g)
    t_chol = time.perf_counter() - t0
    rows = statistics.median(per_row)
    return rows * prob.N + t_chol, rows, t_chol


def cpu_baseline(prob, n_sample=20000):
    cores = os.cpu_count() or 1
    t_iter, _, t_chol = oracle_iteration_seconds(prob, n_sample)
    return {"value": 1.0 / t_iter, "unit": UNIT, "cores": cores, "kind": "oracle",
            "sample": f"{n_sample} of {prob.N} observations (l, g, -H and one line-search l, scaled x{prob.N / n_sample:g}) "
                      f"+ Cholesky solve at the full n_theta={prob.n_theta} ({t_chol:.1f} s)"}


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


# ---------------------------------------------------------------------------
# arms
# ---------------------------------------------------------------------------

def run_reference(args, world, rank):
    """The FP64 CPU oracle as it stands, one bounded sample per step (rank 0 only)."""
    if rank != 0:
        return
    from paper_1404_3177_gb300 import datagen
    prob = datagen.config2()
    n_sample = max(500, int(args.ref_rows))
    cores = os.cpu_count() or 1
    for _ in range(args.warmup):
        oracle_iteration_seconds(prob, n_sample)
    times = []
    for _ in range(args.steps):
        t_iter, _, _ = oracle_iteration_seconds(prob, n_sample)
        times.append(t_iter)
    t = statistics.mean(times)
    v = 1.0 / t
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1000 * t, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": WORKLOAD, "note": CONFIG_NOTE},
            "cpu_baseline": {"value": v, "unit": UNIT, "cores": cores, "kind": "oracle",
                             "sample": f"each step: {n_sample} of {prob.N} observations scaled to N, "
                                       "plus the full-size Cholesky solve"},
            "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def run_ours(args, world, rank, local):
    import torch

    from paper_1404_3177_gb300 import _build, datagen
    from paper_1404_3177_gb300.api import MNL

    _build.build()
    torch.cuda.set_device(local)
    prob = datagen.config2()
    dev = torch.device("cuda", local)
    Xh = torch.from_numpy(prob.X).pin_memory()
    Yh = torch.from_numpy(prob.Y).pin_memory()
    Zh = torch.from_numpy(prob.Z).pin_memory()
    ch = torch.from_numpy(prob.choice).pin_memory()
    X, Y, Z, c = (t.to(dev) for t in (Xh, Yh, Zh, ch))
    n = prob.n_theta
    stream = torch.cuda.current_stream()
    m = MNL(X, Y, Z, c, precision=args.precision, solve=args.solve)
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

    # e2e: through the C ABI with host buffers (H2D of the inputs + one Newton step + D2H of theta)
    # the same step with the float64 Cholesky solve, for comparison (not the headline)
    alt = {}
    if args.solve != "fp64" and args.precision != "fp64":
        from paper_1404_3177_gb300 import _native as nat
        nat.mnl_set_solve(m.h, nat.MNL_SOLVE_FP64)
        step()
        torch.cuda.synchronize()
        a0 = torch.cuda.Event(enable_timing=True)
        a1 = torch.cuda.Event(enable_timing=True)
        a0.record(stream)
        alt_infos = [step() for _ in range(3)]
        a1.record(stream)
        torch.cuda.synchronize()
        alt = {"solve": "fp64", "ms_per_step": a0.elapsed_time(a1) / 3,
               "cholesky_ms": statistics.median(i["t_factor_ms"] for i in alt_infos),
               "solve_ms": statistics.median(i["t_solve_ms"] for i in alt_infos)}
        nat.mnl_set_solve(m.h, nat.SOLVES[args.solve])

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
    h2d = prob.input_bytes() + n * 8
    d2h = n * 8

    if rank != 0:
        return
    pk, pk_kind = peaks()
    med = lambda k: statistics.median(i[k] for i in infos)  # noqa: E731
    N, K, q, f = prob.N, prob.K, prob.p + prob.d, prob.f
    mc = (K - 1) * q
    kern = {
        "pass": med("t_pass_ms"), "build_operands": med("t_build_ms"), "syrk_AtA": med("t_syrk_ms"),
        "syrk_diag_blocks": med("t_band_ms"), "z_blocks": med("t_zblk_ms"), "assemble": med("t_asm_ms"),
        "cholesky": med("t_factor_ms"), "solve": med("t_solve_ms"), "line_search": med("t_ls_ms"),
    }
    mixed_used = infos[-1]["solve_mode"] == 2
    dominant = max(kern, key=kern.get)
    syrk_flops = float(N) * mc * (mc + 1)
    pass_bytes = 4.0 * N * (prob.p + K * (prob.d + f) + 1) + 4.0 * N * K + 4.0 * N * f
    chol_flops = n ** 3 / 3.0
    if args.precision == "fp64":
        syrk_peak, syrk_unit, syrk_bound = FP64_TFLOPS, "TFLOP/s", "alu"
    elif args.precision == "tf32":
        syrk_peak = pk["bf16_tflops_sustained"] / 2.0 if pk.get("bf16_tflops_sustained") else None
        syrk_unit, syrk_bound = "TFLOP/s", "tensor"
    else:
        syrk_peak, syrk_unit, syrk_bound = pk.get("bf16_tflops_sustained"), "TFLOP/s", "tensor"
    traffic = MEASURED_TRAFFIC.get(args.precision, {}) if args.solve == "auto" else {}
    rooflines = {
        "syrk_AtA": {"bound": syrk_bound, "achieved": syrk_flops / (kern["syrk_AtA"] * 1e-3) / 1e12,
                     "peak": syrk_peak, "unit": syrk_unit, "traffic": traffic.get("syrk_AtA")},
        "pass": {"bound": "hbm", "achieved": pass_bytes / (kern["pass"] * 1e-3) / 1e9, "peak": pk["hbm_gbs"],
                 "unit": "GB/s", "traffic": traffic.get("pass")},
        "cholesky": {"bound": "alu", "achieved": chol_flops / (kern["cholesky"] * 1e-3) / 1e12,
                     "peak": FP32_TFLOPS if mixed_used else FP64_TFLOPS, "unit": "TFLOP/s",
                     "traffic": traffic.get("cholesky_mixed") if mixed_used else None,
                     "arith": "f32 factor + f64 refinement" if mixed_used else "f64"},
    }
    for r in rooflines.values():
        r["frac"] = (r["achieved"] / r["peak"]) if r.get("peak") else None
    dom_key = dominant if dominant in rooflines else "syrk_AtA"
    roof = dict(rooflines[dom_key])
    roof["kernel"] = dom_key
    roof["peak_source"] = pk_kind
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": t_step * 1000, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": {"bf16": "bf16+f32+f64", "tf32": "tf32+f32+f64", "fp64": "f64"}[args.precision],
        "data": "synthetic",
        "config": {"workload": WORKLOAD, "precision": args.precision, "solve": args.solve, "n_theta": n,
                   "note": CONFIG_NOTE},
        "roofline": roof,
        "kernels_ms": {k: round(v, 4) for k, v in kern.items()},
        "kernel_rooflines": rooflines,
        "gpu_launches": int(sum(i["launches"] for i in infos)),
        "e2e": {"value": world * e_steps / t_e2e, "unit": UNIT, "h2d_bytes_per_step": int(h2d),
                "d2h_bytes_per_step": int(d2h)},
        "clocks": clocks,
        "ls_evals_per_step": med("ls_evals"),
        "solve_mode_used": {1: "fp64", 2: "mixed"}.get(infos[-1]["solve_mode"]),
        "refine_steps": med("refine_steps"),
        "fallbacks": int(sum(i["fallback"] for i in infos)),
        "fp64_solve_variant": alt or None,
    }
    if not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline(prob, args.ref_rows)
    print(json.dumps(line), flush=True)
    m.close()


# ---------------------------------------------------------------------------
# batched and serving workloads (separate lines; not the default run)
# ---------------------------------------------------------------------------

def run_batch(args):
    """All problems of the batched workload fitted by one mnl_batch_fit: fits/s."""
    import torch

    from paper_1404_3177_gb300 import _build, datagen
    from paper_1404_3177_gb300.api import MNLBatch

    _build.build()
    torch.cuda.set_device(0)
    shapes = datagen.config4_shapes()[: args.count]
    t0 = time.time()
    probs = [datagen.config4_problem(b, sh) for b, sh in enumerate(shapes)]
    gen_s = time.time() - t0
    dev = []
    for pr in probs:
        dev.append(dict(X=torch.from_numpy(pr.X).cuda(), Y=None,
                        Z=torch.from_numpy(pr.Z).cuda() if pr.f else None,
                        choice=torch.from_numpy(pr.choice).cuda(), K=pr.K))
    out = {}
    for prec in args.batch_precisions.split(","):
        with MNLBatch(dev, precision=prec) as b:
            b.fit()  # warm-up (graph capture, lazy module loading)
            torch.cuda.synchronize()
            t = time.perf_counter()
            th, summary, per, rc = b.fit()
            torch.cuda.synchronize()
            dt = time.perf_counter() - t
        out[prec] = {"fits_per_s": len(probs) / dt, "seconds": dt, "iterations": summary["iterations"],
                     "converged": summary["converged"], "failed": summary["failed"],
                     "pass_rows": summary["pass_rows"], "graph_ms": summary["t_graph_ms"]}
    line = {"metric": "batched_fits_per_s", "value": out[args.batch_precisions.split(",")[0]]["fits_per_s"],
            "unit": "fits/s", "n_gpus": 1, "higher_is_better": True, "data": "synthetic",
            "config": {"workload": f"c4_{len(probs)}_problems_N500-50000_K3-30_p2-40_f0-4",
                       "rows_total": int(sum(p.N for p in probs)), "generation_s": round(gen_s, 1)},
            "by_precision": out}
    print(json.dumps(line), flush=True)


def run_serve(args):
    """Poisson arrivals of fit requests (batched-workload sizes plus 2% large ones), p50/p99 latency, fits/s."""
    import torch

    from paper_1404_3177_gb300 import _build, datagen
    from paper_1404_3177_gb300.api import MNLServer

    _build.build()
    torch.cuda.set_device(0)
    arrivals = datagen.config5_arrivals(rate=args.rate, duration=args.duration)
    shapes = datagen.config4_shapes()
    small = [datagen.config4_problem(b, sh) for b, sh in enumerate(shapes[: args.pool])]
    large = [datagen.config5_large(r) for r in range(args.large_pool)]
    res = {}
    for prec in args.serve_precisions.split(","):
        lat, qms, done, ns, nl = [], [], 0, 0, 0
        with MNLServer(precision=prec, mem_budget=80 << 30) as srv:
            pending = {}
            t0 = time.perf_counter()
            i = 0
            ticks = 0
            while i < len(arrivals) or pending:
                now = time.perf_counter() - t0
                while i < len(arrivals) and arrivals[i][0] <= now:
                    is_large = arrivals[i][1]
                    pr = large[nl % len(large)] if is_large else small[ns % len(small)]
                    if is_large:
                        nl += 1
                    else:
                        ns += 1
                    pending[srv.submit(X=pr.X, Z=pr.Z if pr.f else None, choice=pr.choice, K=pr.K)] = is_large
                    i += 1
                srv.step()
                ticks += 1
                for t in list(pending):
                    r = srv.poll(t)
                    if r is not None:
                        lat.append(r[1]["latency_ms"])
                        qms.append(r[1]["queue_ms"])
                        done += 1
                        del pending[t]
            wall = time.perf_counter() - t0
        lat.sort()
        res[prec] = {"requests": len(arrivals), "large": nl, "fits_per_s": done / wall, "wall_s": wall,
                     "ticks": ticks, "p50_ms": lat[len(lat) // 2], "p99_ms": lat[min(len(lat) - 1, int(0.99 * len(lat)))],
                     "queue_p99_ms": sorted(qms)[min(len(qms) - 1, int(0.99 * len(qms)))]}
    first = args.serve_precisions.split(",")[0]
    line = {"metric": "serving_p50_p99_latency_ms", "value": res[first]["p99_ms"], "unit": "ms",
            "higher_is_better": False, "n_gpus": 1, "data": "synthetic",
            "config": {"workload": f"c5_poisson_{args.rate:g}_per_s_{args.duration:g}s_2pct_large",
                       "distinct_small_datasets": args.pool, "distinct_large_datasets": args.large_pool,
                       "mem_budget_gb": 80},
            "by_precision": res}
    print(json.dumps(line), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--precision", default="bf16", choices=["bf16", "tf32", "fp64"])
    ap.add_argument("--solve", default="auto", choices=["auto", "fp64", "mixed"],
                    help="Newton solve: float64 Cholesky, or float32 factor + float64 refinement")
    ap.add_argument("--ref-rows", type=int, default=20000, help="observations in the oracle's bounded sample")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--workload", default="c2", choices=["c2", "batch", "serve"],
                    help="c2: the single large fit (default); batch / serve: the batched and serving workloads")
    ap.add_argument("--count", type=int, default=2048, help="batch: number of problems")
    ap.add_argument("--batch-precisions", default="bf16,fp64")
    ap.add_argument("--serve-precisions", default="bf16,fp64")
    ap.add_argument("--rate", type=float, default=500.0)
    ap.add_argument("--duration", type=float, default=10.0)
    ap.add_argument("--pool", type=int, default=256, help="serve: distinct small request datasets (cycled)")
    ap.add_argument("--large-pool", type=int, default=2)
    args = ap.parse_args()
    if args.workload == "batch":
        return run_batch(args)
    if args.workload == "serve":
        return run_serve(args)
    world, rank, local = dist_init()
    if args.impl == "reference":
        run_reference(args, world, rank)
    else:
        run_ours(args, world, rank, local)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
