#!/usr/bin/env python
"""ILS solves/s on GB300 for the dense 20000 x 500 instance (p = 16000, q = 4000).

One step = one complete solve of a fresh instance through the C ABI: every setup
product (ils_refactor: the Gram matrices A_1^T A_1 and A_2^T A_2, the Cholesky
factorizations of A_1^T A_1 and A^T J A, P = (A_1^T A_1)^{-1} and B = P A_2^T A_2)
followed by ils_solve (A^T J b and the iterations to the tolerance).  The headline
path is mixed-precision SP: FP64-accurate Gram matrices from exact BF16 digit
products on the tcgen05 tensor cores, FP64 Cholesky, FP32 sweeps with P and B, and
FP64 residual refinement.  Plain FP64 SP (the paper's Alg. 1 in FP64 throughout) is
timed the same way on the same instance and reported beside it.  The inputs are
resident in HBM when a step starts; A (80 MB) fits in L2, so L2 is flushed before
every step (a 256 MiB write, outside the timed events).

Usage: python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
Under torchrun every rank runs its own replica (weak scaling); rank 0 prints one
JSON line.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "ILS solves/s at rel err ≤1e-10: mixed+batched+warm vs plain FP64 SP, same GB300"
WORKLOAD = "dense ILS 20000x500 (A_1 16000x500 N(0,1), A_2 4000x500 0.3*N(0,1)), single RHS, seed 1"
TOL_RELRES = 1e-11  # relres target; kappa(A^T J A) ~ 2.5 here, so the error bound is ~2.5e-11
FP64_PEAK_TFLOPS = 1.25  # nominal GB300 FP64 (FMA pipe) rate from the profiling recipe
BF16_PEAK_TFLOPS = 1982.7  # measured cuBLAS BF16 burst rate on this machine (MEASURED_PEAKS.json)


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--cpu-seconds", type=float, default=10.0, help="bound on the CPU oracle sample")
    ap.add_argument("--stream-only", action="store_true",
                    help="only time the matrix-free A_2 stream on the tall 278144 x 500 instance")
    return ap.parse_args()


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def max_over_ranks(value: float, world: int, device=None) -> float:
    """The largest `value` over all ranks (the slowest replica's timed region)."""
    if world <= 1:
        return value
    import torch
    import torch.distributed as dist
    t = torch.tensor([value], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def replica_rate(world: int, steps: int, max_seconds: float) -> float:
    """Whole-job throughput of `world` independent replicas that each ran `steps` steps."""
    return world * steps / max_seconds


def cpu_cores() -> int:
    try:
        return len(os.sched_getaffinity(0))
    except AttributeError:
        return os.cpu_count() or 1


def time_oracle(inst, seconds: float):
    """The CPU oracle's SP solve (as it stands), repeated for about ``seconds``."""
    import oracle
    times = []
    t_end = time.perf_counter() + seconds
    while True:
        t0 = time.perf_counter()
        x, info = oracle.sp_solve(inst.A, inst.b, inst.p, tol=TOL_RELRES)
        times.append(time.perf_counter() - t0)
        if time.perf_counter() > t_end or len(times) >= 50:
            break
    return len(times) / sum(times), len(times), sum(times)


class ClockSampler:
    """nvidia-smi samples of SM clock and throttle reasons while the timed region runs."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.f = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
        self.gpu = gpu_index
        self.p = None

    def start(self):
        try:
            self.p = subprocess.Popen(["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.Q}",
                                       "--format=csv,noheader,nounits", "-lms", "200"],
                                      stdout=self.f, stderr=subprocess.DEVNULL)
        except OSError:
            self.p = None

    def stop(self):
        if self.p is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        time.sleep(0.25)
        self.p.terminate()
        try:
            self.p.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.p.kill()
        self.f.flush()
        self.f.seek(0)
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in self.f.read().splitlines():
            parts = [x.strip() for x in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        os.unlink(self.f.name)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


HBM_PEAK_GBS = 6691.8  # measured STREAM-style copy bandwidth on this machine (MEASURED_PEAKS.json)


def measure_stream(ils, torch, np, dev, reps=20):
    """Time v = A_2^T (A_2 x) streamed from the FP64, FP32 and BF16 row-major copies of A_2 on
    the tall bandwidth instance (A_2 262144 x 500: 1.05 GB in FP64, far above L2), and one
    complete mixed-precision solve of that instance (matrix-free route, BF16 sweeps)."""
    import workloads
    inst = workloads.config2_roofline()
    q, n, p = inst.q, inst.n, inst.p
    At = torch.from_numpy(np.ascontiguousarray(inst.A.T)).to(dev)
    x = torch.from_numpy(np.random.default_rng(0).standard_normal(n)).to(dev)
    v = torch.empty(n, dtype=torch.float64, device=dev)
    out = {}
    for prec, name, elem in ((1, "fp32", 4), (2, "bf16", 2), (0, "fp64", 8)):
        precision = {0: ils.ILS_BF16_REFINE, 1: ils.ILS_FP32_REFINE, 2: ils.ILS_BF16_REFINE}[prec]
        s = ils.Solver(At, p, ils.options(precision=precision, route=ils.ILS_ROUTE_MATRIX_FREE))
        for _ in range(3):
            s.aq_product(x, v, prec=prec)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        e0.record()
        for _ in range(reps):
            s.aq_product(x, v, prec=prec)
        e1.record()
        torch.cuda.synchronize()
        us = e0.elapsed_time(e1) * 1e3 / reps
        gbs = q * n * elem / (us * 1e-6) / 1e9
        out[name] = {"us_per_product": us, "achieved_GBps": gbs, "frac": gbs / HBM_PEAK_GBS,
                     "algorithmic_bytes": q * n * elem}
        if prec == 2:
            import oracle
            b = torch.from_numpy(inst.b).to(dev)
            xs_dev = torch.zeros(n, dtype=torch.float64, device=dev)
            for _ in range(2):
                s.refactor(At)
                info = s.solve(b, xs_dev, tol=TOL_RELRES)
            torch.cuda.synchronize()
            ev = (torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
            ev[0].record()
            s.refactor(At)
            info = s.solve(b, xs_dev, tol=TOL_RELRES)
            ev[1].record()
            torch.cuda.synchronize()
            xs = oracle.normal_equation_solve(inst.A, inst.b, p)
            out["tall_mixed_solve"] = {
                "ms_per_solve": ev[0].elapsed_time(ev[1]), "refinements": info.refinements,
                "relerr_vs_oracle": float(np.linalg.norm(xs_dev.cpu().numpy() - xs) / np.linalg.norm(xs)),
                "workload": "dense 278144x500 (p=16000, q=262144), matrix-free route, BF16 stream sweeps"}
        s.close()
    return out


def run_reference(args, rank, world):
    """Reference arm: the CPU oracle on the host cores (rank 0 only)."""
    if rank != 0:
        return
    import workloads
    inst = workloads.config2()
    per_step = []
    budget = max(2.0, 60.0 / max(args.steps + args.warmup, 1))
    for i in range(args.warmup + args.steps):
        rate, cnt, secs = time_oracle(inst, budget if i >= args.warmup else 0.0)
        if i >= args.warmup:
            per_step.append(secs / cnt)
    value = 1.0 / statistics.mean(per_step)
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": "solves/s", "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 / value, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": WORKLOAD, "method": "SP (Alg. 1)", "tol_relres": TOL_RELRES},
        "cpu_baseline": {"value": value, "unit": "solves/s", "cores": cpu_cores(), "kind": "oracle",
                         "sample": "numpy/LAPACK oracle SP solve of the same instance; each step one or more "
                                   "complete solves (setup included)"},
        "e2e": {"value": value, "unit": "solves/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def main():
    args = parse()
    rank, world, local = dist_env()
    if args.impl == "reference":
        run_reference(args, rank, world)
        return
    import numpy as np
    import torch

    import __graft_entry__
    __graft_entry__.build()
    import paper_2203_15340_gb300 as ils
    import workloads

    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    if args.stream_only:
        print(json.dumps(measure_stream(ils, torch, np, dev, reps=5)), flush=True)
        return
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=dev)

    def barrier():
        if world > 1:
            import torch.distributed as dist
            dist.barrier()

    inst = workloads.config2()
    m, n, p = inst.m, inst.n, inst.p
    At = torch.from_numpy(np.ascontiguousarray(inst.A.T)).to(dev)
    b = torch.from_numpy(inst.b).to(dev)
    x = torch.zeros(n, dtype=torch.float64, device=dev)
    stream = torch.cuda.current_stream(dev)
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)
    import oracle
    xs = oracle.qr_cholesky_solve(inst.A, inst.b, inst.p)

    def measure(opts, steps, with_clocks):
        """Warm up, gate accuracy, then time `steps` complete solves (per-step events)."""
        solver = ils.Solver(At, p, opts, stream=stream)

        def step():
            solver.refactor(At, stream=stream)
            return solver.solve(b, x, tol=TOL_RELRES, stream=stream)

        for _ in range(max(args.warmup, 3)):
            info = step()
        torch.cuda.synchronize()
        relerr = float(np.linalg.norm(x.cpu().numpy() - xs) / np.linalg.norm(xs))
        if not relerr <= 1e-10:
            raise SystemExit(f"accuracy gate failed: relerr {relerr:.3e}")
        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
        phases, infos = [], []
        sampler = ClockSampler(torch.cuda.current_device()) if (rank == 0 and with_clocks) else None
        barrier()
        torch.cuda.synchronize()
        if sampler:
            sampler.start()
        launches0 = ils.binding.kernel_launches()
        wall0 = time.perf_counter()
        for i in range(steps):
            flush.zero_()
            ev[i][0].record(stream)
            info = step()
            ev[i][1].record(stream)
            phases.append(solver.timings())
            infos.append(info.as_dict())
        torch.cuda.synchronize()
        wall = time.perf_counter() - wall0
        launches = ils.binding.kernel_launches() - launches0
        barrier()
        clocks = sampler.stop() if sampler else None
        total_s = max_over_ranks(sum(a.elapsed_time(bb) for a, bb in ev) / 1e3, world, dev)
        ph = {k: statistics.mean(d[k] for d in phases) for k in phases[0]}
        return dict(solver=solver, total_s=total_s, wall=wall, launches=launches, clocks=clocks, relerr=relerr,
                    phases=ph, info=infos[-1], steps=steps)

    mixed = measure(ils.options(precision=ils.ILS_FP32_REFINE, timing=1), args.steps, True)
    plain = measure(ils.options(timing=1), max(3, min(args.steps, 10)), False)
    solver = mixed["solver"]
    value = replica_rate(world, args.steps, mixed["total_s"])
    plain_value = replica_rate(world, plain["steps"], plain["total_s"])

    # ---- end to end through the C ABI with host buffers ----
    A_host = torch.from_numpy(np.ascontiguousarray(inst.A.T)).pin_memory()
    b_host = torch.from_numpy(inst.b.copy()).pin_memory()
    x_host = torch.empty(n, dtype=torch.float64).pin_memory()
    A_dev = torch.empty_like(At)
    b_dev = torch.empty_like(b)
    e2e_steps = max(3, min(args.steps, 10))
    e2e_ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(e2e_steps)]
    for i in range(e2e_steps):
        flush.zero_()
        e2e_ev[i][0].record(stream)
        A_dev.copy_(A_host, non_blocking=True)
        b_dev.copy_(b_host, non_blocking=True)
        solver.refactor(A_dev, stream=stream)
        solver.solve(b_dev, x, tol=TOL_RELRES, stream=stream)
        x_host.copy_(x, non_blocking=True)
        e2e_ev[i][1].record(stream)
    torch.cuda.synchronize()
    e2e_s = max_over_ranks(sum(a.elapsed_time(bb) for a, bb in e2e_ev) / 1e3, world, dev)
    e2e_value = replica_rate(world, e2e_steps, e2e_s)
    h2d = A_host.numel() * 8 + b_host.numel() * 8
    d2h = x_host.numel() * 8

    if rank != 0:
        return
    ms_step = 1e3 * mixed["total_s"] / args.steps
    ph = mixed["phases"]
    # Dominant kernel group of the headline step: the FP64 Cholesky factorizations of
    # A_1^T A_1 and A^T J A (2 n^3 / 3 algorithmic flops), latency-bound FP64 chains.
    chol_ms = ph["cholesky"]
    chol_flops = 2.0 * n ** 3 / 3.0
    chol_ach = chol_flops / (chol_ms * 1e-3) / 1e12
    # Tensor-core Gram A_1^T A_1: algorithmic p n (n+1) flops (FP64-accurate result).
    gram_ms = ph["gram1"]
    gram_flops = float(p) * n * (n + 1)
    n_tiles = (n + 127) // 128
    tensor_flops = 2.0 * 128 * 128 * p * (n_tiles * (n_tiles + 1) // 2) * 55  # executed BF16 MMA flops
    stream = measure_stream(ils, torch, np, dev)
    cpu_rate, cpu_cnt, cpu_secs = time_oracle(inst, args.cpu_seconds)
    line = {
        "metric": METRIC,
        "value": value,
        "unit": "solves/s",
        "n_gpus": world,
        "steps": args.steps,
        "warmup": args.warmup,
        "ms_per_step": ms_step,
        "higher_is_better": True,
        "scaling": "weak",
        "vs_baseline": None,
        "dtype": "f64",
        "data": "synthetic",
        "config": {
            "workload": WORKLOAD,
            "method": "SP (Alg. 1), mixed precision: tensor-core FP64-accurate Grams, FP64 Cholesky, "
                      "FP32 sweeps, FP64 residual refinement",
            "tol_relres": TOL_RELRES,
            "relerr_vs_oracle": mixed["relerr"],
            "refinements": mixed["info"]["refinements"],
            "sp_sweeps": mixed["info"]["outer_iters"],
            "setup_phases_ms": {k: round(v, 4) for k, v in ph.items()},
            "l2": "flushed before every step (256 MiB write outside the timed events)",
            "step": "ils_refactor (all setup products) + ils_solve",
            "wall_s_timed_loop": mixed["wall"],
        },
        "plain_fp64_sp": {
            "value": plain_value, "unit": "solves/s", "ms_per_step": 1e3 * plain["total_s"] / plain["steps"],
            "steps": plain["steps"], "relerr_vs_oracle": plain["relerr"], "outer_iters": plain["info"]["outer_iters"],
            "setup_phases_ms": {k: round(v, 4) for k, v in plain["phases"].items()},
            "speedup_of_headline": value / plain_value,
        },
        "roofline": {
            "kernel": "FP64 Cholesky of A_1^T A_1 and A^T J A (potrf_diag + trsm_panel + syrk_trailing)",
            "bound": "alu",
            "achieved": chol_ach,
            "peak": FP64_PEAK_TFLOPS,
            "peak_source": "nominal FP64 rate of the profiling recipe (FP64 is absent from MEASURED_PEAKS.json)",
            "unit": "TFLOP/s",
            "frac": chol_ach / FP64_PEAK_TFLOPS,
            "traffic": None,
            "kernel_ms": chol_ms,
            "share_of_step": chol_ms / ms_step,
            "note": "latency-bound: 64-cycle dependent FP64 FMA and 440-cycle FP64 rsqrt on the pivot chain",
        },
        "roofline_tensor_gram": {
            "kernel": "gram_split_mma_kernel + digit split + reduce (A_1^T A_1 to FP64 accuracy)",
            "bound": "tensor",
            "achieved": tensor_flops / (gram_ms * 1e-3) / 1e12,
            "peak": BF16_PEAK_TFLOPS,
            "unit": "TFLOP/s (executed BF16 MMA flops)",
            "frac": tensor_flops / (gram_ms * 1e-3) / 1e12 / BF16_PEAK_TFLOPS,
            "fp64_equivalent_tflops": gram_flops / (gram_ms * 1e-3) / 1e12,
            "kernel_ms": gram_ms,
            "share_of_step": gram_ms / ms_step,
        },
        "roofline_stream": {
            "kernel": "aq_stream_kernel (one-pass A_2^T (A_2 x), matrix-free route), tall instance A_2 262144x500",
            "bound": "hbm",
            "achieved": stream["fp32"]["achieved_GBps"],
            "peak": HBM_PEAK_GBS,
            "unit": "GB/s",
            "frac": stream["fp32"]["frac"],
            "traffic": None,
            "by_precision": {k: v for k, v in stream.items() if k in ("fp32", "bf16", "fp64")},
            "note": "FP64 copy is FP64-issue bound (2 FMA per 8 bytes); FP32/BF16 copies stream at HBM speed",
        },
        "tall_config": stream.get("tall_mixed_solve"),
        "cpu_baseline": {
            "value": cpu_rate, "unit": "solves/s", "cores": cpu_cores(), "kind": "oracle",
            "sample": f"{cpu_cnt} complete oracle SP solves of the same instance ({cpu_secs:.1f} s, numpy/LAPACK "
                      "with the default BLAS thread count)",
        },
        "e2e": {"value": e2e_value, "unit": "solves/s", "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h},
        "gpu_launches": int(mixed["launches"]),
        "clocks": mixed["clocks"],
    }
    print(json.dumps(line), flush=True)
    mixed["solver"].close()
    plain["solver"].close()


if __name__ == "__main__":
    main()
