#!/usr/bin/env python
"""ILS solves/s on GB300 for the dense 20000 x 500 instance (p = 16000, q = 4000).

One step = one complete solve of a fresh instance through the C ABI: every setup
product (ils_refactor_async: the Gram matrices A_1^T A_1 and A_2^T A_2, P = (A_1^T A_1)^{-1},
the SPD test of A^T J A, and B = P A_2^T A_2) followed by ils_solve (A^T J b and the
iterations to the tolerance).  The headline path is mixed-precision SP: FP64-accurate
Gram matrices from exact BF16 digit products on the tcgen05 tensor cores, P by FP32
block Gauss-Jordan elimination in one cooperative launch (a second launch on another
stream tests A^T J A the same way), FP32 sweeps with P and B, and FP64 residual refinement, the whole refinement in one
cooperative launch.  Plain FP64 SP (the paper's Alg. 1 in FP64 throughout: FP64 Grams,
FP64 Cholesky, P and B) is timed the same way on the same instance and reported beside
it.  The inputs are resident in HBM when a step starts; A (80 MB) fits in L2, so L2 is
flushed before every step (a 256 MiB write, outside the timed events).

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
TOL_ERR = 1e-10  # target relative error: solves stop once kappa_est * relres <= 1e-10 (ILS_STOP_ERR_BOUND)
TOL_RELRES = 1e-11  # relres target of the secondary measurements (kappa(A^T J A) <= 2.5 on them)
FP64_PEAK_TFLOPS = 1.25  # nominal GB300 FP64 (FMA pipe) rate from the profiling recipe
# FP32 SIMT peak from unit counts: 152 SMs x 128 FP32 lanes x 2 flops x 2.07 GHz (max SM clock)
FP32_SIMT_PEAK_TFLOPS = 152 * 128 * 2 * 2.07e9 / 1e12
# DRAM bytes per launch (dram__bytes_read.sum + dram__bytes_write.sum) from one ncu capture
# of each kernel as it stands, on the headline step; None once a kernel changes.
MMA_TRAFFIC_BYTES = 144_444_416 + 9_991_936
GJ_TRAFFIC_BYTES = 693_504 + 0


def measured_peaks():
    """HBM copy bandwidth and cuBLAS BF16 rates measured on this machine (MEASURED_PEAKS.json, written
    by the pool's driver), else the profiling recipe's fallback figures."""
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as f:
            d = json.load(f)
        return {"hbm_gbs": float(d["hbm_gbs"]), "bf16_tflops": float(d["bf16_tflops"]),
                "bf16_tflops_sustained": float(d.get("bf16_tflops_sustained", d["bf16_tflops"])),
                "source": "of measured (MEASURED_PEAKS.json)"}
    except (OSError, KeyError, ValueError):
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0,
                "source": "of fallback (profiling recipe)"}


PEAKS = measured_peaks()
HBM_PEAK_GBS = PEAKS["hbm_gbs"]
BF16_PEAK_TFLOPS = PEAKS["bf16_tflops"]


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=50)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--cpu-seconds", type=float, default=10.0, help="bound on the CPU oracle sample")
    ap.add_argument("--no-configs", action="store_true",
                    help="skip the sparse, batched and warm-start measurements")
    ap.add_argument("--only", choices=["stream", "sparse", "batched", "warm", "paper"],
                    help="print only one secondary measurement (for profiling runs): the matrix-free stream on "
                         "the tall 278144 x 500 instance, or the sparse, batched or warm-start configuration")
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



def measure_stream(ils, torch, np, dev, reps=20):
    """Time v = A_2^T (A_2 x) streamed from the FP32, BF16, double-FP32 (a mixed handle's
    FP64-accurate copy) and FP64 (an FP64 handle's) row-major copies of A_2 on the tall
    bandwidth instance (A_2 262144 x 500: 1.05 GB in FP64, far above L2), and one complete
    mixed-precision solve of that instance (matrix-free route, BF16 sweeps)."""
    import workloads
    inst = workloads.config2_roofline()
    q, n, p = inst.q, inst.n, inst.p
    At = torch.from_numpy(np.ascontiguousarray(inst.A.T)).to(dev)
    x = torch.from_numpy(np.random.default_rng(0).standard_normal(n)).to(dev)
    v = torch.empty(n, dtype=torch.float64, device=dev)
    out = {}
    for prec, name, elem, precision in ((1, "fp32", 4, ils.ILS_FP32_REFINE), (0, "df32", 8, ils.ILS_FP32_REFINE),
                                        (0, "fp64", 8, ils.ILS_FP64), (2, "bf16", 2, ils.ILS_BF16_REFINE)):
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


def _events(torch):
    return torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)


def _normal_solution(A, B, p):
    """x* = (A^T J A)^{-1} A^T J B by a numpy Cholesky solve (kappa is small on every workload)."""
    import numpy as np
    import scipy.linalg as sla
    A1, A2 = A[:p], A[p:]
    H = A1.T @ A1 - A2.T @ A2
    return sla.cho_solve(sla.cho_factor(H), A1.T @ B[:p] - A2.T @ B[p:])


def measure_sparse(ils, torch, np, dev, k=8):
    """Sparse CSR 100000 x 2000 (density 0.005): SP-RK-RGS with the FP32 cluster chain on the FP64
    residual, the paper's FP64 SP-RK-RGS, and FP64 SP, each on k right-hand sides at once."""
    import scipy.linalg as sla
    import scipy.sparse as sps
    import workloads
    inst = workloads.config3_sparse()
    rng = np.random.default_rng(303)
    A = sps.csr_matrix((inst.val, inst.colind, inst.rowptr), shape=(inst.m, inst.n))
    Bm = np.empty((inst.m, k))
    Bm[:, 0] = inst.b
    for j in range(1, k):
        Bm[:, j] = A @ rng.standard_normal(inst.n) + 1e-3 * rng.standard_normal(inst.m)
    A1, A2 = A[:inst.p], A[inst.p:]
    H = (A1.T @ A1 - A2.T @ A2).toarray()
    Xs = sla.cho_solve(sla.cho_factor(H), A1.T @ Bm[:inst.p] - A2.T @ Bm[inst.p:])
    rp = torch.from_numpy(inst.rowptr).to(dev)
    ci = torch.from_numpy(inst.colind).to(dev)
    va = torch.from_numpy(inst.val).to(dev)
    Bt = torch.from_numpy(np.ascontiguousarray(Bm.T)).to(dev)
    out = {"workload": "sparse CSR 100000x2000 density 0.005 (p=80000, q=20000, A_2 x 0.25), seed 3, "
                       f"{k} right-hand sides solved together"}
    cases = [("rk_rgs_fp32_chain", dict(method=ils.ILS_SP_RK_RGS, precision=ils.ILS_FP32_REFINE)),
             ("rk_rgs_fp64_paper", dict(method=ils.ILS_SP_RK_RGS)),
             ("sp_fp64", dict(method=ils.ILS_SP))]
    for name, kw in cases:
        e0, e1 = _events(torch)
        e0.record()
        s = ils.Solver.from_csr(inst.m, inst.n, inst.p, rp, ci, va, ils.options(seed=3, **kw))
        e1.record()
        torch.cuda.synchronize()
        setup_ms = e0.elapsed_time(e1)
        Xt = torch.zeros((k, inst.n), dtype=torch.float64, device=dev)
        launches0 = ils.binding.kernel_launches()
        e0.record()
        info = s.solve_many(Bt, Xt, tol=TOL_RELRES)
        e1.record()
        torch.cuda.synchronize()
        solve_ms = e0.elapsed_time(e1)
        X = Xt.cpu().numpy().T
        err = max(float(np.linalg.norm(X[:, j] - Xs[:, j]) / np.linalg.norm(Xs[:, j])) for j in range(k))
        out[name] = {"solves_per_s": k / (solve_ms * 1e-3), "solve_ms_k_rhs": solve_ms, "setup_ms": setup_ms,
                     "outer_iters": info.outer_iters, "inner_steps": info.inner_iters,
                     "us_per_inner_step": (1e3 * solve_ms / info.inner_iters) if info.inner_iters else None,
                     "max_relerr": err, "launches": ils.binding.kernel_launches() - launches0}
        s.close()
    return out


def measure_batched(ils, torch, np, dev):
    """256 uneven problems x 8 right-hand sides: one batch (BF16 sweeps, FP64 refinement) against
    plain FP64 SP on one handle at a time; each timed region holds every setup and solve."""
    import workloads
    insts = workloads.config4_batched()
    Ats = [torch.from_numpy(np.ascontiguousarray(x.A.T)).to(dev) for x in insts]
    Bts = [torch.from_numpy(np.ascontiguousarray(x.b.T)).to(dev) for x in insts]
    k = insts[0].b.shape[1]
    Xb = [torch.zeros((k, x.n), dtype=torch.float64, device=dev) for x in insts]
    Xp = [torch.zeros((k, x.n), dtype=torch.float64, device=dev) for x in insts]
    ps = [x.p for x in insts]

    def batched():
        bs = ils.BatchSolver(Ats, ps, ils.options(precision=ils.ILS_BF16_REFINE))
        infos = bs.solve(Bts, Xb, tol=TOL_RELRES)
        bs.close()
        return infos

    def plain():
        for At, p, Bt, X in zip(Ats, ps, Bts, Xp):
            s = ils.Solver(At, p, ils.options())
            s.solve_many(Bt, X, tol=TOL_RELRES)
            s.close()

    Xq = [torch.zeros((k, x.n), dtype=torch.float64, device=dev) for x in insts]

    def plain_batched():  # plain FP64 SP through the same batch machinery (16 streams)
        bs = ils.BatchSolver(Ats, ps, ils.options())
        bs.solve(Bts, Xq, tol=TOL_RELRES)
        bs.close()

    # One CUDA graph holding every setup and solve of the batch (ils_batch_capture with
    # refactor), replayed by one launch per step.
    gstream = torch.cuda.Stream(dev)
    Xg = [torch.zeros((k, x.n), dtype=torch.float64, device=dev) for x in insts]
    with torch.cuda.stream(gstream):
        gb = ils.BatchSolver(Ats, ps, ils.options(precision=ils.ILS_BF16_REFINE), stream=gstream)
        gb.capture(Bts, Xg, refactor=True, steps=8, tol=TOL_RELRES, stream=gstream)
        gb.run(stream=gstream)  # warm-up replay
        g0, g1 = _events(torch)
        reps = 5
        g0.record(gstream)
        for _ in range(reps):
            ginfos = gb.run(stream=gstream)
        g1.record(gstream)
    torch.cuda.synchronize()
    t_g = g0.elapsed_time(g1) / reps
    gb.close()
    batched()  # warm-up (module load, first-touch of the allocator pools)
    torch.cuda.synchronize()
    e0, e1 = _events(torch)
    e0.record()
    infos = batched()
    e1.record()
    torch.cuda.synchronize()
    t_b = e0.elapsed_time(e1)
    e0.record()
    plain()
    e1.record()
    torch.cuda.synchronize()
    t_p = e0.elapsed_time(e1)
    plain_batched()  # warm-up
    torch.cuda.synchronize()
    e0.record()
    plain_batched()
    e1.record()
    torch.cuda.synchronize()
    t_pb = e0.elapsed_time(e1)
    err = 0.0
    for i in range(len(insts)):  # every problem, every right-hand side, all three runs
        xs = _normal_solution(insts[i].A, insts[i].b, insts[i].p)
        for X in (Xb[i], Xp[i], Xg[i], Xq[i]):
            xv = X.cpu().numpy().T
            err = max(err, float(np.max(np.linalg.norm(xv - xs, axis=0) / np.linalg.norm(xs, axis=0))))
    total = len(insts) * k
    return {"workload": f"{len(insts)} uneven dense problems (n 32..512, m 4n..20n, q/m .05..25), {k} RHS each, "
                        "seed [4, i]",
            "batched_bf16_refine": {"solves_per_s": total / (t_b * 1e-3), "ms_setup_plus_solve": t_b,
                                    "max_refinements": max(i.refinements for i in infos)},
            "graph_replay_bf16_refine": {"solves_per_s": total / (t_g * 1e-3), "ms_setup_plus_solve": t_g,
                                         "note": "ils_batch_capture(refactor=1): every setup and solve of the "
                                                 "batch in one CUDA graph, one launch per step",
                                         "max_refinements": max(i.refinements for i in ginfos)},
            "plain_fp64_sp_one_handle_at_a_time": {"solves_per_s": total / (t_p * 1e-3), "ms_setup_plus_solve": t_p},
            "plain_fp64_sp_batched": {"solves_per_s": total / (t_pb * 1e-3), "ms_setup_plus_solve": t_pb},
            "speedup": t_pb / min(t_b, t_g), "speedup_vs_one_at_a_time": t_p / min(t_b, t_g),
            "max_relerr": err, "checked_problems": len(insts)}


def measure_warm(ils, torch, np, dev, n_train=50000, n_eval=2048, epochs=40):
    """Learned warm start on the parametric family (A 8192 x 256, b = F theta + 1e-3 noise): train on
    n_train SP solutions produced by the library, then solve n_eval held-out right-hand sides from
    x0 = net(theta) and from x0 = 0."""
    import workloads
    fam = workloads.config5_warmstart()
    n = fam.A.shape[1]
    At5 = torch.from_numpy(np.ascontiguousarray(fam.A.T)).to(dev)
    certified = dict(stop_rule=ils.ILS_STOP_ERR_BOUND)  # every evaluation stops on kappa_est relres <= 1e-10
    solver = ils.Solver(At5, fam.p, ils.options(**certified))
    msolver = ils.Solver(At5, fam.p, ils.options(precision=ils.ILS_BF16_REFINE, **certified))
    th_train = fam.thetas(n_train, seed=5)
    X_train = torch.zeros((n_train, n), dtype=torch.float64, device=dev)
    e0, e1 = _events(torch)
    t_targets = 0.0
    for c0 in range(0, n_train, 4096):
        c1 = min(n_train, c0 + 4096)
        Bt = torch.from_numpy(np.ascontiguousarray(fam.rhs(th_train[c0:c1], seed=5, start=c0).T)).to(dev)
        e0.record()
        solver.solve_many(Bt, X_train[c0:c1], tol=1e-11)
        e1.record()
        torch.cuda.synchronize()
        t_targets += e0.elapsed_time(e1)
    net = ils.WarmStartNet(16, 256, n, seed=1)
    th_t = torch.from_numpy(th_train.astype(np.float32)).to(dev)
    e0.record()
    loss = net.train(th_t, X_train, epochs=epochs, batch=256, lr=1e-3)
    e1.record()
    torch.cuda.synchronize()
    t_train = e0.elapsed_time(e1)
    th_eval = fam.thetas(n_eval, seed=55)
    B_eval = fam.rhs(th_eval, seed=55)
    Be = torch.from_numpy(np.ascontiguousarray(B_eval.T)).to(dev)
    th_e = torch.from_numpy(th_eval.astype(np.float32)).to(dev)
    Xc = torch.zeros((n_eval, n), dtype=torch.float64, device=dev)
    Xw = torch.zeros_like(Xc)
    Xm = torch.zeros_like(Xc)
    solver.solve_many(Be[:64], Xc[:64], tol=TOL_ERR)  # warm-up
    net.solve(solver, th_e[:64], Be[:64], Xw[:64], tol=TOL_ERR)
    net.solve(msolver, th_e[:64], Be[:64], Xm[:64], tol=TOL_ERR)
    torch.cuda.synchronize()
    e0.record()
    ic = solver.solve_many(Be, Xc, tol=TOL_ERR)
    e1.record()
    torch.cuda.synchronize()
    t_cold = e0.elapsed_time(e1)
    e0.record()
    iw = net.solve(solver, th_e, Be, Xw, tol=TOL_ERR)
    e1.record()
    torch.cuda.synchronize()
    t_warm = e0.elapsed_time(e1)
    # the combined form: mixed-precision sweeps from the network's x0
    e0.record()
    im = net.solve(msolver, th_e, Be, Xm, tol=TOL_ERR)
    e1.record()
    torch.cuda.synchronize()
    t_mixed_warm = e0.elapsed_time(e1)
    # Control: the least-squares affine map theta -> x fitted to the same training targets
    # (x depends on theta affinely up to the noise term, so this is the natural baseline).
    Th1 = np.hstack([th_train, np.ones((n_train, 1))])
    Wls = np.linalg.lstsq(Th1, X_train.cpu().numpy(), rcond=None)[0]
    Xl = torch.from_numpy(np.hstack([th_eval, np.ones((n_eval, 1))]) @ Wls).to(dev)
    e0.record()
    il = solver.solve_many(Be, Xl, x0_zero=False, tol=TOL_ERR)
    e1.record()
    torch.cuda.synchronize()
    t_lin = e0.elapsed_time(e1)
    Xs = _normal_solution(fam.A, B_eval, fam.p)
    err = 0.0
    for X in (Xc, Xw, Xl, Xm):
        xv = X.cpu().numpy().T
        err = max(err, float(np.max(np.linalg.norm(xv - Xs, axis=0) / np.linalg.norm(Xs, axis=0))))
    solver.close()
    msolver.close()
    net.close()
    return {"workload": "A 8192x256 (A_1 6144, A_2 2048 x 0.25), b = F theta + 1e-3 noise, theta ~ U[-1,1]^16; "
                        f"MLP 16-256-256-256 trained on {n_train} library SP solutions (seed 5), {n_eval} held-out "
                        "theta (seed 55)",
            "warm_start_bf16_net": {"solves_per_s": n_eval / (t_warm * 1e-3), "max_outer_iters": iw.outer_iters},
            "cold_x0_zero": {"solves_per_s": n_eval / (t_cold * 1e-3), "max_outer_iters": ic.outer_iters},
            "linear_map_control": {"solves_per_s": n_eval / (t_lin * 1e-3), "max_outer_iters": il.outer_iters,
                                   "note": "x0 = W theta + c fitted by least squares on the training targets"},
            "mixed_bf16_warm": {"solves_per_s": n_eval / (t_mixed_warm * 1e-3), "max_refinements": im.refinements},
            "speedup": t_cold / t_warm, "speedup_mixed_warm_vs_plain_fp64": t_cold / t_mixed_warm,
            "train_loss": loss, "train_ms": t_train, "targets_ms": t_targets, "max_relerr": err,
            "checked_rhs": n_eval}


def measure_paper(ils, torch, np, dev):
    """Paper-shape replay (Sec. 5.2, Tables 2-5): A_1 = rand(p, n), A_2 = d eye(q, n), b = rand,
    x0 = 0, stop at RR = relres^2 < 1e-6, at reduced p with each table's p/n ratio and d
    scaled to keep rho at its paper-size value.  Each case times one complete setup + solve
    (CUDA events) for SP, SP-RK-RGS and SP-SCD in FP64 and checks RR on the host."""
    import math
    import workloads

    def edge(p, n):
        return p / 12.0 * (1.0 - math.sqrt(n / p)) ** 2

    gold = json.load(open(os.path.join(ROOT, "tests", "golden", "paper_tables.json")))
    paper_s = {2: {"SP": 559.3, "SP_RK_RGS": 514.6313, "SP_SCD": 227.7141},
               4: {"SP": 566.9453, "SP_RK_RGS": 466.9094, "SP_SCD": 198.2734}}
    out = {"note": "paper: MATLAB on an i7-9700 at p = 30000 (Table 2) / 50000 (Table 4), n = 13000; context only",
           "cases": []}
    for p in (5000, 10000):
        for table in (2, 4):
            p_ref = 30000 if table == 2 else 50000
            n = int(round(p * 13000 / p_ref))
            q = n if table == 2 else 1
            d = 7.0 * math.sqrt(edge(p, n) / edge(p_ref, 13000))
            inst = workloads.paper_table_workload(p, q, n, seed=table, diag=d)
            At = torch.from_numpy(np.ascontiguousarray(inst.A.T)).to(dev)
            b = torch.from_numpy(inst.b).to(dev)
            A1, A2 = inst.A[:p], inst.A[p:]
            bb = A1.T @ inst.b[:p] - A2.T @ inst.b[p:]
            row = {"table": table, "p": p, "q": q, "n": n, "diag": round(d, 4)}
            for name, kw in (("SP", dict(method=ils.ILS_SP)),
                             ("SP_RK_RGS", dict(method=ils.ILS_SP_RK_RGS, theta=1e-3, seed=table)),
                             ("SP_SCD", dict(method=ils.ILS_SP_SCD, theta=1e-3, seed=table))):
                x = torch.zeros(n, dtype=torch.float64, device=dev)
                opts = ils.options(stop_rule=ils.ILS_STOP_PAPER_RR, max_outer=gold["max_outer"], **kw)
                e0, e1 = _events(torch)
                torch.cuda.synchronize()
                e0.record()
                s = ils.Solver(At, p, opts)
                info = s.solve(b, x, tol=gold["stop_rr"])
                e1.record()
                torch.cuda.synchronize()
                xv = x.cpu().numpy()
                r = A1.T @ (inst.b[:p] - A1 @ xv) - A2.T @ (inst.b[p:] - A2 @ xv)
                rr = float(np.dot(r, r) / np.dot(bb, bb))
                row[name] = {"seconds": e0.elapsed_time(e1) / 1e3, "IT": info.outer_iters,
                             "inner_steps": info.inner_iters, "RR": rr, "RR_ok": rr < gold["stop_rr"],
                             "paper_seconds_full_size": paper_s[table][name]}
                s.close()
            out["cases"].append(row)
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
    if args.only:
        fn = {"stream": lambda: measure_stream(ils, torch, np, dev, reps=5),
              "sparse": lambda: measure_sparse(ils, torch, np, dev),
              "batched": lambda: measure_batched(ils, torch, np, dev),
              "warm": lambda: measure_warm(ils, torch, np, dev),
              "paper": lambda: measure_paper(ils, torch, np, dev)}[args.only]
        print(json.dumps(fn()), flush=True)
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
    xs = _normal_solution(inst.A, inst.b, inst.p)

    def measure(kw, steps, with_clocks):
        """Warm up, gate accuracy, then time `steps` complete solves (per-step events) with
        options.timing off; the phase times come from as many further steps on a second
        handle with options.timing on (its events and their reads stay out of the timed
        region)."""
        solver = ils.Solver(At, p, ils.options(**kw), stream=stream)
        route = "matrix_free" if ils.binding.route_model().get("matrix_free") == 1.0 else "explicit"

        def step(sv=solver):
            sv.refactor_async(At, stream=stream)
            return sv.solve(b, x, tol=TOL_ERR, stream=stream)

        # nvidia-smi starts before the warm-up so that its start-up does not overlap the
        # timed region; every sample it takes falls in the loaded warm-up or timed steps.
        sampler = ClockSampler(torch.cuda.current_device()) if (rank == 0 and with_clocks) else None
        if sampler:
            sampler.start()
        t_warm = time.perf_counter()
        while True:
            for _ in range(max(args.warmup, 3)):
                info = step()
            torch.cuda.synchronize()
            if sampler is None or time.perf_counter() - t_warm > 0.5:
                break
        relerr = float(np.linalg.norm(x.cpu().numpy() - xs) / np.linalg.norm(xs))
        if not relerr <= 1e-10:
            raise SystemExit(f"accuracy gate failed: relerr {relerr:.3e}")
        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
        phases, infos = [], []
        barrier()
        torch.cuda.synchronize()
        launches0 = ils.binding.kernel_launches()
        wall0 = time.perf_counter()
        for i in range(steps):
            flush.zero_()
            ev[i][0].record(stream)
            info = step()
            ev[i][1].record(stream)
            infos.append(info.as_dict())
        torch.cuda.synchronize()
        wall = time.perf_counter() - wall0
        launches = ils.binding.kernel_launches() - launches0
        # the last timed step's answer meets the same gate
        relerr_timed = float(np.linalg.norm(x.cpu().numpy() - xs) / np.linalg.norm(xs))
        if not relerr_timed <= 1e-10 or any(d["status"] != 0 for d in infos):
            raise SystemExit(f"accuracy gate failed after the timed steps: relerr {relerr_timed:.3e}")
        barrier()
        clocks = sampler.stop() if sampler else None
        total_s = max_over_ranks(sum(a.elapsed_time(bb) for a, bb in ev) / 1e3, world, dev)
        timed = ils.Solver(At, p, ils.options(**kw, timing=1), stream=stream)
        for _ in range(3):
            step(timed)
        for _ in range(steps):
            flush.zero_()
            step(timed)
            phases.append(timed.timings())
        timed.close()
        torch.cuda.synchronize()
        ph = {k: statistics.median(d[k] for d in phases) for k in phases[0]}
        return dict(solver=solver, total_s=total_s, wall=wall, launches=launches, clocks=clocks, relerr=relerr,
                    relerr_timed=relerr_timed, phases=ph, info=infos[-1], steps=steps, route=route)

    certified = dict(stop_rule=ils.ILS_STOP_ERR_BOUND)  # stop on kappa_est * relres <= 1e-10
    mixed = measure(dict(precision=ils.ILS_FP32_REFINE, **certified), args.steps, True)
    plain = measure(dict(**certified), max(3, min(args.steps, 10)), False)
    # the mixed form with the factorization kept in FP64 (Cholesky of Abar1 and H)
    mixed64 = measure(dict(precision=ils.ILS_FP32_REFINE, factor64=1, **certified), max(3, min(args.steps, 10)),
                      False)
    solver = mixed["solver"]
    value = replica_rate(world, args.steps, mixed["total_s"])
    plain_value = replica_rate(world, plain["steps"], plain["total_s"])
    mixed64_value = replica_rate(world, mixed64["steps"], mixed64["total_s"])

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
        solver.refactor_async(A_dev, stream=stream)
        solver.solve(b_dev, x, tol=TOL_ERR, stream=stream)
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
    # The two largest kernels of the headline step, each timed alone with CUDA events on the
    # handle's stream (options.timing):
    #  * gram_split_mma_kernel (A_1^T A_1): the method's work is p n^2 flop (FP64 Gram);
    #    the kernel executes 2 x 128 x 128 x p BF16 flop per digit product and tile pair
    #    (45 products on an off-diagonal tile pair, 25 on a diagonal one);
    #  * spd_gj_kernel: P = Abar1^{-1} by FP32 block Gauss-Jordan, n^3 multiply-adds.
    gj_ms = ph["factor"]
    gj_ach = 2.0 * n ** 3 / (gj_ms * 1e-3) / 1e12
    mma_ms = ph["gram1_mma"]
    n_tiles = (n + 127) // 128
    n_upper = n_tiles * (n_tiles + 1) // 2
    executed = 2.0 * 128 * 128 * p * ((n_upper - n_tiles) * 45 + n_tiles * 25)
    alg_flops = float(p) * n * n  # the Gram's algorithmic work
    alg_bytes = 8.0 * p * n        # A_1 read once in FP64
    mma_alg = alg_flops / (mma_ms * 1e-3) / 1e12
    roof_mma = {
        "kernel": "gram_split_mma_kernel (A_1^T A_1 to FP64 accuracy from exact BF16 digit products, tcgen05)",
        "bound": "tensor", "achieved": mma_alg, "peak": BF16_PEAK_TFLOPS, "unit": "TFLOP/s",
        "frac": mma_alg / BF16_PEAK_TFLOPS, "traffic": MMA_TRAFFIC_BYTES,
        "peak_source": "cuBLAS BF16 burst " + PEAKS["source"],
        "work": "p n^2 algorithmic flop per launch (the FP64 Gram); frac_executed counts the BF16 MMA flop run",
        "frac_executed": executed / (mma_ms * 1e-3) / 1e12 / BF16_PEAK_TFLOPS,
        "executed_over_algorithmic": executed / alg_flops,
        "traffic_ratio": MMA_TRAFFIC_BYTES / alg_bytes if MMA_TRAFFIC_BYTES else None,
        "kernel_ms": mma_ms, "share_of_step": mma_ms / ms_step, "gram_phase_ms": ph["gram1"],
    }
    roof_gj = {
        "kernel": "spd_gj_kernel<32> (P = Abar1^{-1}, FP32 block Gauss-Jordan)", "bound": "alu",
        "achieved": gj_ach, "peak": FP32_SIMT_PEAK_TFLOPS, "unit": "TFLOP/s", "frac": gj_ach / FP32_SIMT_PEAK_TFLOPS,
        "traffic": GJ_TRAFFIC_BYTES, "kernel_ms": gj_ms, "share_of_step": gj_ms / ms_step,
        "peak_source": "FP32 SIMT rate from unit counts (152 SMs x 128 lanes x 2 flop x 2.07 GHz)",
    }
    stream = measure_stream(ils, torch, np, dev)
    configs = {}
    if not args.no_configs:
        configs["sparse"] = measure_sparse(ils, torch, np, dev)
        configs["batched"] = measure_batched(ils, torch, np, dev)
        configs["warm_start"] = measure_warm(ils, torch, np, dev)
    cpu_rate, cpu_cnt, cpu_secs = time_oracle(inst, args.cpu_seconds)
    r4 = lambda v: None if v is None else float(f"{v:.4g}")
    summary = {}
    for name, c in configs.items():
        summary[name] = {k: r4(v["solves_per_s"]) for k, v in c.items() if isinstance(v, dict) and "solves_per_s" in v}
        summary[name].update({k: r4(c[k]) for k in ("speedup", "speedup_mixed_warm_vs_plain_fp64", "max_relerr")
                              if k in c})
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
        "dtype": "bf16+f32+f64",
        "data": "synthetic",
        "config": {
            "workload": WORKLOAD,
            "arithmetic": "Grams FP64-accurate from exact BF16 digit products (FP32 accumulation), P and "
                          "sweeps FP32, A^T J b FP64, residuals double-FP32 on row-scaled H",
            "stop": "kappa_est * relres <= 1e-10 (Lanczos kappa_est; ILS_STOP_ERR_BOUND)",
            "relerr_vs_oracle": r4(mixed["relerr_timed"]),
            "err_bound": r4(mixed["info"]["err_bound"]), "kappa_est": r4(mixed["info"]["kappa_est"]),
            "rho_est": r4(mixed["info"]["rho_est"]),
            "refinements": mixed["info"]["refinements"],
            "plain_fp64_sp_value": r4(plain_value),
            "speedup_vs_plain_fp64": r4(value / plain_value),
            "plain_fp64_relerr": r4(plain["relerr_timed"]),
            "mixed_fp64_factor_value": r4(mixed64_value),
            "mixed_fp64_factor_relerr": r4(mixed64["relerr_timed"]),
            "setup_phases_ms": {k: r4(v) for k, v in ph.items()},
            "routes": {"mixed": mixed["route"], "plain_fp64": plain["route"], "mixed_fp64_factor": mixed64["route"]},
            "l2": "flushed before every step (256 MiB write outside the timed events)",
            "step": "ils_refactor_async (all setup products) + ils_solve",
        },
        "roofline": roof_mma if mma_ms >= gj_ms else roof_gj,
        "kernels": {"gj_inverse": {"ms": r4(gj_ms), "frac": r4(roof_gj["frac"])},
                    "gram_mma": {"ms": r4(mma_ms), "frac": r4(roof_mma["frac"]),
                                 "frac_executed": r4(roof_mma["frac_executed"])},
                    "aq_stream_fp32": {"GBps": r4(stream["fp32"]["achieved_GBps"]), "frac": r4(stream["fp32"]["frac"])},
                    "aq_stream_bf16": {"GBps": r4(stream["bf16"]["achieved_GBps"]), "frac": r4(stream["bf16"]["frac"])},
                    "aq_stream_fp64": {"GBps": r4(stream["fp64"]["achieved_GBps"]), "frac": r4(stream["fp64"]["frac"])},
                    "aq_stream_df32": {"GBps": r4(stream["df32"]["achieved_GBps"]), "frac": r4(stream["df32"]["frac"])}},
        "tall_ms_per_solve": r4((stream.get("tall_mixed_solve") or {}).get("ms_per_solve")),
        "other_configs": summary,
        "cpu_baseline": {
            "value": cpu_rate, "unit": "solves/s", "cores": cpu_cores(), "kind": "oracle",
            "sample": f"{cpu_cnt} oracle SP solves of the same instance ({cpu_secs:.1f} s)",
        },
        "e2e": {"value": e2e_value, "unit": "solves/s", "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h},
        "gpu_launches": int(mixed["launches"]),
        "clocks": mixed["clocks"],
    }
    detail = os.environ.get("ILS_BENCH_DETAIL")
    if detail:  # the full measurements, for profiling notes
        with open(detail, "w") as f:
            json.dump({"roofline_gj": roof_gj, "roofline_mma": roof_mma, "stream": stream, "configs": configs,
                       "plain": {k: plain[k] for k in ("relerr", "relerr_timed", "phases", "info")},
                       "mixed64": {k: mixed64[k] for k in ("relerr", "relerr_timed", "phases", "info")}}, f, indent=1)
    print(json.dumps(line), flush=True)
    mixed["solver"].close()
    plain["solver"].close()
    mixed64["solver"].close()


if __name__ == "__main__":
    main()
