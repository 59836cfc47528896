"""Benchmark: JFNK solve time and residual pair-evaluations/s at 181 x 61.

One step = one complete Jacobian-free Newton-Krylov solve of the paper's
collocation system (181 x 61 free-surface and bottom meshes, dx = dy = 0.3,
Gaussian bump 0.2 exp(-(x^2+y^2)), F = 0.7) from the uniform-stream guess to
|F|_inf <= 1e-8, in the mixed form (FP32-compensated pair sums inside the
Jacobian-vector products, FP64 Newton residual, line search, GMRES and
preconditioner).  The preconditioner depends only on the mesh and F and is
factored once before the timed steps (its time is reported separately).

value = pair evaluations performed by all residuals of the step / step time.

--impl reference times the FP64 CPU oracle on the host cores (one full
residual per step) in the same unit.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "JFNK solve time & residual pair-evals/s at 181x61, mixed+learned vs plain FP64"
UNIT = "pair-evals/s"
# algorithmic work of the FP32C pair kernel per (target half point, source node)
# index pair: 46 FP32 ALU instructions + 5 MUFU rsqrt = 51 issue slots
INSTR_PER_INDEX_PAIR = 50  # 45 FP32 operations + 5 reciprocal square roots per index pair
FP32_OPS_PER_INDEX_PAIR = 45
MUFU_PER_INDEX_PAIR = 5  # reciprocal square roots per (target, source) index pair
# dram__bytes_read.sum + dram__bytes_write.sum of one FP32C pair-kernel launch at
# 181x61 from an ncu capture of the current kernel
PAIRS_TRAFFIC = 1.4336e6  # profiles/k_pairs_181x61.md (43 x 87 CTAs)
# dram__bytes_read.sum + dram__bytes_write.sum of one FP32 sweep launch at
# 181x61 from an ncu capture of the current kernel; None until captured
APPLY_TRAFFIC = 500.9e6  # profiles/k_apply_sweep_181x61.md


def _pc_prec(args):
    from paper_1709_08803_gb300 import bfs
    return bfs.BFS_FP32C if args.precond == "fp32" else bfs.BFS_FP64


def _peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as fh:
            return json.load(fh), "measured"
    return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "sm_max_mhz": 2070.0}, "fallback"


def measure_alu_peaks(iters: int = 16384, reps: int = 5) -> dict:
    """Roofline denominators of the pair kernels, measured on this GPU: the best
    of `reps` launches of each pipe probe of the library (FP32 FMA: the issue
    limit of FP32 work; FP32 rsqrt: the special-function unit; FP64 FMA),
    timed with CUDA events on the launching stream, in tera lane-ops/s."""
    import torch
    from paper_1709_08803_gb300 import bfs
    out = torch.empty(bfs.peak_probe_threads(), dtype=torch.float64, device="cuda")
    res = {}
    for kind, name, it in ((0, "ffma", iters), (1, "rsqrt", iters // 4), (2, "dfma", iters // 32),
                           (3, "ffma2", iters)):
        bfs.peak_probe(kind, it, out)
        best = 0.0
        for _ in range(reps):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            ops = bfs.peak_probe(kind, it, out)
            e1.record()
            e1.synchronize()
            best = max(best, ops / (e0.elapsed_time(e1) / 1e3))
        res[name + "_tops"] = best / 1e12
    return res


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled during the timed region."""
    FIELDS = ["clocks.sm", "clocks.max.sm", "power.draw", "clocks_event_reasons.hw_slowdown",
              "clocks_event_reasons.hw_thermal_slowdown", "clocks_event_reasons.sw_thermal_slowdown",
              "clocks_event_reasons.sw_power_cap"]

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), "--query-gpu=" + ",".join(self.FIELDS),
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except Exception:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if not self.proc:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 7:
                continue
            try:
                sm.append(float(parts[0]))
                mx.append(float(parts[1]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[3:7]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        return {"sm_mhz": float(np.median(sm)) if sm else None,
                "sm_max_mhz": float(max(mx)) if mx else None,
                "samples": len(sm), "reasons": sorted(reasons)}


def replica_rate(seconds: float, evals: float, pairs_per_residual: float, dist=None, device: str = "cpu"):
    """Whole-job rate of N independent replicas (one per rank): every rank's
    pair evaluations over the slowest rank's time.  Returns (rate, slowest
    seconds).  With dist (an initialised torch.distributed) the time is the
    max over ranks; every rank gets the same answer."""
    import torch
    world = dist.get_world_size() if dist else 1
    total = float(seconds)
    if dist:
        t = torch.tensor([total], dtype=torch.float64, device=device)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        total = float(t.item())
        dist.barrier()
    return world * evals * pairs_per_residual / total, total


def cpu_oracle_rate(mesh, topo, F, u, reps: int = 1):
    import oracle as O
    P = O.problem(mesh, F)
    O.residual(P, topo, u)  # load + warm
    t0 = time.perf_counter()
    for _ in range(reps):
        O.residual(P, topo, u)
    dt = (time.perf_counter() - t0) / reps
    return mesh.pair_evals() / dt, O.num_threads(), dt


def cpu_oracle_rate_one_thread(mesh, topo, F, u):
    """The same oracle residual on one host thread (the thread count restored)."""
    import oracle as O
    n = O.num_threads()
    O.set_threads(1)
    try:
        rate, _, dt = cpu_oracle_rate(mesh, topo, F, u, reps=1)
    finally:
        O.set_threads(n)
    return rate, dt


def run_reference(args):
    """The oracle on the host cores, same config, metric and unit."""
    import oracle as O
    from paper_1709_08803_gb300 import workloads as W

    O.build()
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return 0
    mesh, topo, F = W.config_paper_scale(0.7)
    u = W.smooth_guess(mesh, 7)
    P = O.problem(mesh, F)
    for _ in range(args.warmup):
        O.residual(P, topo, u)
    times = []
    for _ in range(args.steps):
        t0 = time.perf_counter()
        O.residual(P, topo, u)
        times.append(time.perf_counter() - t0)
    dt = float(np.mean(times))
    value = mesh.pair_evals() / dt
    sample = "one full FP64 residual of the 181x61 system per step (4.849e8 pair evaluations)"
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT,
            "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": dt * 1e3, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": "181x61 free surface + bottom, dx=dy=0.3, bump 0.2, F=0.7; "
                                   "oracle residual on host cores"},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": O.num_threads(), "kind": "oracle",
                             "sample": sample},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line))
    return 0


def residual_rates(mesh, topo, F, steps: int, warmup: int, precs=("fp32c", "df64", "fp64")) -> dict:
    """Residual evaluations of one configuration in each arithmetic: time per
    residual and per pair-kernel launch (CUDA events), pair-evals/s."""
    import torch

    from paper_1709_08803_gb300 import bfs
    from paper_1709_08803_gb300 import workloads as W
    ctx = bfs.Context(mesh, topo, F)
    u = torch.tensor(W.smooth_guess(mesh, 7), dtype=torch.float64, device="cuda")
    out = torch.empty_like(u)
    code = {"fp32c": bfs.BFS_FP32C, "df64": bfs.BFS_DF64, "fp64": bfs.BFS_FP64}
    res = {}
    for name in precs:
        prec = code[name]
        for _ in range(warmup):
            ctx.residual(u, out, precision=prec)
        torch.cuda.synchronize()
        ctx.profile_read()
        ctx.profile_enable(True)
        ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        ev0.record()
        for _ in range(steps):
            ctx.residual(u, out, precision=prec)
        ev1.record()
        ev1.synchronize()
        prof, _ = ctx.profile_read()
        ctx.profile_enable(False)
        ms = ev0.elapsed_time(ev1) / steps
        kern = prof[name][0] / max(prof[name][1], 1)
        res[name] = {"residual_ms": ms, "pair_kernel_ms": kern,
                     "pair_evals_per_s": ctx.pair_evals / (ms / 1e3)}
    ctx.close()
    return res


def run_residual(args):
    """Residual evaluations only (FP32C, then double-float, then FP64) at 181 x 61
    (or 361 x 121 with --config large): the pair-kernel throughput part of the
    metric, with few launches before the first pair kernel (the mode the kernel
    profiles are taken in)."""
    import torch

    import __graft_entry__
    from paper_1709_08803_gb300 import workloads as W

    torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", "0")))
    __graft_entry__.build()
    mesh, topo, F = W.config_large() if args.config == "large" else W.config_paper_scale(args.F)
    res = residual_rates(mesh, topo, F, args.steps, args.warmup)
    alu = measure_alu_peaks()
    peak = alu["ffma2_tops"]
    pairs_per_s = mesh.n_targets * mesh.n_sources / (res["fp32c"]["pair_kernel_ms"] / 1e3)
    ach = FP32_OPS_PER_INDEX_PAIR * pairs_per_s / 1e12
    print(json.dumps({"mode": "residual", "metric": f"residual pair-evals/s at {mesh.N}x{mesh.M}", "unit": UNIT,
                      "value": res["fp32c"]["pair_evals_per_s"], "steps": args.steps, "warmup": args.warmup,
                      "results": res, "roofline": {"bound": "alu", "achieved": ach, "peak": peak,
                                                   "unit": "T FP32 lane-ops/s", "frac": ach / peak,
                                                   "peak_source": "measured packed FP32x2 FMA pipe probe",
                                                   "mufu_frac": MUFU_PER_INDEX_PAIR * pairs_per_s / 1e12
                                                   / alu["rsqrt_tops"],
                                                   "measured_pipes": alu}}))
    return 0


def run_apply(args):
    """Preconditioner sweeps only (z = P^-1 r) at 181 x 61 in the mixed form's
    arithmetic (FP32 sweeps over the FP32 copy of the factors): the dominant
    kernel of the solve, timed alone with CUDA events (burst HBM peak)."""
    import torch

    import __graft_entry__
    from paper_1709_08803_gb300 import bfs
    from paper_1709_08803_gb300 import workloads as W

    torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", "0")))
    __graft_entry__.build()
    mesh, topo, F = W.config_paper_scale(args.F)
    ctx = bfs.Context(mesh, topo, F, bfs.default_options(precond_precision=_pc_prec(args)))
    ctx.precond_factor()
    r = torch.tensor(W.perturbed_guess(mesh, 3, 1.0), dtype=torch.float64, device="cuda")
    z = torch.empty_like(r)
    for _ in range(args.warmup):
        ctx.precond_apply(r, out=z)
    torch.cuda.synchronize()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.nvtx.range_push("timed")
    ev0.record()
    for _ in range(args.steps):
        ctx.precond_apply(r, out=z)
    ev1.record()
    torch.cuda.nvtx.range_pop()
    ev1.synchronize()
    ms = ev0.elapsed_time(ev1) / args.steps
    pinfo = ctx.precond_info()
    h = pinfo["half_band"]
    nb = 3 * (mesh.N + 1)
    blocks = sum(min(k, h) + 1 + min(mesh.M - 1 - k, h) for k in range(mesh.M))
    esz = 4 if args.precond == "fp32" else 8
    nbytes = blocks * nb * nb * esz + 6 * ctx.n * 8
    peaks, src = _peaks()
    hbm = float(peaks.get("hbm_gbs", 6800.0))
    ach = nbytes / (ms / 1e3) / 1e9
    print(json.dumps({"mode": "apply", "metric": "preconditioner sweeps at 181x61", "unit": "ms",
                      "value": ms, "steps": args.steps, "warmup": args.warmup,
                      "sweep_steps": pinfo["sweep_steps"], "sweep_chains": pinfo["chains"],
                      "us_per_sweep_step": ms * 1e3 / pinfo["sweep_steps"],
                      "roofline": {"bound": "hbm", "achieved": ach, "peak": hbm, "unit": "GB/s",
                                   "frac": ach / hbm, "algorithmic_bytes": nbytes,
                                   "peak_source": f"hbm_gbs of the {src} peaks file"}}))
    ctx.close()
    return 0


def run_factor(args):
    """The preconditioner factorisation alone at 181 x 61 (or 361 x 121 with
    --config large) in the mixed form's arithmetic (double-float products and
    inversions for the FP32 sweeps, --precond fp64 for the FP64 one): what a
    new (mesh, F) pays once before its first solve.  Wall time of
    bfs_precond_factor, which synchronises (host table build included)."""
    import torch

    import __graft_entry__
    from paper_1709_08803_gb300 import bfs
    from paper_1709_08803_gb300 import workloads as W

    torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", "0")))
    __graft_entry__.build()
    if args.config == "large":
        mesh, topo, F = W.config_large()
    else:
        mesh, topo, F = W.config_paper_scale(args.F)
    ctx = bfs.Context(mesh, topo, F, bfs.default_options(precond_precision=_pc_prec(args)))
    for _ in range(args.warmup):
        ctx.precond_factor()
    torch.cuda.synchronize()
    times = []
    for _ in range(args.steps):
        t0 = time.perf_counter()
        ctx.precond_factor()
        torch.cuda.synchronize()
        times.append((time.perf_counter() - t0) * 1e3)
    pinfo = ctx.precond_info()
    print(json.dumps({"mode": "factor", "metric": f"preconditioner factorisation at {mesh.N}x{mesh.M}",
                      "unit": "ms", "value": min(times), "mean_ms": sum(times) / len(times), "steps": args.steps,
                      "warmup": args.warmup, "half_band": pinfo["half_band"], "twist": pinfo["twist"],
                      "precond": args.precond, "slice_block": 3 * (mesh.N + 1)}))
    ctx.close()
    return 0


def batch_summary(args, steps: int, warmup: int) -> dict:
    """Batched sweep: args.batch instances (F ~ U[0.5, 1.4], 1-3 Gaussians or a
    ridge, meshes 61x21 ... 241x81) solved in lockstep; one step = one batched
    solve from the uniform-stream guesses.  Preconditioners are factored and
    the persistent kernel's tile shape is tuned before the timed steps."""
    import torch

    from paper_1709_08803_gb300 import bfs
    from paper_1709_08803_gb300 import workloads as W

    meshes, topos, Fs = W.config_batch(seed=3, B=args.batch)
    opts = bfs.default_options(tol=1e-8, krylov_precision=bfs.BFS_FP32C, outer_precision=bfs.BFS_DF64,
                               eta=args.eta, max_newton=30, max_krylov=80, time_budget_s=60.0,
                               precond_precision=_pc_prec(args), refine_below=args.refine_below,
                               stall_newton=3, forcing=args.forcing)
    # the lockstep solve waits for its slowest instance: with 400 GMRES
    # iterations per Newton step (what the supercritical draws need) one more
    # of the 64 converged (13) and the solve ran into its 60 s budget
    t0 = time.perf_counter()
    b = bfs.Batch(meshes, topos, Fs, opts)
    setup_s = time.perf_counter() - t0
    t0 = time.perf_counter()
    tuned_ms = b.autotune()
    tune = b.tuning()
    tune_s = time.perf_counter() - t0
    us0 = b.flat_guesses()
    us = [torch.empty_like(u) for u in us0]
    # warm-up solve (also factors every preconditioner: reported, not timed)
    t0 = time.perf_counter()
    for u, v in zip(us, us0):
        u.copy_(v)
    b.solve(us)
    torch.cuda.synchronize()
    first_s = time.perf_counter() - t0
    for _ in range(max(0, warmup - 1)):
        for u, v in zip(us, us0):
            u.copy_(v)
        b.solve(us)
    torch.cuda.synchronize()
    times, evals, last = [], 0.0, None
    for _ in range(steps):
        for u, v in zip(us, us0):
            u.copy_(v)
        torch.cuda.synchronize()
        ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        ev0.record()
        rc, st = b.solve(us)
        ev1.record()
        ev1.synchronize()
        times.append(ev0.elapsed_time(ev1))
        last = st
        pe = [m.pair_evals() for m in meshes]
        evals += sum(p * (s["residual_evals_fp64"] + s["residual_evals_fp32"]) for p, s in zip(pe, st))
    total_s = sum(times) / 1e3
    conv = [s["status"] == 0 for s in last]
    pair_evals_batched = b.pair_evals
    b.close()
    return {"metric": "batched sweep: pair-evals/s and solves/s", "unit": UNIT,
            "value": evals / total_s, "instances": len(meshes), "steps": steps, "warmup": warmup,
            "ms_per_step": total_s * 1e3 / steps, "solves_per_s": len(meshes) * steps / total_s,
            "converged": int(sum(conv)),
            "failed": [{"i": i, "F": Fs[i], "N": meshes[i].N, "status": last[i]["status"],
                        "fnorm_inf": last[i]["fnorm_inf"]} for i in range(len(meshes)) if not conv[i]],
            "newton_its_max": max(s["newton_its"] for s in last),
            "krylov_its_max": max(s["krylov_its"] for s in last),
            "pair_evals_per_batched_residual": pair_evals_batched,
            "batched_fp32c_residual_ms": tuned_ms, "tuning": tune,
            "setup_s": setup_s, "autotune_s": tune_s, "first_solve_incl_factor_s": first_s,
            "config": {"workload": f"{len(meshes)} instances: F~U[0.5,1.4], 1-3 Gaussians or a ridge, "
                                   "meshes 61x21..241x81, dx=dy=0.3; mixed lockstep JFNK to |F|inf<=1e-8",
                       "l2": "working set > L2 (preconditioners); sources of all instances fit in L2"}}


def run_batch(args):
    import torch

    import __graft_entry__

    torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", "0")))
    __graft_entry__.build()
    sampler = ClockSampler(0)
    sampler.start()
    res = batch_summary(args, args.steps, args.warmup)
    res["clocks"] = sampler.stop()
    print(json.dumps(dict({"mode": "batch"}, **res)))
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--F", type=float, default=0.7)
    ap.add_argument("--eta", type=float, default=1e-2)
    ap.add_argument("--forcing", type=int, default=1, choices=[0, 1],
                    help="GMRES forcing terms: 0 fixed eta, 1 Eisenstat-Walker (the default of the paper's KINSOL)")
    ap.add_argument("--refine-below", type=float, default=1e-5,
                    help="mixed form: FP32C Newton residuals while |F|inf exceeds this, DF64 after (0: DF64 throughout)")
    ap.add_argument("--precond", default="fp32", choices=["fp32", "fp64"],
                    help="storage/arithmetic of the preconditioner sweeps in the mixed form")
    ap.add_argument("--no-plain", action="store_true", help="skip the plain FP64 comparison solve")
    ap.add_argument("--no-cpu", action="store_true", help="skip the CPU oracle baseline")
    ap.add_argument("--no-large", action="store_true", help="skip the 361x121 residual throughput key")
    ap.add_argument("--no-batch", action="store_true", help="skip the batched-sweep key")
    ap.add_argument("--no-learned", action="store_true",
                    help="time the solve from the uniform stream even when trained weights exist")
    ap.add_argument("--mode", default="solve", choices=["solve", "residual", "batch", "apply", "factor"],
                    help="solve: the JFNK step; residual: residual evaluations only; "
                         "batch: the 64-instance batched sweep; apply: preconditioner sweeps only; "
                         "factor: the preconditioner factorisation only")
    ap.add_argument("--batch", type=int, default=64, help="instances in --mode batch")
    ap.add_argument("--config", default="paper", choices=["paper", "large"],
                    help="--mode residual: 181x61 (paper) or 361x121 (large)")
    args = ap.parse_args()
    if args.impl == "reference":
        return run_reference(args)
    if args.mode == "residual":
        return run_residual(args)
    if args.mode == "factor":
        return run_factor(args)
    if args.mode == "apply":
        return run_apply(args)
    if args.mode == "batch":
        return run_batch(args)

    import torch

    import __graft_entry__
    from paper_1709_08803_gb300 import bfs
    from paper_1709_08803_gb300 import workloads as W

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    __graft_entry__.build()

    mesh, topo, F = W.config_paper_scale(args.F)
    opts = bfs.default_options(tol=1e-8, krylov_precision=bfs.BFS_FP32C, outer_precision=bfs.BFS_DF64,
                               eta=args.eta, precond_precision=_pc_prec(args),
                               refine_below=args.refine_below, forcing=args.forcing)
    ctx = bfs.Context(mesh, topo, F, opts)
    pairs_per_residual = ctx.pair_evals
    n_index_pairs = mesh.n_targets * mesh.n_sources

    t0 = time.perf_counter()
    ctx.precond_factor()
    torch.cuda.synchronize()
    factor_ms = (time.perf_counter() - t0) * 1e3

    u0 = ctx.flat_guess()
    u = torch.empty_like(u0)
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")
    stream = torch.cuda.current_stream()

    # mixed+learned: the guess network's output starts Newton (inference is
    # inside the timed step); the uniform stream is the fallback
    from paper_1709_08803_gb300 import surrogate as S
    net, xfeat, cno_launches = None, None, 0
    if not args.no_learned and os.path.exists(S.WEIGHTS):
        params, scale = S.load(S.WEIGHTS)
        net = S.CNO(mesh.M, mesh.N, 1)
        net.set_params(params, scale)
        xfeat = torch.tensor(S.features(mesh, topo, F)[None], device="cuda")
        cno_launches = 9  # input cast, 4 convolutions, 3 activations, fields -> u
    fallbacks = [0]

    def solve_flat():
        u.copy_(u0)
        return ctx.solve(u)

    def solve_learned():
        # bfs_cno_solve: the guess, Newton from it, the uniform stream if that fails
        st = net.solve(ctx, xfeat, u)
        fallbacks[0] += int(st["fallback"])
        if st["status"] != 0:
            raise RuntimeError(f"solve failed: {st}")
        return st

    one_solve = solve_learned if net is not None else solve_flat

    first_ms = None
    for w in range(args.warmup):
        t0 = time.perf_counter()
        one_solve()
        torch.cuda.synchronize()
        if w == 0:  # cold: graph captures and first launches included
            first_ms = (time.perf_counter() - t0) * 1e3
    torch.cuda.synchronize()

    # ---- timed region: K device-resident solves ---------------------------
    sampler = ClockSampler(local)
    sampler.start()
    _, launches0 = ctx.profile_read()
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    step_ms, evals, stats = [], 0, []
    torch.cuda.nvtx.range_push("timed")
    for _ in range(args.steps):
        flush.fill_(1.0)  # L2 flush between steps (not timed)
        ev0 = torch.cuda.Event(enable_timing=True)
        ev1 = torch.cuda.Event(enable_timing=True)
        ev0.record(stream)
        st = one_solve()
        ev1.record(stream)
        ev1.synchronize()
        step_ms.append(ev0.elapsed_time(ev1))
        stats.append(st)
        evals += st["residual_evals_fp64"] + st["residual_evals_fp32"]
    torch.cuda.nvtx.range_pop()
    torch.cuda.synchronize()
    _, launches1 = ctx.profile_read()
    clocks = sampler.stop()

    # the other guess, for comparison (not in the timed region)
    other = None
    if net is not None:
        times_o, st_o = [], None
        for _ in range(max(1, min(args.steps, 3))):
            flush.fill_(1.0)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            st_o = solve_flat()
            e1.record(stream)
            e1.synchronize()
            times_o.append(e0.elapsed_time(e1))
        other = {"guess": "uniform stream", "solve_ms": float(np.mean(times_o)), "newton_its": st_o["newton_its"],
                 "krylov_its": st_o["krylov_its"], "residual_evals_fp64": st_o["residual_evals_fp64"],
                 "residual_evals_fp32": st_o["residual_evals_fp32"]}

    # ---- per-kernel split: the same solves again with CUDA events around the
    # pair kernels and the sweeps (launched one by one: events disable the
    # Arnoldi graphs), outside the timed region ------------------------------
    prof_steps = max(1, min(args.steps, 2))
    ctx.profile_read()
    ctx.profile_enable(True)
    torch.cuda.synchronize()
    t_prof = time.perf_counter()
    for _ in range(prof_steps):
        flush.fill_(1.0)
        one_solve()
    torch.cuda.synchronize()
    prof_wall_ms = (time.perf_counter() - t_prof) * 1e3 / prof_steps
    prof, _ = ctx.profile_read()
    ctx.profile_enable(False)
    (ms64, n64), (ms32, n32), (msdf, ndf) = prof["fp64"], prof["fp32c"], prof["df64"]
    msap, nap = prof["apply"]
    value, total_s = replica_rate(sum(step_ms) / 1e3, evals, pairs_per_residual, dist, "cuda")
    ms_per_step = total_s * 1e3 / args.steps
    status_ok = all(s["status"] == 0 for s in stats)

    # ---- end to end: host inputs in, host solution out --------------------
    e2e_times, e2e_evals = [], 0
    if net is not None:
        # the learned path a user runs: features from pinned host memory, the
        # guess network, the solve, the solution read back
        feat_host = torch.tensor(S.features(mesh, topo, F)[None]).pin_memory()
        out_host = torch.empty(ctx.n, dtype=torch.float64).pin_memory()
        feat_np, out_np = feat_host.numpy(), out_host.numpy()
        h2d, d2h = feat_host.numel() * 4, 8 * ctx.n
        for i in range(max(1, min(args.steps, 3))):
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            st = net.solve_host(ctx, feat_np, out_np)  # bfs_cno_solve_host: copies in and out inside
            fallbacks[0] += int(st["fallback"])
            torch.cuda.synchronize()
            e2e_times.append(time.perf_counter() - t0)
            e2e_evals += st["residual_evals_fp64"] + st["residual_evals_fp32"]
        e2e_entry = "bfs_cno_solve_host: features (pinned host) -> guess network -> bfs_solve (uniform stream as fallback) -> u (pinned host)"
    else:
        u_host = np.ascontiguousarray(u0.cpu().numpy())
        pin = torch.empty(ctx.n, dtype=torch.float64).pin_memory()
        pin_np = pin.numpy()
        h2d, d2h = 8 * ctx.n, 8 * ctx.n
        for i in range(max(1, min(args.steps, 3))):
            pin_np[:] = u_host
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            st = ctx.solve_host(pin_np)
            e2e_times.append(time.perf_counter() - t0)
            e2e_evals += st["residual_evals_fp64"] + st["residual_evals_fp32"]
        e2e_entry = "bfs_solve_host"
    e2e_value, _ = replica_rate(sum(e2e_times), e2e_evals, pairs_per_residual, dist, "cuda")

    # ---- plain FP64 solve for comparison (not in the timed region) --------
    plain = None
    if not args.no_plain and rank == 0:
        # the same Newton-Krylov settings in FP64 throughout (forcing floor 1e-4)
        ctx64 = bfs.Context(mesh, topo, F, bfs.default_options(tol=1e-8, forcing=args.forcing))
        ctx64.precond_factor()
        up = ctx64.flat_guess()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        stp = ctx64.solve(up)
        torch.cuda.synchronize()
        plain = {"solve_ms": (time.perf_counter() - t0) * 1e3, "newton_its": stp["newton_its"],
                 "krylov_its": stp["krylov_its"], "residual_evals_fp64": stp["residual_evals_fp64"],
                 "fnorm_inf": stp["fnorm_inf"],
                 "u_max_abs_diff_vs_mixed": float((up - u).abs().max().item())}
        ctx64.close()

    # ---- roofline of the dominant kernel (FP32C pair kernel) --------------
    peaks, src = _peaks()
    sm_mhz_max = float(peaks.get("sm_max_mhz", 2070.0))
    sms = torch.cuda.get_device_properties(local).multi_processor_count
    alu = measure_alu_peaks()
    avg32 = ms32 / max(n32, 1)
    pairs_per_s = n_index_pairs / (avg32 / 1e3) if n32 else None
    # the binding pipe: the 45 FP32 operations of an index pair on the FMA pipe
    # (128 lane-ops/clk/SM whether packed or not; packing only halves the issue
    # slots), ahead of its 5 reciprocal square roots on the special-function
    # unit (16 lanes/clk/SM)
    achieved = FP32_OPS_PER_INDEX_PAIR * pairs_per_s / 1e12 if n32 else None
    roofline_pairs = {"bound": "alu", "kernel": "k_pairs<float> (FP32C all-pairs quadrature, packed FP32x2)",
                "achieved": achieved, "peak": alu["ffma2_tops"], "unit": "T FP32 lane-ops/s",
                "frac": (achieved / alu["ffma2_tops"]) if achieved else None,
                # dram bytes read + written per launch, from an ncu capture of this kernel at 181x61
                "traffic": PAIRS_TRAFFIC if args.F == 0.7 else None,
                "peak_source": "measured: packed FP32x2 FMA throughput of the library's pipe probe on this "
                               "GPU (best of 5 launches, CUDA events)",
                "mufu": {"achieved": MUFU_PER_INDEX_PAIR * pairs_per_s / 1e12 if n32 else None,
                         "peak": alu["rsqrt_tops"], "unit": "Trsqrt/s",
                         "frac": (MUFU_PER_INDEX_PAIR * pairs_per_s / 1e12 / alu["rsqrt_tops"])
                         if n32 else None,
                         "peak_source": "measured rsqrtf throughput (pipe probe)"},
                "peak_derived": sms * 128 * sm_mhz_max * 1e6 / 1e12,
                "peak_derived_source": f"{sms} SMs x 128 FP32 lanes x {sm_mhz_max:.0f} MHz "
                                       f"(max SM clock, {src} peaks file)",
                "measured_pipes": alu,
                "avg_launch_ms": avg32, "launches": n32,
                "fp64_pair_kernel_avg_ms": ms64 / max(n64, 1) if n64 else None,
                "df64_pair_kernel_avg_ms": msdf / max(ndf, 1) if ndf else None,
                "share_of_step": (ms32 + ms64 + msdf) / (prof_wall_ms * prof_steps)}
    # the preconditioner apply streams every stored factor block once (HBM-bound)
    pinfo = ctx.precond_info()
    h = pinfo["half_band"]
    nb = 3 * (mesh.N + 1)
    blocks = sum(min(k, h) + 1 + min(mesh.M - 1 - k, h) for k in range(mesh.M))
    esz = 4 if args.precond == "fp32" else 8
    apply_bytes = blocks * nb * nb * esz + 6 * ctx.n * 8
    avg_ap = msap / max(nap, 1)
    hbm = float(peaks.get("hbm_gbs", 6800.0))
    roofline_apply = {"bound": "hbm",
                      "kernel": ("k_apply_sweep (FP32 block-banded LU sweeps, task table, bulk-copy ring)"
                                 if esz == 4 else "k_apply_coop (FP64 block-banded LU sweeps)"),
                      "sweep_steps": pinfo["sweep_steps"], "sweep_chains": pinfo["chains"],
                      "us_per_sweep_step": avg_ap * 1e3 / pinfo["sweep_steps"] if nap else None,
                      "achieved": apply_bytes / (avg_ap / 1e3) / 1e9 if nap else None, "peak": hbm,
                      "unit": "GB/s", "frac": (apply_bytes / (avg_ap / 1e3) / 1e9) / hbm if nap else None,
                      # dram bytes read + written per launch, from an ncu capture of this kernel at 181x61
                      "traffic": APPLY_TRAFFIC if (esz == 4 and args.F == 0.7) else None,
                      "algorithmic_bytes": apply_bytes, "avg_launch_ms": avg_ap,
                      "launches": nap, "peak_source": f"hbm_gbs of the {src} peaks file",
                      "share_of_step": msap / (prof_wall_ms * prof_steps)}
    roofline = roofline_apply if msap > ms32 + msdf + ms64 else roofline_pairs
    breakdown = {"source": f"{prof_steps} extra solve(s) with CUDA events around the kernels (Arnoldi "
                           "steps launched one by one), outside the timed region",
                 "solve_ms": prof_wall_ms,
                 "pair_fp32c_ms": ms32 / prof_steps, "pair_df64_ms": msdf / prof_steps,
                 "pair_fp64_ms": ms64 / prof_steps, "precond_apply_ms": msap / prof_steps,
                 "precond_apply_avg_ms": msap / max(nap, 1),
                 "other_ms": prof_wall_ms - (ms32 + msdf + ms64 + msap) / prof_steps}

    cpu = None
    if rank == 0 and not args.no_cpu:
        rate, cores, dt = cpu_oracle_rate(mesh, topo, F, W.smooth_guess(mesh, 7), reps=1)
        rate1, dt1 = cpu_oracle_rate_one_thread(mesh, topo, F, W.smooth_guess(mesh, 7))
        cpu = {"value": rate, "unit": UNIT, "cores": cores, "kind": "oracle",
               "sample": f"one full FP64 oracle residual at 181x61 ({mesh.pair_evals():.3e} pair "
                         f"evaluations, {dt:.2f} s)",
               "one_thread": {"value": rate1, "seconds": dt1}}

    # ---- the large configuration (361 x 121, 7.6e9 pair evaluations per
    # residual): residual throughput beside the oracle's, outside the timed region
    large = None
    if rank == 0 and not args.no_large:
        m5, t5, F5 = W.config_large()
        r5 = residual_rates(m5, t5, F5, steps=5, warmup=2, precs=("fp32c", "df64"))
        large = {"workload": "361x121 free surface + bottom, dx=dy=0.2, x in [-20,52], y in [-12,12], "
                             "F=0.9, bump 0.3 exp(-(x^2+y^2)) + ridge 0.005 exp(-(x-5)^2/2)",
                 "pair_evals_per_residual": m5.pair_evals(),
                 "fp32c_pair_evals_per_s": r5["fp32c"]["pair_evals_per_s"],
                 "fp32c_pair_kernel_ms": r5["fp32c"]["pair_kernel_ms"],
                 "df64_pair_evals_per_s": r5["df64"]["pair_evals_per_s"]}
        if not args.no_cpu:
            rate5, cores5, dt5 = cpu_oracle_rate(m5, t5, F5, W.smooth_guess(m5, 7), reps=1)
            large["oracle_pair_evals_per_s"] = rate5
            large["oracle_cores"] = cores5
            large["oracle_sample"] = f"one full FP64 oracle residual ({dt5:.2f} s)"

    # ---- the batched sweep (64 uneven instances, lockstep): one solve after a
    # warm-up that factors the preconditioners, outside the timed region
    batch = None
    if rank == 0 and world == 1 and not args.no_batch:
        batch = batch_summary(args, steps=1, warmup=1)

    if rank == 0:
        line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": ms_per_step, "higher_is_better": True,
                "scaling": "weak", "vs_baseline": None, "dtype": "f32c+df64+f64", "data": "synthetic",
                "config": {"workload": "181x61 free surface + bottom, dx=dy=0.3, x in [-15,39], "
                                       "y in [-9,9], beta=-1+0.2exp(-(x^2+y^2)), F=%.2f; mixed JFNK "
                                       "solve to |F|inf<=1e-8 from %s" % (
                                           F, "the guess network's output (inference timed; the uniform "
                                              "stream as fallback)" if net is not None else "the uniform stream"),
                           "form": "mixed: FP32C residuals inside Jv; Newton residual and line search in "
                                   "double-float (FP64-accurate, 1e-10 per-row parity); FP64 GMRES and "
                                   "banded-LU factorisation; preconditioner sweeps in %s; Newton residuals in "
                                   "FP32C while |F|inf > %g, double-float after; %s GMRES forcing; %s" % (
                                       "FP32 over FP32 copies of the factors" if args.precond == "fp32" else "FP64",
                                       args.refine_below,
                                       "Eisenstat-Walker" if args.forcing == 1 else "fixed",
                                       "learned initial guess" if net is not None else "no learned guess"),
                           "l2": "flushed between steps (256 MiB write); sources fit in L2",
                           "parallelism": "replicas" if world > 1 else "single GPU",
                           "precond_half_band": int(opts.half_band if opts.half_band > 0 else max(1, round(mesh.M / 20))),
                           "precond_factor_ms_untimed": factor_ms},
                "solve": {"newton_its": stats[-1]["newton_its"], "krylov_its": stats[-1]["krylov_its"],
                          "residual_evals_fp64": stats[-1]["residual_evals_fp64"],
                          "residual_evals_fp32": stats[-1]["residual_evals_fp32"],
                          "fnorm_inf": stats[-1]["fnorm_inf"], "all_converged": status_ok,
                          "guess": "learned" if net is not None else "uniform stream",
                          "learned_fallbacks": fallbacks[0] if net is not None else None,
                          "step_ms": step_ms},
                "first_solve_ms": (factor_ms + first_ms) if first_ms is not None else None,
                "first_solve_parts": {"precond_factor_ms": factor_ms, "first_solve_ms": first_ms,
                                      "note": "untimed: a new (mesh, F) pays the factorisation once; "
                                              "the first solve also captures its step graphs"},
                "step_graphs": ctx.solver_info(),
                "other_guess": other,
                "plain_fp64": plain,
                "step_breakdown": breakdown,
                "roofline": roofline, "roofline_pairs": roofline_pairs, "roofline_apply": roofline_apply,
                "cpu_baseline": cpu,
                "large_361x121": large,
                "batch_64": batch,
                "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": h2d,
                        "d2h_bytes_per_step": d2h, "entry": e2e_entry,
                        "ms_per_step": 1e3 * sum(e2e_times) / len(e2e_times), "steps": len(e2e_times)},
                "gpu_launches": int(launches1 - launches0) + cno_launches * args.steps,
                "launches_before_timed": int(launches0),
                "clocks": clocks}
        print(json.dumps(line))
    if net is not None:
        net.close()
    ctx.close()
    if dist:
        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
