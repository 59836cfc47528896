"""Train the learned initial guess on solutions the solver generates, and
measure what it saves.

    python -m paper_1709_08803_gb300.train_guess --train 2000 --gen-budget 1500 \
        --test 200 --out paper_1709_08803_gb300/weights/cno_181x61.npz --report report.json

1. draws problems from the batched-sweep distribution (F ~ U[0.5, 1.4], 1-3
   Gaussians or a ridge) on the 181 x 61 mesh and solves them with the mixed
   JFNK solver, directly and then by continuation in bump height, until --train
   of them have converged or --gen-budget seconds have passed (draws with no
   steady solution the solver can reach -- most of those near F = 1, with wide
   bumps or with ridges -- are counted and left out of training);
2. trains the network (BF16 tensor-core kernels, Adam) on the converged ones;
3. on the held-out problems, solves each from the uniform stream and from the
   network's guess and reports Newton iterations, Krylov iterations, residual
   evaluations and time for both; the learned guess is accepted only through
   Newton to the same tolerance, and the uniform stream is the fallback when
   it fails.
"""
from __future__ import annotations

import argparse
import json
import sys
import time

import numpy as np


def evaluate(params, scale, n_test: int, seed: int, log=print):
    """n_test held-out draws (attempts, converged or not) of the same
    distribution, three arms: the network's guess (one direct solve;
    continuation from the uniform stream if it fails), continuation from the
    uniform stream (the baseline; a direct solve is tried first), and a single
    direct solve from the uniform stream.  Costs are summed over every solve an
    arm needs."""
    import torch

    from . import surrogate as S
    from . import workloads as W

    mesh = W.config_paper_scale()[0]
    rng = np.random.default_rng(W.SEED_BASE + 9000 + seed)
    probs = [S.sample_problem_desc(rng, mesh) for _ in range(n_test)]
    net = S.CNO(mesh.M, mesh.N, 1)
    net.set_params(params, scale)
    opts = lambda Fb: S.solver_options(F=Fb)
    ctxs, rows = {}, []
    for i, (topo, F, desc) in enumerate(probs):
        c = S.bin_context(ctxs, mesh, topo, F, opts)
        rec = {"F": F, **S.describe(desc)}
        for arm in ("learned", "continuation", "flat"):
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            fallback = False
            if arm == "learned":
                c.set_topography(topo)
                x = torch.tensor(S.features(mesh, topo, F)[None], device="cuda")
                u = net.guess(c, x)
                st = c.solve(u, raise_on_error=False)
                cost = {"newton": st["newton_its"], "krylov": st["krylov_its"],
                        "evals": st["residual_evals_fp64"] + st["residual_evals_fp32"], "stages": 1}
                status = st["status"]
                if status != 0:  # fall back to the method without the network
                    fallback = True
                    u, status, c2 = S.solve_with_continuation(c, topo, direct_first=False)
                    cost = {k: cost[k] + c2[k] for k in cost}
            elif arm == "continuation":
                u, status, cost = S.solve_with_continuation(c, topo)
            else:
                c.set_topography(topo)
                u = c.flat_guess()
                st = c.solve(u, raise_on_error=False)
                status = st["status"]
                cost = {"newton": st["newton_its"], "krylov": st["krylov_its"],
                        "evals": st["residual_evals_fp64"] + st["residual_evals_fp32"], "stages": 1}
            torch.cuda.synchronize()
            rec[arm] = {"status": status, **cost, "ms": (time.perf_counter() - t0) * 1e3, "fallback": fallback}
        rows.append(rec)
        if log and (i + 1) % 20 == 0:
            log(f"evaluated {i + 1}/{n_test}")
    for c in ctxs.values():
        c.close()
    net.close()
    arms = ("learned", "continuation", "flat")
    both = [r for r in rows if r["learned"]["status"] == 0 and r["continuation"]["status"] == 0]
    direct = [r for r in both if not r["learned"]["fallback"]]

    def mean(arm, k, rs):
        return float(np.mean([r[arm][k] for r in rs])) if rs else None

    summary = {
        "test_problems": n_test, "both_converged": len(both),
        "failed": {a: sum(r[a]["status"] != 0 for r in rows) for a in arms},
        "learned_direct_success": sum(r["learned"]["status"] == 0 and not r["learned"]["fallback"] for r in rows),
        "learned_fallbacks": sum(r["learned"]["fallback"] for r in rows),
        "converged": {a: sum(r[a]["status"] == 0 for r in rows) for a in arms},
        "mean_over_both_converged": {a: {k: mean(a, k, both) for k in ("newton", "krylov", "evals", "ms")}
                                     for a in arms},
        "learned_direct_and_continuation_converged": len(direct),
        "mean_over_learned_direct": {a: {k: mean(a, k, direct) for k in ("newton", "krylov", "evals", "ms")}
                                     for a in arms},
    }
    if both:
        m = summary["mean_over_both_converged"]
        summary["newton_saved_vs_continuation"] = m["continuation"]["newton"] - m["learned"]["newton"]
        summary["krylov_saved_vs_continuation"] = m["continuation"]["krylov"] - m["learned"]["krylov"]
        summary["time_ratio_learned_over_continuation"] = m["learned"]["ms"] / m["continuation"]["ms"]
    return summary, rows


def main(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--train", type=int, default=2000, help="converged training solutions wanted")
    ap.add_argument("--gen-budget", type=float, default=None, help="seconds allowed for data generation")
    ap.add_argument("--test", type=int, default=200)
    ap.add_argument("--epochs", type=int, default=60)
    ap.add_argument("--seed", type=int, default=0)
    ap.add_argument("--out", default=None, help="weights file (.npz)")
    ap.add_argument("--report", default=None, help="JSON report")
    a = ap.parse_args(argv)

    import __graft_entry__
    __graft_entry__.build()
    from . import surrogate as S

    log = lambda m: print(m, file=sys.stderr, flush=True)
    t0 = time.time()
    xs, ys, recs = S.generate(a.train, a.seed, time_budget_s=a.gen_budget, log=log)
    n_ok = xs.shape[0]
    gen_s = time.time() - t0
    n_draws_ok = sum(r["status"] == 0 for r in recs)
    log(f"data: {n_ok} solutions ({n_draws_ok} draws converged at full height) of {len(recs)} attempts "
        f"in {gen_s:.1f} s")
    t0 = time.time()
    params, scale, losses = S.train(xs, ys, epochs=a.epochs, seed=a.seed, log=log)
    train_s = time.time() - t0
    out = a.out or S.WEIGHTS
    S.save(out, params, scale, {"losses": losses, "train_size": n_ok, "epochs": a.epochs})
    summary, rows = evaluate(params, scale, a.test, a.seed, log=log)
    rep = {"train_requested": a.train, "train_solutions": n_ok, "train_attempts": len(recs),
           "train_draws_converged": n_draws_ok,
           "attempts": recs,
           "generate_s": gen_s, "train_s": train_s, "final_loss": losses[-1], "loss_curve": losses[::5],
           "weights": out, **summary}
    if a.report:
        with open(a.report, "w") as fh:
            json.dump({"summary": rep, "rows": rows}, fh)
    print(json.dumps(rep))
    return 0


if __name__ == "__main__":
    sys.exit(main())
