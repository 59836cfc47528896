"""Paper-scale solves on the 281 x 281 meshes of Sec. 5 by continuation in
bump height, the paper's route to its large-amplitude solutions.

    python -m paper_1709_08803_gb300.paper_scale --case super \
        --eps 0.1 0.5 1.0 1.25 1.5 1.75 2.0 2.25 2.5 2.75 --max-newton 60 --out super.json

Each stage starts from the previous stage's solution; the preconditioner is
factored once (it does not depend on the bottom, Sec. 4.2).  Reported per
stage: Newton and Krylov iterations, residual evaluations, wall time, the
final residual and the maximum surface height (the quantity Sec. 5 prints:
2.556 for eps = 2.75 in the supercritical case).  Everything runs in the
library's kernels; this module only sequences the calls.
"""
from __future__ import annotations

import argparse
import json
import sys
import time

import numpy as np


def run(case: str, eps_list, half_band: int = 3, tol: float = 1e-8, max_newton: int = 40, log=print):
    import torch

    from . import bfs
    from . import workloads as W

    cfg = W.config_supercritical_281 if case == "super" else W.config_subcritical_281
    mesh, topo, F = cfg(eps_list[0])
    opts = bfs.default_options(tol=tol, krylov_precision=bfs.BFS_FP32C, outer_precision=bfs.BFS_DF64,
                               eta=1e-2, max_newton=max_newton, max_krylov=400, refine_below=1e-5,
                               precond_precision=bfs.BFS_FP32C, half_band=half_band)
    ctx = bfs.Context(mesh, topo, F, opts)
    t0 = time.perf_counter()
    ctx.precond_factor()
    torch.cuda.synchronize()
    factor_s = time.perf_counter() - t0
    log(f"{case} 281x281: {ctx.n} unknowns, {ctx.pair_evals:.3e} pair evaluations per residual, "
        f"preconditioner (half band {half_band}) factored in {factor_s:.1f} s")
    u = ctx.flat_guess()
    stages = []
    for eps in eps_list:
        _, topo_e, _ = cfg(eps)
        ctx.set_topography(topo_e)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        st = ctx.solve(u, raise_on_error=False)
        torch.cuda.synchronize()
        secs = time.perf_counter() - t0
        nv = ctx.unpack(u)
        z = nv["zeta"].cpu().numpy()
        jc = int(np.argmin(np.abs(mesh.y())))
        rec = {"eps": eps, "status": st["status"], "newton": st["newton_its"], "krylov": st["krylov_its"],
               "evals_fp32c": st["residual_evals_fp32"], "evals_fp64": st["residual_evals_fp64"],
               "fnorm_inf": st["fnorm_inf"], "seconds": secs, "zeta_max": float(z.max()),
               "zeta_min": float(z.min()), "centreline_max": float(z[jc].max())}
        stages.append(rec)
        log(json.dumps(rec))
        if st["status"] != 0:
            break
    ctx.close()
    return {"case": case, "mesh": "281x281", "F": F, "half_band": half_band, "factor_s": factor_s,
            "unknowns": mesh.n_unknowns, "pair_evals_per_residual": mesh.pair_evals(), "stages": stages}


def main(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--case", default="super", choices=["super", "sub"])
    ap.add_argument("--eps", type=float, nargs="+", default=[0.1, 0.5, 1.0, 1.5, 2.0, 2.5, 2.75])
    ap.add_argument("--half-band", type=int, default=3)
    ap.add_argument("--max-newton", type=int, default=40)
    ap.add_argument("--out", default=None)
    a = ap.parse_args(argv)
    import __graft_entry__
    __graft_entry__.build()
    rep = run(a.case, a.eps, a.half_band, max_newton=a.max_newton,
              log=lambda m: print(m, file=sys.stderr, flush=True))
    if a.out:
        with open(a.out, "w") as fh:
            json.dump(rep, fh, indent=1)
    print(json.dumps(rep))
    return 0


if __name__ == "__main__":
    sys.exit(main())
