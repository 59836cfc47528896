"""Paper-scale solves on the 281 x 281 meshes of Sec. 5 by continuation in
bump height, the paper's route to its large-amplitude solutions.

    python -m paper_1709_08803_gb300.paper_scale --case super \
        --eps 0.1 0.5 1.0 1.25 1.5 1.75 2.0 2.25 2.5 2.75 --max-newton 60 --out super.json

Each stage starts from the previous stage's solution; the preconditioner is
factored once (it does not depend on the bottom, Sec. 4.2).  Reported per
stage: Newton and Krylov iterations, residual evaluations, wall time, the
final residual, the maximum surface height (the quantity Sec. 5 prints:
2.556 for eps = 2.75 in the supercritical case) and, for supercritical flow,
the apparent wake angle and the wave steepness of Sec. 5.2 (Fig. 6).  The
solve runs in the library's kernels; this module sequences the calls and
post-processes the downloaded surface (wake_metrics).
"""
from __future__ import annotations

import argparse
import json
import math
import sys
import time

import numpy as np


def wake_metrics(x, y, zeta, zeta_x, zeta_y, x_from: float = 15.0, x_to: float = 45.0):
    """Apparent wake angle and wave steepness of a supercritical wave pattern
    (Sec. 5.2, Fig. 6): the angle between the main V-shaped ridge and the
    centreline, and the maximum slope of the surface on the outside of that
    ridge.  The default columns, 15 <= x <= 45 on the 281 x 281 mesh of
    Sec. 5.2, start five bump widths downstream (the ridge is still curved
    nearer the bump) and stop six units short of the downstream edge.

    x (N,), y (M,): node coordinates; zeta, zeta_x, zeta_y: nodal fields
    [M, N] (row j at y[j]).  In every column with x_from <= x <= x_to the
    ridge is the crest of largest height on each side of the centreline,
    located to sub-node accuracy by the parabola through the crest node and
    its two neighbours; a least-squares line y = a + b x through the crests
    of each side gives the angle atan(b).  The steepness is the largest
    |grad zeta| over the nodes of those columns lying farther from the
    centreline than the ridge.  Returns a dict with the angle in degrees
    (mean of the two sides), both sides' angles, the steepness and the rms
    distance of the crests from the fitted lines."""
    x, y = np.asarray(x, float), np.asarray(y, float)
    zeta, zeta_x, zeta_y = (np.asarray(a, float) for a in (zeta, zeta_x, zeta_y))
    cols = np.nonzero((x >= x_from) & (x <= x_to))[0]
    if cols.size < 2:
        raise ValueError("fewer than two columns between x_from and x_to")
    dy = y[1] - y[0]
    angles, rms, steep = [], [], 0.0
    slope = np.hypot(zeta_x, zeta_y)
    for side in (1.0, -1.0):
        rows = np.nonzero(side * y > 0.0)[0]
        if rows.size < 3:
            raise ValueError("fewer than three rows on a side of the centreline")
        yr = np.empty(cols.size)
        for k, i in enumerate(cols):
            col = zeta[rows, i]
            m = int(np.argmax(col))
            off = 0.0
            if 0 < m < rows.size - 1:
                a, b, c = col[m - 1], col[m], col[m + 1]
                den = a - 2.0 * b + c
                if den < 0.0:
                    off = 0.5 * (a - c) / den
            yr[k] = y[rows[m]] + off * dy * (1.0 if rows[1] > rows[0] else -1.0)
        b, a = np.polyfit(x[cols], side * yr, 1)
        angles.append(math.degrees(math.atan(b)))
        rms.append(float(np.sqrt(np.mean((side * yr - (a + b * x[cols])) ** 2))))
        for k, i in enumerate(cols):
            outside = rows[side * y[rows] > side * yr[k]]
            if outside.size:
                steep = max(steep, float(slope[outside, i].max()))
    return {"wake_angle_deg": float(np.mean(angles)), "wake_angle_sides_deg": angles,
            "steepness": steep, "ridge_fit_rms": max(rms)}


def run(case: str, eps_list, half_band: int = 3, tol: float = 1e-8, max_newton: int = 40, log=print,
        F: float | None = None, on_stage=None, refine_below: float = 1e-5, max_krylov: int = 400,
        u0=None, eps0: float | None = None, u_prev=None, eps_prev: float | None = None, secant: bool = True):
    """Continuation in eps from the uniform stream, or from u0 (an unknown
    vector of a converged earlier stage at eps0, host array).  With secant,
    each stage after the second starts from the secant prediction through the
    two previous converged stages, u_k + (u_k - u_{k-1}) (eps - eps_k) /
    (eps_k - eps_{k-1}), instead of u_k alone (u_prev/eps_prev: the stage
    before u0, if known)."""
    import torch

    from . import bfs
    from . import workloads as W

    if case == "super":
        def cfg(e):
            return W.config_supercritical_281(e, 3.0 if F is None else F)
    else:
        cfg = W.config_subcritical_281
    mesh, topo, F0 = cfg(eps_list[0])
    opts = bfs.default_options(tol=tol, krylov_precision=bfs.BFS_FP32C, outer_precision=bfs.BFS_DF64,
                               eta=1e-2, max_newton=max_newton, max_krylov=max_krylov,
                               refine_below=refine_below, precond_precision=bfs.BFS_FP32C,
                               half_band=half_band)
    ctx = bfs.Context(mesh, topo, F0, opts)
    t0 = time.perf_counter()
    ctx.precond_factor()
    torch.cuda.synchronize()
    factor_s = time.perf_counter() - t0
    log(f"{case} 281x281 F={F0}: {ctx.n} unknowns, {ctx.pair_evals:.3e} pair evaluations per residual, "
        f"preconditioner (half band {half_band}) factored in {factor_s:.1f} s")
    u = ctx.flat_guess() if u0 is None else torch.tensor(np.asarray(u0, dtype=np.float64), device="cuda")
    last = (eps0, u.clone()) if u0 is not None else None
    before = (eps_prev, torch.tensor(np.asarray(u_prev, dtype=np.float64), device="cuda")) \
        if (u_prev is not None and eps_prev is not None) else None
    stages = []
    rep = {"case": case, "mesh": "281x281", "F": F0, "half_band": half_band, "tol": tol, "factor_s": factor_s,
           "unknowns": mesh.n_unknowns, "pair_evals_per_residual": mesh.pair_evals(), "stages": stages}
    for eps in eps_list:
        _, topo_e, _ = cfg(eps)
        ctx.set_topography(topo_e)
        if secant and last is not None and before is not None and last[0] != before[0]:
            u.copy_(last[1] + (last[1] - before[1]) * ((eps - last[0]) / (last[0] - before[0])))
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        st = ctx.solve(u, raise_on_error=False)
        torch.cuda.synchronize()
        secs = time.perf_counter() - t0
        nv = {k: v.cpu().numpy() for k, v in ctx.unpack(u).items()}
        z = nv["zeta"]
        jc = int(np.argmin(np.abs(mesh.y())))
        rec = {"eps": eps, "status": st["status"], "newton": st["newton_its"], "krylov": st["krylov_its"],
               "evals_fp32c": st["residual_evals_fp32"], "evals_fp64": st["residual_evals_fp64"],
               "fnorm_inf": st["fnorm_inf"], "seconds": secs, "zeta_max": float(z.max()),
               "zeta_min": float(z.min()), "centreline_max": float(z[jc].max())}
        if case == "super" and st["status"] == 0:
            rec.update(wake_metrics(mesh.x(), mesh.y(), z, nv["zeta_x"], nv["zeta_y"]))
        stages.append(rec)
        log(json.dumps(rec))
        if on_stage:
            on_stage(rep, eps, nv, u.cpu().numpy() if st["status"] == 0 else None)
        if st["status"] != 0:
            break
        before, last = last, (eps, u.clone())
    ctx.close()
    return rep


def wave_heights(x, y, zeta, zeta_x, zeta_y, x_from: float = 5.0, x_to: float = 15.0):
    """Transverse and divergent wave heights of a subcritical wake (Sec. 6,
    Fig. 11), downstream over x_from <= x <= x_to: the transverse height is
    half the crest-to-trough range of zeta on the centreline; the divergent
    height is the highest crest in the sector 12 to 25 degrees off the
    centreline (around the 19.47-degree Kelvin wedge edge, where the divergent
    crests meet the transverse ones); the steepness is the largest |grad zeta|
    in the whole downstream strip."""
    x, y = np.asarray(x, float), np.asarray(y, float)
    zeta = np.asarray(zeta, float)
    cols = (x >= x_from) & (x <= x_to)
    jc = int(np.argmin(np.abs(y)))
    centre = zeta[jc, cols]
    X, Y = np.meshgrid(x, y)
    ang = np.degrees(np.arctan2(np.abs(Y), np.maximum(X, 1e-12)))
    sector = (X >= x_from) & (X <= x_to) & (ang >= 12.0) & (ang <= 25.0)
    strip = (X >= x_from) & (X <= x_to)
    return {"transverse_height": float(0.5 * (centre.max() - centre.min())),
            "divergent_crest": float(zeta[sector].max()),
            "downstream_steepness": float(np.hypot(zeta_x, zeta_y)[strip].max())}


def compare_bump_pressure(eps: float = 0.285, half_band: int = 3, tol: float = 1e-8, max_newton: int = 40,
                          log=print, on_case=None, linear_check: bool = True):
    """Sec. 6, Fig. 11: flow at F = 0.6 over the Gaussian bump (delta = 0.5,
    height eps) and past the applied pressure that gives the same linear wake
    (workloads.gaussian_equivalent_pressure), on the 281 x 281 mesh of
    Sec. 5.1.  One context and one factorisation serve both problems (the
    linear Jacobian depends on neither the bottom nor the pressure, Sec. 4.2).
    Per problem: the solve's counts and wave heights; for the pair, the
    largest departure from the linear relation zeta_bump = zeta_pressure +
    F^2 p relative to the largest bump wave (zero in the linear limit).  With
    linear_check the pair is solved again at eps / 10, where the relation
    should nearly hold."""
    import torch

    from . import bfs
    from . import workloads as W

    mesh, topo_b, F = W.config_subcritical_281(eps)
    opts = bfs.default_options(tol=tol, krylov_precision=bfs.BFS_FP32C, outer_precision=bfs.BFS_DF64,
                               eta=1e-2, max_newton=max_newton, max_krylov=400, refine_below=1e-5,
                               precond_precision=bfs.BFS_FP32C, half_band=half_band)
    ctx = bfs.Context(mesh, topo_b, F, opts)
    t0 = time.perf_counter()
    ctx.precond_factor()
    torch.cuda.synchronize()
    rep = {"case": "bump_vs_pressure", "mesh": "281x281", "F": F, "delta": 0.5,
           "factor_s": time.perf_counter() - t0, "pairs": []}
    log(f"bump vs pressure 281x281 F={F}: preconditioner factored in {rep['factor_s']:.1f} s")
    for e in ([eps, eps / 10.0] if linear_check else [eps]):
        pair = {"eps": e}
        fields = {}
        for kind in ("bump", "pressure"):
            if kind == "bump":
                ctx.set_surface_pressure(None)
                ctx.set_topography(W.config_subcritical_281(e)[1])
            else:
                ctx.set_topography(W.flat_topography(mesh))
                p = W.gaussian_equivalent_pressure(mesh, e, 0.5, F)
                ctx.set_surface_pressure(p)
            u = ctx.flat_guess()
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            st = ctx.solve(u, raise_on_error=False)
            torch.cuda.synchronize()
            secs = time.perf_counter() - t0
            nv = {k: v.cpu().numpy() for k, v in ctx.unpack(u).items()}
            rec = {"status": st["status"], "newton": st["newton_its"], "krylov": st["krylov_its"],
                   "fnorm_inf": st["fnorm_inf"], "seconds": secs, "zeta_max": float(nv["zeta"].max()),
                   "zeta_min": float(nv["zeta"].min())}
            rec.update(wave_heights(mesh.x(), mesh.y(), nv["zeta"], nv["zeta_x"], nv["zeta_y"]))
            pair[kind] = rec
            fields[kind] = nv["zeta"]
            log(json.dumps({"eps": e, kind: rec}))
            if on_case:
                on_case(rep, e, kind, nv)
        if pair["bump"]["status"] == 0 and pair["pressure"]["status"] == 0:
            pz = p.reshape(mesh.M, mesh.N)
            d = fields["bump"] - (fields["pressure"] + F * F * pz)
            pair["linear_relation_defect"] = float(np.abs(d).max() / np.abs(fields["bump"]).max())
        rep["pairs"].append(pair)
        if on_case:
            on_case(rep, e, None, None)
    ctx.set_surface_pressure(None)
    ctx.close()
    return rep


def run_large(log=print, with_plain: bool = True, with_learned: bool = True, max_newton: int = 25,
              max_krylov: int = 400):
    """The large configuration (361 x 121, dx = dy = 0.2, F = 0.9, bump 0.3 plus
    a cross-stream ridge; 7.6e9 pair evaluations per residual): the mixed form
    from the uniform stream and from the guess network's output (accepted only
    through Newton, the uniform stream as fallback), and the plain FP64 form
    from the same start (by continuation in bump height, 1/3, 2/3, 1, when the
    direct solve from the uniform stream fails).  Reports each solve's counts
    and time, and how far the mixed solution lies from the FP64 one."""
    import torch

    from . import bfs
    from . import surrogate as S
    from . import workloads as W

    mesh, topo, F = W.config_large()
    mixed = bfs.default_options(tol=1e-8, krylov_precision=bfs.BFS_FP32C, outer_precision=bfs.BFS_DF64,
                                eta=1e-2, forcing=1, max_newton=max_newton, max_krylov=max_krylov,
                                refine_below=1e-5, precond_precision=bfs.BFS_FP32C)
    rep = {"case": "large", "mesh": "361x121", "F": F, "unknowns": mesh.n_unknowns, "max_krylov": max_krylov,
           "pair_evals_per_residual": mesh.pair_evals(), "solves": {}}
    ctx = bfs.Context(mesh, topo, F, mixed)
    t0 = time.perf_counter()
    ctx.precond_factor()
    torch.cuda.synchronize()
    rep["factor_s_mixed"] = time.perf_counter() - t0
    rep["precond"] = ctx.precond_info()

    def solve(c, u, name):
        torch.cuda.synchronize()
        t = time.perf_counter()
        st = c.solve(u, raise_on_error=False)
        torch.cuda.synchronize()
        rec = {"status": st["status"], "newton": st["newton_its"], "krylov": st["krylov_its"],
               "evals_fp32c": st["residual_evals_fp32"], "evals_fp64": st["residual_evals_fp64"],
               "fnorm_inf": st["fnorm_inf"], "seconds": time.perf_counter() - t}
        rep["solves"][name] = rec
        log(json.dumps({name: rec}))
        return u

    u_flat = solve(ctx, ctx.flat_guess(), "mixed_uniform_stream")
    route = "direct"
    if rep["solves"]["mixed_uniform_stream"]["status"] != 0:
        # the method without the network, as the paper reaches large
        # amplitudes: continuation in bump height, each stage from the last
        t = time.perf_counter()
        u_flat, status, cost = S.solve_with_continuation(ctx, topo, direct_first=False)
        rep["solves"]["mixed_continuation"] = {"status": status, **cost, "seconds": time.perf_counter() - t}
        log(json.dumps({"mixed_continuation": rep["solves"]["mixed_continuation"]}))
        route = "continuation"
    ctx.set_topography(topo)
    if with_learned:
        import os
        if os.path.exists(S.WEIGHTS):
            params, scale = S.load(S.WEIGHTS)
            net = S.CNO(mesh.M, mesh.N, 1)
            net.set_params(params, scale)
            x = torch.tensor(S.features(mesh, topo, F)[None], device="cuda")
            torch.cuda.synchronize()
            t = time.perf_counter()
            u = net.guess(ctx, x)
            torch.cuda.synchronize()
            guess_s = time.perf_counter() - t
            u = solve(ctx, u, "mixed_learned")
            rep["solves"]["mixed_learned"]["guess_s"] = guess_s
            if rep["solves"]["mixed_learned"]["status"] != 0:  # the method without the network
                u = solve(ctx, ctx.flat_guess(), "mixed_learned_fallback")
            net.close()
    z = ctx.unpack(u_flat)["zeta"]
    rep["zeta_max"] = float(z.max())
    ctx.close()
    if with_plain:
        ctx64 = bfs.Context(mesh, topo, F, bfs.default_options(tol=1e-8, forcing=1, max_newton=max_newton,
                                                               max_krylov=400))
        t0 = time.perf_counter()
        ctx64.precond_factor()
        torch.cuda.synchronize()
        rep["factor_s_fp64"] = time.perf_counter() - t0
        if route == "direct":
            u64 = solve(ctx64, ctx64.flat_guess(), "plain_fp64")
        else:
            t = time.perf_counter()
            u64, status, cost = S.solve_with_continuation(ctx64, topo, direct_first=False)
            rep["solves"]["plain_fp64_continuation"] = {"status": status, **cost,
                                                         "seconds": time.perf_counter() - t}
            log(json.dumps({"plain_fp64_continuation": rep["solves"]["plain_fp64_continuation"]}))
        z64 = ctx64.unpack(u64)["zeta"]
        rep["max_abs_zeta_mixed_minus_fp64"] = float((z - z64).abs().max())
        ctx64.close()
    return rep


def run_large_sequenced(log=print, half_band: int = 12, coarse_half_band: int = 6, max_newton: int = 25,
                        max_krylov: int = 150, stages=(1.0 / 3.0, 2.0 / 3.0, 1.0)):
    """Mesh sequencing for the large configuration.  At each bump height of
    the continuation, Newton first runs on the same rectangle at twice the
    spacing (dx = 0.4, 181 x 61), starting from the previous coarse stage.
    It then runs on the 361 x 121 mesh, starting from the coarse solution
    interpolated onto it (sequencing.interpolate_u), with the previous fine
    stage as the fallback start.  The mixed form throughout; half_band slices
    for the fine mesh's preconditioner (twice App. A's b = M/10, which the
    fine mesh needs at F = 0.9).  Stops at the first stage that fails."""
    import torch

    from . import bfs
    from . import surrogate as S
    from . import workloads as W
    from .sequencing import interpolate_u

    mf, topo_f, F = W.config_large()
    mc, topo_c, _ = W.config_large(2)

    def opts(hb):
        return bfs.default_options(tol=1e-8, eta=1e-2, forcing=1, half_band=hb, krylov_precision=bfs.BFS_FP32C,
                                   outer_precision=bfs.BFS_DF64, refine_below=1e-5,
                                   precond_precision=bfs.BFS_FP32C, max_newton=max_newton, max_krylov=max_krylov)

    rep = {"case": "large_sequenced", "F": F, "fine": f"{mf.N}x{mf.M}", "coarse": f"{mc.N}x{mc.M}",
           "half_band": half_band, "coarse_half_band": coarse_half_band, "max_newton": max_newton,
           "max_krylov": max_krylov, "stages": []}
    cc = bfs.Context(mc, topo_c, F, opts(coarse_half_band))
    cf = bfs.Context(mf, topo_f, F, opts(half_band))
    for name, c in (("coarse", cc), ("fine", cf)):
        torch.cuda.synchronize()
        t = time.perf_counter()
        c.precond_factor()
        torch.cuda.synchronize()
        rep[f"factor_s_{name}"] = time.perf_counter() - t

    def solve(c, u):
        torch.cuda.synchronize()
        t = time.perf_counter()
        st = c.solve(u, raise_on_error=False)
        torch.cuda.synchronize()
        z = c.unpack(u)["zeta"]
        return {"status": st["status"], "newton": st["newton_its"], "krylov": st["krylov_its"],
                "fnorm_inf": st["fnorm_inf"], "zeta_max": float(z.max()), "zeta_min": float(z.min()),
                "seconds": time.perf_counter() - t}

    uc, uf_prev = cc.flat_guess(), None
    for s in stages:
        rec = {"scale": s}
        rep["stages"].append(rec)
        cc.set_topography(S.scaled(topo_c, s))
        cf.set_topography(S.scaled(topo_f, s))
        rec["coarse"] = solve(cc, uc)
        log(json.dumps(rec))
        if rec["coarse"]["status"] != 0:
            break
        uf = torch.tensor(interpolate_u(mc, uc.cpu().numpy(), mf), device="cuda")
        rec["fine_from_coarse"] = solve(cf, uf)
        if rec["fine_from_coarse"]["status"] != 0 and uf_prev is not None:
            uf = uf_prev.clone()
            rec["fine_from_previous"] = solve(cf, uf)
        log(json.dumps(rec))
        if rec.get("fine_from_previous", rec["fine_from_coarse"])["status"] != 0:
            break
        uf_prev = uf
    cc.close()
    cf.close()
    return rep


def main(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--case", default="super", choices=["super", "sub", "compare", "large"],
                    help="compare: bump vs equivalent pressure at eps = the first --eps (Sec. 6)")
    ap.add_argument("--eps", type=float, nargs="+", default=[0.1, 0.5, 1.0, 1.5, 2.0, 2.5, 2.75])
    ap.add_argument("--F", type=float, default=None, help="Froude number of the supercritical case (3)")
    ap.add_argument("--half-band", type=int, default=None,
                    help="preconditioner half band in slices (3; 12 for --sequence)")
    ap.add_argument("--max-newton", type=int, default=40)
    ap.add_argument("--max-krylov", type=int, default=400)
    ap.add_argument("--tol", type=float, default=1e-8,
                    help="|F|inf at which a stage has converged (KINSOL's default is about 6e-6)")
    ap.add_argument("--refine-below", type=float, default=1e-5,
                    help="|F|inf below which the Newton residuals switch to double-float")
    ap.add_argument("--save-u", default=None, help="unknown vector of the last converged stage (.npz)")
    ap.add_argument("--start-u", default=None, help="start from a --save-u file instead of the uniform stream")
    ap.add_argument("--no-secant", action="store_true", help="start each stage from the previous solution only")
    ap.add_argument("--no-plain", action="store_true", help="large case: skip the plain FP64 solve")
    ap.add_argument("--sequence", action="store_true",
                    help="large case: mesh sequencing from dx = 0.4 at each continuation stage")
    ap.add_argument("--out", default=None, help="report (JSON), rewritten after every stage")
    ap.add_argument("--fields", default=None, help="surface fields of every converged stage (.npz)")
    ap.add_argument("--analyse", default=None,
                    help="recompute the wake metrics from a --fields file of a supercritical run (no GPU)")
    a = ap.parse_args(argv)
    if a.half_band is None and not (a.case == "large" and a.sequence):
        a.half_band = 3
    if a.analyse:
        from . import workloads as W
        mesh, _, _ = W.config_supercritical_281(0.1, 3.0 if a.F is None else a.F)
        d = np.load(a.analyse)
        for eps in sorted(float(k[len("zeta_eps"):]) for k in d.files if k.startswith("zeta_eps")):
            m = wake_metrics(mesh.x(), mesh.y(), *(d[f"{k}_eps{eps:g}"] for k in ("zeta", "zeta_x", "zeta_y")))
            print(json.dumps({"eps": eps, "zeta_max": float(d[f"zeta_eps{eps:g}"].max()), **m}))
        return 0
    import __graft_entry__
    __graft_entry__.build()
    saved = {}
    if a.case == "large" and a.sequence:
        rep = run_large_sequenced(log=lambda m: print(m, file=sys.stderr, flush=True),
                                  half_band=12 if a.half_band is None else a.half_band,
                                  max_newton=a.max_newton, max_krylov=a.max_krylov)
        if a.out:
            with open(a.out, "w") as fh:
                json.dump(rep, fh, indent=1)
        print(json.dumps(rep))
        return 0
    if a.case == "large":
        rep = run_large(log=lambda m: print(m, file=sys.stderr, flush=True), max_newton=a.max_newton,
                        max_krylov=a.max_krylov, with_plain=not a.no_plain)
        if a.out:
            with open(a.out, "w") as fh:
                json.dump(rep, fh, indent=1)
        print(json.dumps(rep))
        return 0
    if a.case == "compare":
        def on_case(rep, eps, kind, nv):
            if a.out:
                with open(a.out, "w") as fh:
                    json.dump(rep, fh, indent=1)
            if a.fields and kind is not None:
                for k in ("zeta", "zeta_x", "zeta_y"):
                    saved[f"{kind}_{k}_eps{eps:g}"] = nv[k]
                np.savez_compressed(a.fields, **saved)

        rep = compare_bump_pressure(a.eps[0], a.half_band, max_newton=a.max_newton,
                                    log=lambda m: print(m, file=sys.stderr, flush=True), on_case=on_case)
        print(json.dumps(rep))
        return 0

    def on_stage(rep, eps, nv, u):
        if a.out:
            with open(a.out, "w") as fh:
                json.dump(rep, fh, indent=1)
        if a.fields and rep["stages"][-1]["status"] == 0:
            for k in ("zeta", "zeta_x", "zeta_y"):
                saved[f"{k}_eps{eps:g}"] = nv[k]
            np.savez_compressed(a.fields, **saved)
        if a.save_u and u is not None:  # the last two converged stages (for a secant restart)
            prev = saved_u.get("last")
            saved_u["last"] = (u, eps)
            extra = {"u_prev": prev[0], "eps_prev": prev[1]} if prev is not None else {}
            np.savez_compressed(a.save_u, u=u, eps=eps, F=rep["F"], case=rep["case"], **extra)

    u0, eps0, u_prev, eps_prev = None, None, None, None
    saved_u = {}
    if a.start_u:
        d = np.load(a.start_u)
        u0, eps0 = d["u"], float(d["eps"])
        if "u_prev" in d.files:
            u_prev, eps_prev = d["u_prev"], float(d["eps_prev"])
            saved_u["last"] = (u0, eps0)
        print(f"starting from {a.start_u} (eps = {eps0:g})", file=sys.stderr, flush=True)
    rep = run(a.case, a.eps, a.half_band, tol=a.tol, max_newton=a.max_newton,
              log=lambda m: print(m, file=sys.stderr, flush=True), F=a.F, on_stage=on_stage,
              refine_below=a.refine_below, max_krylov=a.max_krylov, u0=u0, eps0=eps0, u_prev=u_prev,
              eps_prev=eps_prev, secant=not a.no_secant)
    print(json.dumps(rep))
    return 0


if __name__ == "__main__":
    sys.exit(main())
