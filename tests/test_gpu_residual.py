"""GPU path vs the FP64 CPU oracle, through the C ABI.

Tolerances (written here, derived in the design notes):
  FP64 residual: |F_gpu - F_oracle| <= 1e-10 * scale_row + 1e-13 per row, where
      scale_row is the sum of |terms| of that row (so the bar stays meaningful
      where F ~ 0).
  FP32C residual: 3e-7 * scale per row, about four times the largest error
      measured (5-8e-8 * scale: per-term FP32 rounding of the near field; the
      two-sum compensation removes the accumulation error).
  Converged zeta at 181 x 61: against the oracle's own root (stored by
      tests/golden/make_paper_scale_roots.py): 1e-8 for the plain FP64 solve,
      1e-6 for the mixed forms after their FP64-accurate final steps.
  Nodal reconstruction: 1e-12 absolute (same trapezoid recurrence).
"""
import math
import os

import numpy as np
import pytest

import oracle as O
from paper_1709_08803_gb300 import workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL64 = 1e-10
TOL32 = 3e-7
GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


@pytest.fixture(scope="module", autouse=True)
def _built():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1709_08803_gb300 import build
    build.build()


def _ctx(mesh, topo, F, **kw):
    from paper_1709_08803_gb300 import bfs
    return bfs.Context(mesh, topo, F, bfs.default_options(**kw))


def _dev(a):
    return torch.tensor(np.asarray(a), dtype=torch.float64, device="cuda")


MESHES = {
    "small_half_31x11": (W.config_small_half()[0], 0.7),
    "ragged_full_23x9": (W.Mesh(N=23, M=9, x1=-3.3, y1=-1.4, dx=0.3, dy=0.35), 0.8),
    "full_61x21": (W.mesh_box(61, 21, 0.3, 0.3), 0.7),
    "half_45x13": (W.Mesh(N=45, M=13, x1=-4.4, y1=0.0, dx=0.4, dy=0.4, half=1), 1.3),
    "minimum_4x3": (W.Mesh(N=4, M=3, x1=-0.6, y1=-0.3, dx=0.3, dy=0.3), 0.9),
}


def _topo(mesh):
    if mesh.N < 8:
        return W.gaussian_bumps(mesh, [(0.05, 0.5, 0.0, 0.0)])
    bumps = [(0.15, 0.8, 0.2, 0.0)] if mesh.half else [(0.15, 0.8, 0.2, 0.3), (0.08, 0.6, -0.5, -0.4)]
    return W.gaussian_bumps(mesh, bumps)


def _guesses(mesh):
    return {"flat": W.flat_guess(mesh), "smooth": W.smooth_guess(mesh, 1),
            "perturbed": W.perturbed_guess(mesh, 2, 1e-2)}


@pytest.mark.parametrize("prec", ["fp64", "df64"])
@pytest.mark.parametrize("name", list(MESHES))
def test_residual_fp64_matches_oracle(name, prec):
    """FP64 and double-float residuals both meet the FP64 bar."""
    from paper_1709_08803_gb300 import bfs
    mesh, F = MESHES[name]
    topo = _topo(mesh)
    ctx = _ctx(mesh, topo, F)
    P = O.problem(mesh, F)
    pr = bfs.BFS_FP64 if prec == "fp64" else bfs.BFS_DF64
    for gname, u in _guesses(mesh).items():
        ref, sc = O.residual(P, topo, u, with_scale=True)
        got = ctx.residual(_dev(u), precision=pr).cpu().numpy()
        err = np.abs(got - ref)
        assert np.all(err <= TOL64 * sc + 1e-13), (name, gname, float((err / (sc + 1e-300)).max()))
        assert ctx.check_finite()


@pytest.mark.parametrize("name", ["small_half_31x11", "full_61x21", "half_45x13"])
def test_residual_fp32c_error_bound(name):
    from paper_1709_08803_gb300 import bfs
    mesh, F = MESHES[name]
    topo = _topo(mesh)
    ctx = _ctx(mesh, topo, F)
    P = O.problem(mesh, F)
    for gname, u in _guesses(mesh).items():
        ref, sc = O.residual(P, topo, u, with_scale=True)
        got = ctx.residual(_dev(u), precision=bfs.BFS_FP32C).cpu().numpy()
        rel = np.abs(got - ref) / (sc + 1e-300)
        print(f"FP32C {name} {gname}: max |dF|/scale = {rel.max():.3e}")
        assert rel.max() <= TOL32, (name, gname, rel.max())


@pytest.mark.parametrize("name", ["small_half_31x11", "ragged_full_23x9"])
def test_unpack_matches_oracle(name):
    mesh, F = MESHES[name]
    ctx = _ctx(mesh, _topo(mesh), F)
    u = W.smooth_guess(mesh, 4)
    ref = O.nodal_values(O.problem(mesh, F), u)
    got = ctx.unpack(_dev(u))
    for k, v in ref.items():
        assert np.abs(got[k].cpu().numpy() - v).max() < 1e-12, k


def test_jvp_matches_oracle_difference_quotient():
    from paper_1709_08803_gb300 import bfs
    mesh, F = MESHES["ragged_full_23x9"]
    topo = _topo(mesh)
    ctx = _ctx(mesh, topo, F)
    P = O.problem(mesh, F)
    u = W.smooth_guess(mesh, 5)
    z = np.random.default_rng(9).standard_normal(mesh.n_unknowns)
    h = 1e-5
    ref = (O.residual(P, topo, u + h * z) - O.residual(P, topo, u)) / h
    Fu = ctx.residual(_dev(u))
    got = ctx.jvp(_dev(u), Fu, _dev(z), h=h, precision=bfs.BFS_FP64).cpu().numpy()
    assert np.abs(got - ref).max() <= 1e-6 * np.abs(ref).max()
    # z = 0 gives exactly zero
    zero = ctx.jvp(_dev(u), Fu, torch.zeros_like(Fu)).cpu().numpy()
    assert not zero.any()


@pytest.mark.parametrize("half_band", [0, 1, 3])
@pytest.mark.parametrize("name", ["ragged_full_23x9", "small_half_31x11"])
def test_precond_apply_matches_dense_solve(name, half_band):
    mesh, F = MESHES[name]
    ctx = _ctx(mesh, _topo(mesh), F)
    ctx.precond_factor(half_band)
    Jb = O.jtilde(O.problem(mesh, F), half_band=half_band)
    r = np.random.default_rng(11).standard_normal(mesh.n_unknowns)
    ref = np.linalg.solve(Jb, r)
    got = ctx.precond_apply(_dev(r)).cpu().numpy()
    assert ctx.check_finite()
    assert np.abs(got - ref).max() <= 1e-9 * np.abs(ref).max()
    # P z = r holds to rounding
    assert np.abs(Jb @ got - r).max() <= 1e-9 * np.abs(r).max() * np.abs(Jb).max()


# Meshes whose slice block (3(N+1) rows) spreads over more than 4 rows per SM
# (the wider register tiles of the sweep kernel) and one beyond them (the
# fallback sweep kernel).
WIDE = {
    "wide_241x3": W.mesh_box(241, 3, 0.4, 0.4),
    "wide_361x3": W.mesh_box(361, 3, 0.4, 0.4),
    "wide_409x3": W.mesh_box(409, 3, 0.4, 0.4),
}


@pytest.mark.parametrize("name", sorted(WIDE))
def test_precond_apply_wide_slices(name):
    mesh = WIDE[name]
    ctx = _ctx(mesh, W.flat_topography(mesh), 0.7)
    ctx.precond_factor(1)
    Jb = O.jtilde(O.problem(mesh, 0.7), half_band=1)
    r = np.random.default_rng(12).standard_normal(mesh.n_unknowns)
    got = ctx.precond_apply(_dev(r)).cpu().numpy()
    assert ctx.check_finite()
    # backward error of an FP64 solve (these blocks are ill-conditioned, so
    # the forward error is not a rounding-level quantity)
    assert np.abs(Jb @ got - r).max() <= 1e-9 * np.abs(r).max() * np.abs(Jb).max()


@pytest.mark.parametrize("half_band", [1, 3])
@pytest.mark.parametrize("name", ["ragged_full_23x9", "small_half_31x11", "wide_241x3", "wide_361x3"])
def test_precond_apply_fp32(name, half_band):
    """FP32 sweeps over an FP32 copy of the FP64 factors.

    Well-conditioned meshes (cond ~1e4): the backward error stays within the
    probabilistic rounding bound 4 sqrt(n) u32 (|P| |z|)_max of a length-n
    sum (Higham and Mary, SIAM J. Sci. Comput. 41, 2019), n = nd nb the
    entries one row sums, u32 = 2^-24.  Wide meshes (cond ~1e7-1e8, where any
    FP32 solve loses most digits): P z must still be within 5 % of r, i.e. the
    FP32 operator keeps the preconditioned spectrum clustered at 1 that the
    preconditioner exists for (Sec. 4.2)."""
    from paper_1709_08803_gb300 import bfs
    mesh = WIDE.get(name) or MESHES[name][0]
    F = MESHES[name][1] if name in MESHES else 0.7
    hb = min(half_band, mesh.M - 1)
    ctx = _ctx(mesh, W.flat_topography(mesh), F, precond_precision=bfs.BFS_FP32C)
    ctx.precond_factor(hb)
    Jb = O.jtilde(O.problem(mesh, F), half_band=hb)
    r = np.random.default_rng(13).standard_normal(mesh.n_unknowns)
    got = ctx.precond_apply(_dev(r)).cpu().numpy()
    assert ctx.check_finite()  # raises BfsError(BFS_ETIMEOUT) if a sweep wait gave up
    res = np.abs(Jb @ got - r).max()
    if name in WIDE:
        assert res <= 0.05 * np.abs(r).max(), res
    else:
        n = (2 * hb + 1) * 3 * (mesh.N + 1)
        u32 = 2.0 ** -24
        bound = 4.0 * math.sqrt(n) * u32 * (np.abs(Jb) @ np.abs(got)).max() + u32 * np.abs(r).max()
        assert res <= bound, (res, bound)


def test_precond_apply_before_factor_is_an_error():
    from paper_1709_08803_gb300 import bfs
    mesh, F = MESHES["minimum_4x3"]
    ctx = _ctx(mesh, _topo(mesh), F)
    with pytest.raises(bfs.BfsError) as e:
        ctx.precond_apply(_dev(np.ones(mesh.n_unknowns)))
    assert e.value.code == bfs.BFS_ENOPREC


def test_nan_input_is_flagged():
    from paper_1709_08803_gb300 import bfs
    mesh, F = MESHES["ragged_full_23x9"]
    ctx = _ctx(mesh, _topo(mesh), F)
    u = W.flat_guess(mesh)
    u[17] = np.nan
    ctx.residual(_dev(u))
    assert not ctx.check_finite()
    assert ctx.check_finite()  # the flag is cleared by the read
    st = ctx.solve(_dev(u), raise_on_error=False)
    assert st["status"] == bfs.BFS_ENAN


@pytest.mark.parametrize("kprec", ["fp64", "fp32c", "fp32c+df64", "fp32c+df64+refine", "fp32c+df64+refine+ew"])
def test_solve_small_config_matches_oracle(kprec):
    """refine: FP32C Newton residuals while |F| > 1e-5, DF64 after, FP32
    preconditioner sweeps (the bench's mixed form)."""
    from paper_1709_08803_gb300 import bfs
    mesh, topo, F = W.config_small_half()
    P = O.problem(mesh, F)
    uref, sref = O.jfnk(P, topo, W.flat_guess(mesh), tol=1e-11)
    assert sref["status"] == 0
    prec = bfs.BFS_FP64 if kprec == "fp64" else bfs.BFS_FP32C
    outer = bfs.BFS_DF64 if "df64" in kprec else bfs.BFS_FP64
    extra = dict(refine_below=1e-5, precond_precision=bfs.BFS_FP32C) if "refine" in kprec else {}
    if kprec.endswith("ew"):  # Eisenstat-Walker forcing terms
        extra["forcing"] = 1
    ctx = _ctx(mesh, topo, F, tol=1e-11, krylov_precision=prec, outer_precision=outer,
               eta=1e-4 if kprec == "fp64" else 1e-2, **extra)
    u = ctx.flat_guess()
    st = ctx.solve(u)
    print(f"solve {kprec}: {st}")
    assert st["status"] == bfs.BFS_OK and st["fnorm_inf"] <= 1e-11
    ug = u.cpu().numpy()
    zg = O.nodal_values(P, ug)["zeta"]
    zr = O.nodal_values(P, uref)["zeta"]
    assert np.abs(zg - zr).max() <= 1e-8
    # the oracle agrees that the GPU iterate is a root
    assert np.abs(O.residual(P, topo, ug)).max() <= 1e-10


def test_solve_limits_and_host_entry():
    from paper_1709_08803_gb300 import bfs
    mesh, topo, F = W.config_small_half()
    ctx = _ctx(mesh, topo, F, max_newton=1, tol=1e-12)
    st = ctx.solve(ctx.flat_guess(), raise_on_error=False)
    assert st["status"] == bfs.BFS_ENOCONV and st["newton_its"] == 1
    ctx2 = _ctx(mesh, topo, F, tol=1e-10)
    uh = W.flat_guess(mesh).copy()
    st2 = ctx2.solve_host(uh)
    assert st2["status"] == bfs.BFS_OK
    assert np.abs(O.residual(O.problem(mesh, F), topo, uh)).max() <= 1e-10
    Fh = ctx2.residual_host(uh)
    assert np.abs(Fh).max() <= 1e-10


# ---------------------------------------------------------------------------
# 181 x 61 (the paper-scale configuration), in the launch configuration the
# benchmark times.
# ---------------------------------------------------------------------------
@pytest.fixture(scope="module")
def paper_scale():
    mesh, topo, F = W.config_paper_scale(0.7)
    P = O.problem(mesh, F)
    u = W.smooth_guess(mesh, 7)
    ref, sc = O.residual(P, topo, u, with_scale=True)
    return mesh, topo, F, P, u, ref, sc


@pytest.mark.parametrize("prec", ["fp64", "df64"])
def test_paper_scale_residual_fp64(paper_scale, prec):
    from paper_1709_08803_gb300 import bfs
    mesh, topo, F, P, u, ref, sc = paper_scale
    ctx = _ctx(mesh, topo, F)
    pr = bfs.BFS_FP64 if prec == "fp64" else bfs.BFS_DF64
    got = ctx.residual(_dev(u), precision=pr).cpu().numpy()
    rel = np.abs(got - ref) / (sc + 1e-300)
    print(f"{prec} 181x61: max |dF|/scale = {rel.max():.3e}")
    assert rel.max() <= TOL64, rel.max()


def test_paper_scale_residual_fp32c(paper_scale):
    from paper_1709_08803_gb300 import bfs
    mesh, topo, F, P, u, ref, sc = paper_scale
    ctx = _ctx(mesh, topo, F)
    got = ctx.residual(_dev(u), precision=bfs.BFS_FP32C).cpu().numpy()
    rel = np.abs(got - ref) / (sc + 1e-300)
    print(f"FP32C 181x61: max |dF|/scale = {rel.max():.3e}, max |dF| = {np.abs(got - ref).max():.3e}")
    assert rel.max() <= TOL32


@pytest.mark.parametrize("form", ["fp64", "mixed", "mixed_refine"])
@pytest.mark.parametrize("F", [0.7, 1.5])
def test_paper_scale_solve_matches_oracle_root(F, form):
    """Converged zeta at 181 x 61 against the FP64 oracle's root of the same
    discrete system (its JFNK with the banded block-LU preconditioner, solved
    to |F|_inf <= 1e-11; Sec. 3.2).  fp64: FP64 residuals, Krylov and sweeps,
    solved to 1e-11 so that only the arithmetic differs: zeta within 1e-8.
    mixed: FP32C Krylov residuals, double-float Newton residuals, to the
    headline tolerance 1e-8: zeta within 1e-6.  mixed_refine (the benchmark's
    form): also FP32C Newton residuals until |F| <= 1e-5 and FP32 sweeps.
    Every converged iterate is also a root of the oracle's own residual."""
    from paper_1709_08803_gb300 import bfs
    mesh, topo, _ = W.config_paper_scale(F)
    P = O.problem(mesh, F)
    key = f"zeta_F{F:g}".replace(".", "p")
    z_orc = np.load(os.path.join(GOLDEN, "paper_scale_181x61_roots.npz"))[key]
    if form == "fp64":
        ctx = _ctx(mesh, topo, F, tol=1e-11)
        bar, res_bar = 1e-8, 1e-9
    else:
        extra = dict(refine_below=1e-5, precond_precision=bfs.BFS_FP32C) if form == "mixed_refine" else {}
        ctx = _ctx(mesh, topo, F, tol=1e-8, krylov_precision=bfs.BFS_FP32C, outer_precision=bfs.BFS_DF64,
                   eta=1e-2, **extra)
        bar, res_bar = 1e-6, 1.5e-8
    u = ctx.flat_guess()
    st = ctx.solve(u)
    ug = u.cpu().numpy()
    res = np.abs(O.residual(P, topo, ug)).max()
    z = O.nodal_values(P, ug)["zeta"].reshape(mesh.M, mesh.N)
    err = np.abs(z - z_orc).max()
    print(f"181x61 F={F} {form}: {st}; |F_oracle(u)|_inf = {res:.2e}, max |zeta - zeta_oracle| = {err:.2e}")
    assert res <= res_bar
    assert err <= bar, err
    ctx.close()


def test_set_topography_and_froude_keep_the_preconditioner():
    """Continuation in bump height (the preconditioner does not depend on the
    bottom) and a Froude-number change (the old factorisation is kept as an
    approximation): both solves reach roots the oracle accepts."""
    from paper_1709_08803_gb300 import bfs
    mesh, topo, F = W.config_small_half()
    ctx = _ctx(mesh, topo, F, tol=1e-10)
    u = ctx.flat_guess()
    assert ctx.solve(u)["status"] == 0
    bigger = W.gaussian_bumps(mesh, [(0.2, 1.0 / math.sqrt(2.0), 0.0, 0.0)])
    ctx.set_topography(bigger)
    st = ctx.solve(u)  # continue from the eps = 0.1 solution
    assert st["status"] == 0
    assert np.abs(O.residual(O.problem(mesh, F), bigger, u.cpu().numpy())).max() <= 1e-10
    ctx.set_froude(0.75)
    st = ctx.solve(u)
    assert st["status"] == 0
    assert np.abs(O.residual(O.problem(mesh, 0.75), bigger, u.cpu().numpy())).max() <= 1e-10
    with pytest.raises(bfs.BfsError):
        ctx.set_froude(0.0)
    # beta is the bottom's height: a bump of 1.1 on the bed at z = -1 tops out at z = 0.1,
    # which F = 0.7 allows (F^2/2 = 0.245) and F = 0.3 does not (0.045)
    tall = W.gaussian_bumps(mesh, [(1.1, 1.0 / math.sqrt(2.0), 0.0, 0.0)])
    assert 0.09 < tall.beta.max() < 0.11
    ctx2 = _ctx(mesh, tall, 0.7)
    with pytest.raises(bfs.BfsError):
        ctx2.set_froude(0.3)
    ctx2.set_froude(0.5)  # F^2/2 = 0.125 is above the top


@pytest.mark.parametrize("name", ["small_half_31x11", "ragged_full_23x9"])
def test_bottom_pressure_matches_oracle(name):
    mesh, F = MESHES[name]
    topo = _topo(mesh)
    ctx = _ctx(mesh, topo, F)
    u = W.smooth_guess(mesh, 6)
    pr, fr = O.bottom_pressure(O.problem(mesh, F), topo, u)
    p, f = ctx.bottom_pressure(_dev(u))
    assert np.abs(p.cpu().numpy() - pr).max() <= 1e-12 * max(1.0, np.abs(pr).max())
    assert np.abs(f - fr).max() <= 1e-10 * max(1.0, np.abs(fr).max())


def test_surface_pressure_residual_and_solve():
    """The pressure-distribution problem (flat bottom, applied surface pressure):
    residual parity with the oracle and a converged solve it accepts."""
    from oracle import linear_fft as LF
    mesh, topo, F = W.config_small_half()
    flat = W.flat_topography(mesh)
    p = LF.equivalent_pressure(lambda X, Y: 0.1 * np.exp(-(X * X + Y * Y)), F, mesh.x(), mesh.y())
    ctx = _ctx(mesh, flat, F, tol=1e-10)
    ctx.set_surface_pressure(p)
    P = O.problem(mesh, F, psurf=p)
    u = W.smooth_guess(mesh, 8)
    ref, sc = O.residual(P, flat, u, with_scale=True)
    got = ctx.residual(_dev(u)).cpu().numpy()
    assert np.all(np.abs(got - ref) <= TOL64 * sc + 1e-13)
    u0 = ctx.flat_guess()
    assert ctx.solve(u0)["status"] == 0
    assert np.abs(O.residual(P, flat, u0.cpu().numpy())).max() <= 1e-10
    ctx.set_surface_pressure(None)
    assert np.abs(ctx.residual(u0).cpu().numpy()).max() > 1e-6  # the forcing is gone


# ---------------------------------------------------------------------------
# Surface tension (Sec. 6: tension times mean curvature in the dynamic
# condition): residual parity, the preconditioner with the linearised term,
# and a converged gravity-capillary solve the oracle accepts.
# ---------------------------------------------------------------------------
@pytest.mark.parametrize("prec", ["fp64", "df64", "fp32c"])
@pytest.mark.parametrize("name", ["ragged_full_23x9", "small_half_31x11", "full_61x21", "minimum_4x3"])
def test_surface_tension_residual_matches_oracle(name, prec):
    from paper_1709_08803_gb300 import bfs
    mesh, F = MESHES[name]
    topo = _topo(mesh)
    tau = 0.3
    ctx = _ctx(mesh, topo, F, surface_tension=tau)
    P = O.problem(mesh, F, tau=tau)
    pr = {"fp64": bfs.BFS_FP64, "df64": bfs.BFS_DF64, "fp32c": bfs.BFS_FP32C}[prec]
    tol = TOL32 if prec == "fp32c" else TOL64
    for gname, u in _guesses(mesh).items():
        ref, sc = O.residual(P, topo, u, with_scale=True)
        got = ctx.residual(_dev(u), precision=pr).cpu().numpy()
        err = np.abs(got - ref)
        assert np.all(err <= tol * sc + 1e-13), (name, gname, float((err / (sc + 1e-300)).max()))


@pytest.mark.parametrize("pcprec", ["fp64", "fp32"])
@pytest.mark.parametrize("half_band", [1, 3])
@pytest.mark.parametrize("name", ["ragged_full_23x9", "small_half_31x11"])
def test_surface_tension_preconditioner(name, half_band, pcprec):
    """tau = 0.02: the discrete gravity-capillary system is ill-conditioned
    well before the critical Bond number 1/3 (cond(P) 4e8 at tau = 0.1 on the
    31 x 11 half mesh against 7e4 at tau = 0.02)."""
    from paper_1709_08803_gb300 import bfs
    mesh, F = MESHES[name]
    tau = 0.02
    pp = bfs.BFS_FP32C if pcprec == "fp32" else bfs.BFS_FP64
    ctx = _ctx(mesh, _topo(mesh), F, surface_tension=tau, precond_precision=pp)
    ctx.precond_factor(half_band)
    Jb = O.jtilde(O.problem(mesh, F, tau=tau), half_band=half_band)
    assert np.abs(Jb - O.jtilde(O.problem(mesh, F), half_band=half_band)).max() > 0.1  # the term is there
    r = np.random.default_rng(14).standard_normal(mesh.n_unknowns)
    got = ctx.precond_apply(_dev(r)).cpu().numpy()
    assert ctx.check_finite()
    res = np.abs(Jb @ got - r).max()
    # With surface tension the library keeps FP64 sweeps even when FP32 ones
    # are requested (the capillary term leaves the factors too ill-conditioned
    # for FP32 copies: an FP32 sweep misses r by 60 % on this mesh).  The
    # factors grow (inverse diagonal blocks up to 1e7), so the bar is the
    # backward error of LU without pivoting across blocks,
    # |r - P z| <= gamma_3n |L||U| |z| (Higham, Accuracy and Stability, Thm. 9.4),
    # with L, U the block factors of the slice-reordered P computed here.
    assert res <= _block_lu_bound(mesh, Jb, half_band, np.linalg.solve(Jb, r)), res


def _block_lu_bound(mesh, Jb, hb, z):
    NB, M = mesh.N + 1, mesh.M
    nb, n = 3 * NB, Jb.shape[0]
    perm = np.array([g * NB * M + l * NB + p for l in range(M) for g in range(3) for p in range(NB)])
    S = Jb[np.ix_(perm, perm)].copy()
    L, U = np.eye(n), np.zeros((n, n))
    for k in range(M):
        ks = slice(k * nb, (k + 1) * nb)
        U[ks, k * nb:] = S[ks, k * nb:]
        Dinv = np.linalg.inv(S[ks, ks])
        for i in range(k + 1, min(M, k + hb + 1)):
            rs = slice(i * nb, (i + 1) * nb)
            L[rs, ks] = S[rs, ks] @ Dinv
            S[rs, k * nb:] -= L[rs, ks] @ S[ks, k * nb:]
    g = 3 * n * 2.0 ** -53
    return g / (1 - g) * (np.abs(L) @ (np.abs(U) @ np.abs(z[perm]))).max()


@pytest.mark.parametrize("form", ["fp64", "mixed"])
def test_surface_tension_solve_is_a_root(form):
    from paper_1709_08803_gb300 import bfs
    mesh, topo, F = W.config_small_half()
    tau = 0.02
    extra = dict(krylov_precision=bfs.BFS_FP32C, outer_precision=bfs.BFS_DF64, eta=1e-2, refine_below=1e-5,
                 precond_precision=bfs.BFS_FP32C) if form == "mixed" else {}
    ctx = _ctx(mesh, topo, F, tol=1e-10, surface_tension=tau, **extra)
    u = ctx.flat_guess()
    st = ctx.solve(u)
    print(f"gravity-capillary solve ({form}): {st}")
    assert st["status"] == 0
    P = O.problem(mesh, F, tau=tau)
    ug = u.cpu().numpy()
    assert np.abs(O.residual(P, topo, ug)).max() <= 1e-10
    # and it is not the pure-gravity solution
    assert np.abs(O.residual(O.problem(mesh, F), topo, ug)).max() > 1e-6


# ---------------------------------------------------------------------------
# 361 x 121 (about 87 000 collocation points, 7.6e9 pair evaluations per
# residual): FP64 and double-float residuals against the full oracle residual,
# and the FP32C error, at a wave-like state.
# ---------------------------------------------------------------------------
@pytest.fixture(scope="module")
def large_case():
    mesh, topo, F = W.config_large()
    P = O.problem(mesh, F)
    u = W.smooth_guess(mesh, 9)
    ref, sc = O.residual(P, topo, u, with_scale=True)
    return mesh, topo, F, u, ref, sc


@pytest.mark.parametrize("prec", ["fp64", "df64", "fp32c"])
def test_large_config_residual(large_case, prec):
    from paper_1709_08803_gb300 import bfs
    mesh, topo, F, u, ref, sc = large_case
    ctx = _ctx(mesh, topo, F)
    pr = {"fp64": bfs.BFS_FP64, "df64": bfs.BFS_DF64, "fp32c": bfs.BFS_FP32C}[prec]
    got = ctx.residual(_dev(u), precision=pr).cpu().numpy()
    rel = np.abs(got - ref) / (sc + 1e-300)
    print(f"361x121 {prec}: max |dF|/scale = {rel.max():.3e}")
    assert rel.max() <= (TOL32 if prec == "fp32c" else TOL64)
    ctx.close()


# ---------------------------------------------------------------------------
# Paper scale (Sec. 5.2): the supercritical 281 x 281 mesh, F = 3, with a bump
# taller than the upstream depth (allowed: the bottom only has to stay below
# F^2/2).  FP64 and double-float residuals against the full oracle residual.
# ---------------------------------------------------------------------------
@pytest.fixture(scope="module")
def paper281():
    mesh, topo, F = W.config_supercritical_281(1.5)
    P = O.problem(mesh, F)
    u = W.smooth_guess(mesh, 10)
    ref, sc = O.residual(P, topo, u, with_scale=True)
    return mesh, topo, F, u, ref, sc


@pytest.mark.parametrize("prec", ["fp64", "df64", "fp32c"])
def test_paper_scale_281_residual(paper281, prec):
    from paper_1709_08803_gb300 import bfs
    mesh, topo, F, u, ref, sc = paper281
    assert float((topo.beta).max()) > 0.0  # the bump rises above z = 0
    ctx = _ctx(mesh, topo, F, half_band=1)
    pr = {"fp64": bfs.BFS_FP64, "df64": bfs.BFS_DF64, "fp32c": bfs.BFS_FP32C}[prec]
    got = ctx.residual(_dev(u), precision=pr).cpu().numpy()
    rel = np.abs(got - ref) / (sc + 1e-300)
    print(f"281x281 {prec}: max |dF|/scale = {rel.max():.3e}")
    assert rel.max() <= (TOL32 if prec == "fp32c" else TOL64)
