"""Pins of the FP64 CPU oracle against what the paper and the mathematics fix.

Each test names the pin it realises and the passage it follows.  None of them
re-types an oracle formula: the expected values come from closed forms,
Green's identity, adaptive quadrature, printed App. B entries, exact identities
of the discretisation (trapezoid, central differences) or the exact linear
solution.
"""
import math
import os

import numpy as np
import pytest

import oracle as O
from oracle import linear_fft as LF
from paper_1709_08803_gb300 import workloads as W

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


# ---------------------------------------------------------------------------
# P1: the uniform stream over a flat bottom solves the discrete system.
# (zeta = 0, phi = psi = x: every integrand has a zero factor, Bernoulli
# gives 1/2 - 1/2, the radiation conditions vanish; Sec. 2.1, 3.1.)
# ---------------------------------------------------------------------------
@pytest.mark.parametrize("half", [0, 1])
@pytest.mark.parametrize("sigma", [-1.0, 1.0])
def test_uniform_stream_is_a_root(half, sigma):
    mesh = W.mesh_box(17, 7, 0.4, 0.3, half=half)
    P = O.problem(mesh, 0.8, sigma=sigma)
    r = O.residual(P, W.flat_topography(mesh), W.flat_guess(mesh))
    assert np.abs(r).max() < 1e-12


# ---------------------------------------------------------------------------
# P2: closed-form integral of S2 over a rectangle (Sec. 3.1) against adaptive
# 2-D quadrature, including rectangles that contain the singular point and
# rectangles with the singular point on an edge (targets on the outer rows).
# ---------------------------------------------------------------------------
@pytest.mark.parametrize("A,B,C,s1,s2,t1,t2", [
    (1.3, 0.4, 1.1, 0.5, 3.0, 0.7, 2.0),
    (1.3, 0.4, 1.1, -2.0, 3.0, -1.5, 2.0),
    (1.0, 0.0, 1.0, -1.0, 2.0, 0.0, 3.0),
    (1.2, -0.5, 1.4, -3.0, -0.2, -2.0, 0.0),
    (1.05, 0.3, 1.02, -6.15, 5.85, -4.0, 0.0),
    (2.0, 1.9, 1.5, -0.3, 0.2, -0.25, 0.35),
])
def test_rect_S2_against_quadrature(A, B, C, s1, s2, t1, t2):
    from scipy import integrate
    f = lambda t, s: 1.0 / math.sqrt(A * s * s + B * s * t + C * t * t)
    ref = 0.0
    for sa, sb in ((s1, min(s2, 0.0)), (max(s1, 0.0), s2)):
        if sb <= sa:
            continue
        for ta, tb in ((t1, min(t2, 0.0)), (max(t1, 0.0), t2)):
            if tb <= ta:
                continue
            ref += integrate.dblquad(f, sa, sb, ta, tb, epsabs=1e-13, epsrel=1e-13)[0]
    assert abs(O.rect_S2(A, B, C, s1, s2, t1, t2) - ref) < 1e-11 * max(1.0, abs(ref))


# ---------------------------------------------------------------------------
# P3: Green's second identity for a harmonic function (Sec. 2.2).
# For u harmonic between two non-flat sheets, with double-layer density u and
# single-layer density grad(u).(outward normal) dS/dxdy, the operator the
# residual is built on must return 2 pi u* at a point of either sheet.  The
# self-sheet double layer has a far field that the truncated mesh cuts off;
# it is added back with the exact solid angle of the rectangle.
# ---------------------------------------------------------------------------
_SING = [((0.2, 0.1, 1.2), 1.0), ((-0.3, 0.2, -2.0), 0.5)]


def _u(x, y, z):
    u = gx = gy = gz = 0.0
    for (sx, sy, sz), q in _SING:
        dx, dy, dz = x - sx, y - sy, z - sz
        r = np.sqrt(dx * dx + dy * dy + dz * dz)
        u = u + q / r
        gx = gx - q * dx / r ** 3
        gy = gy - q * dy / r ** 3
        gz = gz - q * dz / r ** 3
    return u, gx, gy, gz


def _top(x, y):
    e = 0.15 * np.exp(-(x * x + y * y) / 2.0)
    return e, -x * e, -y * e


def _bot(x, y):
    e = 0.2 * np.exp(-((x - 0.5) ** 2 + y * y) / 2.0)
    return -1.0 + e, -(x - 0.5) * e, -y * e


def _omega_rect(s1, s2, t1, t2, c):
    f = lambda s, t: math.atan(s * t / (c * math.sqrt(s * s + t * t + c * c)))
    return f(s2, t2) - f(s1, t2) - f(s2, t1) + f(s1, t1)


def _harmonic_defect(L, h, bottom_sign=1.0):
    N = int(round(2 * L / h)) + 1
    mesh = W.Mesh(N=N, M=N, x1=-L, y1=-L, dx=h, dy=h)
    P = O.problem(mesh, 1.0)
    X, Y = np.meshgrid(mesh.x(), mesh.y())
    zt, ztx, zty = _top(X, Y)
    bt, btx, bty = _bot(X, Y)
    u, gx, gy, gz = _u(X, Y, zt)
    ub, bgx, bgy, bgz = _u(X, Y, bt)
    top = dict(h=zt, hx=ztx, hy=zty, d=u, s=-gx * ztx - gy * zty + gz)
    bot = dict(h=bt, hx=btx, hy=bty, d=ub, s=bottom_sign * (bgx * btx + bgy * bty - bgz))
    k = l = (N - 1) // 2
    xs, ys = -L + (k + 0.5) * h, -L + l * h
    s1, s2, t1, t2 = -L - xs, L - xs, -L - ys, L - ys
    out = []
    for self_bottom in (0, 1):
        if self_bottom:
            z, px, py = _bot(xs, ys)
            uu, g1, g2, g3 = _u(xs, ys, z)
            sd = bottom_sign * (px * g1 + py * g2 - g3)
            far = -1.0
        else:
            z, px, py = _top(xs, ys)
            uu, g1, g2, g3 = _u(xs, ys, z)
            sd = -px * g1 - py * g2 + g3
            far = 0.0
        v, _ = O.bie_point(P, top, bot, self_bottom, dict(x=xs, y=ys, z=z, u=uu, sd=sd, px=px, py=py))
        # far field of the self double layer beyond the mesh: -u* times the
        # integral of K1 (top) or -K1 (bottom) over the flat exterior
        ext = math.copysign(2 * math.pi - _omega_rect(s1, s2, t1, t2, abs(far - z)), far - z)
        v += -uu * ext if not self_bottom else uu * ext
        out.append(v - 2 * math.pi * uu)
    return out


def test_green_identity_harmonic():
    d_top, d_bot = _harmonic_defect(12.0, 0.2)
    # 2 pi u* is about 7 (top) and 5.6 (bottom)
    assert abs(d_top) < 3e-3 and abs(d_bot) < 3e-3
    # the coarse mesh is worse but still close
    c_top, c_bot = _harmonic_defect(6.0, 0.4)
    assert abs(c_top) < 1.5e-2 and abs(c_bot) < 1.5e-2


def test_green_identity_fails_with_inward_bottom_flux():
    """The bottom single-layer density must be the OUTWARD flux
    grad(u).(beta_x, beta_y, -1).  For the flow, grad(Phi - x) . (beta_x,
    beta_y, -1) = -beta_x by the bottom kinematic condition (Sec. 2.1), which
    is why the residual uses sigma = -1 on the printed I4."""
    d_top, d_bot = _harmonic_defect(12.0, 0.2, bottom_sign=-1.0)
    assert abs(d_top) > 0.3 and abs(d_bot) > 0.3


# ---------------------------------------------------------------------------
# Nodal reconstruction: the trapezoid rule is exact for quadratic q (linear
# q_x) and the second-order y stencils are exact for quadratics (Sec. 3.1).
# ---------------------------------------------------------------------------
def test_reconstruction_exact_for_quadratics():
    mesh = W.Mesh(N=13, M=9, x1=-2.0, y1=-1.2, dx=0.35, dy=0.3)
    P = O.problem(mesh, 0.9)
    x, y = mesh.x(), mesh.y()
    X, Y = np.meshgrid(x, y)
    per, blk = mesh.N + 1, (mesh.N + 1) * mesh.M
    u = np.zeros(mesh.n_unknowns)
    coef = [(0.3, -0.2, 0.05, 0.1, -0.07), (1.0, 0.4, -0.03, 0.2, 0.02), (-0.5, 0.1, 0.08, -0.3, 0.04)]
    exact = []
    for f, (a, b, c, d, e) in enumerate(coef):
        q = a + b * X + c * X ** 2 + d * Y + e * Y ** 2
        qx = b + 2 * c * X
        exact.append((q, qx, d + 2 * e * Y))
        for j in range(mesh.M):
            u[f * blk + j * per] = q[j, 0]
            u[f * blk + j * per + 1: f * blk + (j + 1) * per] = qx[j]
    nv = O.nodal_values(P, u)
    assert np.abs(nv["zeta"] - exact[0][0]).max() < 1e-13
    assert np.abs(nv["phi"] - exact[1][0]).max() < 1e-13
    assert np.abs(nv["psi"] - exact[2][0]).max() < 1e-13
    assert np.abs(nv["zeta_y"] - exact[0][2]).max() < 1e-12
    assert np.abs(nv["phi_y"] - exact[1][2]).max() < 1e-12


# ---------------------------------------------------------------------------
# Combined dynamic condition (Sec. 2.1): on a streamsurface of the harmonic
# potential Phi = x + b y + a z (the plane zeta = p x + q y with p + b q = a),
# its kinetic part equals |grad Phi|^2 / 2 = (1 + a^2 + b^2) / 2.
# ---------------------------------------------------------------------------
def test_dynamic_condition_on_streamsurface():
    mesh = W.Mesh(N=11, M=7, x1=-2.0, y1=-0.9, dx=0.4, dy=0.3)
    F, a, b, q = 0.8, 0.3, -0.25, 0.4
    p = a - b * q
    P = O.problem(mesh, F)
    per, blk = mesh.N + 1, (mesh.N + 1) * mesh.M
    u = W.flat_guess(mesh)
    for j, yj in enumerate(mesh.y()):
        u[j * per] = p * mesh.x1 + q * yj
        u[j * per + 1: (j + 1) * per] = p
        u[blk + j * per] = (1 + a * p) * mesh.x1 + (b + a * q) * yj
        u[blk + j * per + 1: blk + (j + 1) * per] = 1 + a * p
    r = O.residual(P, W.flat_topography(mesh), u)
    for l, yl in enumerate(mesh.y()):
        for k in range(mesh.N - 1):
            xs = mesh.x1 + (k + 0.5) * mesh.dx
            zs = p * xs + q * yl
            expect = 0.5 * (1 + a * a + b * b) + zs / F ** 2 - 0.5
            assert abs(r[l * per + 2 + k] - expect) < 1e-13


# ---------------------------------------------------------------------------
# P4: linearisation identity (Sec. 4.2, Fig. 2): at the uniform stream over a
# flat bottom, the finite-difference Jacobian of the NONLINEAR residual equals
# the Jacobian of the LINEAR discrete system of App. B.
# ---------------------------------------------------------------------------
@pytest.mark.parametrize("tau", [0.0, 0.4])
@pytest.mark.parametrize("half", [0, 1])
def test_linearisation_identity(half, tau):
    """tau > 0: the surface-tension term linearises to -tau (zeta_xx + zeta_yy)
    in the linear system, consistently with the nonlinear curvature term."""
    mesh = W.mesh_box(13, 7, 0.4, 0.4, half=half)
    P = O.problem(mesh, 0.7, tau=tau)
    Jfd = O.fd_jacobian(P, W.flat_topography(mesh), W.flat_guess(mesh))
    Jt = O.jtilde(P)
    assert np.abs(Jfd - Jt).max() < 1e-6 * np.abs(Jt).max()


def test_jtilde_block_structure():
    """Sec. 4.2: J23 = J32 and J22 = J33; the (1,3) block is zero; and the
    linear Jacobian does not depend on the sign of I4 (beta_x enters the
    linear system only additively)."""
    mesh = W.mesh_box(11, 5, 0.4, 0.4)
    Jt = O.jtilde(O.problem(mesh, 0.7))
    b = Jt.shape[0] // 3
    assert np.array_equal(Jt[b:2 * b, 2 * b:], Jt[2 * b:, b:2 * b])
    assert np.array_equal(Jt[b:2 * b, b:2 * b], Jt[2 * b:, 2 * b:])
    assert not Jt[:b, 2 * b:].any()
    assert np.array_equal(O.jtilde(O.problem(mesh, 0.7, sigma=1.0)), Jt)


def test_banded_jtilde():
    """App. A: the banded P keeps the slice blocks within half_band of the
    diagonal slice and is J~ there."""
    mesh = W.mesh_box(9, 7, 0.4, 0.4)
    P = O.problem(mesh, 0.7)
    J, Jb = O.jtilde(P), O.jtilde(P, half_band=1)
    per, blk = mesh.N + 1, (mesh.N + 1) * mesh.M
    sl = (np.arange(J.shape[0]) % blk) // per
    keep = np.abs(sl[:, None] - sl[None, :]) <= 1
    assert np.array_equal(Jb[keep], J[keep])
    assert not Jb[~keep].any()
    assert J[~keep].any()


@pytest.mark.parametrize("half", [0, 1])
@pytest.mark.parametrize("h", [0, 1, 2])
def test_jtilde_band_equals_dense_band(half, h):
    """The block-stored banded J~ (for meshes whose dense J~ does not fit in
    memory) holds exactly the band of the dense J~ of the same linear system
    (App. A), block (l, m) being rows of slice l and columns of slice m in the
    order they have in F and in u."""
    mesh = W.mesh_box(13, 7, 0.4, 0.35, half=half)
    P = O.problem(mesh, 0.8, n_rad=0.07)
    J = O.jtilde(P, half_band=h)
    B = O.jtilde_band(P, h)
    NB, M = mesh.N + 1, mesh.M
    nb = 3 * NB
    idx = lambda l: np.array([g * NB * M + l * NB + p for g in range(3) for p in range(NB)])
    scale = np.abs(J).max()
    for l in range(M):
        for m in range(max(0, l - h), min(M, l + h + 1)):
            ref = J[np.ix_(idx(l), idx(m))]
            assert np.abs(B[l, m - l + h] - ref).max() <= 1e-12 * scale, (l, m)
    # and nothing of the dense band is missing from the blocks
    assert sum(np.abs(B[l, m - l + h]).sum() for l in range(M) for m in range(max(0, l - h), min(M, l + h + 1))) \
        == pytest.approx(np.abs(J).sum(), rel=1e-12)
    with pytest.raises(ValueError):
        O.jtilde_band(O.problem(mesh, 0.8, tau=0.01), h)


@pytest.mark.parametrize("half", [0, 1])
def test_band_lu_solves_the_banded_system(half):
    """The block LU of App. A (partial pivoting inside the diagonal blocks)
    solves the banded J~ as a dense library solve does."""
    mesh = W.mesh_box(15, 9, 0.4, 0.4, half=half)
    P = O.problem(mesh, 0.9)
    h = 2
    J = O.jtilde(P, half_band=h)
    B = O.jtilde_band(P, h)
    piv = O.band_factor(P, B)
    r = np.random.default_rng(21).standard_normal(mesh.n_unknowns)
    z = O.band_solve(P, B, piv, r)
    ref = np.linalg.solve(J, r)
    assert np.abs(z - ref).max() <= 1e-10 * np.abs(ref).max()


def test_jfnk_with_banded_block_lu_reaches_the_dense_root():
    """Sec. 3.2 with the block-stored banded preconditioner (the form the
    oracle takes on paper-scale meshes) converges to the root the dense-LU
    preconditioner finds."""
    mesh, topo, F = W.config_small_half()
    P = O.problem(mesh, F)
    u0 = W.flat_guess(mesh)
    ud, sd = O.jfnk(P, topo, u0, half_band=1, tol=1e-11)
    ub, sb = O.jfnk(P, topo, u0, half_band=1, tol=1e-11, banded=True)
    assert sd["status"] == 0 and sb["status"] == 0
    assert np.abs(O.nodal_values(P, ub)["zeta"] - O.nodal_values(P, ud)["zeta"]).max() < 1e-10
    # the preconditioners are the same matrix, so GMRES takes the same path
    assert abs(sb["krylov_its"] - sd["krylov_its"]) <= 2


def _golden_appB():
    rows = []
    with open(os.path.join(GOLDEN, "appB_linear_jacobian.txt")) as fh:
        for line in fh:
            if not line.strip() or line.startswith("#"):
                continue
            lhs, col, expr, cite = [s.strip() for s in line.split("|")]
            eq, k = lhs.split()
            var, nn = col.split()
            rows.append((eq, int(k), var, int(nn), expr, cite))
    return rows


def test_appB_printed_entries():
    mesh = W.Mesh(N=9, M=5, x1=-1.6, y1=-0.8, dx=0.4, dy=0.4)
    Fr, nr = 0.7, 0.05
    J = O.jtilde(O.problem(mesh, Fr, n_rad=nr))
    per, blk = mesh.N + 1, (mesh.N + 1) * mesh.M
    l = 2  # slice l = m = 3 (1-based)
    row_of = {"F5": (0, None), "F6": (0, 1), "F1": (0, 2), "F3": (1, None), "F4": (1, 1),
              "F2": (1, 2), "F8": (2, None), "F9": (2, 1), "F7": (2, 2)}
    field_of = {"zeta": 0, "phi": 1, "psi": 2}
    env = dict(dx=mesh.dx, F=Fr, n=nr, x1=mesh.x1, pi=math.pi)
    entries = _golden_appB()
    assert len(entries) >= 40
    for eq, k, var, nn, expr, cite in entries:
        b, off = row_of[eq]
        r = b * blk + l * per + (0 if off is None else (1 if off == 1 else 2 + (k - 1)))
        if var.endswith("1"):
            c = field_of[var[:-1]] * blk + l * per
        else:
            c = field_of[var[:-1]] * blk + l * per + nn
        expect = eval(expr, {}, env)
        assert abs(J[r, c] - expect) < 1e-12 * max(1.0, abs(expect)), (eq, k, var, nn, cite)


def test_appB_K6_column_sums():
    """App. B prints dF2/dpsi_x(n,m) = dx/2 w(n,m) K6 + dx sum_{i>n} w(i,m) K6
    (and dx/2 sum_{i>=2} w K6 for n = 1), and dF7/dphi_x equal to it; the
    derivative in psi(1,m) is the plain sum of w K6 over the slice (printed 0,
    a misprint: the residual F2 contains (psi - x) K6)."""
    mesh = W.Mesh(N=9, M=5, x1=-1.6, y1=-0.8, dx=0.4, dy=0.4)
    J = O.jtilde(O.problem(mesh, 0.7))
    per, blk = mesh.N + 1, (mesh.N + 1) * mesh.M
    x, y = mesh.x(), mesh.y()
    N, M, dx = mesh.N, mesh.M, mesh.dx

    def w(i, j):  # trapezoid weights (0-based)
        return dx * mesh.dy * (0.5 if i in (0, N - 1) else 1.0) * (0.5 if j in (0, M - 1) else 1.0)

    for (k, l, m) in [(3, 2, 2), (1, 0, 3), (7, 4, 1)]:
        xs, ys = x[0] + (k - 0.5) * dx, y[l]
        K6 = lambda i: (((x[i] - xs) ** 2 + (y[m] - ys) ** 2) + 1.0) ** -1.5
        rF2 = blk + l * per + 2 + (k - 1)
        rF7 = 2 * blk + l * per + 2 + (k - 1)
        for n1 in range(1, N + 1):  # 1-based n
            i0 = n1 - 1
            if n1 == 1:
                expect = sum(0.5 * dx * w(i, m) * K6(i) for i in range(1, N))
            elif n1 < N:
                expect = 0.5 * dx * w(i0, m) * K6(i0) + dx * sum(w(i, m) * K6(i) for i in range(i0 + 1, N))
            else:
                expect = 0.5 * dx * w(i0, m) * K6(i0)
            assert abs(J[rF2, 2 * blk + m * per + n1] - expect) < 1e-13
            assert abs(J[rF7, blk + m * per + n1] - expect) < 1e-13
        s = sum(w(i, m) * K6(i) for i in range(N))
        assert abs(J[rF2, 2 * blk + m * per] - s) < 1e-13
        assert abs(J[rF7, blk + m * per] - s) < 1e-13


# ---------------------------------------------------------------------------
# P5: half domain (y >= 0 mirrored) equals the full domain for symmetric data.
# ---------------------------------------------------------------------------
def test_half_domain_equals_full_domain():
    Mh = 6
    half = W.Mesh(N=15, M=Mh, x1=-2.4, y1=0.0, dx=0.4, dy=0.4, half=1)
    full = W.Mesh(N=15, M=2 * Mh - 1, x1=-2.4, y1=-(Mh - 1) * 0.4, dx=0.4, dy=0.4)
    bump = [(0.15, 0.8, 0.3, 0.0)]
    th, tf = W.gaussian_bumps(half, bump), W.gaussian_bumps(full, bump)
    uh = W.smooth_guess(half, 3)
    per, blk = half.N + 1, (half.N + 1) * Mh
    bf = (half.N + 1) * full.M
    uf = np.zeros(full.n_unknowns)
    for f in range(3):
        for jf in range(full.M):
            jh = abs(jf - (Mh - 1))
            uf[f * bf + jf * per: f * bf + (jf + 1) * per] = uh[f * blk + jh * per: f * blk + (jh + 1) * per]
    rh = O.residual(O.problem(half, 0.7), th, uh)
    rf = O.residual(O.problem(full, 0.7), tf, uf)
    for f in range(3):
        for jh in range(Mh):
            jf = jh + Mh - 1
            a = rh[f * blk + jh * per: f * blk + (jh + 1) * per]
            b = rf[f * bf + jf * per: f * bf + (jf + 1) * per]
            assert np.abs(a - b).max() < 1e-12


# ---------------------------------------------------------------------------
# P7: JFNK (Sec. 3.2) and Newton with the dense finite-difference Jacobian
# converge to the same root; P8: the converged surface respects the height
# bound zeta <= F^2 / 2 (Sec. 5.1: speed^2 >= 0 in Bernoulli).
# ---------------------------------------------------------------------------
@pytest.mark.slow
def test_jfnk_matches_dense_newton_small_config():
    mesh, topo, F = W.config_small_half()
    P = O.problem(mesh, F)
    u0 = W.flat_guess(mesh)
    uj, sj = O.jfnk(P, topo, u0, tol=1e-11)
    ud, sd = O.newton_dense(P, topo, u0, tol=1e-11)
    assert sj["status"] == 0 and sd["status"] == 0
    zj, zd = O.nodal_values(P, uj)["zeta"], O.nodal_values(P, ud)["zeta"]
    assert np.abs(zj - zd).max() < 1e-10
    assert np.abs(uj - ud).max() < 1e-8
    assert zj.max() <= F * F / 2
    # the banded preconditioner of App. A reaches the same root
    ub, sb = O.jfnk(P, topo, u0, half_band=1, tol=1e-11)
    assert sb["status"] == 0
    assert np.abs(O.nodal_values(P, ub)["zeta"] - zj).max() < 1e-10


def test_full_domain_solution_is_symmetric():
    mesh = W.Mesh(N=21, M=9, x1=-3.2, y1=-1.6, dx=0.4, dy=0.4)
    topo = W.gaussian_bumps(mesh, [(0.1, 0.7, 0.0, 0.0)])
    P = O.problem(mesh, 0.7)
    u, st = O.jfnk(P, topo, W.flat_guess(mesh), tol=1e-11)
    assert st["status"] == 0
    z = O.nodal_values(P, u)["zeta"]
    assert np.abs(z - z[::-1, :]).max() < 1e-10


# ---------------------------------------------------------------------------
# P6: small-bump limit against the exact linear solution (Sec. 4.1).
# ---------------------------------------------------------------------------
def test_fft_linear_solution_is_quiet_upstream():
    bf = lambda X, Y: np.exp(-(X * X + Y * Y))
    x, y, z = LF.zeta_linear(bf, 0.7, 400.0, 400.0, 0.1, 0.01)
    up = np.abs(z[:, (x > -150) & (x < -20)]).max()
    dn = np.abs(z[:, (x > 20) & (x < 150)]).max()
    assert up < 0.05 * dn


@pytest.mark.slow
def test_linear_limit_decides_the_I4_sign():
    """Small bump (eps = 1e-3): zeta/eps of the nonlinear discrete solution
    approaches the exact linear solution under mesh refinement with sigma = -1,
    and anti-correlates with it under the printed sigma = +1."""
    F = 0.7
    bf = lambda X, Y: np.exp(-(X * X + Y * Y))
    x, y, z = LF.zeta_linear(bf, F, 409.6, 409.6, 0.1, 0.005)
    res = {}
    for dx, sig in ((0.4, -1.0), (0.3, -1.0), (0.3, 1.0)):
        N, M = int(round(12.0 / dx)) + 1, int(round(3.6 / dx)) + 1
        mesh = W.Mesh(N=N, M=M, x1=-4.8, y1=0.0, dx=dx, dy=dx, half=1)
        topo = W.gaussian_bumps(mesh, [(1e-3, 1 / math.sqrt(2), 0.0, 0.0)])
        zl = LF.sample(x, y, z, mesh.x(), mesh.y())
        u, st = O.jfnk(O.problem(mesh, F, sigma=sig), topo, W.flat_guess(mesh), tol=1e-13)
        assert st["status"] == 0
        zn = O.nodal_values(O.problem(mesh, F), u)["zeta"] / 1e-3
        near = mesh.x() <= 4.0
        err = np.abs(zn[:, near] - zl[:, near]).max() / np.abs(zl).max()
        corr = np.sum(zn * zl) / math.sqrt(np.sum(zn * zn) * np.sum(zl * zl))
        res[(dx, sig)] = (err, corr)
    assert res[(0.3, -1.0)][0] < res[(0.4, -1.0)][0]
    assert res[(0.3, -1.0)][1] > 0.65
    assert res[(0.3, 1.0)][1] < -0.5


def test_dispersion_wavelength_printed():
    """Sec. 5.3: the linear wavelength 2 pi / k at F = 0.6 is about 2.28,
    and the inline-bump separations 9.12 and 10.26 are 4 and 4.5 of them."""
    lam = 2 * math.pi / LF.dispersion_k(0.6)
    assert abs(lam - 2.28) < 0.005
    assert abs(4 * lam - 9.12) < 0.02 and abs(4.5 * lam - 10.26) < 0.02


def test_dense_lu_against_numpy():
    rng = np.random.default_rng(5)
    A = rng.standard_normal((40, 40)) + 10 * np.eye(40)
    b = rng.standard_normal(40)
    assert np.allclose(O.lu_solve_dense(A, b), np.linalg.solve(A, b), rtol=1e-12, atol=1e-12)


# ---------------------------------------------------------------------------
# Bottom pressure (Sec. 2.1): hydrostatic at the uniform stream; on a bottom
# plane that is a streamsurface of Phi = x + b y + a z, p = 1/2 - |grad Phi|^2/2
# - beta/F^2; the force integrates p (beta_x, beta_y, -1) dx dy.
# ---------------------------------------------------------------------------
def test_bottom_pressure_uniform_stream_is_hydrostatic():
    mesh = W.mesh_box(15, 7, 0.4, 0.4)
    F = 0.8
    P = O.problem(mesh, F)
    p, f = O.bottom_pressure(P, W.flat_topography(mesh), W.flat_guess(mesh))
    assert np.abs(p - 1.0 / F ** 2).max() < 1e-12
    area = (mesh.N - 1) * mesh.dx * (mesh.M - 1) * mesh.dy
    assert abs(f[0]) < 1e-12 and abs(f[1]) < 1e-12
    assert abs(f[2] + area / F ** 2) < 1e-9 * area


def test_bottom_pressure_on_streamsurface_plane():
    mesh = W.Mesh(N=11, M=7, x1=-2.0, y1=-0.9, dx=0.4, dy=0.3)
    F, a, b, q = 0.8, 0.05, -0.04, 0.1
    pp = a - b * q  # plane beta = -1.2 + pp x + q y (below z = 0 on this machine)
    P = O.problem(mesh, F)
    X, Y = np.meshgrid(mesh.x(), mesh.y())
    beta = -1.2 + pp * X + q * Y
    topo = W.Topography(beta.ravel(), np.full(beta.size, pp), np.full(beta.size, q))
    per, blk = mesh.N + 1, (mesh.N + 1) * mesh.M
    u = W.flat_guess(mesh)
    for j, yj in enumerate(mesh.y()):
        # psi = Phi on the plane = (1 + a pp) x + (b + a q) y + a (-1.2)
        u[2 * blk + j * per] = (1 + a * pp) * mesh.x1 + (b + a * q) * yj - 1.2 * a
        u[2 * blk + j * per + 1: 2 * blk + (j + 1) * per] = 1 + a * pp
    p, f = O.bottom_pressure(P, topo, u)
    expect = 0.5 - 0.5 * (1 + a * a + b * b) - beta / F ** 2
    assert np.abs(p - expect).max() < 1e-12
    # force components with the trapezoid rule on this plane
    wts = np.outer(np.where((np.arange(mesh.M) == 0) | (np.arange(mesh.M) == mesh.M - 1), 0.5, 1.0),
                   np.where((np.arange(mesh.N) == 0) | (np.arange(mesh.N) == mesh.N - 1), 0.5, 1.0))
    wts = wts * mesh.dx * mesh.dy
    assert abs(f[0] - np.sum(wts * expect * pp)) < 1e-12
    assert abs(f[2] + np.sum(wts * expect)) < 1e-12


# ---------------------------------------------------------------------------
# Sec. 4.1: a surface pressure with p^ = sech(k) b^ / F^2 gives, in the linear
# regime, the bump's wave pattern: zeta_pressure = zeta_bump - F^2 p.  Two
# independent forcing paths of the oracle (bottom integrals vs the dynamic
# condition) must agree through that relation at small amplitude.
# ---------------------------------------------------------------------------
@pytest.mark.slow
def test_pressure_patch_matches_bump_in_linear_regime():
    F, eps = 0.7, 1e-3
    errs = []
    for dx in (0.4, 0.3):
        N, M = int(round(12.0 / dx)) + 1, int(round(3.6 / dx)) + 1
        mesh = W.Mesh(N=N, M=M, x1=-4.8, y1=0.0, dx=dx, dy=dx, half=1)
        bf = lambda X, Y: eps * np.exp(-(X * X + Y * Y))
        topo = W.gaussian_bumps(mesh, [(eps, 1 / math.sqrt(2), 0.0, 0.0)])
        ub, sb = O.jfnk(O.problem(mesh, F), topo, W.flat_guess(mesh), tol=1e-12)
        p = LF.equivalent_pressure(bf, F, mesh.x(), mesh.y())
        up, sp = O.jfnk(O.problem(mesh, F, psurf=p), W.flat_topography(mesh), W.flat_guess(mesh), tol=1e-12)
        assert sb["status"] == 0 and sp["status"] == 0
        zb = O.nodal_values(O.problem(mesh, F), ub)["zeta"]
        zp = O.nodal_values(O.problem(mesh, F), up)["zeta"]
        pred = zb - F * F * p
        errs.append(np.abs(zp - pred).max() / np.abs(pred).max())
    assert errs[0] < 1e-2 and errs[1] < errs[0]


# ---------------------------------------------------------------------------
# Surface tension (Sec. 6: tension times mean curvature in the dynamic
# condition).  The oracle's curvature term, read off as F1(tau) - F1(0) at an
# explicit surface, converges at second order to the mean curvature
# div(grad zeta / sqrt(1 + |grad zeta|^2)) obtained by symbolic
# differentiation of that definition (not of the expanded formula the oracle
# uses), in the full and the half domain.
# ---------------------------------------------------------------------------
def _gaussian_surface_u(mesh, A, s, x0, y0):
    sp = pytest.importorskip("sympy")
    X, Y = sp.symbols("x y", real=True)
    z = A * sp.exp(-((X - x0) ** 2 + (Y - y0) ** 2) / s ** 2)
    zx, zy = sp.diff(z, X), sp.diff(z, Y)
    q = sp.sqrt(1 + zx ** 2 + zy ** 2)
    kappa = sp.diff(zx / q, X) + sp.diff(zy / q, Y)
    f_z, f_zx, f_k = (sp.lambdify((X, Y), e, "numpy") for e in (z, zx, kappa))
    x, y = mesh.x(), mesh.y()
    NB = mesh.N + 1
    u = W.flat_guess(mesh).copy()
    for j in range(mesh.M):  # zeta block: zeta(1) then zeta_x at every node
        u[j * NB] = f_z(x[0], y[j])
        u[j * NB + 1: j * NB + 1 + mesh.N] = f_zx(x, np.full_like(x, y[j]))
    xs = x[:-1] + 0.5 * mesh.dx
    kap = np.array([[f_k(xx, yy) for xx in xs] for yy in y])  # [M, N-1]
    return u, kap


@pytest.mark.parametrize("half", [0, 1])
def test_surface_tension_term_is_the_mean_curvature(half):
    errs = []
    for h in (0.2, 0.1):
        L, H = 4.0, 3.0
        N, M = int(round(2 * L / h)) + 1, (int(round(H / h)) + 1 if half else int(round(2 * H / h)) + 1)
        mesh = W.Mesh(N=N, M=M, x1=-L, y1=0.0 if half else -H, dx=h, dy=h, half=half)
        u, kap = _gaussian_surface_u(mesh, 0.5, 1.3, 0.3, 0.0 if half else 0.4)  # slopes to 0.33
        topo = W.flat_topography(mesh)
        r0 = O.residual(O.problem(mesh, 0.8), topo, u)
        r1 = O.residual(O.problem(mesh, 0.8, tau=1.0), topo, u)
        NB = N + 1
        got = np.array([[-(r1[l * NB + 2 + k] - r0[l * NB + 2 + k]) for k in range(N - 1)] for l in range(M)])
        errs.append(np.abs(got - kap).max() / np.abs(kap).max())
    assert errs[1] < 1e-2, errs
    assert errs[0] / errs[1] > 3.0, errs  # second order


# ---------------------------------------------------------------------------
# P10: preconditioning with the linear Jacobian clusters the spectrum at 1
# (Sec. 4.2, eigenvalue figure: a Gaussian bump eps = 0.1, F = 0.6,
# dx = dy = 0.8, flat-surface iterate; 15 x 15 here instead of 31 x 31).
# ---------------------------------------------------------------------------
def test_linear_preconditioner_clusters_the_spectrum():
    N, dx = 15, 0.8
    mesh = W.Mesh(N=N, M=N, x1=-0.28 * (N - 1) * dx, y1=-0.5 * (N - 1) * dx, dx=dx, dy=dx)
    topo = W.gaussian_bumps(mesh, [(0.1, 1 / math.sqrt(2), 0.0, 0.0)])
    P = O.problem(mesh, 0.6)
    J = O.fd_jacobian(P, topo, W.flat_guess(mesh))
    ev = np.linalg.eigvals(J)
    # unpreconditioned: spread over two decades, almost nothing near 1
    assert np.abs(ev).max() / np.abs(ev).min() > 20
    assert np.mean(np.abs(ev - 1) < 0.1) < 0.05
    # J J~^-1: every eigenvalue within 0.1 of 1
    evp = np.linalg.eigvals(J @ np.linalg.inv(O.jtilde(P)))
    assert np.abs(evp - 1).max() < 0.1
    # the banded preconditioner of App. A keeps most of the cluster
    for hb in (1, 3):
        evb = np.linalg.eigvals(J @ np.linalg.inv(O.jtilde(P, half_band=hb)))
        assert np.mean(np.abs(evb - 1) < 0.1) > 0.9
