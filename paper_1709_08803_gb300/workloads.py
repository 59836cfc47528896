"""Seeded synthetic inputs: meshes, bottom topographies and initial guesses.

This module only builds inputs.  It holds none of the method's arithmetic
(no reconstruction, no kernels, no residual) and is shared by the CUDA path,
the tests and the CPU oracle alike.

Shapes follow the paper's workloads: a rectangular truncated mesh
x_i = x1 + (i-1) dx, y_j = y1 + (j-1) dy (Sec. 3.1) and Gaussian bumps on an
otherwise flat bottom z = -1 (Sec. 2.1, the Gaussian bottom shape), optionally
several of them or a cross-stream ridge.  Nodal arrays are flat float64 of
length N*M with index i + N*j.  The unknown vector u has 3(N+1)M entries laid
out per slice j as [q(x1,y_j), q_x(x_1..x_N, y_j)] for q = zeta, phi, psi
(Sec. 3.1, the vector of unknowns).
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np

SEED_BASE = 170908803


@dataclasses.dataclass(frozen=True)
class Mesh:
    N: int          # nodes in x
    M: int          # nodes in y
    x1: float
    y1: float
    dx: float
    dy: float
    half: int = 0   # 1: y1 = 0 and the flow is mirrored to y < 0

    @property
    def n_unknowns(self) -> int:
        return 3 * (self.N + 1) * self.M

    @property
    def n_targets(self) -> int:
        return (self.N - 1) * self.M

    @property
    def n_sources(self) -> int:
        return self.N * (2 * self.M - 1) if self.half else self.N * self.M

    def x(self) -> np.ndarray:
        return self.x1 + self.dx * np.arange(self.N)

    def y(self) -> np.ndarray:
        return self.y1 + self.dy * np.arange(self.M)

    def pair_evals(self) -> int:
        """Pair evaluations of one residual: four sheet pairings (top/bottom
        target x top/bottom source) over every target and source node."""
        return 4 * self.n_targets * self.n_sources


@dataclasses.dataclass(frozen=True)
class Topography:
    beta: np.ndarray
    beta_x: np.ndarray
    beta_y: np.ndarray


def gaussian_bumps(mesh: Mesh, bumps, ridges=()) -> Topography:
    """beta = -1 + sum eps exp(-((x-b1)^2 + (y-b2)^2) / (2 delta^2))
    + sum a exp(-(x-xr)^2 / (2 dr^2)), with exact derivatives.

    bumps: iterable of (eps, delta, b1, b2); ridges: iterable of (a, dr, xr)
    (a ridge is uniform in y)."""
    X, Y = np.meshgrid(mesh.x(), mesh.y(), indexing="xy")  # shape (M, N)
    beta = -np.ones_like(X)
    bx = np.zeros_like(X)
    by = np.zeros_like(X)
    for eps, delta, b1, b2 in bumps:
        e = eps * np.exp(-((X - b1) ** 2 + (Y - b2) ** 2) / (2.0 * delta * delta))
        beta += e
        bx += -e * (X - b1) / (delta * delta)
        by += -e * (Y - b2) / (delta * delta)
    for a, dr, xr in ridges:
        e = a * np.exp(-((X - xr) ** 2) / (2.0 * dr * dr))
        beta += e
        bx += -e * (X - xr) / (dr * dr)
    return Topography(beta.ravel().copy(), bx.ravel().copy(), by.ravel().copy())


def flat_topography(mesh: Mesh) -> Topography:
    n = mesh.N * mesh.M
    return Topography(-np.ones(n), np.zeros(n), np.zeros(n))


def flat_guess(mesh: Mesh) -> np.ndarray:
    """Uniform stream: zeta = 0, phi = psi = x (so phi_x = psi_x = 1)."""
    u = np.zeros(mesh.n_unknowns)
    per = mesh.N + 1
    blk = per * mesh.M
    for f in (1, 2):
        for j in range(mesh.M):
            s = f * blk + j * per
            u[s] = mesh.x1
            u[s + 1: s + per] = 1.0
    return u


def perturbed_guess(mesh: Mesh, seed: int, amp: float = 1e-3) -> np.ndarray:
    """Flat guess plus amp * N(0,1) in every entry (seeded)."""
    rng = np.random.default_rng(SEED_BASE + seed)
    return flat_guess(mesh) + amp * rng.standard_normal(mesh.n_unknowns)


def smooth_guess(mesh: Mesh, seed: int, amp: float = 0.02) -> np.ndarray:
    """Flat guess plus a seeded smooth wave-like perturbation of zeta_x,
    phi_x, psi_x and the upstream values, of the size a converged wave field
    has (used to exercise the kernels away from the uniform stream)."""
    rng = np.random.default_rng(SEED_BASE + 1000 + seed)
    u = flat_guess(mesh)
    per = mesh.N + 1
    blk = per * mesh.M
    x = mesh.x()
    y = mesh.y()
    for f in range(3):
        k1, k2 = rng.uniform(0.8, 2.5), rng.uniform(0.2, 1.2)
        ph1, ph2 = rng.uniform(0, 2 * math.pi, size=2)
        a = amp * rng.uniform(0.5, 1.5)
        for j in range(mesh.M):
            s = f * blk + j * per
            env = 1.0 / (1.0 + np.exp(-(x - x[0] - 2.0)))  # quiet far upstream
            u[s + 1: s + per] += a * env * np.cos(k1 * x + ph1) * np.cos(k2 * y[j] + ph2)
            u[s] += 0.1 * a * rng.standard_normal()
    return u


# ---------------------------------------------------------------------------
# The configurations the tests and the benchmark run on.
# ---------------------------------------------------------------------------

def config_small_half():
    """31x11 half domain (y >= 0), dx = dy = 0.4, x in [-6, 6], F = 0.7,
    beta = -1 + 0.1 exp(-(x^2 + y^2))."""
    mesh = Mesh(N=31, M=11, x1=-6.0, y1=0.0, dx=0.4, dy=0.4, half=1)
    topo = gaussian_bumps(mesh, [(0.1, 1.0 / math.sqrt(2.0), 0.0, 0.0)])
    return mesh, topo, 0.7


def config_paper_scale(F: float = 0.7):
    """181x61 full mesh, dx = dy = 0.3, x in [-15, 39], y in [-9, 9],
    beta = -1 + 0.2 exp(-(x^2 + y^2)); F = 0.7 or 1.5."""
    mesh = Mesh(N=181, M=61, x1=-15.0, y1=-9.0, dx=0.3, dy=0.3, half=0)
    topo = gaussian_bumps(mesh, [(0.2, 1.0 / math.sqrt(2.0), 0.0, 0.0)])
    return mesh, topo, F


def config_large(coarsen: int = 1):
    """361x121 full mesh, dx = dy = 0.2, x in [-20, 52], y in [-12, 12], F = 0.9,
    bump 0.3 exp(-(x^2 + y^2)) plus a cross-stream ridge 0.005 exp(-(x-5)^2 / 2).
    The ridge height is not given; a two-dimensional ridge blocks steady
    subcritical flow above the hydraulic critical height 1 + F^2/2 - (3/2) F^(2/3)
    of the depth (0.0067 at F = 0.9), so it is taken below that.
    coarsen = c: the same rectangle and bottom at spacing 0.2 c (c divides 120)."""
    if coarsen < 1 or 120 % coarsen:
        raise ValueError("coarsen must divide 120")
    mesh = Mesh(N=360 // coarsen + 1, M=120 // coarsen + 1, x1=-20.0, y1=-12.0, dx=0.2 * coarsen,
                dy=0.2 * coarsen, half=0)
    topo = gaussian_bumps(mesh, [(0.3, 1.0 / math.sqrt(2.0), 0.0, 0.0)], ridges=[(0.005, 1.0, 5.0)])
    return mesh, topo, 0.9


def config_supercritical_281(eps: float = 0.1, F: float = 3.0):
    """The paper's supercritical runs (Sec. 5.2, Figs. 5-6): 281 x 281 nodes,
    x in [-21, 51], y in [-36, 36] (dx = dy = 72/280 = 0.257), F = 3 (Fig. 6
    also F = 4), one Gaussian bump of width delta = 3 at the origin with
    height eps."""
    h = 72.0 / 280.0
    mesh = Mesh(N=281, M=281, x1=-21.0, y1=-36.0, dx=h, dy=h, half=0)
    return mesh, gaussian_bumps(mesh, [(eps, 3.0, 0.0, 0.0)]), float(F)


def config_subcritical_281(eps: float = 0.1):
    """The paper's subcritical runs (Sec. 5.1, Fig. 4): 281 x 281 nodes,
    x in [-7, 17], y in [-12, 12] (dx = dy = 24/280 = 0.0857), F = 0.6, one
    Gaussian bump of width delta = 0.5 at the origin with height eps."""
    h = 24.0 / 280.0
    mesh = Mesh(N=281, M=281, x1=-7.0, y1=-12.0, dx=h, dy=h, half=0)
    return mesh, gaussian_bumps(mesh, [(eps, 0.5, 0.0, 0.0)]), 0.6


def gaussian_equivalent_pressure(mesh: Mesh, eps: float, delta: float, F: float) -> np.ndarray:
    """The applied surface pressure whose linear wake equals that of the
    Gaussian bump beta + 1 = eps exp(-(x^2 + y^2) / (2 delta^2)) (Sec. 6, the
    radial integral for p(x, y); Sec. 4.1: its transform is sech(k) times the
    bump's over F^2):

        p(r) = eps delta^2 / F^2  int_0^inf k sech(k) exp(-delta^2 k^2 / 2) J0(k r) dk.

    An input of the pressure-forced problem (the ship-wake model), evaluated
    once on the host: Simpson's rule in k on [0, k_max] (the Gaussian factor
    is below 1e-19 beyond k_max) at a step resolving J0 at the largest node
    radius, on a radial grid 1/20 of the mesh spacing, interpolated linearly
    to the nodes.  Nodal values, flat, index i + N j."""
    from scipy.special import j0

    X, Y = np.meshgrid(mesh.x(), mesh.y(), indexing="xy")
    r_node = np.hypot(X, Y).ravel()
    r_max = float(r_node.max())
    dr = min(mesh.dx, mesh.dy) / 20.0
    r = np.arange(0.0, r_max + 2.0 * dr, dr)
    k_max = math.sqrt(2.0 * 45.0) / delta
    n_k = int(math.ceil(k_max * max(r_max, 1.0) / 0.05))
    n_k += n_k % 2  # Simpson needs an even number of intervals
    k = np.linspace(0.0, k_max, n_k + 1)
    wk = np.full(n_k + 1, 2.0)
    wk[1::2] = 4.0
    wk[0] = wk[-1] = 1.0
    wk *= (k[1] - k[0]) / 3.0
    g = wk * k / np.cosh(k) * np.exp(-0.5 * (delta * k) ** 2)
    p_r = np.empty(r.size)
    for a in range(0, r.size, 512):
        p_r[a:a + 512] = j0(np.outer(r[a:a + 512], k)) @ g
    p_r *= eps * delta * delta / (F * F)
    return np.interp(r_node, r, p_r)


def mesh_box(N: int, M: int, dx: float, dy: float, half: int = 0, x1: float | None = None) -> Mesh:
    """A mesh of N x M nodes with the upstream edge at about 28% of the
    x-extent upstream of the origin, symmetric in y."""
    if x1 is None:
        x1 = -round(0.28 * (N - 1)) * dx
    y1 = 0.0 if half else -0.5 * (M - 1) * dy
    return Mesh(N=N, M=M, x1=x1, y1=y1, dx=dx, dy=dy, half=half)


def config_batch(seed: int = 3, B: int = 64, sizes=None):
    """Batched-sweep workload: B instances with F ~ U[0.5, 1.4]; the bottom is
    1-3 Gaussians (eps ~ U[0.05, 0.3], delta ~ U[0.5, 2], centres ~ U[-2, 2]^2)
    or a cross-stream ridge (a ~ U[0.05, 0.3], width ~ U[0.5, 2], x_r ~ U[-2, 2]);
    meshes N in {61, 81, ..., 241}, M = (N - 1)/3 + 1, dx = dy = 0.3, full
    domain.  `sizes` overrides the list of N (tests use small meshes).
    Returns (meshes, topographies, Froude numbers)."""
    rng = np.random.default_rng(SEED_BASE + seed)
    Ns = list(sizes) if sizes is not None else list(range(61, 242, 20))
    meshes, topos, Fs = [], [], []
    for _ in range(B):
        N = int(rng.choice(Ns))
        M = (N - 1) // 3 + 1
        mesh = mesh_box(N, M, 0.3, 0.3)
        F = float(rng.uniform(0.5, 1.4))
        if rng.uniform() < 0.8:
            nb = int(rng.integers(1, 4))
            bumps = [(float(rng.uniform(0.05, 0.3)), float(rng.uniform(0.5, 2.0)),
                      float(rng.uniform(-2, 2)), float(rng.uniform(-2, 2))) for _ in range(nb)]
            topo = gaussian_bumps(mesh, bumps)
        else:
            topo = gaussian_bumps(mesh, [], ridges=[(float(rng.uniform(0.05, 0.3)),
                                                     float(rng.uniform(0.5, 2.0)),
                                                     float(rng.uniform(-2, 2)))])
        meshes.append(mesh)
        topos.append(topo)
        Fs.append(F)
    return meshes, topos, Fs
