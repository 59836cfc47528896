"""ctypes binding of the plain-C FP64 oracle (bfs_oracle.c).

TEST INFRASTRUCTURE ONLY: used by tests/, __graft_entry__.smoke() and the CPU
baseline of bench.py.  It shares no code with the CUDA library.

Parity status of each function (how it is pinned, see tests/test_oracle_pins.py):
  residual ........... uniform stream gives 0 (exact), half vs full domain,
                       dynamic condition on a streamsurface of a linear
                       potential, linearisation identity (FD Jacobian at the
                       uniform stream equals the linear Jacobian), linear limit
  bie_point .......... Green's identity for harmonic functions (refinement)
  rect_S2 ............ adaptive 2-D quadrature
  nodal_values ....... exact for quadratic fields
  residual_linear / jtilde ... App. B printed entries that are self-consistent,
                       block symmetries J23 = J32, J22 = J33 (Sec. 4.2)
  lu / jfnk / newton_dense ... dense solve vs numpy; JFNK vs dense FD Newton
  jtilde_band ........ every stored block equals the band of the dense J~
                       (full and half domain)
  band_factor/solve .. the banded block LU solves the banded J~ as the dense
                       LU does; JFNK with it reaches the dense-LU root
  bottom_pressure .... hydrostatic value at the uniform stream; Bernoulli on a
                       streamsurface of a linear potential; force = 0 with
                       no bottom slope
  surface tension .... the curvature term converges at second order to the
                       mean curvature of an explicit surface (differentiated
                       symbolically); linearisation identity with tau
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "bfs_oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")
_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile bfs_oracle.c into liboracle.so (plain gcc, OpenMP, no fast-math)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O3", "-fopenmp", "-fPIC", "-shared", "-std=c99",
                               "-fno-fast-math", _SRC, "-o", tmp, "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


class Problem(ctypes.Structure):
    _fields_ = [("N", ctypes.c_int), ("M", ctypes.c_int), ("half", ctypes.c_int),
                ("x1", ctypes.c_double), ("y1", ctypes.c_double),
                ("dx", ctypes.c_double), ("dy", ctypes.c_double),
                ("F", ctypes.c_double), ("n_rad", ctypes.c_double),
                ("sigma", ctypes.c_double), ("psurf", ctypes.POINTER(ctypes.c_double)),
                ("tau", ctypes.c_double)]


class Stats(ctypes.Structure):
    _fields_ = [("newton_its", ctypes.c_int), ("krylov_its", ctypes.c_int),
                ("residual_evals", ctypes.c_int), ("status", ctypes.c_int),
                ("fnorm_inf", ctypes.c_double), ("fnorm_2", ctypes.c_double)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class Sheet(ctypes.Structure):
    _fields_ = [(n, ctypes.POINTER(ctypes.c_double)) for n in ("h", "hx", "hy", "d", "s")]


class Target(ctypes.Structure):
    _fields_ = [(n, ctypes.c_double) for n in ("x", "y", "z", "u", "sd", "px", "py")]


_D = ctypes.POINTER(ctypes.c_double)
_I = ctypes.POINTER(ctypes.c_int)


def lib():
    global _lib
    with _lock:
        if _lib is None:
            L = ctypes.CDLL(build())
            P = ctypes.POINTER(Problem)
            L.orc_residual.argtypes = [P, _D, _D, _D, _D, _D, _D]
            L.orc_residual_linear.argtypes = [P, _D, _D, _D]
            L.orc_jtilde.argtypes = [P, ctypes.c_int, _D]
            L.orc_jtilde_band.argtypes = [P, ctypes.c_int, _D]
            L.orc_band_factor.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int, _D, _I]
            L.orc_band_solve.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int, _D, _I, _D, _D]
            L.orc_fd_jacobian.argtypes = [P, _D, _D, _D, _D, _D]
            L.orc_nodal_values.argtypes = [P, _D, _D]
            L.orc_rect_S2.argtypes = [ctypes.c_double] * 7
            L.orc_rect_S2.restype = ctypes.c_double
            L.orc_bie_point.argtypes = [P, ctypes.POINTER(Sheet), ctypes.POINTER(Sheet),
                                        ctypes.c_int, ctypes.POINTER(Target), _D]
            L.orc_bie_point.restype = ctypes.c_double
            L.orc_lu_factor.argtypes = [ctypes.c_int, _D, _I]
            L.orc_lu_factor.restype = ctypes.c_int
            L.orc_lu_solve.argtypes = [ctypes.c_int, _D, _I, _D, _D]
            L.orc_jfnk.argtypes = [P, _D, _D, _D, _D, ctypes.c_int, ctypes.c_double,
                                   ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_double,
                                   ctypes.POINTER(Stats)]
            L.orc_jfnk.restype = ctypes.c_int
            L.orc_newton_dense.argtypes = [P, _D, _D, _D, _D, ctypes.c_double, ctypes.c_int,
                                           ctypes.POINTER(Stats)]
            L.orc_newton_dense.restype = ctypes.c_int
            L.orc_bottom_pressure.argtypes = [P, _D, _D, _D, _D, _D, _D]
            L.orc_num_threads.restype = ctypes.c_int
            L.orc_set_threads.argtypes = [ctypes.c_int]
            _lib = L
    return _lib


def _p(a: np.ndarray):
    return a.ctypes.data_as(_D)


def _f64(a) -> np.ndarray:
    return np.ascontiguousarray(a, dtype=np.float64)


def problem(mesh, F: float, sigma: float = -1.0, n_rad: float = 0.05, psurf=None, tau: float = 0.0) -> Problem:
    """psurf: optional applied surface pressure at the nodes (kept alive on the
    returned structure); tau: surface tension parameter (mean-curvature term)."""
    P = Problem(mesh.N, mesh.M, int(mesh.half), mesh.x1, mesh.y1, mesh.dx, mesh.dy,
                float(F), float(n_rad), float(sigma), None, float(tau))
    if psurf is not None:
        P._psurf = _f64(psurf).ravel().copy()
        P.psurf = _p(P._psurf)
    return P


def num_threads() -> int:
    return lib().orc_num_threads()


def set_threads(n: int) -> None:
    lib().orc_set_threads(int(n))


def residual(P: Problem, topo, u, with_scale: bool = False):
    """F(u) in App. B order; optionally the per-row sum of |terms|."""
    b, bx, by, u = _f64(topo.beta), _f64(topo.beta_x), _f64(topo.beta_y), _f64(u)
    n = 3 * (P.N + 1) * P.M
    assert u.size == n and b.size == P.N * P.M
    out = np.empty(n)
    sc = np.empty(n) if with_scale else None
    lib().orc_residual(ctypes.byref(P), _p(b), _p(bx), _p(by), _p(u), _p(out),
                       _p(sc) if sc is not None else None)
    return (out, sc) if with_scale else out


def residual_linear(P: Problem, beta_x, u):
    u = _f64(u)
    bx = _f64(beta_x) if beta_x is not None else None
    out = np.empty(3 * (P.N + 1) * P.M)
    lib().orc_residual_linear(ctypes.byref(P), _p(bx) if bx is not None else None, _p(u), _p(out))
    return out


def jtilde(P: Problem, half_band: int = -1) -> np.ndarray:
    n = 3 * (P.N + 1) * P.M
    J = np.empty((n, n))
    lib().orc_jtilde(ctypes.byref(P), int(half_band), _p(J))
    return J


def jtilde_band(P: Problem, half_band: int) -> np.ndarray:
    """Blocks (l, m), |l - m| <= half_band, of J~ regrouped slice by slice:
    array (M, 2 half_band + 1, nb, nb), block (l, m) at [l, m - l + half_band]."""
    nb = 3 * (P.N + 1)
    B = np.empty((P.M, 2 * half_band + 1, nb, nb))
    if lib().orc_jtilde_band(ctypes.byref(P), int(half_band), _p(B)):
        raise ValueError("banded J~ needs tau = 0 and half_band >= 0")
    return B


def band_factor(P: Problem, B: np.ndarray):
    """Block LU of jtilde_band's blocks in place; returns the pivots."""
    nb = 3 * (P.N + 1)
    h = (B.shape[1] - 1) // 2
    piv = np.empty(P.M * nb, dtype=np.int32)
    if lib().orc_band_factor(P.M, nb, h, _p(B), piv.ctypes.data_as(_I)):
        raise ZeroDivisionError("singular diagonal block")
    return piv


def band_solve(P: Problem, B: np.ndarray, piv: np.ndarray, r) -> np.ndarray:
    """z = P^-1 r with band_factor's factors (r in the order of F, z of u)."""
    h = (B.shape[1] - 1) // 2
    z = np.empty(3 * (P.N + 1) * P.M)
    lib().orc_band_solve(P.N, P.M, h, _p(B), piv.ctypes.data_as(_I), _p(_f64(r)), _p(z))
    return z


def fd_jacobian(P: Problem, topo, u) -> np.ndarray:
    n = 3 * (P.N + 1) * P.M
    J = np.empty((n, n))
    b, bx, by, u = _f64(topo.beta), _f64(topo.beta_x), _f64(topo.beta_y), _f64(u)
    lib().orc_fd_jacobian(ctypes.byref(P), _p(b), _p(bx), _p(by), _p(u), _p(J))
    return J


def nodal_values(P: Problem, u) -> dict:
    n = P.N * P.M
    out = np.empty(8 * n)
    lib().orc_nodal_values(ctypes.byref(P), _p(_f64(u)), _p(out))
    names = ("zeta", "zeta_x", "zeta_y", "phi", "phi_x", "phi_y", "psi", "psi_x")
    return {k: out[i * n:(i + 1) * n].reshape(P.M, P.N) for i, k in enumerate(names)}


def rect_S2(A, B, C, s1, s2, t1, t2) -> float:
    return lib().orc_rect_S2(A, B, C, s1, s2, t1, t2)


def bie_point(P: Problem, top: dict, bot: dict, self_bottom: bool, target: dict):
    """Green's-identity sum at one collocation point (see bfs_oracle.c).
    top/bot: dicts of nodal arrays h, hx, hy, d, s; target: x, y, z, u, sd, px, py.
    Returns (sum, scale)."""
    keep = []

    def sheet(d):
        arrs = [_f64(d[k]).ravel() for k in ("h", "hx", "hy", "d", "s")]
        keep.extend(arrs)
        return Sheet(*[_p(a) for a in arrs])

    st, sb = sheet(top), sheet(bot)
    T = Target(*[float(target[k]) for k in ("x", "y", "z", "u", "sd", "px", "py")])
    sc = ctypes.c_double()
    v = lib().orc_bie_point(ctypes.byref(P), ctypes.byref(st), ctypes.byref(sb),
                            int(bool(self_bottom)), ctypes.byref(T), ctypes.byref(sc))
    return v, sc.value


def bottom_pressure(P: Problem, topo, u):
    """Nodal bottom pressure (M x N) and the force (3,) on the topography."""
    b, bx, by, u = _f64(topo.beta), _f64(topo.beta_x), _f64(topo.beta_y), _f64(u)
    p = np.empty(P.N * P.M)
    f = np.empty(3)
    lib().orc_bottom_pressure(ctypes.byref(P), _p(b), _p(bx), _p(by), _p(u), _p(p), _p(f))
    return p.reshape(P.M, P.N), f


def lu_solve_dense(A: np.ndarray, b: np.ndarray) -> np.ndarray:
    n = A.shape[0]
    LU = np.array(A, dtype=np.float64, order="C", copy=True)
    piv = np.empty(n, dtype=np.int32)
    if lib().orc_lu_factor(n, _p(LU), piv.ctypes.data_as(_I)):
        raise ZeroDivisionError("singular matrix")
    x = np.empty(n)
    lib().orc_lu_solve(n, _p(LU), piv.ctypes.data_as(_I), _p(_f64(b)), _p(x))
    return x


def jfnk(P: Problem, topo, u0, half_band: int = -1, tol: float = 1e-10, max_newton: int = 50,
         restart: int = 50, max_krylov: int = 400, eta: float = 1e-4, banded: bool = False):
    """Damped JFNK solve from u0; returns (u, stats dict).  banded=True takes
    the banded preconditioner in block storage (half_band >= 0), for meshes
    whose dense J~ does not fit in memory."""
    u = _f64(u0).copy()
    b, bx, by = _f64(topo.beta), _f64(topo.beta_x), _f64(topo.beta_y)
    st = Stats()
    hb = int(half_band)
    if banded:
        if hb < 0:
            raise ValueError("banded preconditioner needs half_band >= 0")
        hb = -3 - hb
    lib().orc_jfnk(ctypes.byref(P), _p(b), _p(bx), _p(by), _p(u), hb, tol,
                   max_newton, restart, max_krylov, eta, ctypes.byref(st))
    return u, st.as_dict()


def newton_dense(P: Problem, topo, u0, tol: float = 1e-10, max_newton: int = 30):
    u = _f64(u0).copy()
    b, bx, by = _f64(topo.beta), _f64(topo.beta_x), _f64(topo.beta_y)
    st = Stats()
    lib().orc_newton_dense(ctypes.byref(P), _p(b), _p(bx), _p(by), _p(u), tol, max_newton,
                           ctypes.byref(st))
    return u, st.as_dict()
