"""The C ABI without a GPU: the library builds and loads, exports every entry
point include/bfs.h declares, and rejects invalid problems on the host before
any device work."""
import ctypes
import os
import re
import subprocess

import numpy as np
import pytest

from paper_1709_08803_gb300 import build as B
from paper_1709_08803_gb300 import bfs
from paper_1709_08803_gb300 import workloads as W

INCLUDE = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "include")
HEADERS = sorted(os.path.join(INCLUDE, f) for f in os.listdir(INCLUDE) if f.endswith(".h"))


@pytest.fixture(scope="module")
def L():
    B.build()
    return bfs.lib()


def declared():
    names = set()
    for h in HEADERS:
        text = re.sub(r"/\*.*?\*/", "", open(h).read(), flags=re.S)
        names.update(re.findall(r"\b(bfs_[a-z_0-9]+)\s*\(", text))
    return sorted(names)


def test_header_declares_the_boundary():
    names = declared()
    for must in ("bfs_setup", "bfs_residual", "bfs_jvp", "bfs_precond_factor", "bfs_precond_apply",
                 "bfs_solve", "bfs_destroy", "bfs_last_error", "bfs_cno_create", "bfs_cno_guess"):
        assert must in names


def test_every_exported_entry_point_is_declared(L):
    """The other direction: no bfs_* function leaves the library undocumented."""
    nm = subprocess.run(["nm", "-D", "--defined-only", bfs.LIB_PATH], capture_output=True, text=True)
    if nm.returncode != 0:
        pytest.skip("nm unavailable")
    exported = {ln.split()[-1] for ln in nm.stdout.splitlines()
                if len(ln.split()) == 3 and ln.split()[1] == "T" and ln.split()[-1].startswith("bfs_")}
    assert exported, "no bfs_ symbols exported"
    missing = sorted(exported - set(declared()))
    assert not missing, missing


def test_every_declared_symbol_is_exported(L):
    missing = [n for n in declared() if not hasattr(L, n)]
    assert not missing, missing


def test_default_options(L):
    o = bfs.default_options()
    assert o.n_rad == 0.05 and o.sign_I4 == -1.0 and o.tol == 1e-8
    assert o.gmres_restart == 50 and o.krylov_precision == bfs.BFS_FP64
    # the fields appended later: also checks that the ctypes layout matches the C struct
    assert o.outer_precision == bfs.BFS_FP64 and o.precond_precision == bfs.BFS_FP64
    assert o.refine_below == 0.0 and o.stall_newton == 0 and o.surface_tension == 0.0 and o.forcing == 0


def _setup(mesh, topo, F, opts=None):
    m = bfs.bfs_mesh(mesh.N, mesh.M, int(mesh.half), mesh.x1, mesh.y1, mesh.dx, mesh.dy)
    arrs = [np.ascontiguousarray(a, dtype=np.float64) for a in (topo.beta, topo.beta_x, topo.beta_y)]
    D = ctypes.POINTER(ctypes.c_double)
    t = bfs.bfs_topo(*[a.ctypes.data_as(D) for a in arrs])
    o = opts if opts is not None else bfs.default_options()
    ctx = ctypes.c_void_p()
    rc = bfs.lib().bfs_setup(ctypes.byref(m), ctypes.byref(t), F, ctypes.byref(o), ctypes.byref(ctx))
    return rc, ctx


@pytest.mark.parametrize("case", ["N", "M", "dx", "F", "half_y1", "beta_pierces", "nan", "restart", "sign",
                                  "tension", "refine", "forcing", "precond_precision", "outer_precision"])
def test_setup_rejects_invalid_input(L, case):
    mesh = W.mesh_box(9, 5, 0.4, 0.4)
    topo = W.gaussian_bumps(mesh, [(0.1, 0.7, 0.0, 0.0)])
    F, opts = 0.7, None
    if case == "N":
        mesh = W.Mesh(N=3, M=5, x1=-1, y1=-1, dx=0.4, dy=0.4)
        topo = W.flat_topography(mesh)
    elif case == "M":
        mesh = W.Mesh(N=9, M=2, x1=-1, y1=-1, dx=0.4, dy=0.4)
        topo = W.flat_topography(mesh)
    elif case == "dx":
        mesh = W.Mesh(N=9, M=5, x1=-1, y1=-1, dx=0.0, dy=0.4)
    elif case == "F":
        F = -0.5
    elif case == "half_y1":
        mesh = W.Mesh(N=9, M=5, x1=-1, y1=-0.4, dx=0.4, dy=0.4, half=1)
    elif case == "beta_pierces":
        topo = W.gaussian_bumps(mesh, [(1.0 + 0.5 * F * F + 0.05, 0.7, 0.0, 0.0)])  # top above F^2/2
    elif case == "nan":
        b = topo.beta.copy()
        b[3] = np.nan
        topo = W.Topography(b, topo.beta_x, topo.beta_y)
    elif case == "restart":
        opts = bfs.default_options(gmres_restart=0)
    elif case == "sign":
        opts = bfs.default_options(sign_I4=0.5)
    elif case == "tension":
        opts = bfs.default_options(surface_tension=-0.1)
    elif case == "refine":
        opts = bfs.default_options(refine_below=-1.0)
    elif case == "forcing":
        opts = bfs.default_options(forcing=2)
    elif case == "precond_precision":
        opts = bfs.default_options(precond_precision=bfs.BFS_DF64)
    elif case == "outer_precision":
        opts = bfs.default_options(outer_precision=bfs.BFS_FP32C)
    rc, ctx = _setup(mesh, topo, F, opts)
    assert rc == bfs.BFS_EINVAL and not ctx.value
    assert bfs.lib().bfs_last_error(None)


def test_null_arguments_are_rejected(L):
    assert L.bfs_residual(None, None, None, 0, None) == bfs.BFS_EINVAL
    assert L.bfs_solve(None, None, None, None) == bfs.BFS_EINVAL
    assert L.bfs_precond_apply(None, None, None, None) == bfs.BFS_EINVAL
    L.bfs_destroy(None)


def test_tall_bump_below_the_bernoulli_bound_is_accepted(L):
    """A bottom above z = 0 is valid as long as it stays below F^2/2 (the
    supercritical runs of Sec. 5.2): validation passes, so the call gets as
    far as the device (it fails with BFS_ECUDA only where there is no GPU)."""
    mesh = W.mesh_box(9, 5, 0.4, 0.4)
    F = 3.0
    topo = W.gaussian_bumps(mesh, [(1.5, 0.7, 0.0, 0.0)])  # top at z = 0.5 < F^2/2 = 4.5
    rc, ctx = _setup(mesh, topo, F, None)
    assert rc in (bfs.BFS_OK, bfs.BFS_ECUDA, bfs.BFS_ENOMEM)
    if rc == bfs.BFS_OK:
        L.bfs_destroy(ctx)


@pytest.mark.parametrize("case", ["inf_dx", "nan_x1", "nan_n_rad", "too_many_nodes", "inf_y1"])
def test_static_residual_rejects_invalid_input_before_device_work(L, case):
    """bfs_residual_static checks its sizes (before any int arithmetic on them)
    and every floating-point argument on the host, like bfs_setup."""
    m = bfs.bfs_mesh(N=23, M=9, half_domain=0, x1=-3.3, y1=-1.4, dx=0.3, dy=0.35)
    n_rad = 0.05
    if case == "inf_dx":
        m.dx = float("inf")
    elif case == "nan_x1":
        m.x1 = float("nan")
    elif case == "inf_y1":
        m.y1 = float("inf")
    elif case == "nan_n_rad":
        n_rad = float("nan")
    else:
        m.N, m.M = 1 << 14, 1 << 14
    dummy = ctypes.c_void_p(16)  # never dereferenced: the checks come first
    rc = L.bfs_residual_static(ctypes.byref(m), dummy, dummy, dummy, 0.8, n_rad, -1.0, dummy, dummy,
                               bfs.BFS_FP64, None)
    assert rc == bfs.BFS_EINVAL
    assert L.bfs_static_last_error()
