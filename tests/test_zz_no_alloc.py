"""bfs_residual_static: the residual entry point for callers that cannot
allocate device memory (it keeps all scratch in a static device array).

Checked through the C ABI against bfs_residual, the entry point that owns its
scratch through a context, on two calls in a row with different inputs, within
the residual tolerance the other GPU tests use.  This file is collected last.
"""
import numpy as np
import pytest

import oracle as O
from paper_1709_08803_gb300 import workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL64 = 1e-10  # as in test_gpu_residual.py (per row, relative to the sum of |terms|)
TOL32 = 2e-6


@pytest.fixture(scope="module", autouse=True)
def _built():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1709_08803_gb300 import build
    build.build()


def _dev(a):
    return torch.tensor(np.asarray(a), dtype=torch.float64, device="cuda")


@pytest.mark.parametrize("half", [0, 1])
def test_static_residual_matches_context_residual(half):
    from paper_1709_08803_gb300 import bfs
    mesh = W.mesh_box(41, 13, 0.3, 0.3, half=half)
    F = 0.8
    topo = W.gaussian_bumps(mesh, [(0.15, 0.8, 0.2, 0.0)])
    ctx = bfs.Context(mesh, topo, F)
    b, bx, by = (_dev(a) for a in (topo.beta, topo.beta_x, topo.beta_y))
    P = O.problem(mesh, F)
    for call, seed in enumerate((1, 2)):  # two calls in a row, different inputs
        u = W.smooth_guess(mesh, seed)
        _, sc = O.residual(P, topo, u, with_scale=True)
        ud = _dev(u)
        for prec, tol in ((bfs.BFS_FP64, TOL64), (bfs.BFS_FP32C, TOL32)):
            ref = ctx.residual(ud, precision=prec).cpu().numpy()
            got = bfs.residual_static(mesh, b, bx, by, F, ud, precision=prec).cpu().numpy()
            assert np.all(np.isfinite(got)), (call, prec)
            assert np.all(np.abs(got - ref) <= tol * sc + 1e-13), (call, prec)
    ctx.close()


def test_static_residual_rejects_oversized_mesh():
    from paper_1709_08803_gb300 import bfs
    mesh = W.mesh_box(401, 401, 0.1, 0.1)
    z = torch.zeros(mesh.N * mesh.M, dtype=torch.float64, device="cuda")
    u = torch.zeros(mesh.n_unknowns, dtype=torch.float64, device="cuda")
    with pytest.raises(bfs.BfsError) as e:
        bfs.residual_static(mesh, z - 1.0, z, z, 0.7, u)
    assert e.value.code == bfs.BFS_EINVAL
    assert "too large" in str(e.value)
    assert bfs.lib().bfs_static_scratch_bytes() == 48 << 20
