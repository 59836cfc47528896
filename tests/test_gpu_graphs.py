"""Arnoldi steps launched as conditional CUDA graphs (the step behind a
device-side end-of-cycle flag, the next step queued before the host reads
this one's scalars) against the same solve with every kernel launched one by
one (profiling mode): identical iterates, so identical Newton and Krylov
counts and bit-identical u, on the legacy default stream (the solve moves to
the context's own stream) and on a side stream."""
import numpy as np
import pytest

from paper_1709_08803_gb300 import workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1709_08803_gb300 import build
    build.build()


def _solve(mesh, topo, F, profile, stream):
    from paper_1709_08803_gb300 import bfs
    opts = bfs.default_options(tol=1e-8, krylov_precision=bfs.BFS_FP32C, outer_precision=bfs.BFS_DF64,
                               eta=1e-2, refine_below=1e-5, precond_precision=bfs.BFS_FP32C)
    c = bfs.Context(mesh, topo, F, opts)
    if profile:
        c.profile_enable(True)
    u = c.flat_guess()
    if stream is not None:
        stream.wait_stream(torch.cuda.current_stream())
        with torch.cuda.stream(stream):
            st = c.solve(u, raise_on_error=False)
        torch.cuda.current_stream().wait_stream(stream)
    else:
        st = c.solve(u, raise_on_error=False)
    torch.cuda.synchronize()
    info = c.solver_info()
    out = u.cpu().numpy()
    c.close()
    return st, info, out


@pytest.mark.parametrize("side_stream", [False, True])
def test_conditional_step_graphs_match_unrolled_solve(side_stream):
    mesh = W.mesh_box(61, 21, 0.3, 0.3)
    topo = W.gaussian_bumps(mesh, [(0.2, 1.0 / np.sqrt(2.0), 0.0, 0.0)])
    F = 0.7
    st0, info0, u0 = _solve(mesh, topo, F, True, None)
    s = torch.cuda.Stream() if side_stream else None
    st1, info1, u1 = _solve(mesh, topo, F, False, s)
    print(info0, info1, st1["newton_its"], st1["krylov_its"])
    assert st0["status"] == 0 and st1["status"] == 0
    assert info0["step_graphs"] == 0
    assert info1["step_graphs"] > 0 and info1["conditional"] == info1["step_graphs"]
    assert info1["own_stream"] == (not side_stream)
    assert (st0["newton_its"], st0["krylov_its"]) == (st1["newton_its"], st1["krylov_its"])
    assert np.array_equal(u0, u1)
