"""Timeout path of the device-side waits (failure detection without a GPU fault).

The FP32 preconditioner sweeps are a dataflow kernel: each thread spins on the
tag of the vector entries it multiplies, with a bounded number of polls (the
option wait_polls).  The test prepares the task table on the host so that one
wait names a vector slice no task of that launch writes (bfs_debug_stall_sweep),
then checks that the launch ends by itself, that the host reads BFS_ETIMEOUT,
and that the very next apply on the same context is normal.  Nothing traps,
faults or spins without a limit.
"""
import time

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


@pytest.mark.parametrize("chain", ["top_forward", "middle", "bottom_backward"])
def test_sweep_wait_times_out_and_recovers(chain):
    from paper_1709_08803_gb300 import bfs
    mesh = W.Mesh(N=23, M=9, x1=-3.3, y1=-1.4, dx=0.3, dy=0.35)
    h = 2
    ctx = bfs.Context(mesh, W.flat_topography(mesh), 0.8,
                      bfs.default_options(precond_precision=bfs.BFS_FP32C, wait_polls=4000))
    ctx.precond_factor(h)
    r = torch.tensor(np.random.default_rng(14).standard_normal(mesh.n_unknowns), dtype=torch.float64,
                     device="cuda")
    ref = ctx.precond_apply(r).cpu().numpy()
    assert ctx.check_finite()
    tbl, ntask = bfs.sweep_schedule(mesh.M, h, True)
    assert ntask[1] > 0  # this context runs the two-chain schedule
    nblk, out, k = tbl[:, 2], tbl[:, 1], tbl[:, 0]
    t0 = (mesh.M - h) // 2
    if chain == "top_forward":
        task = int(np.flatnonzero((nblk > 0) & (np.arange(len(tbl)) < ntask[0]))[0])
    elif chain == "middle":
        task = int(np.flatnonzero((out == 1) & (k >= t0) & (k < t0 + h))[0])
    else:
        task = int(np.flatnonzero((out == 1) & (k == mesh.M - 1))[0])
    ctx.debug_stall_sweep(task)
    start = time.perf_counter()
    ctx.precond_apply(r)
    with pytest.raises(bfs.BfsError) as e:
        ctx.check_finite()
    elapsed = time.perf_counter() - start
    assert e.value.code == bfs.BFS_ETIMEOUT
    assert elapsed < 20.0, elapsed
    # the same context, the next call: normal, and the same (deterministic) result
    got = ctx.precond_apply(r).cpu().numpy()
    assert ctx.check_finite()
    assert np.array_equal(got, ref)
    ctx.close()
