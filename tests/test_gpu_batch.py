"""Batched sweeps: the persistent multi-instance pair kernel and the lockstep
batched solve against the single-instance path and the oracle."""
import numpy as np
import pytest

import oracle as O
from paper_1709_08803_gb300 import workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1709_08803_gb300 import build
    build.build()


def _small_batch(B=6, seed=11):
    """Uneven small meshes with modest bumps and subcritical F: problems the
    single-instance solver converges on (config-3's wide random bumps do not
    fit on domains this small)."""
    rng = np.random.default_rng(W.SEED_BASE + seed)
    meshes, topos, Fs = [], [], []
    for i in range(B):
        N = [31, 37, 43, 49][i % 4]
        mesh = W.mesh_box(N, (N - 1) // 3 + 1, 0.3, 0.3)
        eps, delta = float(rng.uniform(0.05, 0.12)), float(rng.uniform(0.5, 0.9))
        meshes.append(mesh)
        topos.append(W.gaussian_bumps(mesh, [(eps, delta, float(rng.uniform(-0.5, 0.5)), 0.0)]))
        Fs.append(0.6 + 0.1 * (i % 3))
    return meshes, topos, Fs


def _dev(a):
    return torch.tensor(np.asarray(a), dtype=torch.float64, device="cuda")


def test_batched_residual_equals_single_instance():
    from paper_1709_08803_gb300 import bfs
    meshes, topos, Fs = _small_batch()
    b = bfs.Batch(meshes, topos, Fs)
    us = [_dev(W.smooth_guess(m, i)) for i, m in enumerate(meshes)]
    for tuned in (False, True):
        if tuned:
            ms = b.autotune()
            t = b.tuning()
            assert ms > 0 and t["tpb"] > 0
        got = b.residual(us)
        for i in range(b.B):
            ref = b.instance_residual(i, us[i], precision=bfs.BFS_FP32C)
            assert torch.equal(got[i], ref), i  # same per-target arithmetic
    # and the FP32C bar against the oracle
    for i in range(b.B):
        P = O.problem(meshes[i], Fs[i])
        r, sc = O.residual(P, topos[i], us[i].cpu().numpy(), with_scale=True)
        rel = np.abs(got[i].cpu().numpy() - r) / (sc + 1e-300)
        assert rel.max() <= 2e-6
    b.close()


def test_batched_solve_matches_single_solves():
    from paper_1709_08803_gb300 import bfs
    meshes, topos, Fs = _small_batch()
    opts = dict(tol=1e-10, krylov_precision=bfs.BFS_FP32C, outer_precision=bfs.BFS_DF64, eta=1e-2)
    b = bfs.Batch(meshes, topos, Fs, bfs.default_options(**opts))
    us = b.flat_guesses()
    rc, stats = b.solve(us)
    assert rc == bfs.BFS_OK, stats
    for i in range(b.B):
        assert stats[i]["status"] == 0 and stats[i]["fnorm_inf"] <= 1e-10
        ctx = bfs.Context(meshes[i], topos[i], Fs[i], bfs.default_options(**opts))
        u1 = ctx.flat_guess()
        st1 = ctx.solve(u1)
        # same iteration; the source splits differ, so the rounding of the
        # partial sums (and the path, slightly) differs
        assert abs(st1["newton_its"] - stats[i]["newton_its"]) <= 1
        assert (u1 - us[i]).abs().max().item() <= 1e-7
        P = O.problem(meshes[i], Fs[i])
        assert np.abs(O.residual(P, topos[i], us[i].cpu().numpy())).max() <= 2e-10
        ctx.close()
    b.close()


def test_batch_rejects_bad_instance():
    from paper_1709_08803_gb300 import bfs
    meshes, topos, Fs = _small_batch(B=3)
    Fs[1] = -1.0
    with pytest.raises(bfs.BfsError) as e:
        bfs.Batch(meshes, topos, Fs)
    assert e.value.code == bfs.BFS_EINVAL and "instance 1" in str(e.value)
