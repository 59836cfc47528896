"""The learned initial guess (the convolutional network's output as Newton's
starting point) on held-out draws of its training distribution.

The network is trained on solutions the solver generates for draws of the
batched-sweep distribution (seed SEED_BASE + 7000); the held-out draws here
come from another seed (SEED_BASE + 9000), as in train_guess.evaluate.  The
guess is accepted only through Newton to the solver's tolerance; when the solve
from it fails, the library falls back to the uniform stream.
"""
import os

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


@pytest.fixture(scope="module")
def net_and_draws():
    from paper_1709_08803_gb300 import surrogate as S
    if not os.path.exists(S.WEIGHTS):
        pytest.skip("no trained weights")
    mesh = W.config_paper_scale()[0]
    params, scale = S.load(S.WEIGHTS)
    net = S.CNO(mesh.M, mesh.N, 1)
    net.set_params(params, scale)
    rng = np.random.default_rng(W.SEED_BASE + 9000)
    draws = []
    while len(draws) < 12:  # held-out subcritical bump draws, the regime where most draws converge
        topo, F, desc = S.sample_problem_desc(rng, mesh)
        if desc[0] == "bumps" and F < 0.8:
            draws.append((topo, F, desc))
    yield mesh, net, draws
    net.close()


def test_learned_guess_on_held_out_draws(net_and_draws):
    """From the guess, Newton converges to the same tolerance on every held-out
    draw that converges from the uniform stream, and on average it needs no
    more Newton steps than from the uniform stream."""
    from paper_1709_08803_gb300 import surrogate as S
    mesh, net, draws = net_and_draws
    ctxs, rows = {}, []
    opts = lambda Fb: S.solver_options(F=Fb)
    for topo, F, desc in draws:
        c = S.bin_context(ctxs, mesh, topo, F, opts)
        c.set_topography(topo)
        u = c.flat_guess()
        flat = c.solve(u, raise_on_error=False)
        if flat["status"] != 0:
            continue
        x = torch.tensor(S.features(mesh, topo, F)[None], device="cuda")
        ul = torch.empty_like(u)
        learned = net.solve(c, x, ul)
        assert learned["status"] == 0 and learned["fnorm_inf"] <= 1e-8
        rows.append((F, flat["newton_its"], learned["newton_its"], flat["krylov_its"], learned["krylov_its"],
                     learned["fallback"]))
    for c in ctxs.values():
        c.close()
    assert len(rows) >= 6, rows
    r = np.array([row[:5] for row in rows], dtype=float)
    saved_newton, saved_krylov = r[:, 1].mean() - r[:, 2].mean(), r[:, 3].mean() - r[:, 4].mean()
    print(f"held-out draws: {len(rows)}; Newton uniform stream {r[:, 1].mean():.2f}, learned {r[:, 2].mean():.2f} "
          f"(saved {saved_newton:.2f}); Krylov {r[:, 3].mean():.1f} vs {r[:, 4].mean():.1f} (saved {saved_krylov:.1f}); "
          f"fallbacks {sum(row[5] for row in rows)}")
    assert saved_newton >= 0.0


def test_failed_guess_falls_back_to_the_uniform_stream(net_and_draws):
    """A guess from which Newton cannot start (non-finite features give a
    non-finite guess) gives way to the method without the network, which
    converges; the host-buffer entry point returns the same solution."""
    from paper_1709_08803_gb300 import bfs
    from paper_1709_08803_gb300 import surrogate as S
    mesh, net, draws = net_and_draws
    topo, F, _ = draws[0]
    c = bfs.Context(mesh, topo, F, S.solver_options(F=F))
    bad = torch.full((1, mesh.M, mesh.N, 4), float("nan"), dtype=torch.float32, device="cuda")
    u = torch.empty(c.n, dtype=torch.float64, device="cuda")
    st = net.solve(c, bad, u)
    assert st["fallback"] and st["status"] == 0
    u_flat = c.flat_guess()
    assert c.solve(u_flat, raise_on_error=False)["status"] == 0
    assert torch.allclose(u, u_flat, rtol=0.0, atol=1e-8)
    # the host-buffer form of the learned solve
    x = torch.tensor(S.features(mesh, topo, F)[None], device="cuda")
    ud = torch.empty_like(u)
    sd = net.solve(c, x, ud)
    uh = np.empty(c.n)
    sh = net.solve_host(c, S.features(mesh, topo, F)[None].copy(), uh)
    assert sd["status"] == 0 and sh["status"] == 0 and sd["fallback"] == sh["fallback"]
    assert np.allclose(uh, ud.cpu().numpy(), rtol=0.0, atol=1e-8)
    c.close()
