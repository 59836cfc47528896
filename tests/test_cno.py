"""The initial-guess network: the FP64 CPU reference is pinned by central
finite differences; the BF16 tensor-core kernels are checked against it."""
import numpy as np
import pytest

from oracle import cno_ref as R

LAYERS = R.LAYERS


def _params(seed=0, scale=1.0):
    rng = np.random.default_rng(seed)
    out = []
    for li, (cin, cout, _) in enumerate(LAYERS):
        real = R.IN_REAL if li == 0 else cin
        w = rng.standard_normal((cout, 9, cin)) * np.sqrt(2.0 / (9 * real)) * scale
        if li == 0:
            w[:, :, R.IN_REAL:] = 0
        out += [w.ravel(), 0.1 * rng.standard_normal(cout)]
    return np.concatenate(out)


def test_reference_gradient_matches_finite_differences():
    rng = np.random.default_rng(1)
    p = _params(1)
    x = rng.standard_normal((2, 7, 11, 4))
    t = rng.standard_normal((2, 7, 11, 3))
    _, g = R.loss_grad(p, x, t, emulate=False)
    idx = rng.choice(p.size, 40, replace=False)
    h = 1e-6
    for i in idx:
        e = np.zeros_like(p)
        e[i] = h
        fd = (R.loss_grad(p + e, x, t, emulate=False)[0] - R.loss_grad(p - e, x, t, emulate=False)[0]) / (2 * h)
        assert abs(fd - g[i]) <= 1e-6 * max(1.0, abs(fd)), (i, fd, g[i])


def test_bf16_rounding_helper():
    v = np.array([1.0, 1.00390625, 1.005859375, -3.1415926, 65504.0])
    r = R.bf16(v)
    assert r[0] == 1.0 and r[1] == 1.0 and r[2] == 1.0078125
    assert abs(r[3] + 3.140625) < 1e-12


@pytest.mark.gpu
def test_gpu_forward_and_gradient_match_reference():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1709_08803_gb300 import build
    build.build()
    from paper_1709_08803_gb300 import surrogate as S
    rng = np.random.default_rng(3)
    p = _params(3).astype(np.float32)
    x = rng.standard_normal((2, 9, 37, 4)).astype(np.float32)
    t = rng.standard_normal((2, 9, 37, 3)).astype(np.float32)
    net = S.CNO(9, 37, 2)
    net.set_params(p)
    y = net.forward(torch.tensor(x, device="cuda")).cpu().numpy()
    yr, _, _ = R.forward(p.astype(np.float64), x.astype(np.float64))
    assert np.abs(y - yr).max() <= 2e-2 * np.abs(yr).max()
    g, loss = net.gradient(torch.tensor(x, device="cuda"), torch.tensor(t, device="cuda"))
    lr, gr = R.loss_grad(p.astype(np.float64), x.astype(np.float64), t.astype(np.float64))
    assert abs(loss - lr) <= 1e-3 * lr
    assert np.linalg.norm(g - gr) <= 3e-2 * np.linalg.norm(gr)
    # a few steps of Adam reduce the loss
    X, T = torch.tensor(x, device="cuda"), torch.tensor(t, device="cuda")
    losses = []
    for _ in range(30):
        net.train_step(X, T, 1e-2)
        losses.append(net.loss())
    assert losses[-1] < 0.7 * losses[0]
    net.close()
