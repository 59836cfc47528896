"""Plain FP64 CPU reference of the initial-guess network (test infrastructure).

TEST INFRASTRUCTURE ONLY: used by tests/ to check the BF16 tensor-core
kernels of csrc/cno.cu.  Four dilated 3x3 convolutions with zero padding and
SiLU between them; parameters in one vector, per layer the weights
[cout][tap][cin] (tap = 3 (dy + 1) + (dx + 1)) then the biases.  With
emulate=True the values the kernels store in BF16 (inputs, weights,
activations, gradients w.r.t. pre-activations) are rounded to BF16 here too,
so that only accumulation order and the exponential differ.
"""
from __future__ import annotations

import numpy as np

LAYERS = [(16, 32, 1), (32, 32, 3), (32, 32, 9), (32, 16, 27)]
IN_REAL, OUT_REAL = 4, 3


def bf16(a):
    """Round to the nearest BF16 (ties to even), returned as float64."""
    f = np.asarray(a, dtype=np.float32)
    u = f.view(np.uint32).astype(np.uint64)
    r = ((u + 0x7FFF + ((u >> 16) & 1)) >> 16) << 16
    return r.astype(np.uint32).view(np.float32).astype(np.float64)


def unpack(p):
    out, off = [], 0
    for cin, cout, d in LAYERS:
        n = cout * 9 * cin
        w = np.asarray(p[off:off + n], dtype=np.float64).reshape(cout, 9, cin)
        b = np.asarray(p[off + n:off + n + cout], dtype=np.float64)
        out.append((w, b, d))
        off += n + cout
    return out


def _shift(a, oy, ox):
    """a[:, y + oy, x + ox, :] with zeros outside."""
    Bt, H, W, C = a.shape
    o = np.zeros_like(a)
    ys0, ys1 = max(0, -oy), min(H, H - oy)
    xs0, xs1 = max(0, -ox), min(W, W - ox)
    if ys0 < ys1 and xs0 < xs1:
        o[:, ys0:ys1, xs0:xs1, :] = a[:, ys0 + oy:ys1 + oy, xs0 + ox:xs1 + ox, :]
    return o


def conv(a, w, d, sign=1):
    z = 0.0
    for t in range(9):
        oy, ox = (t // 3 - 1) * d * sign, (t % 3 - 1) * d * sign
        z = z + _shift(a, oy, ox) @ w[:, t, :].T
    return z


def silu(z):
    return z / (1.0 + np.exp(-z))


def dsilu(z):
    s = 1.0 / (1.0 + np.exp(-z))
    return s * (1.0 + z * (1.0 - s))


def forward(p, x, emulate=True):
    """x: [Bt, H, W, 4] -> (output [Bt, H, W, 16], layer inputs, pre-activations)."""
    r = bf16 if emulate else (lambda v: np.asarray(v, dtype=np.float64))
    a = np.zeros(x.shape[:3] + (16,))
    a[..., :IN_REAL] = x
    a = r(a)
    acts, zs = [a], []
    L = unpack(p)
    for li, (w, b, d) in enumerate(L):
        z = conv(acts[-1], r(w), d) + b
        zs.append(z)
        if li < len(L) - 1:
            acts.append(r(silu(z)))
    return zs[-1], acts, zs


def loss_grad(p, x, t, emulate=True):
    """Mean squared error over the 3 used outputs and its gradient (vector
    laid out like p)."""
    r = bf16 if emulate else (lambda v: np.asarray(v, dtype=np.float64))
    y, acts, zs = forward(p, x, emulate)
    cnt = y.shape[0] * y.shape[1] * y.shape[2] * OUT_REAL
    d = y[..., :OUT_REAL] - t
    loss = float(np.sum(d * d) / cnt)
    gz = np.zeros_like(y)
    gz[..., :OUT_REAL] = 2.0 * d / cnt
    gz = r(gz)
    L = unpack(p)
    grads = [None] * len(L)
    for li in range(len(L) - 1, -1, -1):
        w, b, dil = L[li]
        a = acts[li]
        gw = np.zeros_like(w)
        for tp in range(9):
            oy, ox = (tp // 3 - 1) * dil, (tp % 3 - 1) * dil
            sa = _shift(a, oy, ox)
            gw[:, tp, :] = np.einsum("bhwn,bhwc->nc", gz, sa)
        gb = gz.sum(axis=(0, 1, 2))
        grads[li] = (gw, gb)
        if li == 0:
            break
        ga = conv(gz, np.transpose(r(w), (2, 1, 0)), dil, sign=-1)
        gz = r(ga * dsilu(zs[li - 1]))
    return loss, np.concatenate([np.concatenate([gw.ravel(), gb]) for gw, gb in grads])
