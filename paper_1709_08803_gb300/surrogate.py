"""Learned initial guess for the JFNK solve (an addition; the paper has none).

A small convolutional neural operator (the CUDA kernels behind bfs_cno_* in
csrc/cno.cu: four dilated 3x3 convolutions, BF16 tensor-core contractions with
FP32 accumulation) maps the bottom B = beta + 1, the Froude number and the
node coordinates of a mesh to the nodal fields zeta, phi - x and psi - x.  Its
output is turned into an unknown vector on the device and handed to the
Newton iteration, which accepts it only by converging to the same tolerance;
the uniform-stream guess remains the fallback.

This module holds the ctypes binding (argument marshalling only), the
feature construction, training-data generation with the solver itself, the
training loop (all arithmetic in the CUDA kernels) and the A/B evaluation.
"""
from __future__ import annotations

import ctypes
import math
import os
import time

import numpy as np

from . import bfs
from . import workloads as W

WEIGHTS = os.path.join(os.path.dirname(os.path.abspath(__file__)), "weights", "cno_181x61.npz")
_VP = ctypes.c_void_p


def _lib():
    L = bfs.lib()
    if not getattr(L, "_cno_ready", False):
        C = ctypes.POINTER
        L.bfs_cno_num_params.restype = ctypes.c_int
        L.bfs_cno_create.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int, C(_VP)]
        L.bfs_cno_destroy.argtypes = [_VP]
        L.bfs_cno_last_error.argtypes = [_VP]
        L.bfs_cno_last_error.restype = ctypes.c_char_p
        L.bfs_cno_set_params.argtypes = [_VP, C(ctypes.c_float), C(ctypes.c_float)]
        L.bfs_cno_get_params.argtypes = [_VP, C(ctypes.c_float)]
        L.bfs_cno_forward.argtypes = [_VP, _VP, ctypes.c_int, _VP, _VP]
        L.bfs_cno_gradient.argtypes = [_VP, _VP, _VP, ctypes.c_int, C(ctypes.c_float), C(ctypes.c_float), _VP]
        L.bfs_cno_train_step.argtypes = [_VP, _VP, _VP, ctypes.c_int, ctypes.c_float, _VP]
        L.bfs_cno_read_loss.argtypes = [_VP, C(ctypes.c_float), _VP]
        L.bfs_cno_guess.argtypes = [_VP, _VP, _VP, _VP, _VP]
        L.bfs_cno_solve.argtypes = [_VP, _VP, _VP, _VP, C(bfs.bfs_stats), C(ctypes.c_int), _VP]
        L.bfs_cno_solve_host.argtypes = [_VP, _VP, _VP, _VP, C(bfs.bfs_stats), C(ctypes.c_int), _VP]
        L._cno_ready = True
    return L


# Layer shapes (must match csrc/cno.cu): (cin, cout, dilation)
LAYERS = [(16, 32, 1), (32, 32, 3), (32, 32, 9), (32, 16, 27)]
IN_REAL, OUT_REAL = 4, 3


def num_params() -> int:
    return _lib().bfs_cno_num_params()


def init_params(seed: int = 0) -> np.ndarray:
    """He-style initialisation; padded input channels and unused outputs are 0."""
    rng = np.random.default_rng(W.SEED_BASE + 500 + seed)
    out = []
    for li, (cin, cout, _) in enumerate(LAYERS):
        real_in = IN_REAL if li == 0 else cin
        std = math.sqrt(2.0 / (9 * real_in)) * (0.5 if li == len(LAYERS) - 1 else 1.0)
        w = rng.standard_normal((cout, 9, cin)) * std
        if li == 0:
            w[:, :, IN_REAL:] = 0.0
        if li == len(LAYERS) - 1:
            w[OUT_REAL:, :, :] = 0.0
        out.append(w.ravel())
        out.append(np.zeros(cout))
    p = np.concatenate(out).astype(np.float32)
    assert p.size == num_params()
    return p


class CNO:
    def __init__(self, H: int, Wd: int, batch_max: int = 16):
        import torch
        if not torch.cuda.is_available():
            raise RuntimeError("CUDA device required")
        h = _VP()
        rc = _lib().bfs_cno_create(H, Wd, batch_max, ctypes.byref(h))
        if rc:
            raise bfs.BfsError(rc, _lib().bfs_cno_last_error(None).decode())
        self._n = h
        self.H, self.W, self.batch_max = H, Wd, batch_max
        self.np = num_params()
        self.scale = np.ones(3, dtype=np.float32)

    def _check(self, rc):
        if rc:
            raise bfs.BfsError(rc, _lib().bfs_cno_last_error(self._n).decode())

    def close(self):
        if getattr(self, "_n", None):
            _lib().bfs_cno_destroy(self._n)
            self._n = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _images(self, x, ch: int, Bt: int | None = None) -> int:
        """Checks x is a contiguous float32 CUDA tensor [Bt][H][W][ch] with
        1 <= Bt <= batch_max (and Bt as given); returns Bt."""
        import torch
        bfs._require(isinstance(x, torch.Tensor) and x.is_cuda and x.dtype == torch.float32
                     and x.is_contiguous() and x.dim() == 4 and tuple(x.shape[1:]) == (self.H, self.W, ch),
                     f"expected a contiguous float32 CUDA tensor [Bt, {self.H}, {self.W}, {ch}]")
        n = int(x.shape[0])
        bfs._require(1 <= n <= self.batch_max and (Bt is None or n == Bt),
                     f"batch of {n} images (at most {self.batch_max}, matching the inputs)")
        return n

    def set_params(self, p: np.ndarray, scale=None):
        p = np.ascontiguousarray(p, dtype=np.float32).ravel()
        bfs._require(p.size == self.np, f"expected {self.np} parameters")
        if scale is not None:
            self.scale = np.ascontiguousarray(scale, dtype=np.float32).ravel()
            bfs._require(self.scale.size == 3, "expected 3 output scales")
        F = ctypes.POINTER(ctypes.c_float)
        self._check(_lib().bfs_cno_set_params(self._n, p.ctypes.data_as(F), self.scale.ctypes.data_as(F)))

    def get_params(self) -> np.ndarray:
        p = np.empty(self.np, dtype=np.float32)
        self._check(_lib().bfs_cno_get_params(self._n, p.ctypes.data_as(ctypes.POINTER(ctypes.c_float))))
        return p

    def forward(self, x):
        """x: CUDA float32 [Bt, H, W, 4] -> CUDA float32 [Bt, H, W, 16]."""
        import torch
        Bt = self._images(x, 4)
        y = torch.empty((Bt, self.H, self.W, 16), dtype=torch.float32, device="cuda")
        self._check(_lib().bfs_cno_forward(self._n, _VP(x.data_ptr()), Bt, _VP(y.data_ptr()), bfs._stream(None)))
        return y

    def gradient(self, x, t):
        self._images(t, 3, self._images(x, 4))
        g = np.empty(self.np, dtype=np.float32)
        loss = ctypes.c_float()
        F = ctypes.POINTER(ctypes.c_float)
        self._check(_lib().bfs_cno_gradient(self._n, _VP(x.data_ptr()), _VP(t.data_ptr()), x.shape[0],
                                            g.ctypes.data_as(F), ctypes.byref(loss), bfs._stream(None)))
        return g, loss.value

    def train_step(self, x, t, lr: float):
        self._images(t, 3, self._images(x, 4))
        self._check(_lib().bfs_cno_train_step(self._n, _VP(x.data_ptr()), _VP(t.data_ptr()), x.shape[0],
                                              float(lr), bfs._stream(None)))

    def loss(self) -> float:
        v = ctypes.c_float()
        self._check(_lib().bfs_cno_read_loss(self._n, ctypes.byref(v), bfs._stream(None)))
        return v.value

    def solve(self, ctx: bfs.Context, x, u, stream=None):
        """Solve from the network's guess for features x (CUDA float32 [1, M, N, 4])
        into the device vector u, the uniform stream as fallback; returns the
        summed stats with 'fallback' (the final status is in 'status')."""
        self._images(x, 4, 1)
        st = bfs.bfs_stats()
        fb = ctypes.c_int()
        rc = _lib().bfs_cno_solve(self._n, ctx._ctx, _VP(x.data_ptr()), ctx._vec(u), ctypes.byref(st),
                                  ctypes.byref(fb), bfs._stream(stream))
        if rc not in (0, bfs.BFS_ENOCONV, bfs.BFS_ELINESEARCH, bfs.BFS_EBREAKDOWN, bfs.BFS_ENAN, bfs.BFS_ETIMEOUT):
            self._check(rc)
        d = st.as_dict()
        d["fallback"] = bool(fb.value)
        return d

    def solve_host(self, ctx: bfs.Context, x_host: np.ndarray, u_host: np.ndarray, stream=None):
        """solve on host buffers: features x_host (float32 [M, N, 4] or [1, M, N, 4],
        C-contiguous) in, the solution into u_host (float64, n); both copies in the call."""
        if x_host.dtype != np.float32 or not x_host.flags["C_CONTIGUOUS"] or x_host.size != self.H * self.W * 4:
            raise ValueError("x_host: C-contiguous float32 with M*N*4 values")
        if u_host.dtype != np.float64 or not u_host.flags["C_CONTIGUOUS"] or u_host.size != ctx.n:
            raise ValueError("u_host: C-contiguous float64 of the context's length")
        st = bfs.bfs_stats()
        fb = ctypes.c_int()
        rc = _lib().bfs_cno_solve_host(self._n, ctx._ctx, _VP(x_host.ctypes.data), _VP(u_host.ctypes.data),
                                       ctypes.byref(st), ctypes.byref(fb), bfs._stream(stream))
        if rc not in (0, bfs.BFS_ENOCONV, bfs.BFS_ELINESEARCH, bfs.BFS_EBREAKDOWN, bfs.BFS_ENAN, bfs.BFS_ETIMEOUT):
            self._check(rc)
        d = st.as_dict()
        d["fallback"] = bool(fb.value)
        return d

    def guess(self, ctx: bfs.Context, x, u=None):
        """Unknown vector for ctx from features x (CUDA float32 [1, M, N, 4])."""
        import torch
        self._images(x, 4, 1)
        if u is None:
            u = torch.empty(ctx.n, dtype=torch.float64, device="cuda")
        self._check(_lib().bfs_cno_guess(self._n, ctx._ctx, _VP(x.data_ptr()), ctx._vec(u),
                                         bfs._stream(None)))
        return u


def features(mesh, topo, F: float) -> np.ndarray:
    """Input channels on the nodal grid, [M, N, 4]: B / 0.3, (F - 0.95) / 0.45 and
    the node coordinates scaled to [-1, 1]."""
    X, Y = np.meshgrid(mesh.x(), mesh.y())
    B = (topo.beta + 1.0).reshape(mesh.M, mesh.N)
    xs = (X - 0.5 * (X.max() + X.min())) / (0.5 * (X.max() - X.min()))
    ys = (Y - 0.5 * (Y.max() + Y.min())) / max(1e-12, 0.5 * (Y.max() - Y.min()))
    f = np.stack([B / 0.3, np.full_like(B, (F - 0.95) / 0.45), xs, ys], axis=-1)
    return f.astype(np.float32)


def scaled(topo, s: float):
    """The bottom with every bump height multiplied by s (beta + 1 scales linearly)."""
    return W.Topography(-1.0 + s * (topo.beta + 1.0), s * topo.beta_x, s * topo.beta_y)


def solve_with_continuation(ctx, topo, u0=None, stages=(1.0 / 3.0, 2.0 / 3.0, 1.0), direct_first=True,
                            on_stage=None):
    """Solve on ctx for `topo`: first directly from u0 (the uniform stream when
    None), and if that fails by continuation in bump height through `stages`,
    each stage starting from the previous solution (the paper's route to large
    amplitudes).  Returns (u, status, cost) with cost = summed Newton and Krylov
    iterations, residual evaluations and stages used."""
    cost = {"newton": 0, "krylov": 0, "evals": 0, "stages": 0}

    def add(st):
        cost["newton"] += st["newton_its"]
        cost["krylov"] += st["krylov_its"]
        cost["evals"] += st["residual_evals_fp64"] + st["residual_evals_fp32"]
        cost["stages"] += 1

    if direct_first:
        ctx.set_topography(topo)
        u = ctx.flat_guess() if u0 is None else u0.clone()
        st = ctx.solve(u, raise_on_error=False)
        add(st)
        if st["status"] == 0:
            return u, 0, cost
    u = ctx.flat_guess()
    status = -1
    for sfac in stages:
        ts = scaled(topo, sfac)
        ctx.set_topography(ts)
        st = ctx.solve(u, raise_on_error=False)
        add(st)
        status = st["status"]
        if status != 0:
            break
        if on_stage is not None and sfac < 1.0:
            on_stage(ts, u)
    return u, status, cost


def bin_context(ctxs, mesh, topo, F, opts, bin_width=0.02):
    """A context for F from the per-bin cache (one factored preconditioner per
    bin of Froude numbers; F itself is set exactly).  opts: options, or a
    function of the bin's Froude number returning them."""
    key = int(F / bin_width)
    if key not in ctxs:
        Fb = (key + 0.5) * bin_width
        c = bfs.Context(mesh, topo, Fb, opts(Fb) if callable(opts) else opts)
        c.precond_factor()
        ctxs[key] = c
    c = ctxs[key]
    c.set_froude(F)
    return c


def solver_options(tol: float = 1e-8, budget_s: float = 3.0, F: float | None = None):
    """The mixed form with early exits: GMRES capped per Newton step (80
    iterations for subcritical F; 400 for supercritical F, whose solves need
    50-600 with the linear preconditioner) and the solve abandoned after 3
    consecutive Newton steps whose GMRES ended above tolerance (most draws near
    F = 1 or with wide bumps have no steady solution; this makes a failed
    attempt cost a fraction of a second, not seconds)."""
    sup = F is not None and F > 1.0
    return bfs.default_options(tol=tol, krylov_precision=bfs.BFS_FP32C, outer_precision=bfs.BFS_DF64,
                               eta=1e-2, max_newton=25, max_krylov=400 if sup else 80,
                               time_budget_s=2.0 * budget_s if sup else budget_s,
                               precond_precision=bfs.BFS_FP32C, refine_below=1e-5, stall_newton=3, forcing=1)


def describe(topo_desc) -> dict:
    kind, params = topo_desc
    if kind == "ridge":
        return {"kind": "ridge", "amp": params[0], "width": params[1]}
    return {"kind": f"{len(params)} bumps", "amp": max(b[0] for b in params),
            "width": max(b[1] for b in params)}


def sample_problem_desc(rng, mesh):
    """One draw of the batched-sweep distribution (F, 1-3 bumps or a ridge) on
    `mesh`: (topography, F, description of the draw for the records)."""
    F = float(rng.uniform(0.5, 1.4))
    if rng.uniform() < 0.8:
        nb = int(rng.integers(1, 4))
        bumps = [(float(rng.uniform(0.05, 0.3)), float(rng.uniform(0.5, 2.0)),
                  float(rng.uniform(-2, 2)), float(rng.uniform(-2, 2))) for _ in range(nb)]
        return W.gaussian_bumps(mesh, bumps), F, ("bumps", bumps)
    rd = (float(rng.uniform(0.05, 0.3)), float(rng.uniform(0.5, 2.0)), float(rng.uniform(-2, 2)))
    return W.gaussian_bumps(mesh, [], ridges=[rd]), F, ("ridge", rd)


def generate(n: int, seed: int, mesh=None, tol: float = 1e-8, time_budget_s: float | None = None,
             max_attempts: int | None = None, with_stages: bool = True, log=None):
    """Draw problems from the batched-sweep distribution on `mesh` (default
    181 x 61) and solve each directly, then by continuation in bump height,
    until n solutions have been collected (or the time budget or attempt limit
    runs out).  with_stages also keeps the converged intermediate stages of a
    continuation (the same draw at 1/3 and 2/3 of its bump heights).
    Returns (features [k, M, N, 4], targets [k, M, N, 3] = zeta, phi - x,
    psi - x of the k solutions, records of every attempt)."""
    import torch
    mesh = mesh or W.config_paper_scale()[0]
    rng = np.random.default_rng(W.SEED_BASE + 7000 + seed)
    xs = np.zeros((n, mesh.M, mesh.N, 4), dtype=np.float32)
    ys = np.zeros((n, mesh.M, mesh.N, 3), dtype=np.float32)
    recs, ctxs = [], {}
    opts = lambda Fb: solver_options(tol, F=Fb)
    xg = torch.tensor(mesh.x(), device="cuda").view(1, -1)
    t0 = time.time()
    k = 0
    stage_samples = 0

    def keep(c, topo, F, u):
        nonlocal k
        if k >= n:
            return
        xs[k] = features(mesh, topo, F)
        nv = c.unpack(u)
        ys[k, :, :, 0] = nv["zeta"].float().cpu().numpy()
        ys[k, :, :, 1] = (nv["phi"] - xg).float().cpu().numpy()
        ys[k, :, :, 2] = (nv["psi"] - xg).float().cpu().numpy()
        k += 1

    while k < n:
        if max_attempts is not None and len(recs) >= max_attempts:
            break
        if time_budget_s is not None and time.time() - t0 > time_budget_s:
            break
        topo, F, desc = sample_problem_desc(rng, mesh)
        c = bin_context(ctxs, mesh, topo, F, opts)
        staged = []
        u, status, cost = solve_with_continuation(
            c, topo, on_stage=(lambda ts, us: staged.append((ts, us.clone()))) if with_stages else None)
        recs.append({"F": F, "status": status, **describe(desc), **cost})
        if status == 0:
            keep(c, topo, F, u)
        for ts, us in staged:  # converged intermediate amplitudes of this draw
            keep(c, ts, F, us)
            stage_samples += 1
        if log and len(recs) % 100 == 0:
            log(f"attempted {len(recs)}, collected {k} ({stage_samples} intermediate stages) "
                f"in {time.time() - t0:.1f} s")
    for c in ctxs.values():
        c.close()
    return xs[:k], ys[:k], recs


def train(xs, ys, epochs: int = 60, batch: int = 16, lr: float = 2e-3, seed: int = 0, log=None):
    """Adam on the mean squared error of the scaled targets; returns (params,
    scale, losses).  Only converged samples should be passed."""
    import torch
    n, H, Wd, _ = xs.shape
    scale = np.maximum(ys.reshape(-1, 3).std(axis=0), 1e-6).astype(np.float32)
    net = CNO(H, Wd, batch)
    net.set_params(init_params(seed), scale)
    X = torch.tensor(xs, device="cuda")
    T = torch.tensor(ys / scale, device="cuda")
    g = torch.Generator(device="cpu").manual_seed(seed)
    batch = max(1, min(batch, n))
    steps = epochs * max(1, n // batch)
    losses, k = [], 0
    for ep in range(epochs):
        perm = torch.randperm(n, generator=g)
        ep_loss = []
        for b0 in range(0, n - batch + 1, batch):
            idx = perm[b0:b0 + batch].cuda()
            lr_k = lr * 0.5 * (1 + math.cos(math.pi * k / steps))
            net.train_step(X[idx].contiguous(), T[idx].contiguous(), lr_k)
            k += 1
            if b0 == 0 or b0 + 2 * batch > n:
                ep_loss.append(net.loss())
        losses.append(float(np.mean(ep_loss)))
        if log and (ep % 10 == 0 or ep == epochs - 1):
            log(f"epoch {ep}: loss {losses[-1]:.4e}")
    p = net.get_params()
    net.close()
    return p, scale, losses


def save(path, params, scale, meta: dict):
    os.makedirs(os.path.dirname(path), exist_ok=True)
    np.savez(path, params=params, scale=scale, **{k: np.asarray(v) for k, v in meta.items()})


def load(path=WEIGHTS):
    d = np.load(path)
    return d["params"], d["scale"]
