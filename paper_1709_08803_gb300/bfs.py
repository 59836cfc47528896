"""Python binding of libbfs (include/bfs.h): argument marshalling only.

Every computation runs in the CUDA library; this module converts numpy /
torch arguments to pointers and status codes to exceptions.  It raises
immediately if libbfs.so is missing or CUDA is unavailable: there is no CPU
fallback.  Device buffers are torch CUDA tensors (torch is used for device
memory and streams only).
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libbfs.so")

BFS_OK, BFS_EINVAL, BFS_ECUDA, BFS_ENOMEM, BFS_ENAN = 0, -1, -2, -3, -4
BFS_ENOCONV, BFS_ELINESEARCH, BFS_EBREAKDOWN, BFS_ESINGULAR = -5, -6, -7, -8
BFS_ENOPREC, BFS_ETIMEOUT = -9, -10
BFS_FP64, BFS_FP32C, BFS_DF64 = 0, 1, 2
STATUS_NAMES = {0: "BFS_OK", -1: "BFS_EINVAL", -2: "BFS_ECUDA", -3: "BFS_ENOMEM", -4: "BFS_ENAN",
                -5: "BFS_ENOCONV", -6: "BFS_ELINESEARCH", -7: "BFS_EBREAKDOWN",
                -8: "BFS_ESINGULAR", -9: "BFS_ENOPREC", -10: "BFS_ETIMEOUT"}


class BfsError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"{STATUS_NAMES.get(code, code)}: {msg}")
        self.code = code


class bfs_mesh(ctypes.Structure):
    _fields_ = [("N", ctypes.c_int), ("M", ctypes.c_int), ("half_domain", ctypes.c_int),
                ("x1", ctypes.c_double), ("y1", ctypes.c_double),
                ("dx", ctypes.c_double), ("dy", ctypes.c_double)]


class bfs_topo(ctypes.Structure):
    _fields_ = [("beta", ctypes.POINTER(ctypes.c_double)),
                ("beta_x", ctypes.POINTER(ctypes.c_double)),
                ("beta_y", ctypes.POINTER(ctypes.c_double))]


class bfs_options(ctypes.Structure):
    _fields_ = [("n_rad", ctypes.c_double), ("sign_I4", ctypes.c_double),
                ("half_band", ctypes.c_int), ("tol", ctypes.c_double),
                ("gmres_restart", ctypes.c_int), ("max_newton", ctypes.c_int),
                ("max_krylov", ctypes.c_int), ("eta", ctypes.c_double),
                ("krylov_precision", ctypes.c_int), ("jv_h_rel", ctypes.c_double),
                ("time_budget_s", ctypes.c_double), ("src_splits", ctypes.c_int),
                ("outer_precision", ctypes.c_int), ("precond_precision", ctypes.c_int),
                ("refine_below", ctypes.c_double), ("stall_newton", ctypes.c_int),
                ("surface_tension", ctypes.c_double), ("forcing", ctypes.c_int),
                ("wait_polls", ctypes.c_int)]


class bfs_stats(ctypes.Structure):
    _fields_ = [("newton_its", ctypes.c_int), ("krylov_its", ctypes.c_int),
                ("residual_evals_fp64", ctypes.c_int), ("residual_evals_fp32", ctypes.c_int),
                ("precond_applies", ctypes.c_int),
                ("fnorm_inf", ctypes.c_double), ("fnorm_2", ctypes.c_double),
                ("seconds", ctypes.c_double), ("seconds_residual", ctypes.c_double),
                ("seconds_precond", ctypes.c_double), ("seconds_krylov_other", ctypes.c_double),
                ("status", ctypes.c_int)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


_lib = None
_VP = ctypes.c_void_p


def lib():
    """Load libbfs.so (raises if it was not built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise ImportError(f"libbfs.so not built ({LIB_PATH}); run __graft_entry__.build()")
        L = ctypes.CDLL(LIB_PATH)
        C = ctypes.POINTER
        L.bfs_default_options.argtypes = [C(bfs_options)]
        L.bfs_setup.argtypes = [C(bfs_mesh), C(bfs_topo), ctypes.c_double, C(bfs_options), C(_VP)]
        L.bfs_destroy.argtypes = [_VP]
        L.bfs_last_error.argtypes = [_VP]
        L.bfs_last_error.restype = ctypes.c_char_p
        L.bfs_n_unknowns.argtypes = [_VP]
        L.bfs_pair_evals.argtypes = [_VP]
        L.bfs_pair_evals.restype = ctypes.c_double
        L.bfs_residual.argtypes = [_VP, _VP, _VP, ctypes.c_int, _VP]
        L.bfs_check_finite.argtypes = [_VP, _VP]
        L.bfs_jvp.argtypes = [_VP, _VP, _VP, _VP, _VP, ctypes.c_double, ctypes.c_int, _VP]
        L.bfs_precond_factor.argtypes = [_VP, ctypes.c_int, _VP]
        L.bfs_precond_apply.argtypes = [_VP, _VP, _VP, _VP]
        L.bfs_solve.argtypes = [_VP, _VP, C(bfs_stats), _VP]
        L.bfs_solve_host.argtypes = [_VP, _VP, C(bfs_stats), _VP]
        L.bfs_residual_host.argtypes = [_VP, _VP, _VP, ctypes.c_int, _VP]
        L.bfs_flat_guess.argtypes = [_VP, _VP, _VP]
        L.bfs_unpack.argtypes = [_VP, _VP, _VP, _VP]
        L.bfs_residual_static.argtypes = [C(bfs_mesh), _VP, _VP, _VP, ctypes.c_double, ctypes.c_double,
                                          ctypes.c_double, _VP, _VP, ctypes.c_int, _VP]
        L.bfs_static_last_error.restype = ctypes.c_char_p
        L.bfs_static_scratch_bytes.restype = ctypes.c_size_t
        L.bfs_batch_setup.argtypes = [ctypes.c_int, C(bfs_mesh), C(bfs_topo), C(ctypes.c_double),
                                      C(bfs_options), C(_VP)]
        L.bfs_batch_destroy.argtypes = [_VP]
        L.bfs_batch_last_error.argtypes = [_VP]
        L.bfs_batch_last_error.restype = ctypes.c_char_p
        L.bfs_batch_size.argtypes = [_VP]
        L.bfs_batch_n_unknowns.argtypes = [_VP, ctypes.c_int]
        L.bfs_batch_pair_evals.argtypes = [_VP]
        L.bfs_batch_pair_evals.restype = ctypes.c_double
        L.bfs_batch_instance.argtypes = [_VP, ctypes.c_int]
        L.bfs_batch_instance.restype = _VP
        L.bfs_batch_residual.argtypes = [_VP, C(_VP), C(_VP), _VP]
        L.bfs_batch_autotune.argtypes = [_VP, _VP, C(ctypes.c_double)]
        L.bfs_batch_tuning.argtypes = [_VP, C(ctypes.c_int), C(ctypes.c_int), C(ctypes.c_int),
                                       C(ctypes.c_double)]
        L.bfs_batch_solve.argtypes = [_VP, C(_VP), C(bfs_stats), _VP]
        L.bfs_bottom_pressure.argtypes = [_VP, _VP, _VP, C(ctypes.c_double), _VP]
        L.bfs_set_topography.argtypes = [_VP, C(bfs_topo)]
        L.bfs_set_froude.argtypes = [_VP, ctypes.c_double]
        L.bfs_set_surface_pressure.argtypes = [_VP, _VP]
        L.bfs_profile_enable.argtypes = [_VP, ctypes.c_int]
        L.bfs_profile_read.argtypes = [_VP, ctypes.POINTER(ctypes.c_double),
                                       ctypes.POINTER(ctypes.c_ulonglong)]
        L.bfs_sweep_schedule.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int, C(ctypes.c_int),
                                         ctypes.c_int, C(ctypes.c_int)]
        L.bfs_debug_stall_sweep.argtypes = [_VP, ctypes.c_int]
        L.bfs_precond_info.argtypes = [_VP, C(ctypes.c_int)]
        L.bfs_solver_info.argtypes = [_VP, C(ctypes.c_int)]
        L.bfs_peak_probe.argtypes = [ctypes.c_int, ctypes.c_int, _VP, _VP, C(ctypes.c_double)]
        L.bfs_gj_invert.argtypes = [_VP, _VP, ctypes.c_int, ctypes.c_int, ctypes.c_int, _VP]
        _lib = L
    return _lib


def default_options(**kw) -> bfs_options:
    o = bfs_options()
    lib().bfs_default_options(ctypes.byref(o))
    for k, v in kw.items():
        if not hasattr(o, k):
            raise KeyError(k)
        setattr(o, k, v)
    return o


def _ptr(t) -> int:
    return t.data_ptr()


def _require(ok: bool, msg: str):
    """Argument check that survives python -O: a buffer of the wrong size,
    type or device would otherwise reach the kernels as a raw pointer."""
    if not ok:
        raise ValueError(msg)


def _is_f64_cuda(t, n: int | None = None) -> bool:
    import torch
    return (isinstance(t, torch.Tensor) and t.is_cuda and t.dtype == torch.float64 and t.is_contiguous()
            and (n is None or t.numel() == n))


def _stream(stream):
    import torch
    if stream is None:
        stream = torch.cuda.current_stream()
    return ctypes.c_void_p(stream.cuda_stream)


class Context:
    """A problem set up on the current CUDA device (wraps bfs_ctx)."""

    def __init__(self, mesh, topo, F: float, options: bfs_options | None = None):
        import torch
        if not torch.cuda.is_available():
            raise RuntimeError("CUDA device required: libbfs has no CPU path")
        self.mesh = mesh
        self._h = [np.ascontiguousarray(a, dtype=np.float64) for a in (topo.beta, topo.beta_x, topo.beta_y)]
        m = bfs_mesh(mesh.N, mesh.M, int(mesh.half), mesh.x1, mesh.y1, mesh.dx, mesh.dy)
        D = ctypes.POINTER(ctypes.c_double)
        t = bfs_topo(*[a.ctypes.data_as(D) for a in self._h])
        self.options = options if options is not None else default_options()
        ctx = _VP()
        rc = lib().bfs_setup(ctypes.byref(m), ctypes.byref(t), float(F), ctypes.byref(self.options),
                             ctypes.byref(ctx))
        if rc != BFS_OK:
            raise BfsError(rc, lib().bfs_last_error(None).decode())
        self._ctx = ctx
        self.n = lib().bfs_n_unknowns(ctx)
        self.pair_evals = lib().bfs_pair_evals(ctx)

    def _check(self, rc):
        if rc != BFS_OK:
            raise BfsError(rc, lib().bfs_last_error(self._ctx).decode())

    def close(self):
        if getattr(self, "_ctx", None):
            lib().bfs_destroy(self._ctx)
            self._ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _vec(self, t):
        _require(_is_f64_cuda(t, self.n), f"expected a contiguous float64 CUDA vector of length {self.n}")
        return ctypes.c_void_p(_ptr(t))

    def _host_vec(self, a):
        _require(isinstance(a, np.ndarray) and a.dtype == np.float64 and a.flags.c_contiguous
                 and a.size == self.n, f"expected a contiguous float64 numpy vector of length {self.n}")
        return ctypes.c_void_p(a.ctypes.data)

    # --- the C ABI, one method per entry point -----------------------------
    def residual(self, u, out=None, precision: int = BFS_FP64, stream=None):
        import torch
        if out is None:
            out = torch.empty_like(u)
        self._check(lib().bfs_residual(self._ctx, self._vec(u), self._vec(out), precision, _stream(stream)))
        return out

    def check_finite(self, stream=None) -> bool:
        rc = lib().bfs_check_finite(self._ctx, _stream(stream))
        if rc == BFS_ENAN:
            return False
        self._check(rc)
        return True

    def jvp(self, u, Fu, z, out=None, h: float = 0.0, precision: int = BFS_FP64, stream=None):
        import torch
        if out is None:
            out = torch.empty_like(u)
        self._check(lib().bfs_jvp(self._ctx, self._vec(u), self._vec(Fu), self._vec(z), self._vec(out),
                                  float(h), precision, _stream(stream)))
        return out

    def precond_factor(self, half_band: int = -1, stream=None):
        self._check(lib().bfs_precond_factor(self._ctx, int(half_band), _stream(stream)))

    def precond_apply(self, r, out=None, stream=None):
        import torch
        if out is None:
            out = torch.empty_like(r)
        self._check(lib().bfs_precond_apply(self._ctx, self._vec(r), self._vec(out), _stream(stream)))
        return out

    def precond_info(self) -> dict:
        """Half band, two-ended split (-1: one-ended), sweep chains and the
        dependent steps of the longest chain of the factored preconditioner."""
        info = (ctypes.c_int * 4)()
        self._check(lib().bfs_precond_info(self._ctx, info))
        return {"half_band": info[0], "twist": info[1], "chains": info[2], "sweep_steps": info[3]}

    def solver_info(self) -> dict:
        """How the solves of this context launched their Arnoldi steps: step
        graphs instantiated, how many conditional (queued one step ahead),
        whether graphs are off, whether the context's own stream was used."""
        info = (ctypes.c_int * 4)()
        self._check(lib().bfs_solver_info(self._ctx, info))
        return {"step_graphs": info[0], "conditional": info[1], "graphs_off": bool(info[2]),
                "own_stream": bool(info[3])}

    def debug_stall_sweep(self, task: int):
        """Test hook: the next FP32 sweep launch waits in `task` for a vector no
        task writes (its waits run out after the option wait_polls)."""
        self._check(lib().bfs_debug_stall_sweep(self._ctx, int(task)))

    def solve(self, u, stream=None, raise_on_error: bool = True):
        st = bfs_stats()
        rc = lib().bfs_solve(self._ctx, self._vec(u), ctypes.byref(st), _stream(stream))
        if raise_on_error:
            self._check(rc)
        return st.as_dict()

    def solve_host(self, u_host: np.ndarray, stream=None, raise_on_error: bool = True):
        st = bfs_stats()
        rc = lib().bfs_solve_host(self._ctx, self._host_vec(u_host), ctypes.byref(st), _stream(stream))
        if raise_on_error:
            self._check(rc)
        return st.as_dict()

    def residual_host(self, u_host: np.ndarray, out: np.ndarray | None = None,
                      precision: int = BFS_FP64, stream=None):
        if out is None:
            out = np.empty(self.n)
        self._check(lib().bfs_residual_host(self._ctx, self._host_vec(u_host), self._host_vec(out),
                                            precision, _stream(stream)))
        return out

    def flat_guess(self, out=None, stream=None):
        import torch
        if out is None:
            out = torch.empty(self.n, dtype=torch.float64, device="cuda")
        self._check(lib().bfs_flat_guess(self._ctx, self._vec(out), _stream(stream)))
        return out

    def bottom_pressure(self, u, stream=None):
        """(nodal bottom pressure [M, N] on the device, force (3,) on the host)."""
        import torch
        p = torch.empty(self.mesh.N * self.mesh.M, dtype=torch.float64, device="cuda")
        f = (ctypes.c_double * 3)()
        self._check(lib().bfs_bottom_pressure(self._ctx, self._vec(u), ctypes.c_void_p(_ptr(p)), f,
                                              _stream(stream)))
        return p.view(self.mesh.M, self.mesh.N), np.array(list(f))

    def set_topography(self, topo):
        self._h = [np.ascontiguousarray(a, dtype=np.float64) for a in (topo.beta, topo.beta_x, topo.beta_y)]
        D = ctypes.POINTER(ctypes.c_double)
        t = bfs_topo(*[a.ctypes.data_as(D) for a in self._h])
        self._check(lib().bfs_set_topography(self._ctx, ctypes.byref(t)))

    def set_surface_pressure(self, p=None):
        if p is None:
            self._check(lib().bfs_set_surface_pressure(self._ctx, None))
            return
        self._p = np.ascontiguousarray(p, dtype=np.float64).ravel()
        _require(self._p.size == self.mesh.N * self.mesh.M, "p needs one value per node (N*M)")
        self._check(lib().bfs_set_surface_pressure(self._ctx, ctypes.c_void_p(self._p.ctypes.data)))

    def set_froude(self, F: float):
        self._check(lib().bfs_set_froude(self._ctx, float(F)))

    def profile_enable(self, on: bool = True):
        self._check(lib().bfs_profile_enable(self._ctx, int(bool(on))))

    def profile_read(self):
        """Returns {"fp64"|"fp32c"|"df64": (total ms, launches)} of the pair kernels
        since the last read, and the context's kernel-launch counter."""
        out = (ctypes.c_double * 8)()
        n = ctypes.c_ulonglong()
        self._check(lib().bfs_profile_read(self._ctx, out, ctypes.byref(n)))
        return ({"fp64": (out[0], int(out[1])), "fp32c": (out[2], int(out[3])),
                 "df64": (out[4], int(out[5])), "apply": (out[6], int(out[7]))}, int(n.value))

    def unpack(self, u, stream=None):
        import torch
        NM = self.mesh.N * self.mesh.M
        out = torch.empty(8 * NM, dtype=torch.float64, device="cuda")
        self._check(lib().bfs_unpack(self._ctx, self._vec(u), ctypes.c_void_p(_ptr(out)), _stream(stream)))
        names = ("zeta", "zeta_x", "zeta_y", "phi", "phi_x", "phi_y", "psi", "psi_x")
        return {k: out[i * NM:(i + 1) * NM].view(self.mesh.M, self.mesh.N) for i, k in enumerate(names)}


def residual_static(mesh, beta, beta_x, beta_y, F: float, u, out=None, precision: int = BFS_FP64,
                    n_rad: float = 0.05, sign_I4: float = -1.0, stream=None):
    """bfs_residual_static: F(u) with no device allocation inside the call.
    beta, beta_x, beta_y, u: float64 CUDA tensors (out too, if given)."""
    import torch
    if out is None:
        out = torch.empty_like(u)
    NM = mesh.N * mesh.M
    for t in (beta, beta_x, beta_y):
        _require(_is_f64_cuda(t, NM), f"beta, beta_x, beta_y: contiguous float64 CUDA arrays of N*M = {NM}")
    n = 3 * (mesh.N + 1) * mesh.M
    for t in (u, out):
        _require(_is_f64_cuda(t, n), f"u, out: contiguous float64 CUDA vectors of length {n}")
    m = bfs_mesh(mesh.N, mesh.M, int(mesh.half), mesh.x1, mesh.y1, mesh.dx, mesh.dy)
    rc = lib().bfs_residual_static(ctypes.byref(m), ctypes.c_void_p(_ptr(beta)), ctypes.c_void_p(_ptr(beta_x)),
                                   ctypes.c_void_p(_ptr(beta_y)), float(F), float(n_rad), float(sign_I4),
                                   ctypes.c_void_p(_ptr(u)), ctypes.c_void_p(_ptr(out)), int(precision),
                                   _stream(stream))
    if rc != BFS_OK:
        raise BfsError(rc, lib().bfs_static_last_error().decode())
    return out


def sweep_schedule(M: int, half_band: int, twisted: bool):
    """Task table of the FP32 preconditioner sweeps (host only, no GPU): an
    (ntasks, 16) int array of {k, out, nblk, 0, m[4], vec[4], uid[4]} rows and
    the number of tasks of each CTA group."""
    L = lib()
    cnt = (ctypes.c_int * 2)()
    n = L.bfs_sweep_schedule(int(M), int(half_band), int(bool(twisted)), None, 0, cnt)
    if n < 0:
        raise BfsError(n, "invalid sweep schedule arguments")
    buf = (ctypes.c_int * (16 * max(n, 1)))()
    n2 = L.bfs_sweep_schedule(int(M), int(half_band), int(bool(twisted)), buf, n, cnt)
    if n2 != n:
        raise BfsError(n2, "sweep schedule changed between calls")
    return np.frombuffer(buf, dtype=np.int32, count=16 * n).reshape(n, 16).copy(), (cnt[0], cnt[1])


def peak_probe(kind: int, iters: int, out, stream=None) -> float:
    """Launch one roofline probe (0 FP32 FMA, 1 FP32 rsqrt, 2 FP64 FMA) writing
    into the device tensor `out` (peak_probe_threads() float64 entries);
    returns the lane operations the launch executes."""
    ops = ctypes.c_double()
    rc = lib().bfs_peak_probe(int(kind), int(iters), ctypes.c_void_p(out.data_ptr()), _stream(stream),
                              ctypes.byref(ops))
    if rc:
        raise BfsError(rc, "peak probe failed")
    return ops.value


def gj_invert(A, method: int, stream=None):
    """Inverses of the (n, n) or (2, n, n) float64 CUDA tensor A by the
    factorisation's Gauss-Jordan kernels (method 0: FP64 rows kernel, 1:
    blocked double-float, clustered panels where they fit, 2: blocked
    double-float with one CTA per panel); raises BfsError on a failure code."""
    import torch
    A = A.contiguous()
    nmat = 1 if A.dim() == 2 else A.shape[0]
    out = torch.empty_like(A)
    rc = lib().bfs_gj_invert(ctypes.c_void_p(A.data_ptr()), ctypes.c_void_p(out.data_ptr()), int(A.shape[-1]),
                             int(nmat), int(method), _stream(stream))
    if rc != BFS_OK:
        raise BfsError(rc, f"bfs_gj_invert(n={A.shape[-1]}, nmat={nmat}, method={method})")
    return out


def peak_probe_threads() -> int:
    return int(lib().bfs_peak_probe_threads())


class Batch:
    """Many independent problems solved together (wraps bfs_batch)."""

    def __init__(self, meshes, topos, Fs, options: bfs_options | None = None):
        import torch
        if not torch.cuda.is_available():
            raise RuntimeError("CUDA device required: libbfs has no CPU path")
        B = len(meshes)
        _require(len(topos) == B and len(Fs) == B, "meshes, topos and Fs differ in length")
        self.meshes = list(meshes)
        D = ctypes.POINTER(ctypes.c_double)
        self._h = []
        ms = (bfs_mesh * B)()
        ts = (bfs_topo * B)()
        for i, (m, t) in enumerate(zip(meshes, topos)):
            arrs = [np.ascontiguousarray(a, dtype=np.float64) for a in (t.beta, t.beta_x, t.beta_y)]
            self._h.append(arrs)
            ms[i] = bfs_mesh(m.N, m.M, int(m.half), m.x1, m.y1, m.dx, m.dy)
            ts[i] = bfs_topo(*[a.ctypes.data_as(D) for a in arrs])
        F = (ctypes.c_double * B)(*[float(f) for f in Fs])
        self.options = options if options is not None else default_options()
        h = _VP()
        rc = lib().bfs_batch_setup(B, ms, ts, F, ctypes.byref(self.options), ctypes.byref(h))
        if rc != BFS_OK:
            raise BfsError(rc, lib().bfs_batch_last_error(None).decode())
        self._b = h
        self.B = B
        self.n = [lib().bfs_batch_n_unknowns(h, i) for i in range(B)]
        self.pair_evals = lib().bfs_batch_pair_evals(h)

    def _check(self, rc):
        if rc != BFS_OK:
            raise BfsError(rc, lib().bfs_batch_last_error(self._b).decode())

    def close(self):
        if getattr(self, "_b", None):
            lib().bfs_batch_destroy(self._b)
            self._b = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _ptrs(self, ts):
        _require(len(ts) == self.B, f"expected {self.B} vectors")
        for i, (t, n) in enumerate(zip(ts, self.n)):
            _require(_is_f64_cuda(t, n), f"vector {i}: expected a contiguous float64 CUDA vector of length {n}")
        return (_VP * self.B)(*[_ptr(t) for t in ts])

    def flat_guesses(self):
        import torch
        out = []
        for i in range(self.B):
            u = torch.empty(self.n[i], dtype=torch.float64, device="cuda")
            rc = lib().bfs_flat_guess(lib().bfs_batch_instance(self._b, i), ctypes.c_void_p(_ptr(u)),
                                      _stream(None))
            self._check(rc)
            out.append(u)
        return out

    def residual(self, us, outs=None, stream=None):
        import torch
        if outs is None:
            outs = [torch.empty_like(u) for u in us]
        self._check(lib().bfs_batch_residual(self._b, self._ptrs(us), self._ptrs(outs), _stream(stream)))
        return outs

    def instance_residual(self, i, u, precision: int = BFS_FP64, stream=None):
        import torch
        _require(0 <= i < self.B, f"instance {i} is not in the batch")
        _require(_is_f64_cuda(u, self.n[i]), f"instance {i}: expected a contiguous float64 CUDA vector of length {self.n[i]}")
        out = torch.empty_like(u)
        self._check(lib().bfs_residual(lib().bfs_batch_instance(self._b, i), ctypes.c_void_p(_ptr(u)),
                                       ctypes.c_void_p(_ptr(out)), precision, _stream(stream)))
        return out

    def autotune(self, stream=None) -> float:
        ms = ctypes.c_double()
        self._check(lib().bfs_batch_autotune(self._b, _stream(stream), ctypes.byref(ms)))
        return ms.value

    def tuning(self) -> dict:
        v, tpb, tpt = ctypes.c_int(), ctypes.c_int(), ctypes.c_int()
        ms = (ctypes.c_double * 8)()
        self._check(lib().bfs_batch_tuning(self._b, ctypes.byref(v), ctypes.byref(tpb), ctypes.byref(tpt), ms))
        return {"variant": v.value, "tpb": tpb.value, "tpt": tpt.value, "ms_per_variant": list(ms)[:5]}

    def solve(self, us, stream=None, raise_on_error: bool = False):
        st = (bfs_stats * self.B)()
        rc = lib().bfs_batch_solve(self._b, self._ptrs(us), st, _stream(stream))
        if raise_on_error:
            self._check(rc)
        return rc, [x.as_dict() for x in st]
