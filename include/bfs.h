/*
 * bfs.h -- C ABI of the GB300 boundary-integral JFNK solver for steady 3-D
 * free-surface flow over bottom topography (Buttle, Pethiyagoda, Moroney &
 * McCue, arXiv:1709.08803).
 *
 * Conventions shared by every call:
 *   - Return value: BFS_OK (0) on success, a negative BFS_E* code otherwise.
 *     No exception crosses the ABI.  bfs_last_error(ctx) gives a message for
 *     the last failing call on ctx (bfs_last_error(NULL) for bfs_setup).
 *   - Vectors of unknowns u and residuals F are FP64 arrays of length
 *     n = 3(N+1)M (bfs_n_unknowns).
 *       u, per slice j = 1..M, for q = zeta, then phi, then psi (three blocks
 *       of (N+1)M):  [ q(x1, y_j), q_x(x_1, y_j), ..., q_x(x_N, y_j) ]
 *       (Sec. 3.1, the vector of unknowns).
 *       F, per slice l, in three blocks: [F5, F6, F1(1..N-1)],
 *       [F3, F4, F2(1..N-1)], [F8, F9, F7(1..N-1)]  (App. B, the order of the
 *       vector function): F1 the combined dynamic condition (Sec. 2.1), F2
 *       and F7 the boundary integral equation collocated at the half mesh
 *       points of the free surface and of the bottom (Sec. 2.2, 3.1), F3-F6,
 *       F8, F9 the radiation conditions of Scullen (Sec. 3.1).
 *   - Pointers called "device" must be CUDA device memory of the current
 *     device (e.g. torch tensor data_ptr()); "host" pointers are ordinary
 *     host memory.  The caller owns every buffer it passes; the context owns
 *     all the memory it allocates and frees it in bfs_destroy.
 *   - stream is a cudaStream_t (NULL = the legacy default stream).  Calls
 *     that take a stream are asynchronous on it unless stated otherwise.
 *   - A context is used from one host thread and one stream at a time.
 */
#ifndef BFS_H
#define BFS_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

enum {
    BFS_OK = 0,
    BFS_EINVAL = -1,      /* invalid argument (sizes, spacing, F, topography) */
    BFS_ECUDA = -2,       /* a CUDA runtime call failed */
    BFS_ENOMEM = -3,      /* device allocation failed */
    BFS_ENAN = -4,        /* a residual or update was not finite */
    BFS_ENOCONV = -5,     /* Newton iteration limit reached */
    BFS_ELINESEARCH = -6, /* line search found no sufficient decrease */
    BFS_EBREAKDOWN = -7,  /* GMRES breakdown without convergence */
    BFS_ESINGULAR = -8,   /* zero pivot while factoring the preconditioner */
    BFS_ENOPREC = -9,     /* preconditioner applied before it was factored */
    BFS_ETIMEOUT = -10    /* wall-clock budget of bfs_solve exhausted */
};

/* Arithmetic of the boundary-integral pair sums. */
enum {
    BFS_FP64 = 0,  /* FP64 throughout */
    BFS_FP32C = 1, /* pair terms in FP32 with compensated (two-sum) accumulation,
                      reduced and finished in FP64 */
    BFS_DF64 = 2   /* pair terms in double-float arithmetic (pairs of FP32 values
                      carrying about 46 bits) on the FP32 pipes; FP64-accurate
                      to the 1e-10 per-row bar, reduced and finished in FP64 */
};

/* Truncated mesh x_i = x1 + (i-1) dx, i = 1..N; y_j = y1 + (j-1) dy, j = 1..M
   (Sec. 3.1).  half_domain = 1 solves only y >= 0 (y1 must be 0) for flows
   symmetric in y: the rows j >= 2 are mirrored to y < 0 as extra sources. */
typedef struct {
    int N, M;
    int half_domain;
    double x1, y1, dx, dy;
} bfs_mesh;

/* Bottom z = beta(x, y) and its exact derivatives at the N*M nodes, index
   i + N*j (0-based), HOST arrays, copied by bfs_setup.  beta tends to -1 far
   away (Sec. 2.1) and must stay below F^2/2: Bernoulli bounds every surface
   height by F^2/2 (the speed cannot be imaginary), so a bottom reaching it
   pierces the surface.  A bottom above z = 0 is allowed (the supercritical
   solutions of Sec. 5.2 flow over bumps taller than the upstream depth). */
typedef struct {
    const double *beta, *beta_x, *beta_y;
} bfs_topo;

typedef struct {
    double n_rad;         /* radiation decay rate n (Sec. 3.1; 0.05) */
    double sign_I4;       /* sign of the bottom single layer I4: -1 from Green's
                             identity with outward normals (default), +1 as printed */
    int half_band;        /* preconditioner half band width in slices (App. A) */
    double tol;           /* bfs_solve stops when |F|_inf <= tol */
    int gmres_restart;    /* Krylov vectors per GMRES cycle */
    int max_newton;       /* Newton iteration limit */
    int max_krylov;       /* Krylov iterations per Newton step */
    double eta;           /* GMRES relative tolerance (forcing term) */
    int krylov_precision; /* BFS_FP64 or BFS_FP32C for the residuals inside
                             the Jacobian-vector products; the Newton residual
                             and the line search are always FP64 */
    double jv_h_rel;      /* FD step: h = jv_h_rel (1 + |u|_2) / |z|_2; <= 0 picks
                             sqrt(eps) of the Krylov precision's arithmetic */
    double time_budget_s; /* bfs_solve wall-clock limit (<= 0: none) */
    int src_splits;       /* source splits of the pair kernels (<= 0: automatic) */
    int outer_precision;  /* BFS_FP64 (default) or BFS_DF64 for the Newton residual
                             and the line search */
    int precond_precision; /* BFS_FP64 (default) or BFS_FP32C: storage and arithmetic
                              of the preconditioner sweeps.  The factorisation is FP64
                              either way; FP32C sweeps an FP32 copy of the factors
                              (the preconditioner only steers GMRES, the Newton
                              residual and the converged u do not depend on it).
                              With surface_tension > 0 the sweeps stay FP64: the
                              capillary term leaves the factors too ill-conditioned
                              for FP32 copies. */
    double refine_below;   /* > 0 with outer_precision != krylov_precision: the Newton
                              residual and the line search use the Krylov arithmetic
                              while |F|_inf > refine_below, then switch to
                              outer_precision for the final steps (iterative
                              refinement); they switch earlier when a full Newton
                              step in the Krylov arithmetic lowers |F|_2 by less
                              than 10 % or its line search fails (the Krylov
                              arithmetic's rounding then limits progress).
                              Convergence is only ever accepted on an
                              outer_precision residual.  0 (default): always outer. */
    int stall_newton;      /* > 0: give up with BFS_ENOCONV once GMRES has ended above
                              its forcing tolerance (max_krylov reached) in this many
                              consecutive Newton steps -- the signature of a problem
                              with no nearby steady solution.  0 (default): off. */
    double surface_tension; /* tau >= 0: the dynamic condition gains -tau * kappa,
                              kappa the mean curvature operator div(grad zeta /
                              sqrt(1 + |grad zeta|^2)) at the half points (the
                              extension Sec. 6 proposes); the preconditioner gains the
                              linearised term -tau (zeta_xx + zeta_yy).  0 (default). */
    int forcing;           /* GMRES relative tolerance of Newton step k: 0 (default) the
                              fixed eta; 1 Eisenstat-Walker choice 1 (the KINSOL
                              default of Sec. 5's solver), eta_k = | |F_k| - |F_{k-1} +
                              J s_{k-1}| | / |F_{k-1}|, safeguarded by eta_{k-1}^1.618
                              when that exceeds 0.1, kept in [eta, 0.9]; eta_0 =
                              max(eta, 0.1) */
    int wait_polls;        /* polls of a device-side wait (the tags of the preconditioner
                              sweeps, the grid barriers of the cooperative kernels) before
                              it gives up: the kernel raises the context's timeout bit,
                              returns, and bfs_check_finite / bfs_solve report
                              BFS_ETIMEOUT.  <= 0 (default): about one second per wait. */
} bfs_options;

typedef struct {
    int newton_its, krylov_its;
    int residual_evals_fp64, residual_evals_fp32;
    int precond_applies;
    double fnorm_inf, fnorm_2; /* of the final FP64 residual */
    double seconds;            /* wall time of bfs_solve */
    double seconds_residual, seconds_precond, seconds_krylov_other;
    int status;                /* same as the return value */
} bfs_stats;

typedef struct bfs_ctx bfs_ctx;

/* Fills *o with the defaults (n = 0.05, sign_I4 = -1, half_band =
   max(1, round(M/20)), tol = 1e-8, restart 50, 60 Newton steps, 200 Krylov
   iterations, eta = 1e-4, FP64 Krylov residuals). */
void bfs_default_options(bfs_options *o);

/* Validates the problem, allocates device memory on the current device,
   uploads the topography and precomputes the parts of the bottom integral
   that depend only on the bottom (the single-layer sum over the bottom seen
   from bottom collocation points, Sec. 3.1).  Synchronous.  Errors:
   BFS_EINVAL for N < 4, M < 3, dx or dy <= 0, F <= 0, half_domain with
   y1 != 0, beta >= F^2/2 anywhere or a non-finite input; BFS_ENOMEM; BFS_ECUDA. */
int bfs_setup(const bfs_mesh *mesh, const bfs_topo *topo, double F, const bfs_options *opt,
              bfs_ctx **out);

void bfs_destroy(bfs_ctx *ctx);

/* Replace the topography of a context (HOST arrays as in bfs_setup) and
   recompute its bottom-only integral part; the factored preconditioner stays
   valid because the linearised Jacobian does not depend on the bottom
   (Sec. 4.2).  This is the continuation step in bump height that the
   paper's large-amplitude solutions rely on (Sec. 5).  Synchronous; errors as
   bfs_setup's topography checks. */
int bfs_set_topography(bfs_ctx *ctx, const bfs_topo *topo);

/* Apply a pressure distribution p(x, y) to the free surface (the ship-wake
   model the paper relates to the bump in Sec. 4.1 and 6): p adds to the
   combined dynamic condition, p* being the mean of the two nodes around each
   half point.  p: HOST array of N*M nodal values (index i + N*j), copied; NULL
   removes it.  The preconditioner is unchanged (p does not depend on u).
   Synchronous; BFS_EINVAL for a non-finite value. */
int bfs_set_surface_pressure(bfs_ctx *ctx, const double *p);

/* Change the Froude number.  The factored preconditioner (formed for the
   previous F) is kept as an approximation and stays usable; call
   bfs_precond_factor to refresh it.  Synchronous.  BFS_EINVAL, with the
   context unchanged, for F <= 0 or an F whose F^2/2 the current bottom
   reaches (the bound bfs_setup checks). */
int bfs_set_froude(bfs_ctx *ctx, double F);
const char *bfs_last_error(const bfs_ctx *ctx);
int bfs_n_unknowns(const bfs_ctx *ctx);
/* Pair evaluations of one residual: 4 (N-1)M x (number of sources). */
double bfs_pair_evals(const bfs_ctx *ctx);

/* Fu = F(u), the nonlinear residual (Sec. 3.1; App. B order).  u, Fu: device,
   length n.  precision: BFS_FP64, BFS_FP32C or BFS_DF64.  Asynchronous; a non-finite
   entry raises the context's NaN flag (read by bfs_check_finite). */
int bfs_residual(bfs_ctx *ctx, const double *u, double *Fu, int precision, void *stream);

/* Synchronises stream and returns BFS_ETIMEOUT if a device-side wait gave up
   (see wait_polls; the sweep vectors are then reset, so the next call runs
   normally), else BFS_ENAN if any residual evaluated since the previous call
   was non-finite, else BFS_OK; clears the flags. */
int bfs_check_finite(bfs_ctx *ctx, void *stream);

/* Jz = (F(u + h z) - Fu) / h, the finite-difference Jacobian-vector product
   (Sec. 3.2).  u, Fu, z, Jz: device, length n; Fu must be F(u) in FP64.
   h <= 0 picks h = h_rel (1 + |u|_2) / |z|_2 on the device.  The perturbed
   residual uses `precision`.  Jz = 0 when z = 0. */
int bfs_jvp(bfs_ctx *ctx, const double *u, const double *Fu, const double *z, double *Jz,
            double h, int precision, void *stream);

/* Forms the Jacobian of the linearised discrete system (Sec. 4.2, App. B),
   keeps the slice blocks within half_band of the diagonal (App. A), reorders
   it slice by slice into 3(N+1) x 3(N+1) blocks and factors it by block LU
   with partial pivoting inside each diagonal block.  Depends on the mesh, F
   and n only.  half_band < 0 uses the option's value.  Synchronous.
   Errors: BFS_ESINGULAR, BFS_ENOMEM, BFS_ECUDA. */
int bfs_precond_factor(bfs_ctx *ctx, int half_band, void *stream);

/* Shape of the factored preconditioner: info[0] the half band h, info[1] the
   first middle slice t of the two-ended order (-1: one-ended), info[2] the
   chains the FP32 sweeps run side by side (0: FP64 sweeps), info[3] the
   dependent steps of the longest chain (tasks of the sweep table; 2M for the
   FP64 sweeps).  BFS_ENOPREC before bfs_precond_factor. */
int bfs_precond_info(const bfs_ctx *ctx, int *info4);

/* How bfs_solve launched its Arnoldi steps (for tests and reports): info4[0]
   step graphs instantiated (one per Krylov index and base residual buffer,
   kept until a captured argument changes), info4[1] how many of them are
   conditional (the step behind a device-side end-of-cycle flag, so the next
   step is queued before the host reads this one's scalars), info4[2] 1 if
   graphs are off for this context (a capture failed; steps launched one by
   one), info4[3] 1 if a solve was handed the legacy default stream and ran on
   the context's own stream (graphs cannot be captured on the legacy stream).
   Profiling (bfs_profile_enable) launches steps one by one without graphs. */
int bfs_solver_info(const bfs_ctx *ctx, int *info4);

/* z = P^{-1} r with the factored preconditioner.  r, z: device, length n,
   in the order of u (r may equal z).  BFS_ENOPREC before bfs_precond_factor. */
int bfs_precond_apply(bfs_ctx *ctx, const double *r, double *z, void *stream);

/* Damped inexact Newton with backtracking line search and right-
   preconditioned restarted GMRES on finite-difference Jacobian-vector
   products (Sec. 3.2), in place on the device vector u_inout (length n).
   Factors the preconditioner first if needed.  Synchronous; st may be NULL.
   Returns BFS_OK when |F|_inf <= tol, else BFS_ENOCONV, BFS_ELINESEARCH,
   BFS_EBREAKDOWN, BFS_ENAN or BFS_ETIMEOUT (u_inout then holds the last
   accepted iterate). */
int bfs_solve(bfs_ctx *ctx, double *u_inout, bfs_stats *st, void *stream);

/* bfs_solve on a HOST vector: copies u_host to the device, solves and copies
   the result back (both copies inside the call).  Synchronous. */
int bfs_solve_host(bfs_ctx *ctx, double *u_host_inout, bfs_stats *st, void *stream);

/* bfs_residual on HOST vectors (copies in and out inside the call). Synchronous. */
int bfs_residual_host(bfs_ctx *ctx, const double *u_host, double *F_host, int precision,
                      void *stream);

/* Writes the uniform-stream guess (zeta = 0, phi = psi = x) into the device
   vector u (length n). */
int bfs_flat_guess(bfs_ctx *ctx, double *u, void *stream);

/* Nodal fields from u (device in, device out): out holds 8 arrays of N*M
   (index i + N*j): zeta, zeta_x, zeta_y, phi, phi_x, phi_y, psi, psi_x
   (trapezoid reconstruction in x, second-order differences in y). */
int bfs_unpack(bfs_ctx *ctx, const double *u, double *out, void *stream);

/* Pressure on the bottom and the force of the fluid on the topography
   (Sec. 2.1: Bernoulli's equation along the bottom, from the bottom potential
   psi of u).  u: device vector; p: device array of N*M nodal pressures (index
   i + N*j); force_host (may be NULL): 3 host doubles, the trapezoid integral of
   p (beta_x, beta_y, -1) dx dy (x: drag, z: vertical; the half domain reports
   the whole mirrored domain and a zero y component).  Synchronous when
   force_host is given. */
int bfs_bottom_pressure(bfs_ctx *ctx, const double *u, double *p, double *force_host, void *stream);

/* The task table of the FP32 preconditioner sweeps for M slices and half band
   half_band (App. A), without a GPU: the one-ended block LU (twisted = 0: the
   forward chain, then the backward chain) or the two-ended one (twisted = 1:
   a chain from each end, the middle system, the chains back outwards; the
   order bfs_precond_factor takes when the FP32 sweeps can run it).  Writes
   the tasks as 16 ints each into tasks_out (room for cap tasks; NULL to only
   count them): {k, out, nblk, 0, m[4], vec[4], uid[4]} -- task uid u writes
   slice k of y (out 0, adding the right-hand side) or z (out 1) as
   sum_p sign_p B(k, m[p]) v_p, v_p being z_{m[p]} if vec bit 0 is set (else
   y_{m[p]}), sign + if vec bit 1 is set, and written by task uid[p]; vec bits
   2-3 say where the kernel's threads find v_p (0: loaded at the end of the
   step before; 1: held in registers since it was the critical vector of an
   earlier task, bits 4-5 its index, newest first; 2: the critical vector,
   written by the group's previous task and polled last).  Group 0's
   tasks come first; ntask_out (optional, 2 ints) receives the tasks per group.
   Returns the number of tasks, or BFS_EINVAL (half_band > 3, M < 1, or
   cap too small). */
int bfs_sweep_schedule(int M, int half_band, int twisted, int *tasks_out, int cap, int *ntask_out);

/* Test hook for the timeout path of the sweeps' waits: the next FP32 sweep
   launch of ctx (bfs_precond_apply or an Arnoldi step launched directly, not
   replayed from a graph) waits, in task `task` of the table above, for a
   vector slice no task of that launch writes, so that its waits run out after
   wait_polls polls and it returns with the timeout bit raised.  The table is
   restored right after that launch; bfs_check_finite then returns
   BFS_ETIMEOUT and resets the sweep vectors, and the next apply is normal.
   BFS_EINVAL unless the preconditioner is factored with FP32 task-table
   sweeps and the task multiplies at least one block. */
int bfs_debug_stall_sweep(bfs_ctx *ctx, int task);

/* The inversions of the block factorisation (App. B: the inverted diagonal
   blocks D_k^-1 of the block LU, and the two-ended order's middle system) on
   caller matrices.  A: DEVICE, nmat (1 or 2) consecutive n x n row-major FP64
   matrices, read only; Ainv: DEVICE, the same layout, receives the inverses.
   method 0: FP64 Gauss-Jordan with partial pivoting, rows spread over the
   GPU, one exchange between CTAs per column (the factorisation's kernel when
   the sweeps are FP64); method 1: blocked Gauss-Jordan in double-float
   arithmetic (panels of 64 columns spread over a cluster of 8 CTAs' shared
   memory from 128 rows up, else panels of up to 64 columns in one CTA; then
   one rank-panel product per panel; the kernel when the sweeps are FP32);
   method 2: method 1 with one CTA per panel at every size.  All pivot on the
   unused row with the largest |entry|, ties to the lowest row; methods 1 and
   2 compare the magnitudes to 12 significant bits.  Allocates its own scratch and synchronises stream.
   BFS_EINVAL for a bad argument or an n the method's tiles do not take
   (method 0: n > 16 rows per CTA; methods 1 and 2: n > 2048, or a panel of
   16 columns does not fit in one CTA), BFS_ESINGULAR for a zero pivot,
   BFS_ETIMEOUT if a wait between CTAs gave up (method 0). */
int bfs_gj_invert(const double *A, double *Ainv, int n, int nmat, int method, void *stream);

/* Profiling.  bfs_profile_enable(ctx, 1) records a CUDA event pair on the
   launching stream around every pair-kernel launch and every preconditioner
   apply of the context; bfs_profile_read waits for the recorded events and
   returns, in out8, {total ms and launch count} of the FP64, FP32C and DF64
   pair kernels and of the preconditioner apply, in that order, then forgets
   them.  *launches (optional)
   receives the number of kernels the context has launched since bfs_setup. */
int bfs_profile_enable(bfs_ctx *ctx, int on);
int bfs_profile_read(bfs_ctx *ctx, double *out8, unsigned long long *launches);

/* Roofline probes (measurement only; the paper has no counterpart): one launch
   of a kernel that streams a single instruction kind through its pipe with
   no dependence between consecutive instructions and a full SM of warps:
   kind 0 FP32 fused multiply-add, 1 FP32 reciprocal square root (the
   special-function unit), 2 FP64 fused multiply-add, 3 packed FP32x2 fused
   multiply-add (two lane operations per instruction).  out: DEVICE buffer of
   bfs_peak_probe_threads() doubles (results kept live); *lane_ops receives
   the lane operations the launch executes, so that lane_ops / (its CUDA-event
   time) is the pipe's throughput.  Asynchronous on stream.  BFS_EINVAL for an
   unknown kind, iters < 1 or out NULL. */
int bfs_peak_probe(int kind, int iters, void *out, void *stream, double *lane_ops);
int bfs_peak_probe_threads(void);

/* Batched sweeps (an addition: the paper solves one problem at a
   time).  A batch holds B independent problems -- each its own mesh, bottom
   and Froude number -- and evaluates the FP32C residuals that their Krylov
   iterations need in ONE persistent-kernel launch per step: CTAs take
   (instance, target tile, source split) items from a queue, largest
   instances first, so uneven meshes share the GPU evenly.  That batched
   residual is captured once as a CUDA graph and replayed.
     bfs_batch_setup: B problems (arrays of B meshes, topographies and F; the
       same options for all).  Each instance owns a context; errors as
       bfs_setup, prefixed with the instance index (bfs_batch_last_error(NULL)).
     bfs_batch_residual: Fu[i] = F(u[i]) in FP32C for every instance; u, Fu:
       HOST arrays of B DEVICE pointers.  Asynchronous.
     bfs_batch_autotune: times the persistent kernel's tile shapes on the batch
       and keeps the fastest (*ms_out: its batched-residual time).  Synchronous.
     bfs_batch_tuning: the chosen shape and the time of every candidate
       (ms_per_variant: 8 entries, -1 where not run).
     bfs_batch_solve: bfs_solve for every instance, in lockstep (u: host array of
       B device pointers; st: B stats or NULL).  Factors preconditioners that
       are not yet factored.  Synchronous.  Returns BFS_OK when every instance
       converged, otherwise the status of a failing instance (each instance's
       own status is in st[i].status).
     bfs_batch_instance: the context of instance i (owned by the batch), for
       the single-instance calls. */
typedef struct bfs_batch bfs_batch;
int bfs_batch_setup(int B, const bfs_mesh *meshes, const bfs_topo *topos, const double *F,
                    const bfs_options *opt, bfs_batch **out);
void bfs_batch_destroy(bfs_batch *b);
const char *bfs_batch_last_error(const bfs_batch *b);
int bfs_batch_size(const bfs_batch *b);
int bfs_batch_n_unknowns(const bfs_batch *b, int i);
double bfs_batch_pair_evals(const bfs_batch *b);
bfs_ctx *bfs_batch_instance(bfs_batch *b, int i);
int bfs_batch_residual(bfs_batch *b, const double *const *u, double *const *Fu, void *stream);
int bfs_batch_autotune(bfs_batch *b, void *stream, double *ms_out);
int bfs_batch_tuning(const bfs_batch *b, int *variant, int *tpb, int *tpt, double *ms_per_variant);
int bfs_batch_solve(bfs_batch *b, double *const *u, bfs_stats *st, void *stream);

/* Residual for callers that cannot allocate device memory.  The paper has no
   counterpart: this is a library convenience.  Code that runs where a device
   allocation is not allowed (inside a host callback, under a memory pool that
   must not grow, or without ever creating a bfs_ctx) gets the F(u) that
   bfs_residual computes for a context with the default options (no surface
   tension, no applied surface pressure), from the same kernels, with every
   piece of scratch kept in one
   static device array of bfs_static_scratch_bytes() bytes (48 MiB) that each
   GPU loading the library holds until the process exits.  No cudaMalloc,
   cudaFree or allocating library routine is called.
     mesh: as for bfs_setup (host struct); beta, beta_x, beta_y: DEVICE arrays
     of N*M (index i + N*j); u, Fu: DEVICE vectors of length 3(N+1)M in the
     layouts above; n_rad and sign_I4 as in bfs_options; precision BFS_FP64 or
     BFS_FP32C.  Asynchronous on stream.
   The bottom-only part of the bottom integral is recomputed on every call
   (FP64), so a call costs about one FP64 residual more than bfs_residual.
   Limits and errors: BFS_EINVAL (message from bfs_static_last_error) for
   invalid arguments or a mesh whose scratch exceeds the static array (about
   N*M <= 60000 nodes); BFS_ECUDA if the device address of the array cannot
   be obtained.  The first call on each device looks that address up (with the
   device current) and caches it: make that first call before any stream
   capture, and do not use this entry point across a cudaDeviceReset of the
   device (the cached address belongs to the context the reset destroys).  All calls share the array, which keeps the last call's contents
   (the NaN flag is cleared on entry; nothing else needs clearing): calls
   that overlap on the GPU (unordered streams) race and give wrong results;
   calls ordered in one stream are safe.  A non-finite result is not reported
   through a context; check Fu. */
int bfs_residual_static(const bfs_mesh *mesh, const double *beta, const double *beta_x,
                        const double *beta_y, double F, double n_rad, double sign_I4,
                        const double *u, double *Fu, int precision, void *stream);
const char *bfs_static_last_error(void);
size_t bfs_static_scratch_bytes(void);

#ifdef __cplusplus
}
#endif
#endif /* BFS_H */
