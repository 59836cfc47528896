// Internal declarations of the GB300 boundary-integral JFNK library.
// Everything here is private to libbfs; the public ABI is include/bfs.h.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <string>
#include <vector>

#include "bfs.h"

namespace bfs {

// Per-source record (16 values, FP64 or FP32).  Lengths are in units of dx,
// measured from the mesh centre, so that horizontal offsets between nodes
// and half points are exact in FP32 when dx == dy.
//   0 xs   1 ys   2 zeta/dx   3 (beta+1)/dx
//   4 zeta_x  5 zeta_y  6 beta_x  7 beta_y
//   8 w1 f   9 w2 zeta_x   10 w1 g   11 w2 sigma beta_x
//   12 w1    13 w2   14,15 unused
// with f = phi - x, g = psi - x, w the trapezoid weight, w1 = w/dx^2 (double
// layer, K1 scales as 1/dx^2) and w2 = w/dx (single layer and S2).
constexpr int REC = 16;

// Per-target record (16 values) for the half point (k, l):
//   0 xt  1 yt  2 zeta*/dx  3 (beta*+1)/dx  4 zeta_x*  5 zeta_y*  6 f*  7 g*
//   8 A  9 B  10 C   (S2 coefficients of the free surface at the target)
//   11 zeta*/dx + 1/dx   12 (beta*+1)/dx - 1/dx   13 phi_x*  14 phi_y*  15 unused
constexpr int TREC = 16;

// Accumulators written by the pair kernels, per split and target:
//   0  double layer at top targets (top and bottom sheets)
//   1  single layer at top targets (top and bottom sheets)
//   2  sum of w S2 at top targets
//   3  double layer at bottom targets (top and bottom sheets)
//   4  single layer of the top sheet at bottom targets
constexpr int NACC = 5;

// One instance of a batched sweep as the persistent pair kernel sees it.
struct BatchInst {
    const float *src;
    const float *tgt;
    double *part;
    int *flag;  // the instance's status word (bit 2: a wait timed out)
    int Nt, per_split;
};

struct BatchVariant {
    int tpb, tpt;
};

// One step of the FP32 preconditioner sweeps (apply.cu): the slice k whose
// rows it finishes and the stored blocks (k, m[p]) it multiplies.
//   out 0: y_k = r_k - sum_p B(k, m_p) v_p;  out 1: z_k = sum_p +-B(k, m_p) v_p
//   vec[p] bit 0: v_p is z_{m_p} (else y_{m_p}); bit 1: sign + (else -);
//          bits 2-3: where a thread finds its columns of v_p (SW_EARLY, SW_WIN,
//          SW_CRIT); bits 4-5: the register-window index (SW_WIN)
//   uid[p]: the task that wrote v_p (tasks are numbered group 0 first)
constexpr int SW_BMAX = 4;
constexpr int SW_HW = 2;  // register window: the last SW_HW critical vectors
enum { SW_EARLY = 0, SW_WIN = 1, SW_CRIT = 2 };
struct SweepTask {
    int k, out, nblk, pad;
    int m[SW_BMAX], vec[SW_BMAX], uid[SW_BMAX];
};

struct SweepPlan {
    int twist = -1;          // first middle slice of the two-ended order, or -1
    int groups = 1;          // chains run side by side (CTA groups)
    int ntask[2] = {0, 0};   // tasks per group
    std::vector<SweepTask> tasks;
};

struct PairPlan {
    int tpb;        // threads per CTA
    int tpt;        // targets per thread
    int chunk;      // sources staged per shared-memory chunk
    int splits;     // source splits (grid.y)
    int per_split;  // sources per split (multiple of chunk)
    int tiles;      // target tiles (grid.x)
};

}  // namespace bfs

struct bfs_ctx {
    // problem
    int N, M, half;
    double x1, y1, dx, dy, F;
    double beta_max;  // highest bottom node; a valid F keeps it below F^2/2
    bfs_options opt;
    int n, Nt, NM, Ns, Ns_cap;
    double xc, yc;  // centre of the mesh (physical)
    int device;

    // residual buffers
    double *d_beta, *d_bx, *d_by;  // NM each
    double *d_nodal;               // 8 NM: zeta, zx, zy, phi, phx, phy, psi, psx
    double *d_src64;               // Ns_cap * REC
    float *d_src32;                // Ns_cap * REC
    double *d_tgt64;               // Nt * TREC
    float *d_tgt32;                // Nt * TREC
    double *d_part;                // max splits * NACC * Nt
    double *d_constB;              // Nt: bottom-only single-layer part at bottom targets
    double *d_psurf;               // NM applied surface pressure, or nullptr
    int *d_flag;                   // non-finite flag
    float *d_srcdf;                // Ns_cap * 32 double-float source records
    float *d_tgtdf;                // Nt * 32 double-float target records
    bfs::PairPlan plan64, plan32, plandf;
    size_t part_cap;

    // Jacobian-vector product scratch
    double *d_up, *d_Fp;  // n each
    double *d_scal;       // 16 scalars

    // Newton / GMRES workspace
    int m_alloc;
    double *d_V;      // (m+1) n Krylov basis
    double *d_H;      // Hessenberg, column j at d_H + j (m+1)
    double *d_giv;    // cs[m], sn[m], g[m+1], y[m], h[m+1], h2[m+1]
    double *d_red;    // reduction partials
    unsigned int *d_tailbar;  // grid barrier of the fused Arnoldi tail
    int tail_grid;            // its grid (0: the kernels one by one)
    double *d_sbase;  // one allocation holding the n-vectors below
    double *d_F, *d_du, *d_ut, *d_Ft, *d_z, *d_w, *d_F32, *d_uio;  // n each
    double *h_pin;    // pinned host scalars

    // preconditioner
    int pc_ready, pc_h, nb, apply_grid;
    double *d_pc;      // M * (2h+1) * nb * nb  block-banded factors
    float *d_pc32;     // FP32 copy of d_pc (precond_precision FP32C)
    unsigned long long *d_flow;  // tagged y and z of the FP32 sweeps, 2 M nb, then the tag word
    unsigned long long flow_count;  // FP32 sweep launches since the tags were reset
    int capturing;               // a CUDA graph is being captured on the solver stream
    int pc_twist;                // two-ended factor order: first middle slice; -1: one-ended
    bfs::SweepTask *d_tasks;     // task table of the FP32 sweeps
    std::vector<bfs::SweepTask> h_tasks;
    int sweep_table;             // 1: the task-table kernel runs the FP32 sweeps
    int sweep_groups, sweep_ntask[2], sweep_ntags, sweep_rpc, sweep_nslot;
    size_t sweep_dyn;
    int dbg_stall_task;          // test hook: task whose first wait is made unsatisfiable, or -1

    // Arnoldi steps of bfs_solve replayed as CUDA graphs, one per (Krylov
    // index j, base residual buffer); cleared whenever a captured argument
    // could change (factor, F, topography, surface pressure, u buffer)
    std::vector<cudaGraphExec_t> gm_exec;
    std::vector<unsigned long long> gm_nlaunch, gm_nflow;
    // gm_iscond[key]: the step sits in a conditional node behind a guard that
    // reads the device-side end-of-cycle flag, so the next step can be queued
    // before this one's scalars reach the host; gm_cond: 1 while such graphs
    // instantiate, -1 once one failed (plain step graphs from then on)
    std::vector<char> gm_iscond;
    int gm_cond;
    cudaEvent_t gm_ev;
    // solves handed the legacy default stream run here (graph capture needs a
    // stream of its own), joined to the caller's stream by join_ev
    cudaStream_t own_stream;
    cudaEvent_t join_ev;
    const double *gm_u;
    int gm_warm, gm_disabled;
    int ldp32;                   // padded row length of d_pc32
    int flow_checked;
    double *d_gj;      // Gauss-Jordan work matrices and GEMM scratch
    void *d_gjscr;     // dataflow Gauss-Jordan: candidate slots, perm / pinv
    double *d_gjdata;  // dataflow Gauss-Jordan: candidate rows
    double *d_rowsum5; // Nt
    int *d_pivflag;
    double *d_perm_a, *d_perm_b;  // n each

    // profiling: launch counter and CUDA-event timing of the pair kernels
    unsigned long long launches;
    int prof_on;
    std::vector<cudaEvent_t> ev_pool;
    std::vector<int> ev_kind;  // per recorded pair: 0 FP64, 1 FP32C
    size_t ev_used;

    std::string err;
};

namespace bfs {

// residual.cu
int residual_launch(bfs_ctx *c, const double *u, double *Fu, int precision, cudaStream_t s);
int unpack_launch(bfs_ctx *c, const double *u, cudaStream_t s, int which = 3);
int constB_launch(bfs_ctx *c, cudaStream_t s);
PairPlan make_plan(int Nt, int Ns, int tpb, int tpt, int chunk, int splits_req, int sms);
void plans_for(int Nt, int Ns, int splits_req, int sms, PairPlan *p64, PairPlan *p32);

int finish_launch(bfs_ctx *c, double *Fu, int precision, cudaStream_t s);

// apply.cu
int precond_make_f32(bfs_ctx *c, cudaStream_t s);
int apply_flow_launch(bfs_ctx *c, const double *r, double *z, cudaStream_t s);
int flow_wrap_check(bfs_ctx *c, cudaStream_t s);
int flow_reset(bfs_ctx *c, cudaStream_t s);
int sweep_plan(int M, int h, int twisted, SweepPlan &P);
int sweep_twist_ok(bfs_ctx *c, int h);
extern const BatchVariant kBatchVariants[];
extern const int kNumBatchVariants;
int batch_pairs_occupancy(int v, int *blocks_per_sm);
void batch_pairs_launch(int v, int grid, const BatchInst *inst, const int4 *items, int n_items,
                        unsigned int *counter, const unsigned char *mask, cudaStream_t s);

// pairs_df64.cu
PairPlan plan_df(int Nt, int Ns, int splits_req, int sms);
int pairs_df_launch(bfs_ctx *c, cudaStream_t s);

// solver.cu
// GMRES state of one instance between device phases (see solver.cu).
struct Gm {
    enum State { BEGIN, ARNOLDI, CYCLE_END, RESTART, DONE };
    const double *u, *F, *Fbase;
    double target, res;
    int maxit, its, j, status, precs, jvs;
    State state;
};
void gm_start(bfs_ctx *c, Gm &g, const double *u, const double *F, const double *Fbase,
              double fnorm2, double eta, int maxit, cudaStream_t s);
void gm_cycle_begin(bfs_ctx *c, Gm &g, double beta, cudaStream_t s);
int gm_arnoldi_pre(bfs_ctx *c, Gm &g, cudaStream_t s);
int gm_arnoldi_sweep(bfs_ctx *c, Gm &g, cudaStream_t s);
// several instances' Arnoldi steps at once (up to GM_BMAX per launch)
constexpr int GM_BMAX = 64;
int gm_multi_pre(bfs_ctx *const *cs, Gm *const *gs, int cnt, cudaStream_t s);
int gm_multi_post(bfs_ctx *const *cs, Gm *const *gs, int cnt, cudaStream_t s);
int gm_arnoldi_post(bfs_ctx *c, Gm &g, cudaStream_t s);
void gm_arnoldi_host(bfs_ctx *c, Gm &g, double hn, double res);
int gm_cycle_end(bfs_ctx *c, Gm &g, cudaStream_t s);
int gm_restart_post(bfs_ctx *c, Gm &g, cudaStream_t s);
int jv_prep(bfs_ctx *c, const double *u, const double *z, double h, int precision, cudaStream_t s,
            bool unorm_ready);
int jv_post(bfs_ctx *c, const double *Fu, double *Jz, cudaStream_t s);
void solver_axpby(bfs_ctx *c, double *y, const double *x, const double *z, double a, double b,
                  cudaStream_t s);
int jvp_launch(bfs_ctx *c, const double *u, const double *Fu, const double *z, double *Jz,
               double h, int precision, cudaStream_t s, bool unorm_ready = false);
int solve_device(bfs_ctx *c, double *u, bfs_stats *st, cudaStream_t s);
void gm_graphs_clear(bfs_ctx *c);
int alloc_solver(bfs_ctx *c);
void norms_launch(bfs_ctx *c, const double *v, int n, double *d_out2, double *d_outinf, cudaStream_t s);

// precond.cu
int precond_factor(bfs_ctx *c, int half_band, cudaStream_t s);
int precond_apply(bfs_ctx *c, const double *r, double *z, cudaStream_t s);
void precond_free(bfs_ctx *c);

int num_sms(int device);
// records an event pair around a pair-kernel launch when profiling is on
cudaEvent_t prof_event(bfs_ctx *c);
}  // namespace bfs

#define BFS_CUDA_TRY(ctx, call)                                                      \
    do {                                                                             \
        cudaError_t e_ = (call);                                                     \
        if (e_ != cudaSuccess) {                                                     \
            (ctx)->err = std::string(#call) + ": " + cudaGetErrorString(e_);         \
            return BFS_ECUDA;                                                        \
        }                                                                            \
    } while (0)
