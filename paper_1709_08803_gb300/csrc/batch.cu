// Batched sweeps: many independent problems (uneven meshes, Froude numbers,
// topographies) solved together on one GPU.
//
// Each instance keeps its own context (records, preconditioner, Krylov
// workspace).  What is shared is the dominant work: every FP32C residual the
// Krylov iterations need, for all instances at once, is ONE launch of a
// persistent pair kernel whose CTAs take (instance, target tile, source split)
// work items from a queue until it is empty.  Items have near-equal cost (each
// instance's sources are split into chunks of the same length), and are
// queued largest instance first, so meshes from 61 x 21 to 241 x 81 balance
// across the SMs.  The whole batched residual (per-instance record builds,
// queue reset, the persistent kernel, per-instance finishes) is captured once
// as a CUDA graph and replayed.  The tile shape of the persistent kernel is
// chosen by timing the candidates on the batch itself.
//
// The Newton-Krylov iteration runs the instances in lockstep through the
// GMRES phases of solver.cu: every phase is launched for all instances that
// need it, their residuals are evaluated together, and the host reads all
// their scalars with one synchronisation.
#include <math.h>
#include <string.h>

#include <algorithm>
#include <chrono>
#include <new>
#include <numeric>
#include <string>
#include <vector>

#include "bfs_internal.cuh"

struct bfs_batch {
    int B;
    std::vector<bfs_ctx *> c;
    bfs::BatchInst *d_inst;
    int4 *d_items[8];
    int n_items[8];
    unsigned int *d_counter;
    unsigned char *d_mask, *h_mask;
    double *h_sc;      // pinned: 4 scalars per instance
    int variant, grid;
    double tune_ms[8];
    cudaStream_t cap;  // capture stream
    cudaGraphExec_t g_up;  // FP32C residual of every instance's d_up into its d_Fp
    std::string err;
};

namespace {
thread_local std::string g_batch_err;

int berr(bfs_batch *b, int code, const std::string &m)
{
    if (b) b->err = m;
    else g_batch_err = m;
    return code;
}

void free_batch(bfs_batch *b)
{
    if (!b) return;
    for (bfs_ctx *c : b->c) bfs_destroy(c);
    cudaFree(b->d_inst);
    for (int v = 0; v < 8; v++) cudaFree(b->d_items[v]);
    cudaFree(b->d_counter);
    cudaFree(b->d_mask);
    if (b->h_mask) cudaFreeHost(b->h_mask);
    if (b->h_sc) cudaFreeHost(b->h_sc);
    if (b->g_up) cudaGraphExecDestroy(b->g_up);
    if (b->cap) cudaStreamDestroy(b->cap);
}

// Work items of variant v: every (instance, tile, split), largest instances first.
int build_items(bfs_batch *b, int v)
{
    const bfs::BatchVariant var = bfs::kBatchVariants[v];
    std::vector<int> order(b->B);
    std::iota(order.begin(), order.end(), 0);
    std::stable_sort(order.begin(), order.end(), [&](int x, int y) {
        return (double)b->c[x]->Nt * b->c[x]->Ns > (double)b->c[y]->Nt * b->c[y]->Ns;
    });
    std::vector<int4> items;
    for (int i : order) {
        const bfs_ctx *c = b->c[i];
        const int tiles = (c->Nt + var.tpb * var.tpt - 1) / (var.tpb * var.tpt);
        for (int sp = 0; sp < c->plan32.splits; sp++)
            for (int t = 0; t < tiles; t++) items.push_back(make_int4(i, t, sp, 0));
    }
    b->n_items[v] = (int)items.size();
    if (cudaMalloc(&b->d_items[v], sizeof(int4) * items.size()) != cudaSuccess ||
        cudaMemcpy(b->d_items[v], items.data(), sizeof(int4) * items.size(), cudaMemcpyHostToDevice) !=
            cudaSuccess)
        return berr(b, BFS_ENOMEM, "batch work items: allocation failed");
    return BFS_OK;
}

int grid_for_variant(int v)
{
    int per_sm = 0;
    if (bfs::batch_pairs_occupancy(v, &per_sm) || per_sm < 1) return 0;
    int dev = 0;
    cudaGetDevice(&dev);
    return bfs::num_sms(dev) * per_sm;
}

// The batched FP32C residual of the instances whose mask byte is set:
// u[i] -> F[i].  Launches only (capturable).
int batched_residual32(bfs_batch *b, const std::vector<const double *> &u, const std::vector<double *> &F,
                       int v, int grid, cudaStream_t s)
{
    int rc;
    for (int i = 0; i < b->B; i++)
        if ((rc = bfs::unpack_launch(b->c[i], u[i], s, 2))) return berr(b, rc, b->c[i]->err);
    if (cudaMemsetAsync(b->d_counter, 0, sizeof(unsigned int), s) != cudaSuccess)
        return berr(b, BFS_ECUDA, "queue reset failed");
    bfs::batch_pairs_launch(v, grid, b->d_inst, b->d_items[v], b->n_items[v], b->d_counter, b->d_mask, s);
    for (int i = 0; i < b->B; i++)
        if ((rc = bfs::finish_launch(b->c[i], F[i], BFS_FP32C, s))) return berr(b, rc, b->c[i]->err);
    if (cudaGetLastError() != cudaSuccess) return berr(b, BFS_ECUDA, "batched residual launch failed");
    return BFS_OK;
}

int set_mask(bfs_batch *b, const std::vector<char> &on, cudaStream_t s)
{
    for (int i = 0; i < b->B; i++) b->h_mask[i] = on[i] ? 1 : 0;
    if (cudaMemcpyAsync(b->d_mask, b->h_mask, b->B, cudaMemcpyHostToDevice, s) != cudaSuccess)
        return berr(b, BFS_ECUDA, "mask upload failed");
    return BFS_OK;
}

// Graph of the batched FP32C residual d_up[i] -> d_Fp[i] (every instance).
int capture_up_graph(bfs_batch *b)
{
    if (b->g_up) {
        cudaGraphExecDestroy(b->g_up);
        b->g_up = nullptr;
    }
    std::vector<const double *> u(b->B);
    std::vector<double *> F(b->B);
    for (int i = 0; i < b->B; i++) {
        u[i] = b->c[i]->d_up;
        F[i] = b->c[i]->d_Fp;
    }
    cudaGraph_t g;
    if (cudaStreamBeginCapture(b->cap, cudaStreamCaptureModeThreadLocal) != cudaSuccess)
        return berr(b, BFS_ECUDA, "stream capture failed to start");
    int rc = batched_residual32(b, u, F, b->variant, b->grid, b->cap);
    cudaError_t e = cudaStreamEndCapture(b->cap, &g);
    if (rc) return rc;
    if (e != cudaSuccess) return berr(b, BFS_ECUDA, "stream capture failed");
    e = cudaGraphInstantiate(&b->g_up, g, 0);
    cudaGraphDestroy(g);
    if (e != cudaSuccess) return berr(b, BFS_ECUDA, "graph instantiation failed");
    return BFS_OK;
}

int read_batch(bfs_batch *b, const std::vector<int> &who, int off, int cnt, cudaStream_t s)
{
    for (int i : who)
        if (cudaMemcpyAsync(b->h_sc + 4 * i, b->c[i]->d_scal + off, sizeof(double) * cnt,
                            cudaMemcpyDeviceToHost, s) != cudaSuccess)
            return berr(b, BFS_ECUDA, "scalar read failed");
    if (cudaStreamSynchronize(s) != cudaSuccess) return berr(b, BFS_ECUDA, "synchronisation failed");
    return BFS_OK;
}
}  // namespace

extern "C" {

const char *bfs_batch_last_error(const bfs_batch *b) { return b ? b->err.c_str() : g_batch_err.c_str(); }

void bfs_batch_destroy(bfs_batch *b)
{
    if (!b) return;
    free_batch(b);
    delete b;
}

int bfs_batch_setup(int B, const bfs_mesh *meshes, const bfs_topo *topos, const double *F,
                    const bfs_options *opt, bfs_batch **out)
{
    if (!out) return berr(nullptr, BFS_EINVAL, "out is NULL");
    *out = nullptr;
    if (B < 1 || B > 4096 || !meshes || !topos || !F) return berr(nullptr, BFS_EINVAL, "bad batch arguments");
    bfs_batch *b = new (std::nothrow) bfs_batch();
    if (!b) return berr(nullptr, BFS_ENOMEM, "host allocation failed");
    b->B = B;
    bfs_options base;
    if (opt) base = *opt;
    else bfs_default_options(&base);
    for (int i = 0; i < B; i++) {
        bfs_options o = base;
        // equal-length source splits (4 chunks of 128) so that work items cost the same
        const int Ns = meshes[i].half_domain ? meshes[i].N * (2 * meshes[i].M - 1) : meshes[i].N * meshes[i].M;
        o.src_splits = std::max(1, ((Ns + 127) / 128 + 3) / 4);
        if (o.half_band < 0) o.half_band = std::max(1, (int)lround(meshes[i].M / 20.0));
        bfs_ctx *c = nullptr;
        int rc = bfs_setup(&meshes[i], &topos[i], F[i], &o, &c);
        if (rc) {
            std::string m = std::string("instance ") + std::to_string(i) + ": " + bfs_last_error(nullptr);
            free_batch(b);
            delete b;
            return berr(nullptr, rc, m);
        }
        b->c.push_back(c);
    }
    std::vector<bfs::BatchInst> inst(B);
    for (int i = 0; i < B; i++) {
        inst[i].src = b->c[i]->d_src32;
        inst[i].flag = b->c[i]->d_flag;
        inst[i].tgt = b->c[i]->d_tgt32;
        inst[i].part = b->c[i]->d_part;
        inst[i].Nt = b->c[i]->Nt;
        inst[i].per_split = b->c[i]->plan32.per_split;
    }
    auto fail = [&](int code, const std::string &m) {
        free_batch(b);
        delete b;
        cudaGetLastError();
        return berr(nullptr, code, m);
    };
    if (cudaMalloc(&b->d_inst, sizeof(bfs::BatchInst) * B) != cudaSuccess ||
        cudaMemcpy(b->d_inst, inst.data(), sizeof(bfs::BatchInst) * B, cudaMemcpyHostToDevice) != cudaSuccess ||
        cudaMalloc(&b->d_counter, sizeof(unsigned int)) != cudaSuccess ||
        cudaMalloc(&b->d_mask, B) != cudaSuccess || cudaMallocHost(&b->h_mask, B) != cudaSuccess ||
        cudaMallocHost(&b->h_sc, sizeof(double) * 4 * B) != cudaSuccess ||
        cudaStreamCreateWithFlags(&b->cap, cudaStreamNonBlocking) != cudaSuccess)
        return fail(BFS_ENOMEM, "batch allocation failed");
    for (int v = 0; v < bfs::kNumBatchVariants; v++)
        if (build_items(b, v)) return fail(BFS_ENOMEM, b->err);
    b->variant = 0;
    b->grid = grid_for_variant(0);
    if (b->grid < 1) return fail(BFS_ECUDA, "persistent pair kernel cannot be resident");
    memset(b->h_mask, 1, B);
    if (cudaMemcpy(b->d_mask, b->h_mask, B, cudaMemcpyHostToDevice) != cudaSuccess)
        return fail(BFS_ECUDA, "mask upload failed");
    *out = b;
    return BFS_OK;
}

int bfs_batch_size(const bfs_batch *b) { return b ? b->B : 0; }

int bfs_batch_n_unknowns(const bfs_batch *b, int i) { return (b && i >= 0 && i < b->B) ? b->c[i]->n : 0; }

double bfs_batch_pair_evals(const bfs_batch *b)
{
    double s = 0.0;
    if (b)
        for (bfs_ctx *c : b->c) s += bfs_pair_evals(c);
    return s;
}

bfs_ctx *bfs_batch_instance(bfs_batch *b, int i) { return (b && i >= 0 && i < b->B) ? b->c[i] : nullptr; }

int bfs_batch_residual(bfs_batch *b, const double *const *u, double *const *Fu, void *stream)
{
    if (!b || !u || !Fu) return berr(b, BFS_EINVAL, "NULL argument");
    cudaStream_t s = (cudaStream_t)stream;
    std::vector<const double *> uu(u, u + b->B);
    std::vector<double *> FF(Fu, Fu + b->B);
    int rc = set_mask(b, std::vector<char>(b->B, 1), s);
    if (rc) return rc;
    return batched_residual32(b, uu, FF, b->variant, b->grid, s);
}

int bfs_batch_autotune(bfs_batch *b, void *stream, double *ms_out)
{
    if (!b) return BFS_EINVAL;
    cudaStream_t s = (cudaStream_t)stream;
    std::vector<const double *> u(b->B);
    std::vector<double *> F(b->B);
    for (int i = 0; i < b->B; i++) {
        bfs_ctx *c = b->c[i];
        int rc = bfs_flat_guess(c, c->d_up, stream);
        if (rc) return berr(b, rc, c->err);
        u[i] = c->d_up;
        F[i] = c->d_Fp;
    }
    int rc = set_mask(b, std::vector<char>(b->B, 1), s);
    if (rc) return rc;
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    double best = 1e30;
    int bestv = 0;
    for (int v = 0; v < bfs::kNumBatchVariants; v++) {
        const int grid = grid_for_variant(v);
        b->tune_ms[v] = -1.0;
        if (grid < 1) continue;
        if ((rc = batched_residual32(b, u, F, v, grid, s))) break;  // warm
        cudaEventRecord(e0, s);
        for (int r = 0; r < 3; r++)
            if ((rc = batched_residual32(b, u, F, v, grid, s))) break;
        cudaEventRecord(e1, s);
        if (rc || cudaEventSynchronize(e1) != cudaSuccess) break;
        float ms = 0.f;
        cudaEventElapsedTime(&ms, e0, e1);
        b->tune_ms[v] = ms / 3.0;
        if (ms / 3.0 < best) { best = ms / 3.0; bestv = v; }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (rc) return rc;
    b->variant = bestv;
    b->grid = grid_for_variant(bestv);
    if (b->g_up) {
        cudaGraphExecDestroy(b->g_up);
        b->g_up = nullptr;
    }
    if (ms_out) *ms_out = best;
    return BFS_OK;
}

int bfs_batch_tuning(const bfs_batch *b, int *variant, int *tpb, int *tpt, double *ms_per_variant)
{
    if (!b) return BFS_EINVAL;
    if (variant) *variant = b->variant;
    if (tpb) *tpb = bfs::kBatchVariants[b->variant].tpb;
    if (tpt) *tpt = bfs::kBatchVariants[b->variant].tpt;
    if (ms_per_variant)
        for (int v = 0; v < bfs::kNumBatchVariants; v++) ms_per_variant[v] = b->tune_ms[v];
    return BFS_OK;
}

int bfs_batch_solve(bfs_batch *b, double *const *u, bfs_stats *st, void *stream)
{
    using clk = std::chrono::steady_clock;
    if (!b || !u) return berr(b, BFS_EINVAL, "NULL argument");
    const auto t0 = clk::now();
    cudaStream_t s = (cudaStream_t)stream;
    const int B = b->B;
    int rc;
    for (int i = 0; i < B; i++) {
        bfs_ctx *c = b->c[i];
        if ((rc = bfs::alloc_solver(c))) return berr(b, rc, c->err);
        if (!c->pc_ready && (rc = bfs::precond_factor(c, c->opt.half_band, s))) return berr(b, rc, c->err);
    }
    if (!b->g_up && (rc = capture_up_graph(b))) return rc;
    const bfs_options &o = b->c[0]->opt;
    const bool k32 = o.krylov_precision == BFS_FP32C;
    // per instance: arithmetic of the Newton residual (the Krylov one while
    // |F| > refine_below, then the outer one)
    const int outer = o.outer_precision;
    std::vector<int> cur(B, (o.refine_below > 0.0 && o.krylov_precision != outer) ? o.krylov_precision : outer);
    std::vector<bfs_stats> S(B);
    std::vector<bfs::Gm> g(B);
    std::vector<int> status(B, 1);  // 1 running, else final status
    std::vector<double> f2(B), finf(B), mu(B);
    std::vector<int> stalls(B, 0);
    // forcing terms per instance (Eisenstat-Walker choice 1 when o.forcing == 1)
    std::vector<double> eta(B, o.forcing == 1 ? std::max(o.eta, 0.1) : o.eta), prev_f2(B, -1.0), prev_lin(B, 0.0);
    std::vector<int> all(B);
    std::iota(all.begin(), all.end(), 0);

    auto outer_residuals = [&](const std::vector<int> &who, bool trial) -> int {
        for (int i : who) {
            bfs_ctx *c = b->c[i];
            const double *x = trial ? c->d_ut : u[i];
            double *y = trial ? c->d_Ft : c->d_F;
            if ((rc = bfs::residual_launch(c, x, y, cur[i], s))) return berr(b, rc, c->err);
            if (cur[i] == BFS_FP32C) S[i].residual_evals_fp32++;
            else S[i].residual_evals_fp64++;
            bfs::norms_launch(c, y, c->n, c->d_scal + 10, c->d_scal + 11, s);
        }
        return read_batch(b, who, 10, 2, s);
    };
    // residuals inside the Krylov phases: FP32C instances through the graph
    auto krylov_residuals = [&](const std::vector<int> &who) -> int {
        if (who.empty()) return BFS_OK;
        if (k32) {
            std::vector<char> on(B, 0);
            for (int i : who) on[i] = 1;
            if ((rc = set_mask(b, on, s))) return rc;
            if (cudaGraphLaunch(b->g_up, s) != cudaSuccess) return berr(b, BFS_ECUDA, "graph launch failed");
            for (int i : who) S[i].residual_evals_fp32++;
            return BFS_OK;
        }
        for (int i : who) {
            bfs_ctx *c = b->c[i];
            if ((rc = bfs::residual_launch(c, c->d_up, c->d_Fp, o.krylov_precision, s))) return berr(b, rc, c->err);
            S[i].residual_evals_fp64++;
        }
        return BFS_OK;
    };

    for (int i = 0; i < B; i++) {
        cudaMemsetAsync(b->c[i]->d_flag, 0, sizeof(int), s);
        cudaMemsetAsync(b->c[i]->d_tailbar, 0, 2 * sizeof(unsigned int), s);
    }
    if ((rc = outer_residuals(all, false))) return rc;
    for (int i = 0; i < B; i++) { f2[i] = b->h_sc[4 * i]; finf[i] = b->h_sc[4 * i + 1]; }

    for (int k = 0;; k++) {
        {
            // instances close enough for the final arithmetic switch to it
            std::vector<int> sw;
            for (int i = 0; i < B; i++)
                if (status[i] == 1 && cur[i] != outer && isfinite(finf[i]) &&
                    (finf[i] <= o.refine_below || finf[i] <= o.tol)) {
                    cur[i] = outer;
                    sw.push_back(i);
                }
            if (!sw.empty()) {
                if ((rc = outer_residuals(sw, false))) return rc;
                for (int i : sw) { f2[i] = b->h_sc[4 * i]; finf[i] = b->h_sc[4 * i + 1]; }
            }
        }
        std::vector<int> act;
        for (int i = 0; i < B; i++) {
            if (status[i] != 1) continue;
            S[i].fnorm_2 = f2[i];
            S[i].fnorm_inf = finf[i];
            if (!isfinite(f2[i]) || !isfinite(finf[i])) status[i] = BFS_ENAN;
            else if (finf[i] <= o.tol) status[i] = BFS_OK;
            else if (k >= o.max_newton) status[i] = BFS_ENOCONV;
            else if (o.time_budget_s > 0.0 &&
                     std::chrono::duration<double>(clk::now() - t0).count() > o.time_budget_s)
                status[i] = BFS_ETIMEOUT;
            else act.push_back(i);
        }
        if (act.empty()) break;
        // base residuals of the finite differences, in the Krylov arithmetic
        std::vector<int> base;
        for (int i : act)
            if (cur[i] != o.krylov_precision) base.push_back(i);
        if (!base.empty()) {
            if (k32) {
                std::vector<char> on(B, 0);
                for (int i : base) on[i] = 1;
                if ((rc = set_mask(b, on, s))) return rc;
                std::vector<const double *> uu(B);
                std::vector<double *> FF(B);
                for (int i = 0; i < B; i++) { uu[i] = u[i]; FF[i] = b->c[i]->d_F32; }
                if ((rc = batched_residual32(b, uu, FF, b->variant, b->grid, s))) return rc;
                for (int i : base) S[i].residual_evals_fp32++;
            } else {
                for (int i : base) {
                    bfs_ctx *c = b->c[i];
                    if ((rc = bfs::residual_launch(c, u[i], c->d_F32, o.krylov_precision, s))) return berr(b, rc, c->err);
                    S[i].residual_evals_fp64++;
                }
            }
        }
        for (int i : act) {
            bfs_ctx *c = b->c[i];
            bfs::Gm gi{};
            gi.precs = g[i].precs;
            gi.jvs = g[i].jvs;
            g[i] = gi;
            if (o.forcing == 1 && prev_f2[i] > 0.0) {
                double e = fabs(f2[i] - prev_lin[i]) / prev_f2[i];
                const double sg = pow(eta[i], 1.6180339887498949);
                if (sg > 0.1) e = std::max(e, sg);
                eta[i] = std::min(0.9, std::max(o.eta, e));
            }
            bfs::gm_start(c, g[i], u[i], c->d_F, cur[i] != o.krylov_precision ? c->d_F32 : c->d_F, f2[i], eta[i],
                          o.max_krylov, s);
        }
        if ((rc = read_batch(b, act, 8, 1, s))) return rc;
        for (int i : act) bfs::gm_cycle_begin(b->c[i], g[i], b->h_sc[4 * i], s);
        // lockstep GMRES
        while (true) {
            std::vector<int> arn, rst, live;
            for (int i : act) {
                if (g[i].state == bfs::Gm::CYCLE_END &&
                    (rc = bfs::gm_cycle_end(b->c[i], g[i], s)))
                    return berr(b, rc, b->c[i]->err);
            }
            for (int i : act) {
                if (g[i].state == bfs::Gm::ARNOLDI) arn.push_back(i);
                else if (g[i].state == bfs::Gm::RESTART) rst.push_back(i);
            }
            if (arn.empty() && rst.empty()) break;
            // the sweeps per instance, then |z|, h, u + h z for all in one launch pair
            std::vector<bfs_ctx *> acs;
            std::vector<bfs::Gm *> ags;
            for (int i : arn) {
                if ((rc = bfs::gm_arnoldi_sweep(b->c[i], g[i], s))) return berr(b, rc, b->c[i]->err);
                acs.push_back(b->c[i]);
                ags.push_back(&g[i]);
            }
            if (!arn.empty() && (rc = bfs::gm_multi_pre(acs.data(), ags.data(), (int)arn.size(), s)))
                return berr(b, rc, acs[0]->err);
            live = arn;
            live.insert(live.end(), rst.begin(), rst.end());
            if ((rc = krylov_residuals(live))) return rc;
            // Jz, CGS2, v_{j+1} and Givens for all in one cooperative launch
            if (!arn.empty() && (rc = bfs::gm_multi_post(acs.data(), ags.data(), (int)arn.size(), s)))
                return berr(b, rc, acs[0]->err);
            for (int i : rst)
                if ((rc = bfs::gm_restart_post(b->c[i], g[i], s))) return berr(b, rc, b->c[i]->err);
            if ((rc = read_batch(b, live, 8, 2, s))) return rc;
            for (int i : arn) bfs::gm_arnoldi_host(b->c[i], g[i], b->h_sc[4 * i], b->h_sc[4 * i + 1]);
            for (int i : rst) bfs::gm_cycle_begin(b->c[i], g[i], b->h_sc[4 * i], s);
        }
        std::vector<int> ls;
        for (int i : act) {
            S[i].krylov_its += g[i].its;
            stalls[i] = g[i].res > g[i].target ? stalls[i] + 1 : 0;
            if (g[i].status != BFS_OK) status[i] = g[i].status;
            else if (o.stall_newton > 0 && stalls[i] >= o.stall_newton) status[i] = BFS_ENOCONV;
            else { ls.push_back(i); mu[i] = 1.0; }
        }
        // lockstep backtracking line search
        while (!ls.empty()) {
            for (int i : ls) {
                bfs_ctx *c = b->c[i];
                bfs::solver_axpby(c, c->d_ut, u[i], c->d_du, 1.0, mu[i], s);
            }
            if ((rc = outer_residuals(ls, true))) return rc;
            std::vector<int> next;
            for (int i : ls) {
                bfs_ctx *c = b->c[i];
                const double t2 = b->h_sc[4 * i], tinf = b->h_sc[4 * i + 1];
                if (isfinite(t2) && t2 <= (1.0 - 1e-4 * mu[i]) * f2[i]) {
                    prev_f2[i] = f2[i];
                    prev_lin[i] = (1.0 - mu[i]) * f2[i] + mu[i] * g[i].res;
                    f2[i] = t2;
                    finf[i] = tinf;
                    cudaMemcpyAsync(u[i], c->d_ut, sizeof(double) * c->n, cudaMemcpyDeviceToDevice, s);
                    std::swap(c->d_F, c->d_Ft);
                    S[i].newton_its = k + 1;
                } else {
                    mu[i] *= 0.5;
                    if (mu[i] >= 1e-4) next.push_back(i);
                    else status[i] = BFS_ELINESEARCH;
                }
            }
            ls.swap(next);
        }
    }
    const double secs = std::chrono::duration<double>(clk::now() - t0).count();
    int worst = BFS_OK;
    for (int i = 0; i < B; i++) {
        S[i].status = status[i];
        S[i].seconds = secs;
        S[i].precond_applies = g[i].precs;
        if (st) st[i] = S[i];
        if (status[i] != BFS_OK) worst = status[i];
    }
    if (cudaStreamSynchronize(s) != cudaSuccess) return berr(b, BFS_ECUDA, "synchronisation failed");
    if (worst != BFS_OK) b->err = "at least one instance did not converge (see its status)";
    return worst;
}

}  // extern "C"
