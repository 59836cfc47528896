// C ABI of libbfs (declared and documented in include/bfs.h).
#include <math.h>
#include <stdio.h>
#include <string.h>

#include <new>
#include <vector>

#include "bfs_internal.cuh"

namespace {
thread_local std::string g_setup_err;

__global__ void k_flat_guess(double *u, int N, int M, double x1)
{
    const int NB = N + 1, n = 3 * NB * M;
    for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < n; e += gridDim.x * blockDim.x) {
        int g = e / (NB * M), p = (e % (NB * M)) % NB;
        u[e] = g == 0 ? 0.0 : (p == 0 ? x1 : 1.0);
    }
}

void free_all(bfs_ctx *c)
{
    if (!c) return;
    bfs::precond_free(c);
    cudaFree(c->d_beta);
    cudaFree(c->d_nodal);
    cudaFree(c->d_src64);
    cudaFree(c->d_src32);
    cudaFree(c->d_tgt64);
    cudaFree(c->d_tgt32);
    cudaFree(c->d_srcdf);
    cudaFree(c->d_tgtdf);
    cudaFree(c->d_part);
    cudaFree(c->d_constB);
    cudaFree(c->d_psurf);
    cudaFree(c->d_flag);
    cudaFree(c->d_up);
    cudaFree(c->d_scal);
    cudaFree(c->d_red);
    cudaFree(c->d_tailbar);
    cudaFree(c->d_V);
    cudaFree(c->d_H);
    cudaFree(c->d_giv);
    cudaFree(c->d_sbase);
    if (c->h_pin) cudaFreeHost(c->h_pin);
    if (c->gm_ev) cudaEventDestroy(c->gm_ev);
    c->gm_ev = nullptr;
    if (c->join_ev) cudaEventDestroy(c->join_ev);
    c->join_ev = nullptr;
    if (c->own_stream) {
        cudaStreamSynchronize(c->own_stream);
        cudaStreamDestroy(c->own_stream);
    }
    c->own_stream = nullptr;
    for (cudaEvent_t e : c->ev_pool) cudaEventDestroy(e);
    c->ev_pool.clear();
}

int set_err(bfs_ctx *c, int code, const std::string &msg)
{
    if (c) c->err = msg;
    else g_setup_err = msg;
    return code;
}
}  // namespace

namespace bfs {
int num_sms(int device)
{
    int v = 0;
    cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, device);
    return v > 0 ? v : 1;
}
}  // namespace bfs

extern "C" {

void bfs_default_options(bfs_options *o)
{
    if (!o) return;
    memset(o, 0, sizeof(*o));
    o->n_rad = 0.05;
    o->sign_I4 = -1.0;
    o->half_band = -1;  // resolved in bfs_setup: max(1, round(M / 20))
    o->tol = 1e-8;
    o->gmres_restart = 50;
    o->max_newton = 60;
    o->max_krylov = 200;
    o->eta = 1e-4;
    o->krylov_precision = BFS_FP64;
    o->jv_h_rel = 0.0;
    o->time_budget_s = 0.0;
    o->src_splits = 0;
    o->outer_precision = BFS_FP64;
    o->precond_precision = BFS_FP64;
    o->refine_below = 0.0;
    o->stall_newton = 0;
    o->surface_tension = 0.0;
    o->forcing = 0;
}

const char *bfs_last_error(const bfs_ctx *c) { return c ? c->err.c_str() : g_setup_err.c_str(); }

int bfs_n_unknowns(const bfs_ctx *c) { return c ? c->n : 0; }

double bfs_pair_evals(const bfs_ctx *c) { return c ? 4.0 * (double)c->Nt * (double)c->Ns : 0.0; }

int bfs_setup(const bfs_mesh *mesh, const bfs_topo *topo, double F, const bfs_options *opt,
              bfs_ctx **out)
{
    if (!out) return set_err(nullptr, BFS_EINVAL, "out is NULL");
    *out = nullptr;
    if (!mesh || !topo || !topo->beta || !topo->beta_x || !topo->beta_y)
        return set_err(nullptr, BFS_EINVAL, "mesh or topography is NULL");
    const int N = mesh->N, M = mesh->M;
    if (N < 4 || M < 3) return set_err(nullptr, BFS_EINVAL, "need N >= 4 and M >= 3");
    if ((long long)N * M > (1LL << 26)) return set_err(nullptr, BFS_EINVAL, "mesh too large");
    if (!(mesh->dx > 0.0) || !(mesh->dy > 0.0) || !isfinite(mesh->dx) || !isfinite(mesh->dy) ||
        !isfinite(mesh->x1) || !isfinite(mesh->y1))
        return set_err(nullptr, BFS_EINVAL, "dx and dy must be positive and finite");
    if (!(F > 0.0) || !isfinite(F)) return set_err(nullptr, BFS_EINVAL, "F must be positive");
    if (mesh->half_domain && mesh->y1 != 0.0)
        return set_err(nullptr, BFS_EINVAL, "half_domain requires y1 == 0");
    bfs_options o;
    if (opt) o = *opt;
    else bfs_default_options(&o);
    if (o.half_band < 0) o.half_band = std::max(1, (int)lround(M / 20.0));
    if (o.gmres_restart < 1 || o.gmres_restart > 120)
        return set_err(nullptr, BFS_EINVAL, "gmres_restart must be in [1, 120]");
    if (o.sign_I4 != 1.0 && o.sign_I4 != -1.0)
        return set_err(nullptr, BFS_EINVAL, "sign_I4 must be +1 or -1");
    if (o.krylov_precision != BFS_FP64 && o.krylov_precision != BFS_FP32C && o.krylov_precision != BFS_DF64)
        return set_err(nullptr, BFS_EINVAL, "unknown krylov_precision");
    if (!(o.refine_below >= 0.0)) return set_err(nullptr, BFS_EINVAL, "refine_below must be >= 0");
    if (o.forcing != 0 && o.forcing != 1) return set_err(nullptr, BFS_EINVAL, "forcing must be 0 or 1");
    if (!(o.surface_tension >= 0.0) || !isfinite(o.surface_tension))
        return set_err(nullptr, BFS_EINVAL, "surface_tension must be finite and >= 0");
    if (o.precond_precision != BFS_FP64 && o.precond_precision != BFS_FP32C)
        return set_err(nullptr, BFS_EINVAL, "precond_precision must be BFS_FP64 or BFS_FP32C");
    if (o.outer_precision != BFS_FP64 && o.outer_precision != BFS_DF64)
        return set_err(nullptr, BFS_EINVAL, "outer_precision must be BFS_FP64 or BFS_DF64");
    const size_t NM = (size_t)N * M;
    double beta_max = -INFINITY;
    for (size_t q = 0; q < NM; q++) {
        if (!isfinite(topo->beta[q]) || !isfinite(topo->beta_x[q]) || !isfinite(topo->beta_y[q]))
            return set_err(nullptr, BFS_EINVAL, "topography has a non-finite value");
        if (!(topo->beta[q] < 0.5 * F * F))
            return set_err(nullptr, BFS_EINVAL, "the bottom reaches F^2/2, above any possible free surface");
        beta_max = std::max(beta_max, topo->beta[q]);
    }

    bfs_ctx *c = new (std::nothrow) bfs_ctx();
    if (!c) return set_err(nullptr, BFS_ENOMEM, "host allocation failed");
    c->N = N; c->M = M; c->half = mesh->half_domain ? 1 : 0;
    c->x1 = mesh->x1; c->y1 = mesh->y1; c->dx = mesh->dx; c->dy = mesh->dy; c->F = F;
    c->beta_max = beta_max;
    c->opt = o;
    c->pc_twist = -1;
    c->dbg_stall_task = -1;
    c->n = 3 * (N + 1) * M;
    c->Nt = (N - 1) * M;
    c->NM = (int)NM;
    c->Ns = c->half ? N * (2 * M - 1) : N * M;
    cudaGetDevice(&c->device);
    const int sms = bfs::num_sms(c->device);
    bfs::plans_for(c->Nt, c->Ns, o.src_splits, sms, &c->plan64, &c->plan32);
    if (o.src_splits <= 0) {
        // FP32C: down to one chunk of sources per split while the split partial
        // sums stay below 2^20 target slots (40 MB): many short CTAs, so that the
        // last wave of the launch is a small part of it (the split count changes
        // only how the chunk totals are grouped: a two-sum within a split, FP64
        // across splits; the 181 x 61 residuals came out identical)
        const int nchunks = (c->Ns + c->plan32.chunk - 1) / c->plan32.chunk;
        const int fine = std::min(nchunks, std::max(c->plan32.splits, (1 << 20) / std::max(c->Nt, 1)));
        if (fine > c->plan32.splits)
            c->plan32 = bfs::make_plan(c->Nt, c->Ns, c->plan32.tpb, c->plan32.tpt, c->plan32.chunk, fine, sms);
    }
    c->plandf = bfs::plan_df(c->Nt, c->Ns, o.src_splits, sms);
    c->Ns_cap = std::max(c->plan64.splits * c->plan64.per_split, c->plan32.splits * c->plan32.per_split);
    c->Ns_cap = std::max(c->Ns_cap, c->plandf.splits * c->plandf.per_split);
    c->part_cap = (size_t)std::max(std::max(c->plan64.splits, c->plan32.splits), c->plandf.splits) *
                  bfs::NACC * c->Nt;

    auto fail = [&](int code, const std::string &m) {
        free_all(c);
        delete c;
        cudaGetLastError();
        return set_err(nullptr, code, m);
    };
#define ALLOC(ptr, bytes)                                                       \
    if (cudaMalloc(&(ptr), (bytes)) != cudaSuccess) return fail(BFS_ENOMEM, "device allocation failed: " #ptr);
    ALLOC(c->d_beta, sizeof(double) * 3 * NM);
    c->d_bx = c->d_beta + NM;
    c->d_by = c->d_beta + 2 * NM;
    ALLOC(c->d_nodal, sizeof(double) * 8 * NM);
    ALLOC(c->d_src64, sizeof(double) * bfs::REC * (size_t)c->Ns_cap);
    ALLOC(c->d_src32, sizeof(float) * bfs::REC * (size_t)c->Ns_cap);
    ALLOC(c->d_tgt64, sizeof(double) * bfs::TREC * (size_t)c->Nt);
    ALLOC(c->d_tgt32, sizeof(float) * bfs::TREC * (size_t)c->Nt);
    ALLOC(c->d_srcdf, sizeof(float) * 32 * (size_t)c->Ns_cap);
    ALLOC(c->d_tgtdf, sizeof(float) * 32 * (size_t)c->Nt);
    ALLOC(c->d_part, sizeof(double) * c->part_cap);
    ALLOC(c->d_constB, sizeof(double) * (size_t)c->Nt);
    ALLOC(c->d_flag, sizeof(int));
    ALLOC(c->d_up, sizeof(double) * 2 * (size_t)c->n);
    c->d_Fp = c->d_up + c->n;
    ALLOC(c->d_scal, sizeof(double) * 32);
    ALLOC(c->d_red, sizeof(double) * 128 * 256);
#undef ALLOC
    if (cudaMemcpy(c->d_beta, topo->beta, sizeof(double) * NM, cudaMemcpyHostToDevice) ||
        cudaMemcpy(c->d_bx, topo->beta_x, sizeof(double) * NM, cudaMemcpyHostToDevice) ||
        cudaMemcpy(c->d_by, topo->beta_y, sizeof(double) * NM, cudaMemcpyHostToDevice) ||
        cudaMemset(c->d_flag, 0, sizeof(int)) || cudaMemset(c->d_scal, 0, sizeof(double) * 32))
        return fail(BFS_ECUDA, "upload failed");
    // bottom-only constant: needs the source and target records of any u
    double *u0 = c->d_Fp;
    k_flat_guess<<<(c->n + 255) / 256, 256>>>(u0, N, M, c->x1);
    c->launches++;
    if (bfs::unpack_launch(c, u0, 0) || bfs::constB_launch(c, 0) ||
        cudaDeviceSynchronize() != cudaSuccess)
        return fail(BFS_ECUDA, std::string("setup kernels failed: ") + c->err);
    *out = c;
    return BFS_OK;
}

int bfs_set_topography(bfs_ctx *c, const bfs_topo *topo)
{
    if (!c || !topo || !topo->beta || !topo->beta_x || !topo->beta_y)
        return set_err(c, BFS_EINVAL, "NULL argument");
    const size_t NM = (size_t)c->NM;
    double beta_max = -INFINITY;
    for (size_t q = 0; q < NM; q++) {
        if (!isfinite(topo->beta[q]) || !isfinite(topo->beta_x[q]) || !isfinite(topo->beta_y[q]))
            return set_err(c, BFS_EINVAL, "topography has a non-finite value");
        if (!(topo->beta[q] < 0.5 * c->F * c->F))
            return set_err(c, BFS_EINVAL, "the bottom reaches F^2/2, above any possible free surface");
        beta_max = std::max(beta_max, topo->beta[q]);
    }
    BFS_CUDA_TRY(c, cudaDeviceSynchronize());
    bfs::gm_graphs_clear(c);
    BFS_CUDA_TRY(c, cudaMemcpy(c->d_beta, topo->beta, sizeof(double) * NM, cudaMemcpyHostToDevice));
    BFS_CUDA_TRY(c, cudaMemcpy(c->d_bx, topo->beta_x, sizeof(double) * NM, cudaMemcpyHostToDevice));
    BFS_CUDA_TRY(c, cudaMemcpy(c->d_by, topo->beta_y, sizeof(double) * NM, cudaMemcpyHostToDevice));
    c->beta_max = beta_max;
    double *u0 = c->d_Fp;
    k_flat_guess<<<(c->n + 255) / 256, 256>>>(u0, c->N, c->M, c->x1);
    c->launches++;
    if (bfs::unpack_launch(c, u0, 0) || bfs::constB_launch(c, 0)) return BFS_ECUDA;
    BFS_CUDA_TRY(c, cudaDeviceSynchronize());
    return BFS_OK;
}

int bfs_set_surface_pressure(bfs_ctx *c, const double *p)
{
    if (!c) return BFS_EINVAL;
    cudaDeviceSynchronize();
    bfs::gm_graphs_clear(c);
    if (!p) {
        cudaFree(c->d_psurf);
        c->d_psurf = nullptr;
        return BFS_OK;
    }
    for (int q = 0; q < c->NM; q++)
        if (!isfinite(p[q])) return set_err(c, BFS_EINVAL, "surface pressure has a non-finite value");
    BFS_CUDA_TRY(c, cudaDeviceSynchronize());
    if (!c->d_psurf && cudaMalloc(&c->d_psurf, sizeof(double) * (size_t)c->NM) != cudaSuccess) {
        cudaGetLastError();
        return set_err(c, BFS_ENOMEM, "device allocation failed");
    }
    BFS_CUDA_TRY(c, cudaMemcpy(c->d_psurf, p, sizeof(double) * (size_t)c->NM, cudaMemcpyHostToDevice));
    return BFS_OK;
}

int bfs_set_froude(bfs_ctx *c, double F)
{
    if (!c) return BFS_EINVAL;
    if (!(F > 0.0) || !isfinite(F)) return set_err(c, BFS_EINVAL, "F must be positive");
    if (!(c->beta_max < 0.5 * F * F))
        return set_err(c, BFS_EINVAL, "the bottom reaches F^2/2, above any possible free surface");
    BFS_CUDA_TRY(c, cudaDeviceSynchronize());
    bfs::gm_graphs_clear(c);  // F is an argument of the captured finish kernels
    c->F = F;
    return BFS_OK;
}

void bfs_destroy(bfs_ctx *c)
{
    if (!c) return;
    cudaDeviceSynchronize();
    bfs::gm_graphs_clear(c);
    free_all(c);
    delete c;
}

int bfs_residual(bfs_ctx *c, const double *u, double *Fu, int precision, void *stream)
{
    if (!c || !u || !Fu) return set_err(c, BFS_EINVAL, "NULL argument");
    if (precision != BFS_FP64 && precision != BFS_FP32C && precision != BFS_DF64)
        return set_err(c, BFS_EINVAL, "bad precision");
    return bfs::residual_launch(c, u, Fu, precision, (cudaStream_t)stream);
}

int bfs_check_finite(bfs_ctx *c, void *stream)
{
    if (!c) return BFS_EINVAL;
    int flag = 0;
    cudaStream_t s = (cudaStream_t)stream;
    BFS_CUDA_TRY(c, cudaMemcpyAsync(&flag, c->d_flag, sizeof(int), cudaMemcpyDeviceToHost, s));
    BFS_CUDA_TRY(c, cudaStreamSynchronize(s));
    BFS_CUDA_TRY(c, cudaMemsetAsync(c->d_flag, 0, sizeof(int), s));
    if (flag & 2) {
        // entries a timed-out sweep left behind must not match a later launch's tags
        int rc = bfs::flow_reset(c, s);
        if (rc) return rc;
        return set_err(c, BFS_ETIMEOUT, "a device-side wait timed out");
    }
    if (flag) return set_err(c, BFS_ENAN, "a residual entry was not finite");
    return BFS_OK;
}

int bfs_jvp(bfs_ctx *c, const double *u, const double *Fu, const double *z, double *Jz, double h,
            int precision, void *stream)
{
    if (!c || !u || !Fu || !z || !Jz) return set_err(c, BFS_EINVAL, "NULL argument");
    if (precision != BFS_FP64 && precision != BFS_FP32C && precision != BFS_DF64)
        return set_err(c, BFS_EINVAL, "bad precision");
    return bfs::jvp_launch(c, u, Fu, z, Jz, h, precision, (cudaStream_t)stream);
}

int bfs_precond_factor(bfs_ctx *c, int half_band, void *stream)
{
    if (!c) return BFS_EINVAL;
    return bfs::precond_factor(c, half_band, (cudaStream_t)stream);
}

int bfs_precond_info(const bfs_ctx *c, int *info)
{
    if (!c || !info) return BFS_EINVAL;
    if (!c->pc_ready) return BFS_ENOPREC;
    info[0] = c->pc_h;
    info[1] = c->pc_twist;
    info[2] = c->sweep_table ? c->sweep_groups : (c->d_pc32 ? 1 : 0);
    info[3] = c->sweep_table ? std::max(c->sweep_ntask[0], c->sweep_ntask[1]) : 2 * c->M;
    return BFS_OK;
}

int bfs_solver_info(const bfs_ctx *c, int *info)
{
    if (!c || !info) return BFS_EINVAL;
    int graphs = 0, cond = 0;
    for (size_t k = 0; k < c->gm_exec.size(); k++)
        if (c->gm_exec[k]) {
            graphs++;
            cond += c->gm_iscond[k] ? 1 : 0;
        }
    info[0] = graphs;
    info[1] = cond;
    info[2] = c->gm_disabled;
    info[3] = c->own_stream ? 1 : 0;
    return BFS_OK;
}

int bfs_precond_apply(bfs_ctx *c, const double *r, double *z, void *stream)
{
    if (!c || !r || !z) return set_err(c, BFS_EINVAL, "NULL argument");
    if (r == z) {
        int rc = bfs::precond_apply(c, r, c->d_Fp, (cudaStream_t)stream);
        if (rc) return rc;
        BFS_CUDA_TRY(c, cudaMemcpyAsync(z, c->d_Fp, sizeof(double) * c->n, cudaMemcpyDeviceToDevice,
                                        (cudaStream_t)stream));
        return BFS_OK;
    }
    return bfs::precond_apply(c, r, z, (cudaStream_t)stream);
}

int bfs_solve(bfs_ctx *c, double *u, bfs_stats *st, void *stream)
{
    if (!c || !u) return set_err(c, BFS_EINVAL, "NULL argument");
    int rc = bfs::solve_device(c, u, st, (cudaStream_t)stream);
    if (rc && c->err.empty()) {
        const char *m = rc == BFS_ENOCONV ? "Newton iteration limit reached"
                        : rc == BFS_ELINESEARCH ? "line search failed"
                        : rc == BFS_ENAN ? "non-finite residual"
                        : rc == BFS_ETIMEOUT ? "time budget exhausted"
                        : rc == BFS_EBREAKDOWN ? "GMRES breakdown" : "solve failed";
        c->err = m;
    }
    return rc;
}

int bfs_solve_host(bfs_ctx *c, double *u_host, bfs_stats *st, void *stream)
{
    if (!c || !u_host) return set_err(c, BFS_EINVAL, "NULL argument");
    cudaStream_t s = (cudaStream_t)stream;
    int rc = bfs::alloc_solver(c);
    if (rc) return rc;
    double *u = c->d_uio;  // the context's own device copy of the iterate
    cudaError_t e = cudaMemcpyAsync(u, u_host, sizeof(double) * c->n, cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) rc = bfs_solve(c, u, st, stream);
    else rc = set_err(c, BFS_ECUDA, "upload of u failed");
    if (cudaMemcpyAsync(u_host, u, sizeof(double) * c->n, cudaMemcpyDeviceToHost, s) != cudaSuccess ||
        cudaStreamSynchronize(s) != cudaSuccess)
        rc = rc ? rc : set_err(c, BFS_ECUDA, "download of u failed");
    return rc;
}

int bfs_residual_host(bfs_ctx *c, const double *u_host, double *F_host, int precision, void *stream)
{
    if (!c || !u_host || !F_host) return set_err(c, BFS_EINVAL, "NULL argument");
    cudaStream_t s = (cudaStream_t)stream;
    double *u = c->d_up, *F = c->d_Fp;  // context scratch, unused outside bfs_jvp
    BFS_CUDA_TRY(c, cudaMemcpyAsync(u, u_host, sizeof(double) * c->n, cudaMemcpyHostToDevice, s));
    int rc = bfs_residual(c, u, F, precision, stream);
    if (rc) return rc;
    BFS_CUDA_TRY(c, cudaMemcpyAsync(F_host, F, sizeof(double) * c->n, cudaMemcpyDeviceToHost, s));
    BFS_CUDA_TRY(c, cudaStreamSynchronize(s));
    return BFS_OK;
}

int bfs_flat_guess(bfs_ctx *c, double *u, void *stream)
{
    if (!c || !u) return set_err(c, BFS_EINVAL, "NULL argument");
    k_flat_guess<<<(c->n + 255) / 256, 256, 0, (cudaStream_t)stream>>>(u, c->N, c->M, c->x1);
    c->launches++;
    BFS_CUDA_TRY(c, cudaGetLastError());
    return BFS_OK;
}

int bfs_unpack(bfs_ctx *c, const double *u, double *out, void *stream)
{
    if (!c || !u || !out) return set_err(c, BFS_EINVAL, "NULL argument");
    cudaStream_t s = (cudaStream_t)stream;
    int rc = bfs::unpack_launch(c, u, s);
    if (rc) return rc;
    BFS_CUDA_TRY(c, cudaMemcpyAsync(out, c->d_nodal, sizeof(double) * 8 * (size_t)c->NM,
                                    cudaMemcpyDeviceToDevice, s));
    return BFS_OK;
}

int bfs_profile_enable(bfs_ctx *c, int on)
{
    if (!c) return BFS_EINVAL;
    c->prof_on = on ? 1 : 0;
    c->ev_used = 0;
    c->ev_kind.clear();
    return BFS_OK;
}

int bfs_profile_read(bfs_ctx *c, double *out8, unsigned long long *launches)
{
    if (!c) return BFS_EINVAL;
    if (launches) *launches = c->launches;
    if (!out8) return BFS_OK;
    for (int i = 0; i < 8; i++) out8[i] = 0.0;
    for (size_t i = 0; i < c->ev_kind.size(); i++) {
        float ms = 0.0f;
        BFS_CUDA_TRY(c, cudaEventSynchronize(c->ev_pool[2 * i + 1]));
        BFS_CUDA_TRY(c, cudaEventElapsedTime(&ms, c->ev_pool[2 * i], c->ev_pool[2 * i + 1]));
        int k = c->ev_kind[i];
        out8[2 * k] += ms;
        out8[2 * k + 1] += 1.0;
    }
    c->ev_used = 0;
    c->ev_kind.clear();
    return BFS_OK;
}

}  // extern "C"
