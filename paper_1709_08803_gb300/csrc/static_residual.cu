// bfs_residual_static: the nonlinear residual without any device allocation.
//
// Some callers cannot allocate device memory at the point where they need a
// residual: code that runs inside a host callback or another library's
// allocation-free region, code under a memory pool that must not grow, or
// callers that never create a bfs_ctx at all.  This entry point computes the
// same F(u) as bfs_residual, with the same kernels, but keeps every piece of
// scratch (nodal fields, source and target records, split partial sums, the
// bottom-only constant and the NaN flag) in one file-scope device array,
// g_static_scratch, of BFS_STATIC_SCRATCH_BYTES bytes.  Every GPU that loads
// the library holds that array until the process exits.
//
// The residual is the one of a context with the default options: no surface
// tension and no applied surface pressure.
//
// In host code the name g_static_scratch is only a host-side stand-in for
// the symbol, not a device address; its device address is looked up once per
// device (cudaGetSymbolAddress, with that device current) on the first call
// on that device, and cached.  That first call should therefore come before
// any stream capture.  The cached address belongs to the device's current
// primary context: after a cudaDeviceReset of that device it is stale, so the
// entry point must not be used across a reset.  All calls share the one array: calls whose work
// overlaps on the GPU (different streams, no ordering between them) race on
// it and give wrong results.  Calls in one stream are ordered and safe.
#include <math.h>
#include <string.h>

#include <mutex>
#include <string>

#include "bfs_internal.cuh"

#define BFS_STATIC_SCRATCH_BYTES (48u << 20)  // 48 MiB

static __device__ __align__(256) unsigned char g_static_scratch[BFS_STATIC_SCRATCH_BYTES];

namespace {
constexpr int MAX_DEVICES = 64;
std::mutex g_mu;
unsigned char *g_addr[MAX_DEVICES];
thread_local std::string g_static_err;

int fail(int code, const std::string &m)
{
    g_static_err = m;
    return code;
}

size_t align256(size_t b) { return (b + 255) & ~size_t(255); }
}  // namespace

extern "C" const char *bfs_static_last_error(void) { return g_static_err.c_str(); }

extern "C" size_t bfs_static_scratch_bytes(void) { return BFS_STATIC_SCRATCH_BYTES; }

extern "C" int bfs_residual_static(const bfs_mesh *mesh, const double *beta, const double *beta_x,
                                   const double *beta_y, double F, double n_rad, double sign_I4,
                                   const double *u, double *Fu, int precision, void *stream)
{
    if (!mesh || !beta || !beta_x || !beta_y || !u || !Fu)
        return fail(BFS_EINVAL, "NULL argument");
    const int N = mesh->N, M = mesh->M;
    if (N < 4 || M < 3) return fail(BFS_EINVAL, "need N >= 4 and M >= 3");
    // before any int arithmetic on the sizes: the same node limit as bfs_setup
    if ((size_t)N * (size_t)M > ((size_t)1 << 26)) return fail(BFS_EINVAL, "mesh too large");
    if (!(mesh->dx > 0.0) || !(mesh->dy > 0.0) || !isfinite(mesh->dx) || !isfinite(mesh->dy) ||
        !isfinite(mesh->x1) || !isfinite(mesh->y1))
        return fail(BFS_EINVAL, "dx and dy must be positive and finite, x1 and y1 finite");
    if (!(F > 0.0) || !isfinite(F)) return fail(BFS_EINVAL, "F must be positive");
    if (!isfinite(n_rad)) return fail(BFS_EINVAL, "n_rad must be finite");
    if (mesh->half_domain && mesh->y1 != 0.0) return fail(BFS_EINVAL, "half_domain requires y1 == 0");
    if (sign_I4 != 1.0 && sign_I4 != -1.0) return fail(BFS_EINVAL, "sign_I4 must be +1 or -1");
    if (precision != BFS_FP64 && precision != BFS_FP32C) return fail(BFS_EINVAL, "bad precision");

    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= MAX_DEVICES)
        return fail(BFS_ECUDA, "no usable current device");

    // A context on the host stack whose device pointers all point into the
    // static array; no device memory is allocated.
    bfs_ctx c{};
    c.N = N; c.M = M; c.half = mesh->half_domain ? 1 : 0;
    c.x1 = mesh->x1; c.y1 = mesh->y1; c.dx = mesh->dx; c.dy = mesh->dy; c.F = F;
    bfs_default_options(&c.opt);
    c.opt.n_rad = n_rad;
    c.opt.sign_I4 = sign_I4;
    c.n = 3 * (N + 1) * M;
    c.Nt = (N - 1) * M;
    c.NM = N * M;
    c.Ns = c.half ? N * (2 * M - 1) : N * M;
    c.device = dev;
    bfs::plans_for(c.Nt, c.Ns, 0, bfs::num_sms(dev), &c.plan64, &c.plan32);
    c.Ns_cap = std::max(c.plan64.splits * c.plan64.per_split, c.plan32.splits * c.plan32.per_split);
    c.part_cap = (size_t)std::max(c.plan64.splits, c.plan32.splits) * bfs::NACC * c.Nt;

    const size_t NM = (size_t)N * M;
    size_t off[9], need = 0;
    const size_t sz[9] = {
        align256(sizeof(double) * 8 * NM),                        // nodal
        align256(sizeof(double) * bfs::REC * (size_t)c.Ns_cap),    // src64
        align256(sizeof(float) * bfs::REC * (size_t)c.Ns_cap),     // src32
        align256(sizeof(double) * bfs::TREC * (size_t)c.Nt),       // tgt64
        align256(sizeof(float) * bfs::TREC * (size_t)c.Nt),        // tgt32
        align256(sizeof(double) * c.part_cap),                     // partial sums
        align256(sizeof(double) * (size_t)c.Nt),                   // bottom-only constant
        align256(sizeof(int)),                                     // NaN flag
        0};
    for (int i = 0; i < 8; i++) { off[i] = need; need += sz[i]; }
    if (need > BFS_STATIC_SCRATCH_BYTES)
        return fail(BFS_EINVAL, "mesh too large for bfs_residual_static: needs " +
                                    std::to_string(need) + " bytes of scratch, the static array holds " +
                                    std::to_string((size_t)BFS_STATIC_SCRATCH_BYTES));

    unsigned char *base;
    {
        std::lock_guard<std::mutex> lk(g_mu);
        if (!g_addr[dev]) {
            void *p = nullptr;
            cudaError_t e = cudaGetSymbolAddress(&p, g_static_scratch);
            if (e != cudaSuccess || !p)
                return fail(BFS_ECUDA, std::string("cudaGetSymbolAddress: ") + cudaGetErrorString(e));
            g_addr[dev] = (unsigned char *)p;
        }
        base = g_addr[dev];
    }
    c.d_nodal = (double *)(base + off[0]);
    c.d_src64 = (double *)(base + off[1]);
    c.d_src32 = (float *)(base + off[2]);
    c.d_tgt64 = (double *)(base + off[3]);
    c.d_tgt32 = (float *)(base + off[4]);
    c.d_part = (double *)(base + off[5]);
    c.d_constB = (double *)(base + off[6]);
    c.d_flag = (int *)(base + off[7]);
    c.d_beta = const_cast<double *>(beta);
    c.d_bx = const_cast<double *>(beta_x);
    c.d_by = const_cast<double *>(beta_y);

    cudaStream_t s = (cudaStream_t)stream;
    // the flag keeps the previous call's value: clear it
    if (cudaMemsetAsync(c.d_flag, 0, sizeof(int), s) != cudaSuccess)
        return fail(BFS_ECUDA, "clearing the NaN flag failed");
    // the bottom-only constant depends on the topography of this call
    int rc = bfs::unpack_launch(&c, u, s);
    if (!rc) rc = bfs::constB_launch(&c, s);
    if (!rc) rc = bfs::residual_launch(&c, u, Fu, precision, s);
    if (rc) return fail(rc, c.err);
    return BFS_OK;
}
