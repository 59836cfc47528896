// Jacobian-free Newton-Krylov driver (Buttle et al., arXiv:1709.08803, Sec. 3.2):
// damped Newton u <- u + mu du with a backtracking line search, du from
// right-preconditioned restarted GMRES (Saad & Schultz) on J P^-1, and
// J P^-1 v approximated by the forward difference (F(u + h P^-1 v) - F(u)) / h.
//
// Every vector operation runs on the device in FP64: Arnoldi with classical
// Gram-Schmidt applied twice, Givens rotations, the triangular solve and the
// update.  The host only reads one scalar per Arnoldi step (the GMRES residual
// estimate) and one per line-search trial.
#include <math.h>
#include <chrono>

#include "bfs_internal.cuh"

namespace bfs {

constexpr int RED_BLOCKS = 256;
constexpr int RED_TPB = 256;

__device__ __forceinline__ double warp_sum(double v)
{
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    return v;
}

__device__ __forceinline__ double warp_max(double v)
{
    for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_down_sync(0xffffffffu, v, o));
    return v;
}

// partial[j * RED_BLOCKS + b] = sum over block b's slice of V_j . w   (grid: RED_BLOCKS x cnt)
__global__ void k_dots(const double *__restrict__ V, size_t ldv, const double *__restrict__ w,
                       int n, double *__restrict__ partial)
{
    __shared__ double sh[RED_TPB / 32];
    const int j = blockIdx.y;
    const double *v = V + (size_t)j * ldv;
    double acc = 0.0;
    for (int i = blockIdx.x * RED_TPB + threadIdx.x; i < n; i += RED_BLOCKS * RED_TPB)
        acc = fma(v[i], w[i], acc);
    acc = warp_sum(acc);
    if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = acc;
    __syncthreads();
    if (threadIdx.x < 32) {
        double t = threadIdx.x < RED_TPB / 32 ? sh[threadIdx.x] : 0.0;
        t = warp_sum(t);
        if (threadIdx.x == 0) partial[(size_t)j * RED_BLOCKS + blockIdx.x] = t;
    }
}

// out[j] = sum_b partial[j * RED_BLOCKS + b]   (one block per j, fixed order)
__global__ void k_dots_final(const double *__restrict__ partial, double *__restrict__ out)
{
    __shared__ double sh[RED_BLOCKS / 32];
    const int j = blockIdx.x;
    double t = partial[(size_t)j * RED_BLOCKS + threadIdx.x];
    t = warp_sum(t);
    if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = t;
    __syncthreads();
    if (threadIdx.x < 32) {
        double q = threadIdx.x < RED_BLOCKS / 32 ? sh[threadIdx.x] : 0.0;
        q = warp_sum(q);
        if (threadIdx.x == 0) out[j] = q;
    }
}

// out2 = |v|_2^2 partials (slot 0) and |v|_inf partials (slot 1)
__global__ void k_norms(const double *__restrict__ v, int n, double *__restrict__ partial)
{
    __shared__ double s2[RED_TPB / 32], si[RED_TPB / 32];
    double a = 0.0, m = 0.0;
    for (int i = blockIdx.x * RED_TPB + threadIdx.x; i < n; i += RED_BLOCKS * RED_TPB) {
        double x = v[i];
        a = fma(x, x, a);
        m = fmax(m, fabs(x));
        if (x != x) m = x;  // propagate NaN
    }
    a = warp_sum(a);
    m = warp_max(m);
    if ((threadIdx.x & 31) == 0) { s2[threadIdx.x >> 5] = a; si[threadIdx.x >> 5] = m; }
    __syncthreads();
    if (threadIdx.x < 32) {
        double p = threadIdx.x < RED_TPB / 32 ? s2[threadIdx.x] : 0.0;
        double q = threadIdx.x < RED_TPB / 32 ? si[threadIdx.x] : 0.0;
        p = warp_sum(p);
        q = warp_max(q);
        if (threadIdx.x == 0) { partial[blockIdx.x] = p; partial[RED_BLOCKS + blockIdx.x] = q; }
    }
}

__global__ void k_norms_final(const double *__restrict__ partial, double *out2, double *outinf)
{
    __shared__ double s2[RED_BLOCKS / 32], si[RED_BLOCKS / 32];
    double p = partial[threadIdx.x], q = partial[RED_BLOCKS + threadIdx.x];
    p = warp_sum(p);
    q = warp_max(q);
    if ((threadIdx.x & 31) == 0) { s2[threadIdx.x >> 5] = p; si[threadIdx.x >> 5] = q; }
    __syncthreads();
    if (threadIdx.x < 32) {
        p = threadIdx.x < RED_BLOCKS / 32 ? s2[threadIdx.x] : 0.0;
        q = threadIdx.x < RED_BLOCKS / 32 ? si[threadIdx.x] : 0.0;
        p = warp_sum(p);
        q = warp_max(q);
        if (threadIdx.x == 0) {
            if (out2) *out2 = sqrt(p);
            if (outinf) *outinf = q;
        }
    }
}

void norms_launch(bfs_ctx *c, const double *v, int n, double *d_out2, double *d_outinf,
                  cudaStream_t s)
{
    k_norms<<<RED_BLOCKS, RED_TPB, 0, s>>>(v, n, c->d_red);
    c->launches++;
    k_norms_final<<<1, RED_BLOCKS, 0, s>>>(c->d_red, d_out2, d_outinf);
    c->launches++;
}

// y = a x + b z, with a and/or b read from device scalars when the pointer is given
__global__ void k_axpby(double *y, const double *x,
                        const double *z, int n, double a, double b,
                        const double *__restrict__ dscale_b)
{
    double bb = dscale_b ? b * *dscale_b : b;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x)
        y[i] = a * x[i] + bb * z[i];
}

// h = h_rel (1 + |u|) / |z| into sc[4]; 1/h into sc[5]; sc[6] = 1 when z == 0.
__global__ void k_jv_step(double *sc, double h_fixed, double h_rel)
{
    double nu = sc[0], nz = sc[1];
    double h = h_fixed > 0.0 ? h_fixed : (nz > 0.0 ? h_rel * (1.0 + nu) / nz : 0.0);
    sc[4] = h;
    sc[5] = h > 0.0 ? 1.0 / h : 0.0;
    sc[6] = (nz > 0.0) ? 0.0 : 1.0;
}

// Jz = (Fp - Fu) / h
__global__ void k_jv_diff(double *__restrict__ Jz, const double *__restrict__ Fp,
                          const double *__restrict__ Fu, int n, const double *__restrict__ sc)
{
    double ih = sc[5];
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x)
        Jz[i] = (Fp[i] - Fu[i]) * ih;
}

static int grid_for(int n) { return (n + 255) / 256 < 1184 ? (n + 255) / 256 : 1184; }

void solver_axpby(bfs_ctx *c, double *y, const double *x, const double *z, double a, double b,
                  cudaStream_t s)
{
    k_axpby<<<grid_for(c->n), 256, 0, s>>>(y, x, z, c->n, a, b, nullptr);
    c->launches++;
}

// First half of a Jacobian-vector product: h from |u| and |z| on the device,
// u + h z into the context's perturbed-point buffer d_up.
int jv_prep(bfs_ctx *c, const double *u, const double *z, double h, int precision, cudaStream_t s,
            bool unorm_ready)
{
    const int n = c->n;
    double h_rel = c->opt.jv_h_rel;
    if (!(h_rel > 0.0)) h_rel = precision == BFS_FP32C ? 3.4526698e-4 : 1.4901161193847656e-8;
    if (!(h > 0.0)) {
        if (!unorm_ready) norms_launch(c, u, n, c->d_scal + 0, nullptr, s);
        norms_launch(c, z, n, c->d_scal + 1, nullptr, s);
    }
    k_jv_step<<<1, 1, 0, s>>>(c->d_scal, h, h_rel);
    c->launches++;
    // u + h z (a zero z gives h = 0 and Jz = 0)
    k_axpby<<<grid_for(n), 256, 0, s>>>(c->d_up, u, z, n, 1.0, 1.0, c->d_scal + 4);
    c->launches++;
    BFS_CUDA_TRY(c, cudaGetLastError());
    return BFS_OK;
}

// Second half, after F(u + h z) is in d_Fp: Jz = (F(u + h z) - Fu) / h.
int jv_post(bfs_ctx *c, const double *Fu, double *Jz, cudaStream_t s)
{
    k_jv_diff<<<grid_for(c->n), 256, 0, s>>>(Jz, c->d_Fp, Fu, c->n, c->d_scal);
    c->launches++;
    BFS_CUDA_TRY(c, cudaGetLastError());
    return BFS_OK;
}

int jvp_launch(bfs_ctx *c, const double *u, const double *Fu, const double *z, double *Jz,
               double h, int precision, cudaStream_t s, bool unorm_ready)
{
    int rc = jv_prep(c, u, z, h, precision, s, unorm_ready);
    if (!rc) rc = residual_launch(c, c->d_up, c->d_Fp, precision, s);
    if (!rc) rc = jv_post(c, Fu, Jz, s);
    return rc;
}

// w -= V[0..cnt) h   (h on the device)
__global__ void k_gemv_sub(double *__restrict__ w, const double *__restrict__ V, size_t ldv,
                           const double *__restrict__ h, int cnt, int n)
{
    __shared__ double hs[128];
    for (int j = threadIdx.x; j < cnt; j += blockDim.x) hs[j] = h[j];
    __syncthreads();
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        double acc = w[i];
        for (int j = 0; j < cnt; j++) acc = fma(-hs[j], V[(size_t)j * ldv + i], acc);
        w[i] = acc;
    }
}

// x = V[0..cnt) y
__global__ void k_gemv(double *__restrict__ x, const double *__restrict__ V, size_t ldv,
                       const double *__restrict__ y, int cnt, int n)
{
    __shared__ double ys[128];
    for (int j = threadIdx.x; j < cnt; j += blockDim.x) ys[j] = y[j];
    __syncthreads();
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        double acc = 0.0;
        for (int j = 0; j < cnt; j++) acc = fma(ys[j], V[(size_t)j * ldv + i], acc);
        x[i] = acc;
    }
}

// V_{j+1} = w / |w| (|w| at *nrm; a zero norm leaves zeros)
__global__ void k_scale_into(double *__restrict__ out, const double *__restrict__ w, int n,
                             const double *__restrict__ nrm)
{
    double s = *nrm > 0.0 ? 1.0 / *nrm : 0.0;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x)
        out[i] = w[i] * s;
}

// Givens step for column j: H(0..j, j) = h + h2, H(j+1, j) = |w|; rotate with
// the stored rotations, form the new one, update g; residual estimate |g_{j+1}|
// goes to res.  Layout of giv: cs[m] sn[m] g[m+1] y[m] h[m+1] h2[m+1].
__device__ void givens_step(double *H, double *giv, int m, int j, double hn, double *res)
{
    double *cs = giv, *sn = giv + m, *g = giv + 2 * m, *h = giv + 4 * m + 1,
           *h2 = giv + 5 * m + 2;
    double *col = H + (size_t)j * (m + 1);
    for (int i = 0; i <= j; i++) col[i] = h[i] + h2[i];
    col[j + 1] = hn;
    for (int i = 0; i < j; i++) {
        double a = col[i], b = col[i + 1];
        col[i] = cs[i] * a + sn[i] * b;
        col[i + 1] = -sn[i] * a + cs[i] * b;
    }
    double a = col[j], b = col[j + 1];
    double d = hypot(a, b);
    cs[j] = d > 0.0 ? a / d : 1.0;
    sn[j] = d > 0.0 ? b / d : 0.0;
    col[j] = d;
    col[j + 1] = 0.0;
    g[j + 1] = -sn[j] * g[j];
    g[j] = cs[j] * g[j];
    *res = fabs(g[j + 1]);
}

__global__ void k_givens(double *H, double *giv, int m, int j, const double *hn, double *res)
{
    givens_step(H, giv, m, j, *hn, res);
}

// ---------------------------------------------------------------------------
// The tail of an Arnoldi step in one cooperative launch: two classical
// Gram-Schmidt passes of w against V[0..cnt) (h, then h2), |w|, v_cnt = w/|w|
// and the Givens step of column cnt-1.  CTA b owns the slice [b chunk,
// (b+1) chunk) of the vectors; each dot product is reduced in a fixed order
// (warp shuffles inside a CTA, then one CTA per dot over the CTA partials),
// so the result does not depend on timing; values other CTAs wrote in this
// launch are read past L1.  Six grid barriers, each a
// bounded spin (about a second) that raises bit 2 of the flag on timeout.
// ---------------------------------------------------------------------------
struct TailBar {
    unsigned int count, gen;
};

__device__ bool tail_sync(TailBar *b, int *flag, unsigned int spin, unsigned int arrivals)
{
    __shared__ int ok;
    __syncthreads();
    if (threadIdx.x == 0) {
        ok = 1;
        volatile unsigned int *vgen = &b->gen;
        const unsigned int g = *vgen;
        __threadfence();
        const unsigned int arrived = atomicAdd(&b->count, 1u);
        if (arrived == arrivals - 1) {
            atomicExch(&b->count, 0u);
            __threadfence();
            atomicAdd(&b->gen, 1u);
        } else {
            unsigned int spins = 0;
            while (*vgen == g) {
                if (++spins > spin) {
                    atomicOr(flag, 2);
                    ok = 0;
                    break;
                }
                __nanosleep(20);
            }
        }
        __threadfence();
    }
    __syncthreads();
    return ok;
}

constexpr int TAIL_TPB = 256;

struct TailArgs {
    const double *V;
    double *w, *Vnext, *H, *giv, *part, *hn, *res;
    int n, cnt, m;
    TailBar *bar;
    int *flag;
    unsigned int spin;
    // when Fp is set, w = (Fp - Fu) / h first (the Jv difference, 1/h in jsc[5])
    const double *Fp, *Fu, *jsc;
};

// One Arnoldi tail over G CTAs (this one: b) that share a.bar.
__device__ void arnoldi_tail(const TailArgs &a, int G, int b)
{
    __shared__ double hs[128];
    __shared__ double red[TAIL_TPB / 32];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int n = a.n, cnt = a.cnt, m = a.m;
    const int chunk = (n + G - 1) / G, e0 = b * chunk, e1 = min(n, e0 + chunk);
    if (a.Fp) {
        const double ih = a.jsc[5];
        for (int e = e0 + tid; e < e1; e += TAIL_TPB) a.w[e] = (a.Fp[e] - a.Fu[e]) * ih;
        __syncthreads();
    }
    double *h = a.giv + 4 * m + 1, *h2 = a.giv + 5 * m + 2;
    auto block_sum = [&](double v) {  // every thread gets the CTA total
        v = warp_sum(v);
        __syncthreads();
        if (lane == 0) red[warp] = v;
        __syncthreads();
        double t = tid < TAIL_TPB / 32 ? red[tid] : 0.0;
        if (warp == 0) t = warp_sum(t);
        if (tid == 0) red[0] = t;
        __syncthreads();
        return red[0];
    };
    for (int pass = 0; pass < 2; pass++) {
        double *hp = pass ? h2 : h;
        // partial dots of this CTA's slice, one warp per dot
        for (int i = warp; i < cnt; i += TAIL_TPB / 32) {
            const double *vi = a.V + (size_t)i * n;
            double acc = 0.0;
            for (int e = e0 + lane; e < e1; e += 32) acc = fma(vi[e], a.w[e], acc);
            acc = warp_sum(acc);
            if (lane == 0) a.part[(size_t)i * G + b] = acc;
        }
        if (!tail_sync(a.bar, a.flag, a.spin, (unsigned int)G)) return;
        // dot i reduced by CTA i (fixed order over the CTA partials)
        for (int i = b; i < cnt; i += G) {
            double v = 0.0;
            for (int q = tid; q < G; q += TAIL_TPB) v += __ldcg(a.part + (size_t)i * G + q);
            v = block_sum(v);
            if (tid == 0) hp[i] = v;
        }
        if (!tail_sync(a.bar, a.flag, a.spin, (unsigned int)G)) return;
        for (int i = tid; i < cnt; i += TAIL_TPB) hs[i] = __ldcg(hp + i);
        __syncthreads();
        for (int e = e0 + tid; e < e1; e += TAIL_TPB) {
            double acc = a.w[e];
            for (int i = 0; i < cnt; i++) acc = fma(-hs[i], a.V[(size_t)i * n + e], acc);
            a.w[e] = acc;
        }
        __syncthreads();  // the next pass reads w with a different thread mapping
    }
    // |w|
    double s2 = 0.0;
    for (int e = e0 + tid; e < e1; e += TAIL_TPB) s2 = fma(a.w[e], a.w[e], s2);
    s2 = block_sum(s2);
    if (tid == 0) a.part[b] = s2;
    if (!tail_sync(a.bar, a.flag, a.spin, (unsigned int)G)) return;
    if (b == 0) {
        double v = 0.0;
        for (int q = tid; q < G; q += TAIL_TPB) v += __ldcg(a.part + q);
        v = block_sum(v);
        if (tid == 0) *a.hn = sqrt(v);
    }
    if (!tail_sync(a.bar, a.flag, a.spin, (unsigned int)G)) return;
    const double hn = __ldcg(a.hn);
    const double sc = hn > 0.0 ? 1.0 / hn : 0.0;
    for (int e = e0 + tid; e < e1; e += TAIL_TPB) a.Vnext[e] = a.w[e] * sc;
    if (b == 0 && tid == 0) givens_step(a.H, a.giv, m, cnt - 1, hn, a.res);
}

__global__ void __launch_bounds__(TAIL_TPB) k_arnoldi_tail(TailArgs a)
{
    arnoldi_tail(a, gridDim.x, blockIdx.x);
}

// The tails of several instances in one cooperative launch: CTAs
// start[q] .. start[q+1]-1 run instance q's tail on its own barrier.
struct MtailSet {
    TailArgs a[GM_BMAX];
    int start[GM_BMAX + 1];
    int cnt;
};

__global__ void __launch_bounds__(TAIL_TPB) k_marnoldi_tail(const __grid_constant__ MtailSet s)
{
    int q = 0;
    while (q + 1 < s.cnt && (int)blockIdx.x >= s.start[q + 1]) q++;
    arnoldi_tail(s.a[q], s.start[q + 1] - s.start[q], (int)blockIdx.x - s.start[q]);
}

// g = (beta, 0, ..., 0) and V_0 scale factor
__global__ void k_gmres_init(double *giv, int m, const double *beta)
{
    double *g = giv + 2 * m;
    for (int i = 0; i <= m; i++) g[i] = 0.0;
    g[0] = *beta;
}

// Back substitution H(0..k,0..k) y = g(0..k) into y
__global__ void k_trisolve(const double *H, double *giv, int m, int k)
{
    double *g = giv + 2 * m, *y = giv + 3 * m + 1;
    for (int i = k - 1; i >= 0; i--) {
        double s = g[i];
        for (int q = i + 1; q < k; q++) s -= H[(size_t)q * (m + 1) + i] * y[q];
        y[i] = s / H[(size_t)i * (m + 1) + i];
    }
}

int alloc_solver(bfs_ctx *c)
{
    if (c->d_V) return BFS_OK;
    const int m = c->opt.gmres_restart, n = c->n;
    c->m_alloc = m;
    BFS_CUDA_TRY(c, cudaMalloc(&c->d_V, sizeof(double) * (size_t)(m + 1) * n));
    BFS_CUDA_TRY(c, cudaMalloc(&c->d_H, sizeof(double) * (size_t)(m + 1) * m));
    BFS_CUDA_TRY(c, cudaMalloc(&c->d_giv, sizeof(double) * (size_t)(6 * m + 4)));
    BFS_CUDA_TRY(c, cudaMalloc(&c->d_sbase, sizeof(double) * (size_t)8 * n));
    double *b = c->d_sbase;
    c->d_F = b; c->d_du = b + n; c->d_ut = b + 2 * (size_t)n; c->d_Ft = b + 3 * (size_t)n;
    c->d_z = b + 4 * (size_t)n; c->d_w = b + 5 * (size_t)n; c->d_F32 = b + 6 * (size_t)n;
    c->d_uio = b + 7 * (size_t)n;
    BFS_CUDA_TRY(c, cudaMallocHost(&c->h_pin, sizeof(double) * 16));
    // the fused Arnoldi tail: one CTA per SM (its partials, one per CTA and
    // dot, fit the reduction scratch of 32768 doubles for up to 128 dots)
    BFS_CUDA_TRY(c, cudaMalloc(&c->d_tailbar, 2 * sizeof(unsigned int)));
    BFS_CUDA_TRY(c, cudaMemset(c->d_tailbar, 0, 2 * sizeof(unsigned int)));
    {
        int per_sm = 0;
        const int G = num_sms(c->device);
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_arnoldi_tail, TAIL_TPB, 0) == cudaSuccess &&
            per_sm >= 1 && (size_t)G * 129 <= 128 * 256)
            c->tail_grid = G;
        else
            cudaGetLastError();
    }
    return BFS_OK;
}

static int read_scalars(bfs_ctx *c, const double *d, int cnt, cudaStream_t s)
{
    BFS_CUDA_TRY(c, cudaMemcpyAsync(c->h_pin, d, sizeof(double) * cnt, cudaMemcpyDeviceToHost, s));
    BFS_CUDA_TRY(c, cudaStreamSynchronize(s));
    return BFS_OK;
}

// CGS2 orthogonalisation of w against V[0..cnt); h + h2 in giv; |w| in d_scal[8]
static void arnoldi_orth(bfs_ctx *c, int cnt, cudaStream_t s)
{
    const int m = c->m_alloc, n = c->n;
    double *h = c->d_giv + 4 * m + 1, *h2 = c->d_giv + 5 * m + 2;
    const size_t ldv = (size_t)n;
    for (int pass = 0; pass < 2; pass++) {
        double *hp = pass ? h2 : h;
        k_dots<<<dim3(RED_BLOCKS, cnt), RED_TPB, 0, s>>>(c->d_V, ldv, c->d_w, n, c->d_red);
        c->launches++;
        k_dots_final<<<cnt, RED_BLOCKS, 0, s>>>(c->d_red, hp);
        c->launches++;
        k_gemv_sub<<<grid_for(n), 256, 0, s>>>(c->d_w, c->d_V, ldv, hp, cnt, n);
        c->launches++;
    }
    norms_launch(c, c->d_w, n, c->d_scal + 8, nullptr, s);
}

// Device copy of the host's end-of-cycle test, for step graphs that are
// queued before the previous step's scalars reach the host.  Scalars:
// sc[2] GMRES target, sc[3] iteration limit, sc[7] end-of-cycle flag,
// sc[8] |w|, sc[9] |g_{j+1}|, sc[14] Krylov iterations so far.
__global__ void k_gm_set(double *sc, double target, double maxit)
{
    sc[2] = target;
    sc[3] = maxit;
}

__global__ void k_gm_cycle(double *sc, double its)
{
    sc[7] = 0.0;
    sc[14] = its;
}

// After the Arnoldi step that produced v_{j1}: count it and end the cycle on
// convergence, a non-finite residual, an invariant subspace, a full basis or
// the iteration limit (the tests of gm_arnoldi_host).
__global__ void k_gm_flag(double *sc, int j1, int m)
{
    const double its = sc[14] + 1.0;
    sc[14] = its;
    const double hn = sc[8], res = sc[9];
    const bool stop = !isfinite(res) || res <= sc[2] || hn == 0.0 || j1 >= m || its >= sc[3];
    sc[7] = stop ? 1.0 : 0.0;
}

// Guard of a step graph: its body runs unless the previous step ended the cycle.
__global__ void k_gm_guard(cudaGraphConditionalHandle h, const double *sc)
{
    cudaGraphSetConditional(h, sc[7] != 0.0 ? 0u : 1u);
}

// ---------------------------------------------------------------------------
// GMRES as a sequence of device phases with host decisions between them.  A
// single solve drives one instance; the batched solve drives many in lockstep
// and evaluates their residuals together.  Device scalars: d_scal[8] = |w|
// (or beta at a cycle start), d_scal[9] = |g_{j+1}|.
// ---------------------------------------------------------------------------
void gm_start(bfs_ctx *c, Gm &g, const double *u, const double *F, const double *Fbase,
              double fnorm2, double eta, int maxit, cudaStream_t s)
{
    const int n = c->n;
    g.u = u; g.F = F; g.Fbase = Fbase;
    g.target = eta * fnorm2;
    g.maxit = maxit;
    g.its = 0; g.j = 0; g.res = 0.0; g.state = Gm::BEGIN; g.status = BFS_OK;
    k_gm_set<<<1, 1, 0, s>>>(c->d_scal, g.target, (double)maxit);
    c->launches++;
    cudaMemsetAsync(c->d_du, 0, sizeof(double) * n, s);
    norms_launch(c, u, n, c->d_scal + 0, nullptr, s);  // |u| is fixed during the solve
    k_axpby<<<grid_for(n), 256, 0, s>>>(c->d_w, F, F, n, -1.0, 0.0, nullptr);  // r = -F
    c->launches++;
    norms_launch(c, c->d_w, n, c->d_scal + 8, nullptr, s);
}

// With beta = |r| read: finish, or start a cycle (V_0 = r / beta, g = beta e_1).
void gm_cycle_begin(bfs_ctx *c, Gm &g, double beta, cudaStream_t s)
{
    const int m = c->m_alloc, n = c->n;
    if (!isfinite(beta)) { g.status = BFS_ENAN; g.state = Gm::DONE; return; }
    g.res = beta;  // the true residual of the current iterate
    if (beta <= g.target || g.its >= g.maxit) { g.state = Gm::DONE; return; }
    k_scale_into<<<grid_for(n), 256, 0, s>>>(c->d_V, c->d_w, n, c->d_scal + 8);
    c->launches++;
    k_gmres_init<<<1, 1, 0, s>>>(c->d_giv, m, c->d_scal + 8);
    c->launches++;
    k_gm_cycle<<<1, 1, 0, s>>>(c->d_scal, (double)g.its);
    c->launches++;
    g.j = 0;
    g.state = Gm::ARNOLDI;
}

// Arnoldi step, before the residual: z = P^-1 v_j, then u + h z into d_up.
int gm_arnoldi_sweep(bfs_ctx *c, Gm &g, cudaStream_t s)
{
    int rc = precond_apply(c, c->d_V + (size_t)g.j * c->n, c->d_z, s);
    if (rc) return rc;
    g.precs++;
    return BFS_OK;
}

int gm_arnoldi_pre(bfs_ctx *c, Gm &g, cudaStream_t s)
{
    int rc = gm_arnoldi_sweep(c, g, s);
    if (rc) return rc;
    return jv_prep(c, g.u, c->d_z, 0.0, c->opt.krylov_precision, s, true);
}

// Arnoldi step, after F(u + h z) is in d_Fp: w = J z, CGS2, V_{j+1}, Givens.
int gm_arnoldi_post(bfs_ctx *c, Gm &g, cudaStream_t s)
{
    const int m = c->m_alloc, n = c->n;
    int rc = jv_post(c, g.Fbase, c->d_w, s);
    if (rc) return rc;
    g.jvs++;
    if (c->tail_grid > 0 && g.j + 1 <= 128) {
        TailArgs ta;
        ta.V = c->d_V; ta.w = c->d_w; ta.Vnext = c->d_V + (size_t)(g.j + 1) * n;
        ta.H = c->d_H; ta.giv = c->d_giv; ta.part = c->d_red; ta.hn = c->d_scal + 8; ta.res = c->d_scal + 9;
        ta.n = n; ta.cnt = g.j + 1; ta.m = m;
        ta.bar = reinterpret_cast<TailBar *>(c->d_tailbar);
        ta.flag = c->d_flag;
        ta.spin = c->opt.wait_polls > 0 ? (unsigned int)c->opt.wait_polls : (1u << 24);
        ta.Fp = ta.Fu = ta.jsc = nullptr;
        void *args[] = {&ta};
        BFS_CUDA_TRY(c, cudaLaunchCooperativeKernel((const void *)k_arnoldi_tail, dim3(c->tail_grid),
                                                    dim3(TAIL_TPB), args, 0, s));
        c->launches++;
        return BFS_OK;
    }
    arnoldi_orth(c, g.j + 1, s);
    k_scale_into<<<grid_for(n), 256, 0, s>>>(c->d_V + (size_t)(g.j + 1) * n, c->d_w, n, c->d_scal + 8);
    c->launches++;
    k_givens<<<1, 1, 0, s>>>(c->d_H, c->d_giv, m, g.j, c->d_scal + 8, c->d_scal + 9);
    c->launches++;
    BFS_CUDA_TRY(c, cudaGetLastError());
    return BFS_OK;
}

// ---------------------------------------------------------------------------
// The Arnoldi step of several instances at once (the lockstep batched solve):
// after each instance's sweep, k_mjv_norms + k_mjv_axpy form |z|, h and
// u + h z for all of them (the reductions and arithmetic of norms_launch,
// k_jv_step and k_axpby); after the batched residual, k_marnoldi_tail forms
// Jz, CGS2, v_{j+1} and the Givens step for all, each instance on a CTA group
// of its own, sized to its unknowns.
// ---------------------------------------------------------------------------
struct MjvInst {
    const double *u, *z;
    double *up, *red, *sc;
    int n;
    double h_rel;
};

struct MjvSet {
    MjvInst in[GM_BMAX];
    int cnt;
};

__global__ void __launch_bounds__(RED_TPB) k_mjv_norms(const __grid_constant__ MjvSet s)
{
    __shared__ double s2[RED_TPB / 32];
    const MjvInst &q = s.in[blockIdx.y];
    double a = 0.0;
    for (int i = blockIdx.x * RED_TPB + threadIdx.x; i < q.n; i += RED_BLOCKS * RED_TPB) a = fma(q.z[i], q.z[i], a);
    a = warp_sum(a);
    if ((threadIdx.x & 31) == 0) s2[threadIdx.x >> 5] = a;
    __syncthreads();
    if (threadIdx.x < 32) {
        double p = threadIdx.x < RED_TPB / 32 ? s2[threadIdx.x] : 0.0;
        p = warp_sum(p);
        if (threadIdx.x == 0) q.red[blockIdx.x] = p;
    }
}

__global__ void __launch_bounds__(RED_BLOCKS) k_mjv_axpy(const __grid_constant__ MjvSet s)
{
    __shared__ double s2[RED_BLOCKS / 32];
    __shared__ double hsh;
    const MjvInst &q = s.in[blockIdx.y];
    double p = q.red[threadIdx.x];
    p = warp_sum(p);
    if ((threadIdx.x & 31) == 0) s2[threadIdx.x >> 5] = p;
    __syncthreads();
    if (threadIdx.x < 32) {
        p = threadIdx.x < RED_BLOCKS / 32 ? s2[threadIdx.x] : 0.0;
        p = warp_sum(p);
        if (threadIdx.x == 0) {
            const double nz = sqrt(p), nu = q.sc[0];
            const double h = nz > 0.0 ? q.h_rel * (1.0 + nu) / nz : 0.0;
            hsh = h;
            if (blockIdx.x == 0) {
                q.sc[1] = nz;
                q.sc[4] = h;
                q.sc[5] = h > 0.0 ? 1.0 / h : 0.0;
                q.sc[6] = nz > 0.0 ? 0.0 : 1.0;
            }
        }
    }
    __syncthreads();
    const double a = 1.0, bb = 1.0 * hsh;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < q.n; i += gridDim.x * blockDim.x)
        q.up[i] = a * q.u[i] + bb * q.z[i];
}

int gm_multi_pre(bfs_ctx *const *cs, Gm *const *gs, int cnt, cudaStream_t s)
{
    for (int o = 0; o < cnt; o += GM_BMAX) {
        MjvSet set;
        set.cnt = std::min(GM_BMAX, cnt - o);
        int nmax = 0;
        for (int q = 0; q < set.cnt; q++) {
            bfs_ctx *c = cs[o + q];
            double h_rel = c->opt.jv_h_rel;
            if (!(h_rel > 0.0)) h_rel = c->opt.krylov_precision == BFS_FP32C ? 3.4526698e-4 : 1.4901161193847656e-8;
            set.in[q] = MjvInst{gs[o + q]->u, c->d_z, c->d_up, c->d_red, c->d_scal, c->n, h_rel};
            nmax = std::max(nmax, c->n);
        }
        k_mjv_norms<<<dim3(RED_BLOCKS, set.cnt), RED_TPB, 0, s>>>(set);
        k_mjv_axpy<<<dim3(std::min(grid_for(nmax), 256), set.cnt), RED_BLOCKS, 0, s>>>(set);
        for (int q = 0; q < set.cnt; q++) cs[o + q]->launches += 2;
        BFS_CUDA_TRY(cs[o], cudaGetLastError());
    }
    return BFS_OK;
}

int gm_multi_post(bfs_ctx *const *cs, Gm *const *gs, int cnt, cudaStream_t s)
{
    int per_sm = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_marnoldi_tail, TAIL_TPB, 0) != cudaSuccess) {
        cudaGetLastError();
        per_sm = 0;
    }
    for (int o = 0; o < cnt; o += GM_BMAX) {
        const int k = std::min(GM_BMAX, cnt - o);
        bool multi = per_sm > 0;
        double ntot = 0.0;
        for (int q = 0; q < k; q++) {
            multi = multi && cs[o + q]->tail_grid > 0 && gs[o + q]->j + 1 <= 128;
            ntot += cs[o + q]->n;
        }
        if (!multi) {  // one instance at a time
            for (int q = 0; q < k; q++) {
                int rc = gm_arnoldi_post(cs[o + q], *gs[o + q], s);
                if (rc) return rc;
            }
            continue;
        }
        const int sms = num_sms(cs[o]->device), cap = per_sm * sms;
        const double target = std::min(2.0 * sms, (double)cap - k);
        MtailSet set;
        set.cnt = k;
        set.start[0] = 0;
        for (int q = 0; q < k; q++) {
            bfs_ctx *c = cs[o + q];
            Gm &g = *gs[o + q];
            const int G = std::max(1, (int)(target * c->n / ntot));
            set.start[q + 1] = set.start[q] + G;
            TailArgs &ta = set.a[q];
            ta.V = c->d_V; ta.w = c->d_w; ta.Vnext = c->d_V + (size_t)(g.j + 1) * c->n;
            ta.H = c->d_H; ta.giv = c->d_giv; ta.part = c->d_red; ta.hn = c->d_scal + 8; ta.res = c->d_scal + 9;
            ta.n = c->n; ta.cnt = g.j + 1; ta.m = c->m_alloc;
            ta.bar = reinterpret_cast<TailBar *>(c->d_tailbar);
            ta.flag = c->d_flag;
            ta.spin = c->opt.wait_polls > 0 ? (unsigned int)c->opt.wait_polls : (1u << 24);
            ta.Fp = c->d_Fp; ta.Fu = g.Fbase; ta.jsc = c->d_scal;
            g.jvs++;
            c->launches++;
        }
        if (set.start[k] > cap) {  // cannot happen: target <= cap - k
            cs[o]->err = "multi-instance Arnoldi tail: more CTA groups than can be resident";
            return BFS_ECUDA;
        }
        void *args[] = {&set};
        BFS_CUDA_TRY(cs[o], cudaLaunchCooperativeKernel((const void *)k_marnoldi_tail, dim3(set.start[k]),
                                                        dim3(TAIL_TPB), args, 0, s));
    }
    return BFS_OK;
}

// With (|w|, |g_{j+1}|) read: count the step; end the cycle on convergence,
// an invariant subspace, a full basis or the iteration limit.
void gm_arnoldi_host(bfs_ctx *c, Gm &g, double hn, double res)
{
    g.its++;
    g.j++;
    g.res = res;
    if (!isfinite(res)) { g.status = BFS_ENAN; g.state = Gm::DONE; return; }
    if (res <= g.target || hn == 0.0 || g.j >= c->m_alloc || g.its >= g.maxit) g.state = Gm::CYCLE_END;
}

// End of a cycle: du += P^-1 V y.  Then either done, or a restart needs
// J du (prepared here: u + h du into d_up; the caller evaluates its residual).
int gm_cycle_end(bfs_ctx *c, Gm &g, cudaStream_t s)
{
    const int m = c->m_alloc, n = c->n;
    k_trisolve<<<1, 1, 0, s>>>(c->d_H, c->d_giv, m, g.j);
    c->launches++;
    k_gemv<<<grid_for(n), 256, 0, s>>>(c->d_w, c->d_V, (size_t)n, c->d_giv + 3 * m + 1, g.j, n);
    c->launches++;
    int rc = precond_apply(c, c->d_w, c->d_z, s);
    if (rc) return rc;
    g.precs++;
    k_axpby<<<grid_for(n), 256, 0, s>>>(c->d_du, c->d_du, c->d_z, n, 1.0, 1.0, nullptr);
    c->launches++;
    if (g.res <= g.target || g.its >= g.maxit) {
        g.state = Gm::DONE;
        return BFS_OK;
    }
    g.state = Gm::RESTART;
    return jv_prep(c, g.u, c->d_du, 0.0, c->opt.krylov_precision, s, true);
}

// Restart, after F(u + h du) is in d_Fp: r = -F - J du, |r| into d_scal[8].
int gm_restart_post(bfs_ctx *c, Gm &g, cudaStream_t s)
{
    int rc = jv_post(c, g.Fbase, c->d_w, s);
    if (rc) return rc;
    g.jvs++;
    k_axpby<<<grid_for(c->n), 256, 0, s>>>(c->d_w, g.F, c->d_w, c->n, -1.0, -1.0, nullptr);
    c->launches++;
    norms_launch(c, c->d_w, c->n, c->d_scal + 8, nullptr, s);
    g.state = Gm::BEGIN;
    return BFS_OK;
}

void gm_graphs_clear(bfs_ctx *c)
{
    for (cudaGraphExec_t e : c->gm_exec)
        if (e) cudaGraphExecDestroy(e);
    c->gm_exec.clear();
    c->gm_nlaunch.clear();
    c->gm_nflow.clear();
    c->gm_iscond.clear();
    c->gm_u = nullptr;
}

// The Arnoldi step of Krylov index g.j as a graph (captured on first use):
// P^-1 v_j, u + h z, F(u + h z), J z, CGS2, v_{j+1}, Givens -- about twenty
// kernels launched as one.  Preferred form: the step inside a conditional IF
// node behind a one-thread guard that reads the end-of-cycle flag the
// previous step left (k_gm_flag closes the body), so that a step can be
// queued speculatively and does nothing if the cycle has ended.  Falls back
// to the plain step graph if the conditional form does not instantiate, and
// returns null when graphs are off (profiling, or a capture that failed): the
// caller then launches the kernels one by one.
static int capture_step(bfs_ctx *c, Gm &g, cudaStream_t s)
{
    int rc = gm_arnoldi_pre(c, g, s);
    if (!rc) rc = residual_launch(c, c->d_up, c->d_Fp, c->opt.krylov_precision, s);
    if (!rc) rc = gm_arnoldi_post(c, g, s);
    return rc;
}

static cudaGraphExec_t arnoldi_graph_cond(bfs_ctx *c, Gm &g, cudaStream_t s)
{
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t ex = nullptr;
    bool ok = cudaGraphCreate(&graph, 0) == cudaSuccess;
    cudaGraphConditionalHandle h = 0;
    cudaGraphNode_t guard = nullptr, cond = nullptr;
    double *sc = c->d_scal;
    if (ok) ok = cudaGraphConditionalHandleCreate(&h, graph, 0, 0) == cudaSuccess;
    if (ok) {
        cudaKernelNodeParams kp = {};
        void *kargs[] = {&h, &sc};
        kp.func = (void *)k_gm_guard;
        kp.gridDim = dim3(1);
        kp.blockDim = dim3(1);
        kp.kernelParams = kargs;
        ok = cudaGraphAddKernelNode(&guard, graph, nullptr, 0, &kp) == cudaSuccess;
    }
    cudaGraph_t body = nullptr;
    if (ok) {
        cudaGraphNodeParams cp = {};
        cp.type = cudaGraphNodeTypeConditional;
        cp.conditional.handle = h;
        cp.conditional.type = cudaGraphCondTypeIf;
        cp.conditional.size = 1;
        ok = cudaGraphAddNode(&cond, graph, &guard, nullptr, 1, &cp) == cudaSuccess;
        if (ok) body = cp.conditional.phGraph_out[0];
    }
    if (ok) ok = cudaStreamBeginCaptureToGraph(s, body, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal) ==
                 cudaSuccess;
    if (ok) {
        c->capturing = 1;
        int rc = capture_step(c, g, s);
        if (!rc) {
            k_gm_flag<<<1, 1, 0, s>>>(c->d_scal, g.j + 1, c->m_alloc);
            c->launches++;
        }
        cudaGraph_t out = nullptr;
        const cudaError_t e = cudaStreamEndCapture(s, &out);
        c->capturing = 0;
        ok = !rc && e == cudaSuccess;
    }
    if (ok) ok = cudaGraphInstantiate(&ex, graph, 0) == cudaSuccess;
    if (!ok) {
        if (ex) cudaGraphExecDestroy(ex);
        ex = nullptr;
        c->err.clear();
    }
    if (graph) cudaGraphDestroy(graph);
    cudaGetLastError();
    return ex;
}

static cudaGraphExec_t arnoldi_graph(bfs_ctx *c, Gm &g, cudaStream_t s, size_t &key)
{
    if (c->prof_on || c->gm_disabled || !c->gm_warm) return nullptr;
    if (g.u != c->gm_u) {
        gm_graphs_clear(c);
        c->gm_u = g.u;
    }
    key = 2 * (size_t)g.j + (g.Fbase == c->d_F ? 0 : 1);
    if (key >= c->gm_exec.size()) {
        c->gm_exec.resize(key + 1, nullptr);
        c->gm_nlaunch.resize(key + 1, 0);
        c->gm_nflow.resize(key + 1, 0);
        c->gm_iscond.resize(key + 1, 0);
    }
    if (c->gm_exec[key]) return c->gm_exec[key];
    const unsigned long long l0 = c->launches, f0 = c->flow_count;
    const int p0 = g.precs, j0 = g.jvs;
    cudaGraphExec_t ex = nullptr;
    if (c->gm_cond >= 0) {
        ex = arnoldi_graph_cond(c, g, s);
        c->gm_cond = ex ? 1 : -1;
    }
    const bool iscond = ex != nullptr;
    if (!ex) {
        c->launches = l0;
        c->flow_count = f0;
        g.precs = p0;
        g.jvs = j0;
        if (cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal) != cudaSuccess) {
            cudaGetLastError();
            c->gm_disabled = 1;
            return nullptr;
        }
        c->capturing = 1;
        int rc = capture_step(c, g, s);
        cudaGraph_t graph = nullptr;
        cudaError_t e = cudaStreamEndCapture(s, &graph);
        c->capturing = 0;
        if (!rc && e == cudaSuccess && graph && cudaGraphInstantiate(&ex, graph, 0) == cudaSuccess) {
        } else {
            ex = nullptr;
            c->gm_disabled = 1;  // launch one by one from now on
            c->err.clear();
        }
        if (graph) cudaGraphDestroy(graph);
        cudaGetLastError();
    }
    const unsigned long long nl = c->launches - l0, nf = c->flow_count - f0;
    c->launches = l0;
    c->flow_count = f0;
    g.precs = p0;
    g.jvs = j0;
    if (ex) {
        c->gm_exec[key] = ex;
        c->gm_nlaunch[key] = nl;
        c->gm_nflow[key] = nf;
        c->gm_iscond[key] = iscond ? 1 : 0;
    }
    return ex;
}

// One instance: the phases above with the residual evaluated in between.
// With conditional step graphs the loop keeps one step queued ahead: step j's
// scalars (end-of-cycle flag, |w|, |g_{j+1}|) are copied to pinned memory
// behind an event, step j+1 is launched, and only then does the host wait --
// on the event, not the stream -- so the GPU never idles on the round trip.
// A step queued past the end of a cycle finds the flag set and does nothing.
static int gmres(bfs_ctx *c, Gm &g, cudaStream_t s, double beta_known)
{
    int rc;
    const int kp = c->opt.krylov_precision, m = c->m_alloc;
    // |r| of the first cycle is |F|_2, which the caller already holds bit for
    // bit (the same norm kernel on -F): no round trip for it
    if (beta_known >= 0.0) {
        gm_cycle_begin(c, g, beta_known, s);
    } else {
        if ((rc = read_scalars(c, c->d_scal + 8, 1, s))) return rc;
        gm_cycle_begin(c, g, c->h_pin[0], s);
    }
    int queued = -1;  // Krylov index whose conditional step graph is already in the stream
    size_t qkey = 0;
    while (g.state != Gm::DONE) {
        if (g.state == Gm::ARNOLDI) {
            size_t key = 0;
            cudaGraphExec_t ex = nullptr;
            if (queued == g.j) {
                key = qkey;
                ex = c->gm_exec[key];
            } else {
                ex = arnoldi_graph(c, g, s, key);
                if (ex) {
                    if ((rc = flow_wrap_check(c, s))) return rc;
                    BFS_CUDA_TRY(c, cudaGraphLaunch(ex, s));
                    if (c->gm_iscond[key]) c->launches++;  // the guard
                } else {
                    if ((rc = gm_arnoldi_pre(c, g, s))) return rc;
                    if ((rc = residual_launch(c, c->d_up, c->d_Fp, kp, s))) return rc;
                    if ((rc = gm_arnoldi_post(c, g, s))) return rc;
                    c->gm_warm = 1;
                }
            }
            queued = -1;
            if (ex) {  // the step ran: its guard saw the flag that the previous step left clear
                c->launches += c->gm_nlaunch[key];
                c->flow_count += c->gm_nflow[key];
                g.precs++;
                g.jvs++;
            }
            if (ex && c->gm_iscond[key]) {
                if (!c->gm_ev) BFS_CUDA_TRY(c, cudaEventCreateWithFlags(&c->gm_ev, cudaEventDisableTiming));
                BFS_CUDA_TRY(c, cudaMemcpyAsync(c->h_pin + 4, c->d_scal + 7, 3 * sizeof(double),
                                                cudaMemcpyDeviceToHost, s));
                BFS_CUDA_TRY(c, cudaEventRecord(c->gm_ev, s));
                if (g.j + 1 < m && g.its + 1 < g.maxit) {
                    Gm gn = g;
                    gn.j = g.j + 1;
                    size_t k2 = 0;
                    cudaGraphExec_t ex2 = arnoldi_graph(c, gn, s, k2);
                    if (ex2 && c->gm_iscond[k2]) {
                        if ((rc = flow_wrap_check(c, s))) return rc;
                        BFS_CUDA_TRY(c, cudaGraphLaunch(ex2, s));
                        c->launches++;
                        queued = gn.j;
                        qkey = k2;
                    }
                }
                BFS_CUDA_TRY(c, cudaEventSynchronize(c->gm_ev));
                const bool stop = c->h_pin[4] != 0.0;
                gm_arnoldi_host(c, g, c->h_pin[5], c->h_pin[6]);
                // the device flag decides whether the queued step ran; the tests agree
                if (stop && g.state == Gm::ARNOLDI) g.state = Gm::CYCLE_END;
                if (g.state != Gm::ARNOLDI) queued = -1;
            } else {
                if ((rc = read_scalars(c, c->d_scal + 8, 2, s))) return rc;
                gm_arnoldi_host(c, g, c->h_pin[0], c->h_pin[1]);
            }
        } else if (g.state == Gm::CYCLE_END) {
            if ((rc = gm_cycle_end(c, g, s))) return rc;
        } else if (g.state == Gm::RESTART) {
            if ((rc = residual_launch(c, c->d_up, c->d_Fp, kp, s))) return rc;
            if ((rc = gm_restart_post(c, g, s))) return rc;
            if ((rc = read_scalars(c, c->d_scal + 8, 1, s))) return rc;
            gm_cycle_begin(c, g, c->h_pin[0], s);
        } else {
            break;
        }
    }
    return g.status;
}

static int solve_on(bfs_ctx *c, double *u, bfs_stats *st, cudaStream_t s);

// The legacy default stream cannot be captured into graphs, so a solve handed
// it runs on the context's own non-blocking stream, ordered after the
// caller's earlier work and before its later work by an event each way.
int solve_device(bfs_ctx *c, double *u, bfs_stats *st, cudaStream_t s)
{
    if (s != nullptr && s != cudaStreamLegacy) return solve_on(c, u, st, s);
    if (!c->own_stream) {
        BFS_CUDA_TRY(c, cudaStreamCreateWithFlags(&c->own_stream, cudaStreamNonBlocking));
        BFS_CUDA_TRY(c, cudaEventCreateWithFlags(&c->join_ev, cudaEventDisableTiming));
    }
    BFS_CUDA_TRY(c, cudaEventRecord(c->join_ev, s));
    BFS_CUDA_TRY(c, cudaStreamWaitEvent(c->own_stream, c->join_ev, 0));
    const int rc = solve_on(c, u, st, c->own_stream);
    BFS_CUDA_TRY(c, cudaEventRecord(c->join_ev, c->own_stream));
    BFS_CUDA_TRY(c, cudaStreamWaitEvent(s, c->join_ev, 0));
    return rc;
}

static int solve_on(bfs_ctx *c, double *u, bfs_stats *st, cudaStream_t s)
{
    using clk = std::chrono::steady_clock;
    const auto t0 = clk::now();
    const int n = c->n;
    int rc = alloc_solver(c);
    if (rc) return rc;
    if (!c->pc_ready && (rc = precond_factor(c, c->opt.half_band, s))) return rc;
    bfs_stats S{};
    Gm g{};
    auto finish = [&](int status) {
        S.status = status;
        S.seconds = std::chrono::duration<double>(clk::now() - t0).count();
        S.precond_applies = g.precs;
        if (c->opt.krylov_precision == BFS_FP32C) S.residual_evals_fp32 += g.jvs;
        else S.residual_evals_fp64 += g.jvs;
        if (st) *st = S;
        return status;
    };
    BFS_CUDA_TRY(c, cudaMemsetAsync(c->d_flag, 0, sizeof(int), s));
    // a barrier left half-way, or sweep entries left, by a timed-out launch must not carry over
    BFS_CUDA_TRY(c, cudaMemsetAsync(c->d_tailbar, 0, 2 * sizeof(unsigned int), s));
    if ((rc = flow_reset(c, s))) return finish(rc);
    // arithmetic of the Newton residual and line search: the Krylov one while
    // |F| is large (refine_below > 0), the outer one for the final steps
    const int outer = c->opt.outer_precision;
    int cur = (c->opt.refine_below > 0.0 && c->opt.krylov_precision != outer) ? c->opt.krylov_precision : outer;
    auto count = [&](int prec) {
        if (prec == BFS_FP32C) S.residual_evals_fp32++;
        else S.residual_evals_fp64++;
    };
    if ((rc = residual_launch(c, u, c->d_F, cur, s))) return finish(rc);
    count(cur);
    norms_launch(c, c->d_F, n, c->d_scal + 10, c->d_scal + 11, s);
    if ((rc = read_scalars(c, c->d_scal + 10, 2, s))) return finish(rc);
    double f2 = c->h_pin[0], finf = c->h_pin[1];
    int stalls = 0;
    // forcing terms (Eisenstat-Walker choice 1 when opt.forcing == 1)
    const double eta_min = c->opt.eta;
    double eta_k = c->opt.forcing == 1 ? std::max(eta_min, 0.1) : eta_min;
    double prev_f2 = -1.0, prev_lin = 0.0, last_mu = 0.0;
    for (int k = 0;; k++) {
        if (c->opt.forcing == 1 && prev_f2 > 0.0) {
            const double prev_eta = eta_k;
            double e = fabs(f2 - prev_lin) / prev_f2;
            const double sg = pow(prev_eta, 1.6180339887498949);
            if (sg > 0.1) e = std::max(e, sg);
            eta_k = std::min(0.9, std::max(eta_min, e));
        }
        // switch to the outer arithmetic for the final steps: below refine_below,
        // at the tolerance, or when a full Newton step in the Krylov arithmetic
        // reduced |F|_2 by less than 10 % (its rounding, not the linearisation,
        // then limits progress)
        const bool stagnant = prev_f2 > 0.0 && last_mu == 1.0 && f2 > 0.9 * prev_f2;
        if (cur != outer && isfinite(finf) &&
            (finf <= c->opt.refine_below || finf <= c->opt.tol || stagnant)) {
            if ((rc = residual_launch(c, u, c->d_F, outer, s))) return finish(rc);
            count(outer);
            norms_launch(c, c->d_F, n, c->d_scal + 10, c->d_scal + 11, s);
            if ((rc = read_scalars(c, c->d_scal + 10, 2, s))) return finish(rc);
            f2 = c->h_pin[0];
            finf = c->h_pin[1];
            cur = outer;
        }
        S.fnorm_2 = f2;
        S.fnorm_inf = finf;
        if (!isfinite(f2) || !isfinite(finf)) return finish(BFS_ENAN);
        if (finf <= c->opt.tol) return finish(BFS_OK);
        if (k >= c->opt.max_newton) return finish(BFS_ENOCONV);
        if (c->opt.time_budget_s > 0.0 &&
            std::chrono::duration<double>(clk::now() - t0).count() > c->opt.time_budget_s)
            return finish(BFS_ETIMEOUT);
        // the finite difference must subtract a residual of the same arithmetic
        const double *Fbase = c->d_F;
        if (c->opt.krylov_precision != cur) {
            if ((rc = residual_launch(c, u, c->d_F32, c->opt.krylov_precision, s))) return finish(rc);
            count(c->opt.krylov_precision);
            Fbase = c->d_F32;
        }
        Gm gk{};
        gk.precs = g.precs;
        gk.jvs = g.jvs;
        gm_start(c, gk, u, c->d_F, Fbase, f2, eta_k, c->opt.max_krylov, s);
        rc = gmres(c, gk, s, f2);
        S.krylov_its += gk.its;
        g.precs = gk.precs;
        g.jvs = gk.jvs;
        if (rc) return finish(rc);
        stalls = gk.res > gk.target ? stalls + 1 : 0;
        if (c->opt.stall_newton > 0 && stalls >= c->opt.stall_newton) {
            c->err = "GMRES stalled above its tolerance in consecutive Newton steps";
            return finish(BFS_ENOCONV);
        }
        double mu = 1.0;
        bool ok = false;
        while (mu >= 1e-4) {
            k_axpby<<<grid_for(n), 256, 0, s>>>(c->d_ut, u, c->d_du, n, 1.0, mu, nullptr);
            c->launches++;
            if ((rc = residual_launch(c, c->d_ut, c->d_Ft, cur, s))) return finish(rc);
            count(cur);
            norms_launch(c, c->d_Ft, n, c->d_scal + 12, c->d_scal + 13, s);
            // the sweeps' timeout bit travels with the trial's norms (one round trip)
            int *hflag = reinterpret_cast<int *>(c->h_pin + 3);
            BFS_CUDA_TRY(c, cudaMemcpyAsync(hflag, c->d_flag, sizeof(int), cudaMemcpyDeviceToHost, s));
            if ((rc = read_scalars(c, c->d_scal + 12, 2, s))) return finish(rc);
            if (*hflag & 2) {
                c->err = "a wait in the preconditioner sweeps timed out";
                return finish(BFS_ETIMEOUT);
            }
            if (isfinite(c->h_pin[0]) && c->h_pin[0] <= (1.0 - 1e-4 * mu) * f2) {
                ok = true;
                break;
            }
            mu *= 0.5;
        }
        if (!ok) {
            if (cur == outer) return finish(BFS_ELINESEARCH);
            // no sufficient decrease in the Krylov arithmetic: its rounding is the
            // limit; continue with the outer arithmetic from the same iterate
            if ((rc = residual_launch(c, u, c->d_F, outer, s))) return finish(rc);
            count(outer);
            norms_launch(c, c->d_F, n, c->d_scal + 10, c->d_scal + 11, s);
            if ((rc = read_scalars(c, c->d_scal + 10, 2, s))) return finish(rc);
            f2 = c->h_pin[0];
            finf = c->h_pin[1];
            cur = outer;
            prev_f2 = -1.0;
            continue;
        }
        // |F + J (mu du)| estimated from the GMRES residual of the full step
        last_mu = mu;
        prev_f2 = f2;
        prev_lin = (1.0 - mu) * f2 + mu * gk.res;
        f2 = c->h_pin[0];
        finf = c->h_pin[1];
        BFS_CUDA_TRY(c, cudaMemcpyAsync(u, c->d_ut, sizeof(double) * n, cudaMemcpyDeviceToDevice, s));
        // copy rather than swap: d_F stays the buffer the Arnoldi graphs captured
        BFS_CUDA_TRY(c, cudaMemcpyAsync(c->d_F, c->d_Ft, sizeof(double) * n, cudaMemcpyDeviceToDevice, s));
        S.newton_its = k + 1;
    }
}

}  // namespace bfs
