// Nonlinear residual F(u) of the boundary-integral collocation scheme
// (Buttle et al., arXiv:1709.08803, Sec. 2.2 and 3.1; ordering App. B).
//
// One residual is four launches on the caller's stream:
//   k_unpack   trapezoid reconstruction of nodal zeta, phi, psi from u (Sec. 3.1)
//   k_records  y-derivatives, source records (nodes and, in the half domain,
//              their mirror images) and half-point target records
//   k_pairs    the all-pairs quadrature: every half point of the free surface
//              and of the bottom against every node of both sheets, with the
//              (phi - phi*) / (psi - psi*) and S2 singularity subtractions
//   k_finish   split reduction in FP64, closed-form I2'', the -2 pi (phi*-x*)
//              term, the combined dynamic condition and the radiation rows
#include <math.h>

#include <algorithm>

#include "bfs_internal.cuh"

namespace bfs {

// ---------------------------------------------------------------------------
// Unpack: per slice j and field q, q(x1) followed by q_x at the N nodes; the
// nodal values follow by the trapezoid rule along x (Sec. 3.1).
// ---------------------------------------------------------------------------
__global__ void k_unpack(const double *__restrict__ u, double *__restrict__ nodal, int N, int M,
                         double dx)
{
    // one warp per (field, slice): inclusive shuffle scan of the trapezoid increments
    const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, lane = threadIdx.x & 31;
    if (warp >= 3 * M) return;
    const int f = warp / M, j = warp - f * M;
    const size_t NM = (size_t)N * M;
    const double *s = u + (size_t)f * (N + 1) * M + (size_t)j * (N + 1);
    double *q = nodal + (size_t)(3 * f) * NM + (size_t)j * N;
    double *qx = nodal + (size_t)(3 * f + 1) * NM + (size_t)j * N;
    double carry = s[0];
    for (int i0 = 0; i0 < N; i0 += 32) {
        const int i = i0 + lane;
        const double cur = i < N ? s[1 + i] : 0.0;
        double inc = (i >= 1 && i < N) ? 0.5 * dx * (s[i] + cur) : 0.0;
        for (int o = 1; o < 32; o <<= 1) {
            const double v = __shfl_up_sync(0xffffffffu, inc, o);
            if (lane >= o) inc += v;
        }
        const double val = carry + inc;
        if (i < N) {
            q[i] = val;
            qx[i] = cur;
        }
        carry = __shfl_sync(0xffffffffu, val, 31);
    }
}

// Second-order y-derivative at node (i, j); the half domain mirrors the
// field across y = 0 (derivative 0 on that row).
// (the FP64 pipe of this GPU is slow, so the record kernel multiplies by
// reciprocals computed once on the host: i2dy = 1 / (2 dy))
__device__ __forceinline__ double ydiff(const double *q, int N, int M, int half, double i2dy, int i,
                                        int j)
{
    if (j == 0) {
        if (half) return 0.0;
        return (-3.0 * q[i] + 4.0 * q[i + N] - q[i + 2 * N]) * i2dy;
    }
    if (j == M - 1)
        return (3.0 * q[i + (size_t)N * (M - 1)] - 4.0 * q[i + (size_t)N * (M - 2)] +
                q[i + (size_t)N * (M - 3)]) * i2dy;
    return (q[i + (size_t)N * (j + 1)] - q[i + (size_t)N * (j - 1)]) * i2dy;
}

struct RecArgs {
    int N, M, half, Ns, Ns_cap, Nt;
    int w64, w32;  // which source-record copies to write (a residual reads one)
    double x1, y1, dx, dy, sigma, jc, ry;
    double idx, i2dy;  // 1 / dx, 1 / (2 dy)
};

// Builds source records [0, Ns_cap) and target records [0, Nt) in FP64 and FP32.
__global__ void k_records(double *nodal, const double *__restrict__ beta,
                          const double *__restrict__ bx, const double *__restrict__ by,
                          double *__restrict__ src64, float *__restrict__ src32,
                          double *__restrict__ tgt64, float *__restrict__ tgt32, RecArgs a)
{
    int e = blockIdx.x * blockDim.x + threadIdx.x;
    const int N = a.N, M = a.M;
    const size_t NM = (size_t)N * M;
    const double *z = nodal, *zx = nodal + NM, *ph = nodal + 3 * NM, *phx = nodal + 4 * NM;
    const double *ps = nodal + 6 * NM;
    double r[REC];
    if (e < a.Ns_cap) {
        if (e < a.Ns) {
            int img = e >= (int)NM;
            int i, j;
            if (!img) { i = e % N; j = e / N; }
            else { int q = e - (int)NM; i = q % N; j = 1 + q / N; }
            size_t q = (size_t)j * N + i;
            double zy = ydiff(z, N, M, a.half, a.i2dy, i, j);
            if (!img) {  // the nodal y-derivatives are also an output (bfs_unpack)
                nodal[2 * NM + q] = zy;
                nodal[5 * NM + q] = ydiff(ph, N, M, a.half, a.i2dy, i, j);
            }
            double x = a.x1 + i * a.dx;
            double cx = (i == 0 || i == N - 1) ? 0.5 : 1.0;
            double cy = a.half ? ((j == M - 1) ? 0.5 : 1.0) : ((j == 0 || j == M - 1) ? 0.5 : 1.0);
            double w = a.dx * a.dy * cx * cy;
            double w1 = w * a.idx * a.idx, w2 = w * a.idx;
            double ysg = img ? -1.0 : 1.0;
            double f = ph[q] - x, g = ps[q] - x;
            r[0] = (double)i - 0.5 * (N - 1);
            r[1] = (ysg * j - a.jc) * a.ry;
            r[2] = z[q] * a.idx;
            r[3] = (beta[q] + 1.0) * a.idx;
            r[4] = zx[q];
            r[5] = ysg * zy;
            r[6] = bx[q];
            r[7] = ysg * by[q];
            r[8] = w1 * f;
            r[9] = w2 * zx[q];
            r[10] = w1 * g;
            r[11] = w2 * a.sigma * bx[q];
            r[12] = w1;
            r[13] = w2;
            r[14] = ysg * j - a.jc;  // row coordinate in mesh units (exact)
            r[15] = 0.0;
        } else {  // padding: far away, zero weight
            for (int k = 0; k < REC; k++) r[k] = 0.0;
            r[0] = 1.0e6;
        }
        if (a.w64)
            for (int k = 0; k < REC; k++) src64[(size_t)e * REC + k] = r[k];
        if (a.w32) {  // sources in interleaved pairs for the packed FP32x2 pair kernel
            float *d = src32 + (size_t)(e >> 1) * REC * 2 + (e & 1);
            for (int k = 0; k < REC; k++) d[2 * k] = k == 10 ? -(float)r[k] : (float)r[k];
        }
        return;
    }
    e -= a.Ns_cap;
    if (e >= a.Nt) return;
    int k = e % (N - 1), l = e / (N - 1);
    size_t qa = (size_t)l * N + k, qb = qa + 1;
    double xa = a.x1 + k * a.dx, xb = xa + a.dx;
    double zs = 0.5 * (z[qa] + z[qb]);
    double zxs = 0.5 * (zx[qa] + zx[qb]);
    double zys = 0.5 * (ydiff(z, N, M, a.half, a.i2dy, k, l) + ydiff(z, N, M, a.half, a.i2dy, k + 1, l));
    double pxs = 0.5 * (phx[qa] + phx[qb]);
    double pys = 0.5 * (ydiff(ph, N, M, a.half, a.i2dy, k, l) + ydiff(ph, N, M, a.half, a.i2dy, k + 1, l));
    double fs = 0.5 * ((ph[qa] - xa) + (ph[qb] - xb));
    double gs = 0.5 * ((ps[qa] - xa) + (ps[qb] - xb));
    double bs = 0.5 * (beta[qa] + beta[qb]);
    r[0] = (double)k + 0.5 - 0.5 * (N - 1);
    r[1] = ((double)l - a.jc) * a.ry;
    r[2] = zs * a.idx;
    r[3] = (bs + 1.0) * a.idx;
    r[4] = zxs;
    r[5] = zys;
    r[6] = fs;
    r[7] = gs;
    r[8] = 1.0 + zxs * zxs;
    r[9] = 2.0 * zxs * zys;
    r[10] = 1.0 + zys * zys;
    r[11] = zs * a.idx + a.idx;
    r[12] = (bs + 1.0) * a.idx - a.idx;
    r[13] = pxs;
    r[14] = pys;
    r[15] = (double)l - a.jc;  // row coordinate in mesh units (exact)
    for (int q = 0; q < TREC; q++) {
        tgt64[(size_t)e * TREC + q] = r[q];
        tgt32[(size_t)e * TREC + q] = (float)r[q];
    }
}

// ---------------------------------------------------------------------------
// All-pairs quadrature.
// ---------------------------------------------------------------------------
__device__ __forceinline__ float rsq(float x) { return rsqrtf(x); }
__device__ __forceinline__ double rsq(double x) { return rsqrt(x); }

template <typename R> struct Vec;
template <> struct Vec<float> { typedef float4 T; static constexpr int W = 4; };
template <> struct Vec<double> { typedef double2 T; static constexpr int W = 2; };

// Knuth's two-sum: hi + lo == a + b exactly.
__device__ __forceinline__ void two_sum_acc(float &hi, float &lo, float b)
{
    float s = hi + b;
    float bp = s - hi;
    float err = (hi - (s - bp)) + (b - bp);
    hi = s;
    lo += err;
}

// One tile of the all-pairs sum: targets [tile * TPB * TPT, +TPB * TPT) against
// the sources of split `split`; writes that split's partial sums.
template <typename R, int TPB, int TPT, int CH, bool COMP>
__device__ __forceinline__ void pair_tile(const R *__restrict__ src, int per_split,
                                          const R *__restrict__ tgt, int Nt,
                                          double *__restrict__ part, int tile, int split, R *sh)
{
    typedef typename Vec<R>::T V;
    constexpr int VW = Vec<R>::W;
    const R *sb = src + (size_t)split * per_split * REC;

    R tx[TPT], ty[TPT], tz[TPT], tB[TPT], tf[TPT], tg[TPT];
    R cA[TPT], cB[TPT], cC[TPT], cTB[TPT], cBT[TPT];
    int tid[TPT];
#pragma unroll
    for (int p = 0; p < TPT; p++) {
        int t = tile * TPB * TPT + p * TPB + threadIdx.x;
        tid[p] = t;
        const R *tr = tgt + (size_t)min(t, Nt - 1) * TREC;
        tx[p] = tr[0]; ty[p] = tr[1]; tz[p] = tr[2]; tB[p] = tr[3];
        tf[p] = tr[6]; tg[p] = tr[7]; cA[p] = tr[8]; cB[p] = tr[9]; cC[p] = tr[10];
        cTB[p] = tr[11]; cBT[p] = tr[12];
    }
    R hi[TPT][NACC], lo[TPT][NACC];
#pragma unroll
    for (int p = 0; p < TPT; p++)
#pragma unroll
        for (int q = 0; q < NACC; q++) { hi[p][q] = R(0); lo[p][q] = R(0); }

    for (int c0 = 0; c0 < per_split; c0 += CH) {
        __syncthreads();
        const V *g = reinterpret_cast<const V *>(sb + (size_t)c0 * REC);
        V *sv = reinterpret_cast<V *>(sh);
        for (int e = threadIdx.x; e < CH * REC / VW; e += TPB) sv[e] = g[e];
        __syncthreads();
        R l[TPT][NACC];
#pragma unroll
        for (int p = 0; p < TPT; p++)
#pragma unroll
            for (int q = 0; q < NACC; q++) l[p][q] = R(0);
#pragma unroll 2
        for (int s = 0; s < CH; s++) {
            const R *r = sh + s * REC;
            const R xs = r[0], ys = r[1], zs = r[2], bs = r[3];
            const R zxs = r[4], zys = r[5], bxs = r[6], bys = r[7];
            const R w1f = r[8], w2zx = r[9], w1g = r[10], w2sb = r[11];
            const R w1 = r[12], w2 = r[13];
#pragma unroll
            for (int p = 0; p < TPT; p++) {
                const R sx = xs - tx[p], sy = ys - ty[p];
                const R syy = sy * sy;
                const R rho2 = fma(sx, sx, syy);
                // top target, top source: w (f - f*) K1 + w zeta_x K2, and w S2
                {
                    const R d = zs - tz[p];
                    const R ri = rsq(fma(d, d, rho2));
                    const R ri3 = ri * ri * ri;
                    const R num = fma(-sy, zys, fma(-sx, zxs, d));
                    const R dens = fma(-tf[p], w1, w1f);
                    l[p][0] = fma(dens * num, ri3, l[p][0]);
                    l[p][1] = fma(w2zx, ri, l[p][1]);
                    const R qf = fma(sx, fma(cA[p], sx, cB[p] * sy), cC[p] * syy);
                    l[p][2] = fma(w2, rsq(qf), l[p][2]);
                }
                // top target, bottom source: -w g K1(beta) + w sigma beta_x K2(beta)
                {
                    const R d = bs - cTB[p];
                    const R ri = rsq(fma(d, d, rho2));
                    const R ri3 = ri * ri * ri;
                    const R num = fma(-sy, bys, fma(-sx, bxs, d));
                    l[p][0] = fma(-(w1g * num), ri3, l[p][0]);
                    l[p][1] = fma(w2sb, ri, l[p][1]);
                }
                // bottom target, top source: w f K1 + w zeta_x K2
                {
                    const R d = zs - cBT[p];
                    const R ri = rsq(fma(d, d, rho2));
                    const R ri3 = ri * ri * ri;
                    const R num = fma(-sy, zys, fma(-sx, zxs, d));
                    l[p][3] = fma(w1f * num, ri3, l[p][3]);
                    l[p][4] = fma(w2zx, ri, l[p][4]);
                }
                // bottom target, bottom source: -w (g - g*) K1(beta)
                {
                    const R d = bs - tB[p];
                    const R ri = rsq(fma(d, d, rho2));
                    const R ri3 = ri * ri * ri;
                    const R num = fma(-sy, bys, fma(-sx, bxs, d));
                    const R dens = fma(-tg[p], w1, w1g);
                    l[p][3] = fma(-(dens * num), ri3, l[p][3]);
                }
            }
        }
#pragma unroll
        for (int p = 0; p < TPT; p++)
#pragma unroll
            for (int q = 0; q < NACC; q++) {
                if constexpr (COMP) two_sum_acc(hi[p][q], lo[p][q], l[p][q]);
                else hi[p][q] += l[p][q];
            }
    }
#pragma unroll
    for (int p = 0; p < TPT; p++) {
        if (tid[p] >= Nt) continue;
#pragma unroll
        for (int q = 0; q < NACC; q++)
            part[((size_t)split * NACC + q) * Nt + tid[p]] = (double)hi[p][q] + (double)lo[p][q];
    }
}

// ---------------------------------------------------------------------------
// FP32C all-pairs with the packed FP32x2 arithmetic of sm_100-class GPUs: one
// instruction applies the same operation to two sources, so the 45 FP32
// operations of an index pair take 23 issue slots (the five reciprocal square
// roots stay scalar on the special-function unit); the FMA pipe still spends
// one lane-cycle per operation, and it is the kernel's limit.  The quadratic
// form of S2 is taken as s^2 + t^2 + (zeta_x* s + zeta_y* t)^2 (three
// operations on the shared s^2 + t^2 instead of four).  Sources are staged in
// shared memory as interleaved pairs (value v of sources 2i and 2i+1 side by
// side, one 64-bit word), the target values are broadcast into both halves
// once per tile, and the offsets are taken target minus source so that no
// operand needs a negation; the density w g of the bottom double layer is
// negated while staging for the same reason.  The sums are those of
// pair_tile<float>: each half accumulates its sources over a chunk, the halves
// are added and the chunk total enters the two-sum accumulator.
// ---------------------------------------------------------------------------
struct f2 {
    unsigned long long v;
};
__device__ __forceinline__ f2 f2_pack(float a, float b)
{
    f2 r;
    asm("mov.b64 %0, {%1, %2};" : "=l"(r.v) : "f"(a), "f"(b));
    return r;
}
__device__ __forceinline__ void f2_unpack(f2 x, float &a, float &b)
{
    asm("mov.b64 {%0, %1}, %2;" : "=f"(a), "=f"(b) : "l"(x.v));
}
__device__ __forceinline__ f2 f2_fma(f2 a, f2 b, f2 c)
{
    f2 d;
    asm("fma.rn.ftz.f32x2 %0, %1, %2, %3;" : "=l"(d.v) : "l"(a.v), "l"(b.v), "l"(c.v));
    return d;
}
__device__ __forceinline__ f2 f2_mul(f2 a, f2 b)
{
    f2 d;
    asm("mul.rn.ftz.f32x2 %0, %1, %2;" : "=l"(d.v) : "l"(a.v), "l"(b.v));
    return d;
}
__device__ __forceinline__ f2 f2_sub(f2 a, f2 b)
{
    f2 d;
    asm("sub.rn.ftz.f32x2 %0, %1, %2;" : "=l"(d.v) : "l"(a.v), "l"(b.v));
    return d;
}
__device__ __forceinline__ f2 f2_rsq(f2 x)
{
    float a, b;
    f2_unpack(x, a, b);
    return f2_pack(rsqrtf(a), rsqrtf(b));
}

// Two shared-memory chunk buffers filled by 1-D bulk copies (cp.async.bulk,
// completion counted in bytes on an mbarrier per buffer): the copy of the
// next chunk is in flight while the CTA works on the current one.  `seq`
// counts the chunks this CTA has consumed (persistent CTAs run several tiles),
// which fixes each chunk's buffer and mbarrier phase.  Waits are bounded: on
// timeout bit 2 of *flag is raised, the CTA drains its copy and gives up the
// tile (its partial sums are then not written).
struct ChunkRing {
    float *buf;                     // two buffers of `floats` floats, back to back
    unsigned long long *bar;        // two mbarriers
    unsigned int seq;
    unsigned int floats;
    __device__ __forceinline__ float *at(unsigned int q) const { return buf + (size_t)(q & 1) * floats; }
};

__device__ __forceinline__ unsigned int smem_addr(const void *p)
{
    return (unsigned int)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ void chunk_ring_init(ChunkRing &r)
{
    if (threadIdx.x == 0) {
        for (int i = 0; i < 2; i++)
            asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_addr(&r.bar[i])) : "memory");
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncthreads();
}

__device__ __forceinline__ void chunk_issue(ChunkRing &r, unsigned int q, const float *src, unsigned int bytes)
{
    // thread 0 only; the generic-proxy reads of this buffer happened before a
    // __syncthreads, the fence orders them before the async-proxy writes
    const unsigned int b = smem_addr(&r.bar[q & 1]);
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(b), "r"(bytes) : "memory");
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                     smem_addr(r.at(q))),
                 "l"(src), "r"(bytes), "r"(b)
                 : "memory");
}

__device__ __forceinline__ bool chunk_wait(const ChunkRing &r, unsigned int q)
{
    const unsigned int b = smem_addr(&r.bar[q & 1]), parity = (q >> 1) & 1;
    for (unsigned int i = 0; i < (1u << 22); i++) {
        unsigned int done;
        asm volatile(
            "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}"
            : "=r"(done)
            : "r"(b), "r"(parity)
            : "memory");
        if (done) return true;
    }
    return false;
}

template <int TPB, int TPT, int CH>
__device__ __forceinline__ void pair_tile_x2(const float *__restrict__ src, int per_split,
                                             const float *__restrict__ tgt, int Nt,
                                             double *__restrict__ part, int tile, int split, ChunkRing &ring,
                                             int *flag)
{
    static_assert(CH % 2 == 0, "sources are taken in pairs");
    constexpr unsigned int CHUNK_BYTES = CH * REC * sizeof(float);
    const float *sb = src + (size_t)split * per_split * REC;
    const int nch = per_split / CH;
    // target values broadcast into both halves; -f* for the top double layer
    f2 TX[TPT], TY[TPT], TZ[TPT], TB[TPT], NTF[TPT], TG[TPT], ZX[TPT], ZY[TPT], CTB[TPT], CBT[TPT];
    int tid[TPT];
#pragma unroll
    for (int p = 0; p < TPT; p++) {
        int t = tile * TPB * TPT + p * TPB + threadIdx.x;
        tid[p] = t;
        const float *tr = tgt + (size_t)min(t, Nt - 1) * TREC;
        TX[p] = f2_pack(tr[0], tr[0]); TY[p] = f2_pack(tr[1], tr[1]);
        TZ[p] = f2_pack(tr[2], tr[2]); TB[p] = f2_pack(tr[3], tr[3]);
        NTF[p] = f2_pack(-tr[6], -tr[6]); TG[p] = f2_pack(tr[7], tr[7]);
        ZX[p] = f2_pack(tr[4], tr[4]); ZY[p] = f2_pack(tr[5], tr[5]);
        CTB[p] = f2_pack(tr[11], tr[11]); CBT[p] = f2_pack(tr[12], tr[12]);
    }
    float hi[TPT][NACC], lo[TPT][NACC];
#pragma unroll
    for (int p = 0; p < TPT; p++)
#pragma unroll
        for (int q = 0; q < NACC; q++) { hi[p][q] = 0.f; lo[p][q] = 0.f; }

    const unsigned int q0 = ring.seq;
    if (threadIdx.x == 0) chunk_issue(ring, q0, sb, CHUNK_BYTES);
    for (int c = 0; c < nch; c++) {
        const unsigned int q = q0 + c;
        // the next chunk into the other buffer (read by every thread before the
        // __syncthreads that ended the previous chunk)
        if (threadIdx.x == 0 && c + 1 < nch) chunk_issue(ring, q + 1, sb + (size_t)(c + 1) * CH * REC, CHUNK_BYTES);
        if (!__syncthreads_and(chunk_wait(ring, q))) {
            if (threadIdx.x == 0) {
                atomicOr(flag, 2);
                if (c + 1 < nch) chunk_wait(ring, q + 1);  // drain the copy in flight
            }
            ring.seq = q0 + nch;
            return;
        }
        const f2 *sp2 = reinterpret_cast<const f2 *>(ring.at(q));
        f2 L[TPT][NACC];
#pragma unroll
        for (int p = 0; p < TPT; p++)
#pragma unroll
            for (int qq = 0; qq < NACC; qq++) L[p][qq].v = 0ull;
#pragma unroll 2
        for (int i = 0; i < CH / 2; i++) {
            const f2 *r = sp2 + i * REC;
            const f2 xs = r[0], ys = r[1], zs = r[2], bs = r[3];
            const f2 zxs = r[4], zys = r[5], bxs = r[6], bys = r[7];
            const f2 w1f = r[8], w2zx = r[9], nw1g = r[10], w2sb = r[11];
            const f2 w1 = r[12], w2 = r[13];
#pragma unroll
            for (int p = 0; p < TPT; p++) {
                const f2 sx = f2_sub(TX[p], xs), sy = f2_sub(TY[p], ys);  // target minus source
                const f2 rho2 = f2_fma(sx, sx, f2_mul(sy, sy));
                // top target, top source: w (f - f*) K1 + w zeta_x K2, and w S2
                {
                    const f2 d = f2_sub(zs, TZ[p]);
                    const f2 ri = f2_rsq(f2_fma(d, d, rho2));
                    const f2 ri3 = f2_mul(f2_mul(ri, ri), ri);
                    const f2 num = f2_fma(sy, zys, f2_fma(sx, zxs, d));
                    const f2 dens = f2_fma(NTF[p], w1, w1f);
                    L[p][0] = f2_fma(f2_mul(dens, num), ri3, L[p][0]);
                    L[p][1] = f2_fma(w2zx, ri, L[p][1]);
                    // A s^2 + B s t + C t^2 = s^2 + t^2 + (zeta_x* s + zeta_y* t)^2
                    const f2 mq = f2_fma(ZX[p], sx, f2_mul(ZY[p], sy));
                    L[p][2] = f2_fma(w2, f2_rsq(f2_fma(mq, mq, rho2)), L[p][2]);
                }
                // top target, bottom source: -w g K1(beta) + w sigma beta_x K2(beta)
                {
                    const f2 d = f2_sub(bs, CTB[p]);
                    const f2 ri = f2_rsq(f2_fma(d, d, rho2));
                    const f2 ri3 = f2_mul(f2_mul(ri, ri), ri);
                    const f2 num = f2_fma(sy, bys, f2_fma(sx, bxs, d));
                    L[p][0] = f2_fma(f2_mul(nw1g, num), ri3, L[p][0]);
                    L[p][1] = f2_fma(w2sb, ri, L[p][1]);
                }
                // bottom target, top source: w f K1 + w zeta_x K2
                {
                    const f2 d = f2_sub(zs, CBT[p]);
                    const f2 ri = f2_rsq(f2_fma(d, d, rho2));
                    const f2 ri3 = f2_mul(f2_mul(ri, ri), ri);
                    const f2 num = f2_fma(sy, zys, f2_fma(sx, zxs, d));
                    L[p][3] = f2_fma(f2_mul(w1f, num), ri3, L[p][3]);
                    L[p][4] = f2_fma(w2zx, ri, L[p][4]);
                }
                // bottom target, bottom source: -w (g - g*) K1(beta)
                {
                    const f2 d = f2_sub(bs, TB[p]);
                    const f2 ri = f2_rsq(f2_fma(d, d, rho2));
                    const f2 ri3 = f2_mul(f2_mul(ri, ri), ri);
                    const f2 num = f2_fma(sy, bys, f2_fma(sx, bxs, d));
                    const f2 densn = f2_fma(TG[p], w1, nw1g);  // g* w - w g
                    L[p][3] = f2_fma(f2_mul(densn, num), ri3, L[p][3]);
                }
            }
        }
#pragma unroll
        for (int p = 0; p < TPT; p++)
#pragma unroll
            for (int qq = 0; qq < NACC; qq++) {
                float a, b;
                f2_unpack(L[p][qq], a, b);
                two_sum_acc(hi[p][qq], lo[p][qq], a + b);
            }
        __syncthreads();  // every thread is done with this buffer before it is refilled
    }
    ring.seq = q0 + nch;
    // the split's sums as hi/lo float pairs (8 bytes, like the FP64 partials of the
    // other kernels): k_finish adds them in double-float on the FP32 pipes
    float2 *pf = reinterpret_cast<float2 *>(part);
#pragma unroll
    for (int p = 0; p < TPT; p++) {
        if (tid[p] >= Nt) continue;
#pragma unroll
        for (int q = 0; q < NACC; q++) pf[((size_t)split * NACC + q) * Nt + tid[p]] = make_float2(hi[p][q], lo[p][q]);
    }
}

template <typename R, int TPB, int TPT, int CH, bool COMP>
__global__ void __launch_bounds__(TPB)
k_pairs(const R *__restrict__ src, int per_split, const R *__restrict__ tgt, int Nt,
        double *__restrict__ part, int *flag)
{
    if constexpr (sizeof(R) == 4 && COMP) {
        __shared__ __align__(128) float sh[2 * CH * REC];
        __shared__ __align__(8) unsigned long long bar[2];
        ChunkRing ring{sh, bar, 0u, (unsigned int)(CH * REC)};
        chunk_ring_init(ring);
        pair_tile_x2<TPB, TPT, CH>(src, per_split, tgt, Nt, part, blockIdx.x, blockIdx.y, ring, flag);
    } else {
        __shared__ __align__(16) R sh[CH * REC];
        pair_tile<R, TPB, TPT, CH, COMP>(src, per_split, tgt, Nt, part, blockIdx.x, blockIdx.y, sh);
    }
}

// ---------------------------------------------------------------------------
// Closed-form integral of S2 = (A s^2 + B s t + C t^2)^(-1/2) over a rectangle
// (Sec. 3.1).  The antiderivative printed in the paper is
//   t/sqrt(A) ln(2As + Bt + 2 sqrt(A Q)) + s/sqrt(C) ln(2Ct + Bs + 2 sqrt(C Q));
// where the log argument would cancel (2As + Bt < 0) it is evaluated through
// (2As + Bt + 2 sqrt(AQ)) (2 sqrt(AQ) - 2As - Bt) = (4AC - B^2) t^2 as
// ln((4AC - B^2) t^2 / (2 sqrt(AQ) - 2As - Bt)), and t ln(.) -> 0 at t = 0.
// ---------------------------------------------------------------------------
__device__ double antideriv_S2(double A, double B, double C, double s, double t)
{
    const double Q = A * s * s + B * s * t + C * t * t;
    const double D = 4.0 * A * C - B * B;
    double g = 0.0;
    if (t != 0.0) {
        const double lin = 2.0 * A * s + B * t, r = 2.0 * sqrt(A * Q);
        // lin + r = D t^2 / (r - lin): one logarithm, no cancellation when lin < 0
        const double L = log((lin >= 0.0) ? lin + r : D * t * t / (r - lin));
        g += t * rsqrt(A) * L;
    }
    if (s != 0.0) {
        const double lin = 2.0 * C * t + B * s, r = 2.0 * sqrt(C * Q);
        const double L = log((lin >= 0.0) ? lin + r : D * s * s / (r - lin));
        g += s * rsqrt(C) * L;
    }
    return g;
}

// One of the two logarithmic terms of antideriv_S2 at corner (s, t): which = 0
// the t term, 1 the s term (their sum is antideriv_S2).
__device__ double antideriv_S2_term(double A, double B, double C, double s, double t, int which)
{
    const double Q = A * s * s + B * s * t + C * t * t;
    const double D = 4.0 * A * C - B * B;
    if (which == 0) {
        if (t == 0.0) return 0.0;
        const double lin = 2.0 * A * s + B * t, r = 2.0 * sqrt(A * Q);
        return t * rsqrt(A) * log((lin >= 0.0) ? lin + r : D * t * t / (r - lin));
    }
    if (s == 0.0) return 0.0;
    const double lin = 2.0 * C * t + B * s, r = 2.0 * sqrt(C * Q);
    return s * rsqrt(C) * log((lin >= 0.0) ? lin + r : D * s * s / (r - lin));
}

__device__ double rect_S2(double A, double B, double C, double s1, double s2, double t1, double t2)
{
    return antideriv_S2(A, B, C, s2, t2) - antideriv_S2(A, B, C, s1, t2) -
           antideriv_S2(A, B, C, s2, t1) + antideriv_S2(A, B, C, s1, t1);
}

struct FinArgs {
    int N, M, Nt, splits, half;
    int part_f2;  // the partials are hi/lo float pairs (FP32C pair kernels), not FP64
    double x1, y1, dx, dy, ylo, yhi, xhi, F, n_rad, tau;
    double iF2;  // 1 / F^2 (the FP64 pipe of this GPU is slow: no division per target)
};

// Second y-difference of nodal zeta at node (i, j): central inside,
// second-order one-sided on an outer row (first order when M = 3), mirror
// ghost on y = 0 of the half domain.
__device__ __forceinline__ double zeta_yy(const double *__restrict__ z, int N, int M, int half, double dy, int i,
                                          int j)
{
    const double *c = z + i;
    double v;
    if (j == 0) {
        if (half) v = 2.0 * (c[(size_t)N] - c[0]);
        else if (M >= 4) v = 2.0 * c[0] - 5.0 * c[(size_t)N] + 4.0 * c[2 * (size_t)N] - c[3 * (size_t)N];
        else v = c[0] - 2.0 * c[(size_t)N] + c[2 * (size_t)N];
    } else if (j == M - 1) {
        const double *e = c + (size_t)(M - 1) * N;
        if (M >= 4) v = 2.0 * e[0] - 5.0 * e[-(long)N] + 4.0 * e[-2 * (long)N] - e[-3 * (long)N];
        else v = e[0] - 2.0 * e[-(long)N] + e[-2 * (long)N];
    } else {
        const double *e = c + (size_t)j * N;
        v = e[-(long)N] - 2.0 * e[0] + e[(size_t)N];
    }
    return v / (dy * dy);
}

constexpr int FIN_LANES = 8;  // lanes per target in k_finish: one FP64 logarithm of the closed
                               // form each (4 corners x 2 terms), a short dependent chain per lane

// a + b in double-float: Knuth's two-sum of the high parts, the low parts added,
// renormalised (the explicit _rn operations keep the compiler from contracting)
__device__ __forceinline__ float2 fin_df_add(float2 a, float2 b)
{
    const float t = __fadd_rn(a.x, b.x);
    const float bb = __fsub_rn(t, a.x);
    const float err = __fadd_rn(__fsub_rn(a.x, __fsub_rn(t, bb)), __fsub_rn(b.x, bb));
    const float l = __fadd_rn(err, __fadd_rn(a.y, b.y));
    const float h = __fadd_rn(t, l);
    return make_float2(h, __fsub_rn(l, __fsub_rn(h, t)));
}

// F2 / F7 / F1 at every half point (FIN_LANES lanes per target share the
// split partial sums and take one logarithm each of the closed-form integral),
// radiation rows per slice.
__global__ void k_finish(const double *__restrict__ part, const double *__restrict__ tgt,
                         const double *__restrict__ constB, const double *__restrict__ nodal,
                         const double *__restrict__ psurf, double *__restrict__ Fu,
                         int *__restrict__ flag, FinArgs a)
{
    const double TWO_PI = 6.283185307179586476925286766559;
    const int g = blockIdx.x * blockDim.x + threadIdx.x;
    const int e = g / FIN_LANES, q4 = g % FIN_LANES;
    const int N = a.N, M = a.M;
    const size_t blk = (size_t)(N + 1) * M;
    bool bad = false;
    const bool is_t = e < a.Nt;
    const int et = is_t ? e : 0;
    double acc[NACC];
#pragma unroll
    for (int q = 0; q < NACC; q++) acc[q] = 0.0;
    if (a.part_f2) {
        // hi/lo pairs summed in double-float (Knuth's two-sum on the FP32 pipes; an
        // FP64 addition costs this GPU the pipe time of 64 FP32 ones), lanes joined
        // by an xor tree, then one FP64 rounding
        const float2 *pf = reinterpret_cast<const float2 *>(part);
        float2 d[NACC];
#pragma unroll
        for (int q = 0; q < NACC; q++) d[q] = make_float2(0.f, 0.f);
        if (is_t) {
#pragma unroll 2
            for (int s = q4; s < a.splits; s += FIN_LANES)
#pragma unroll
                for (int q = 0; q < NACC; q++) d[q] = fin_df_add(d[q], pf[((size_t)s * NACC + q) * a.Nt + et]);
        }
#pragma unroll
        for (int o = 1; o < FIN_LANES; o <<= 1)
#pragma unroll
            for (int q = 0; q < NACC; q++) {
                const float2 od = make_float2(__shfl_xor_sync(0xffffffffu, d[q].x, o),
                                              __shfl_xor_sync(0xffffffffu, d[q].y, o));
                d[q] = fin_df_add(d[q], od);
            }
        if (q4 == 0)
#pragma unroll
            for (int q = 0; q < NACC; q++) acc[q] = (double)d[q].x + (double)d[q].y;
    } else if (is_t) {
#pragma unroll 2
        for (int s = q4; s < a.splits; s += FIN_LANES)
#pragma unroll
            for (int q = 0; q < NACC; q++) acc[q] += part[((size_t)s * NACC + q) * a.Nt + et];
    }
    const int k = et % (N - 1), l = et / (N - 1);
    const double *r = tgt + (size_t)et * TREC;
    const double A = r[8], B = r[9], C = r[10];
    const double xs = a.x1 + (k + 0.5) * a.dx, ys = a.y1 + l * a.dy;
    // lane q4: corner q4 >> 1 of the rectangle, (s2,t2) +, (s1,t2) -, (s2,t1) -, (s1,t1) +,
    // and term q4 & 1 of its antiderivative
    const int cq = q4 >> 1;
    const double sc = (cq & 1) ? a.x1 - xs : a.xhi - xs;
    const double tc = (cq & 2) ? a.ylo - ys : a.yhi - ys;
    double g2 = is_t ? antideriv_S2_term(A, B, C, sc, tc, q4 & 1) : 0.0;
    if ((cq == 1) || (cq == 2)) g2 = -g2;
#pragma unroll
    for (int o = 1; o < FIN_LANES; o <<= 1) {
        g2 += __shfl_xor_sync(0xffffffffu, g2, o);
        if (!a.part_f2)
#pragma unroll
            for (int q = 0; q < NACC; q++) acc[q] += __shfl_xor_sync(0xffffffffu, acc[q], o);
    }
    if (is_t && q4 == 0) {
        const double zs = r[2] * a.dx, zxs = r[4], zys = r[5], fs = r[6], gs = r[7];
        const double pxs = r[13], pys = r[14];
        const double F2 = acc[0] + acc[1] - zxs * acc[2] + zxs * g2 - TWO_PI * fs;
        const double F7 = acc[3] + acc[4] + constB[e] - TWO_PI * gs;
        const double num = (1.0 + zxs * zxs) * pys * pys + (1.0 + zys * zys) * pxs * pxs -
                           2.0 * zxs * zys * pxs * pys;
        double F1 = 0.5 * num / (1.0 + zxs * zxs + zys * zys) + zs * a.iF2 - 0.5;
        if (a.tau != 0.0) {  // surface tension: -tau times the mean curvature at the half point
            const size_t NM = (size_t)N * M, qa = (size_t)l * N + k;
            const double zxx = (nodal[NM + qa + 1] - nodal[NM + qa]) / a.dx;
            const double zxy = (nodal[2 * NM + qa + 1] - nodal[2 * NM + qa]) / a.dx;
            const double zyy = 0.5 * (zeta_yy(nodal, N, M, a.half, a.dy, k, l) +
                                      zeta_yy(nodal, N, M, a.half, a.dy, k + 1, l));
            const double w = 1.0 + zxs * zxs + zys * zys;
            F1 -= a.tau * ((1.0 + zys * zys) * zxx - 2.0 * zxs * zys * zxy + (1.0 + zxs * zxs) * zyy) / (w * sqrt(w));
        }
        if (psurf) {  // applied surface pressure at the half point (Sec. 4.1)
            const size_t qa = (size_t)l * N + k;
            F1 += 0.5 * (psurf[qa] + psurf[qa + 1]);
        }
        const size_t row = (size_t)l * (N + 1) + 2 + k;
        Fu[row] = F1;
        Fu[blk + row] = F2;
        Fu[2 * blk + row] = F7;
        bad = !isfinite(F1) || !isfinite(F2) || !isfinite(F7);
    } else if (!is_t && q4 == 0 && e < a.Nt + M) {
        // radiation conditions of Scullen at x1 (Sec. 3.1); second derivatives
        // are forward differences of the first derivatives
        const int lsl = e - a.Nt;
        const size_t NM = (size_t)N * M, qq = (size_t)lsl * N, row = (size_t)lsl * (N + 1);
        const double x1 = a.x1, n = a.n_rad, h = a.dx;
        for (int f = 0; f < 3; f++) {
            const double v1 = nodal[(3 * f) * NM + qq];
            const double d1 = nodal[(3 * f + 1) * NM + qq], d2 = nodal[(3 * f + 1) * NM + qq + 1];
            double Fa, Fb;
            if (f == 0) {
                Fa = x1 * d1 + n * v1;
                Fb = x1 * (d2 - d1) / h + n * d1;
            } else {
                Fa = x1 * (d1 - 1.0) + n * (v1 - x1);
                Fb = x1 * (d2 - d1) / h + n * (d1 - 1.0);
            }
            Fu[f * blk + row] = Fa;
            Fu[f * blk + row + 1] = Fb;
            bad = bad || !isfinite(Fa) || !isfinite(Fb);
        }
    }
    if (bad) atomicOr(flag, 1);
}

// Bottom-only part of the bottom single layer seen from bottom half points:
//   sigma [ sum w beta_x K2(beta; beta*) - beta_x* sum w S2_beta ] + sigma beta_x* I2''_beta
// It depends on the topography alone, so it is evaluated once (FP64).
__global__ void k_constB(const double *__restrict__ src, int Ns, const double *__restrict__ tgt,
                         const double *__restrict__ bx, const double *__restrict__ by,
                         double *__restrict__ out, FinArgs a, double sigma)
{
    int e = blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= a.Nt) return;
    const int N = a.N;
    int k = e % (N - 1), l = e / (N - 1);
    size_t qa = (size_t)l * N + k, qb = qa + 1;
    const double bxs = 0.5 * (bx[qa] + bx[qb]), bys = 0.5 * (by[qa] + by[qb]);
    const double A = 1.0 + bxs * bxs, B = 2.0 * bxs * bys, C = 1.0 + bys * bys;
    const double *t = tgt + (size_t)e * TREC;
    const double tx = t[0], ty = t[1], tb = t[3];
    double sK = 0.0, sS = 0.0;
    for (int s = 0; s < Ns; s++) {
        const double *r = src + (size_t)s * REC;
        const double sx = r[0] - tx, sy = r[1] - ty, d = r[3] - tb;
        sK += r[11] * rsqrt(sx * sx + sy * sy + d * d);
        sS += r[13] * rsqrt(A * sx * sx + B * sx * sy + C * sy * sy);
    }
    const double xs = a.x1 + (k + 0.5) * a.dx, ys = a.y1 + l * a.dy;
    const double I2pp = rect_S2(A, B, C, a.x1 - xs, a.xhi - xs, a.ylo - ys, a.yhi - ys);
    out[e] = sK - sigma * bxs * sS + sigma * bxs * I2pp;
}

// ---------------------------------------------------------------------------
// Host side
// ---------------------------------------------------------------------------
static RecArgs rec_args(const bfs_ctx *c)
{
    RecArgs a;
    a.N = c->N; a.M = c->M; a.half = c->half; a.Ns = c->Ns; a.Ns_cap = c->Ns_cap; a.Nt = c->Nt;
    a.x1 = c->x1; a.y1 = c->y1; a.dx = c->dx; a.dy = c->dy; a.sigma = c->opt.sign_I4;
    a.jc = c->half ? 0.0 : 0.5 * (c->M - 1);
    a.ry = c->dy / c->dx;
    a.idx = 1.0 / c->dx;
    a.i2dy = 1.0 / (2.0 * c->dy);
    a.w64 = a.w32 = 1;
    return a;
}

static FinArgs fin_args(const bfs_ctx *c, int splits, int part_f2 = 0)
{
    FinArgs a;
    a.N = c->N; a.M = c->M; a.Nt = c->Nt; a.splits = splits; a.half = c->half;
    a.part_f2 = part_f2;
    a.tau = c->opt.surface_tension;
    a.x1 = c->x1; a.y1 = c->y1; a.dx = c->dx; a.dy = c->dy;
    a.iF2 = 1.0 / (c->F * c->F);
    a.yhi = c->y1 + (c->M - 1) * c->dy;
    a.ylo = c->half ? -a.yhi : c->y1;
    a.xhi = c->x1 + (c->N - 1) * c->dx;
    a.F = c->F; a.n_rad = c->opt.n_rad;
    return a;
}

// Source splits of a pair-kernel launch: about eight CTAs' worth of (target
// tile, source split) items per SM, small enough that the block scheduler,
// refilling each SM as its CTAs finish, evens out the load.  splits_req > 0
// asks for a split count instead.
PairPlan make_plan(int Nt, int Ns, int tpb, int tpt, int chunk, int splits_req, int sms)
{
    PairPlan p;
    p.tpb = tpb; p.tpt = tpt; p.chunk = chunk;
    p.tiles = (Nt + tpb * tpt - 1) / (tpb * tpt);
    int nchunks = (Ns + chunk - 1) / chunk;
    int want = splits_req > 0 ? splits_req : (sms * 8 + p.tiles - 1) / p.tiles;
    if (want < 1) want = 1;
    if (want > nchunks) want = nchunks;
    int cps = (nchunks + want - 1) / want;
    p.splits = (nchunks + cps - 1) / cps;
    p.per_split = cps * chunk;
    return p;
}

int unpack_launch(bfs_ctx *c, const double *u, cudaStream_t s, int which)
{
    k_unpack<<<(3 * c->M * 32 + 127) / 128, 128, 0, s>>>(u, c->d_nodal, c->N, c->M, c->dx);
    c->launches++;
    RecArgs ra = rec_args(c);
    ra.w64 = which & 1;
    ra.w32 = (which >> 1) & 1;
    int tot = c->Ns_cap + c->Nt;
    k_records<<<(tot + 255) / 256, 256, 0, s>>>(c->d_nodal, c->d_beta, c->d_bx, c->d_by, c->d_src64,
                                                 c->d_src32, c->d_tgt64, c->d_tgt32, ra);
    c->launches++;
    BFS_CUDA_TRY(c, cudaGetLastError());
    return BFS_OK;
}

// Launch configurations of the pair kernels.
constexpr int P64_TPB = 128, P64_TPT = 1, P64_CH = 32;
constexpr int P32_TPB = 128, P32_TPT = 2, P32_CH = 128;

int residual_launch(bfs_ctx *c, const double *u, double *Fu, int precision, cudaStream_t s)
{
    // FP32C pairs read the FP32 source records, FP64 and double-float ones the FP64 records
    int rc = unpack_launch(c, u, s, precision == BFS_FP32C ? 2 : 1);
    if (rc) return rc;
    const PairPlan &p = precision == BFS_FP32C ? c->plan32 : (precision == BFS_DF64 ? c->plandf : c->plan64);
    dim3 grid(p.tiles, p.splits);
    cudaEvent_t ev1 = nullptr;
    if (c->prof_on) {
        cudaEvent_t ev0 = prof_event(c);
        ev1 = prof_event(c);
        c->ev_kind.push_back(precision == BFS_FP32C ? 1 : (precision == BFS_DF64 ? 2 : 0));
        cudaEventRecord(ev0, s);
    }
    if (precision == BFS_DF64) {
        if ((rc = pairs_df_launch(c, s))) return rc;
    } else if (precision == BFS_FP32C)
        k_pairs<float, P32_TPB, P32_TPT, P32_CH, true>
            <<<grid, P32_TPB, 0, s>>>(c->d_src32, p.per_split, c->d_tgt32, c->Nt, c->d_part, c->d_flag);
    else
        k_pairs<double, P64_TPB, P64_TPT, P64_CH, false>
            <<<grid, P64_TPB, 0, s>>>(c->d_src64, p.per_split, c->d_tgt64, c->Nt, c->d_part, c->d_flag);
    if (precision != BFS_DF64) c->launches++;
    if (ev1) cudaEventRecord(ev1, s);
    FinArgs fa = fin_args(c, p.splits, precision == BFS_FP32C);
    int tot = FIN_LANES * (c->Nt + c->M);
    k_finish<<<(tot + 127) / 128, 128, 0, s>>>(c->d_part, c->d_tgt64, c->d_constB, c->d_nodal, c->d_psurf, Fu,
                                               c->d_flag, fa);
    c->launches++;
    BFS_CUDA_TRY(c, cudaGetLastError());
    return BFS_OK;
}

int finish_launch(bfs_ctx *c, double *Fu, int precision, cudaStream_t s)
{
    const PairPlan &p = precision == BFS_FP32C ? c->plan32 : (precision == BFS_DF64 ? c->plandf : c->plan64);
    FinArgs fa = fin_args(c, p.splits, precision == BFS_FP32C);
    int tot = FIN_LANES * (c->Nt + c->M);
    k_finish<<<(tot + 127) / 128, 128, 0, s>>>(c->d_part, c->d_tgt64, c->d_constB, c->d_nodal, c->d_psurf, Fu,
                                               c->d_flag, fa);
    c->launches++;
    BFS_CUDA_TRY(c, cudaGetLastError());
    return BFS_OK;
}

// Persistent multi-instance FP32C pair kernel: CTAs take (instance, target
// tile, source split) items from a queue until it is empty; items of masked
// instances are skipped.
template <int TPB, int TPT>
__global__ void __launch_bounds__(TPB)
k_pairs_batch(const BatchInst *__restrict__ inst, const int4 *__restrict__ items, int n_items,
              unsigned int *__restrict__ counter, const unsigned char *__restrict__ mask)
{
    __shared__ __align__(128) float sh[2 * P32_CH * REC];
    __shared__ __align__(8) unsigned long long bar[2];
    __shared__ int it;
    ChunkRing ring{sh, bar, 0u, (unsigned int)(P32_CH * REC)};
    chunk_ring_init(ring);
    while (true) {
        if (threadIdx.x == 0) it = (int)atomicAdd(counter, 1u);
        __syncthreads();
        const int w = it;
        __syncthreads();
        if (w >= n_items) return;
        const int4 item = items[w];
        if (!mask[item.x]) continue;
        const BatchInst I = inst[item.x];
        pair_tile_x2<TPB, TPT, P32_CH>(I.src, I.per_split, I.tgt, I.Nt, I.part, item.y, item.z, ring, I.flag);
    }
}

const BatchVariant kBatchVariants[] = {{128, 2}, {256, 1}, {64, 2}, {128, 1}, {64, 4}};
const int kNumBatchVariants = 5;

int batch_pairs_occupancy(int v, int *blocks_per_sm)
{
    cudaError_t e = cudaErrorInvalidValue;
    switch (v) {
    case 0: e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks_per_sm, k_pairs_batch<128, 2>, 128, 0); break;
    case 1: e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks_per_sm, k_pairs_batch<256, 1>, 256, 0); break;
    case 2: e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks_per_sm, k_pairs_batch<64, 2>, 64, 0); break;
    case 3: e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks_per_sm, k_pairs_batch<128, 1>, 128, 0); break;
    case 4: e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks_per_sm, k_pairs_batch<64, 4>, 64, 0); break;
    }
    return e == cudaSuccess ? 0 : -1;
}

void batch_pairs_launch(int v, int grid, const BatchInst *inst, const int4 *items, int n_items,
                        unsigned int *counter, const unsigned char *mask, cudaStream_t s)
{
    switch (v) {
    case 0: k_pairs_batch<128, 2><<<grid, 128, 0, s>>>(inst, items, n_items, counter, mask); break;
    case 1: k_pairs_batch<256, 1><<<grid, 256, 0, s>>>(inst, items, n_items, counter, mask); break;
    case 2: k_pairs_batch<64, 2><<<grid, 64, 0, s>>>(inst, items, n_items, counter, mask); break;
    case 3: k_pairs_batch<128, 1><<<grid, 128, 0, s>>>(inst, items, n_items, counter, mask); break;
    case 4: k_pairs_batch<64, 4><<<grid, 64, 0, s>>>(inst, items, n_items, counter, mask); break;
    }
}

int constB_launch(bfs_ctx *c, cudaStream_t s)
{
    FinArgs fa = fin_args(c, 1);
    k_constB<<<(c->Nt + 127) / 128, 128, 0, s>>>(c->d_src64, c->Ns, c->d_tgt64, c->d_bx, c->d_by,
                                                 c->d_constB, fa, c->opt.sign_I4);
    c->launches++;
    BFS_CUDA_TRY(c, cudaGetLastError());
    return BFS_OK;
}

cudaEvent_t prof_event(bfs_ctx *c)
{
    if (c->ev_used == c->ev_pool.size()) {
        cudaEvent_t e;
        cudaEventCreate(&e);
        c->ev_pool.push_back(e);
    }
    return c->ev_pool[c->ev_used++];
}

void plans_for(int Nt, int Ns, int splits_req, int sms, PairPlan *p64, PairPlan *p32)
{
    *p64 = make_plan(Nt, Ns, P64_TPB, P64_TPT, P64_CH, splits_req, sms);
    *p32 = make_plan(Nt, Ns, P32_TPB, P32_TPT, P32_CH, splits_req, sms);
}

}  // namespace bfs
