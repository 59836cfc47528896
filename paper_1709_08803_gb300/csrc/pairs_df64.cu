// Double-float ("df64") all-pairs quadrature: the FP64-accurate residual on
// the FP32 pipes.
//
// GB300 executes two FP64 fused multiply-adds per SM per clock against 128 in
// FP32, so the FP64 pair kernel is bound by that pipe.  Here every FP64 quantity
// of the pair sum is carried as an unevaluated sum hi + lo of two floats
// (Dekker 1971; Knuth's two-sum; two-product by fused multiply-add), which
// keeps about 46 significant bits: per term a relative error near 1e-13,
// well inside the 1e-10 per-row parity bar of the FP64 residual.  The sums
// are the same four sheet pairings, singularity subtractions and S2 term as
// the FP64 and FP32C kernels (Sec. 2.2 and 3.1 of the paper).
//
// Horizontal offsets are exact in single precision: records carry the node
// column and row positions in mesh units (half-integers), the x offset is in
// units of dx and the y offset is (row difference) * dy/dx, applied as a
// double-float factor.
#include <math.h>

#include "bfs_internal.cuh"

namespace bfs {

struct df {
    float hi, lo;
};

__device__ __forceinline__ df mk(float h, float l) { return df{h, l}; }

// |a| >= |b| (or a == 0)
__device__ __forceinline__ df fast_two_sum(float a, float b)
{
    float s = a + b;
    return mk(s, b - (s - a));
}

__device__ __forceinline__ df df_add(df a, df b)
{
    float s = a.hi + b.hi;
    float bb = s - a.hi;
    float e = (a.hi - (s - bb)) + (b.hi - bb);
    e += a.lo + b.lo;
    return fast_two_sum(s, e);
}

__device__ __forceinline__ df df_neg(df a) { return mk(-a.hi, -a.lo); }
__device__ __forceinline__ df df_sub(df a, df b) { return df_add(a, df_neg(b)); }

__device__ __forceinline__ df df_add_f(df a, float b)
{
    float s = a.hi + b;
    float bb = s - a.hi;
    float e = (a.hi - (s - bb)) + (b - bb);
    e += a.lo;
    return fast_two_sum(s, e);
}

__device__ __forceinline__ df df_mul(df a, df b)
{
    float p = a.hi * b.hi;
    float e = fmaf(a.hi, b.hi, -p);
    e = fmaf(a.hi, b.lo, e);
    e = fmaf(a.lo, b.hi, e);
    return fast_two_sum(p, e);
}

__device__ __forceinline__ df df_mulf(df a, float b)
{
    float p = a.hi * b;
    float e = fmaf(a.hi, b, -p);
    e = fmaf(a.lo, b, e);
    return fast_two_sum(p, e);
}

// The same three without the final renormalisation (the pair stays an exact
// unevaluated sum, its low part up to about 2^-22 of the high one), for the
// quantities of the pair sum that cannot cancel: sums of squares, powers of
// 1/r, and products entering a renormalising accumulation.
__device__ __forceinline__ df df_add_s(df a, df b)
{
    float s = a.hi + b.hi;
    float bb = s - a.hi;
    float e = (a.hi - (s - bb)) + (b.hi - bb);
    e += a.lo + b.lo;
    return mk(s, e);
}

__device__ __forceinline__ df df_mul_s(df a, df b)
{
    float p = a.hi * b.hi;
    float e = fmaf(a.hi, b.hi, -p);
    e = fmaf(a.hi, b.lo, e);
    e = fmaf(a.lo, b.hi, e);
    return mk(p, e);
}

__device__ __forceinline__ df df_sqr_s(df a)
{
    float p = a.hi * a.hi;
    float e = fmaf(a.hi, a.hi, -p);
    e = fmaf(2.0f * a.hi, a.lo, e);
    return mk(p, e);
}

__device__ __forceinline__ df df_sqr(df a)
{
    float p = a.hi * a.hi;
    float e = fmaf(a.hi, a.hi, -p);
    e = fmaf(2.0f * a.hi, a.lo, e);
    return fast_two_sum(p, e);
}

// 1/sqrt(a): single-precision seed, one Newton step carried in double-float
// (the step's residual 1 - a y0^2 is formed from the exact square of y0).
__device__ __forceinline__ df df_rsqrt(df a)
{
    const float y0 = rsqrtf(a.hi);
    const float p = y0 * y0;
    const df y2 = mk(p, fmaf(y0, y0, -p));
    const df q = df_mul(a, y2);
    const float e = (1.0f - q.hi) - q.lo;
    return mk(y0, 0.5f * y0 * e);
}

__device__ __forceinline__ df ld2(const float *p) { return mk(p[0], p[1]); }

// Double-float source and target records (32 floats each):
// source: 0 column, 1 row (mesh units, exact), then hi/lo pairs of
//   2 zeta/dx  4 (beta+1)/dx  6 zeta_x  8 zeta_y dy/dx  10 beta_x  12 beta_y dy/dx
//   14 w1 f  16 w2 zeta_x  18 w1 g  20 w2 sigma beta_x  22 w1  24 w2
// target: 0 column, 1 row, then 2 zeta*/dx  4 zeta*/dx + 1/dx  6 (beta*+1)/dx - 1/dx
//   8 (beta*+1)/dx  10 f*  12 g*  14 A  16 B dy/dx  18 C (dy/dx)^2
constexpr int DREC = 32;

__device__ __forceinline__ void split2(double v, float *o)
{
    float h = (float)v;
    o[0] = h;
    o[1] = (float)(v - (double)h);
}

__global__ void k_records_df(const double *__restrict__ src64, const double *__restrict__ tgt64,
                             float *__restrict__ srcdf, float *__restrict__ tgtdf, int Ns_cap, int Nt,
                             double ry)
{
    int e = blockIdx.x * blockDim.x + threadIdx.x;
    if (e < Ns_cap) {
        const double *r = src64 + (size_t)e * REC;
        float *o = srcdf + (size_t)e * DREC;
        o[0] = (float)r[0];
        o[1] = (float)r[14];
        split2(r[2], o + 2);
        split2(r[3], o + 4);
        split2(r[4], o + 6);
        split2(r[5] * ry, o + 8);
        split2(r[6], o + 10);
        split2(r[7] * ry, o + 12);
        split2(r[8], o + 14);
        split2(r[9], o + 16);
        split2(r[10], o + 18);
        split2(r[11], o + 20);
        split2(r[12], o + 22);
        split2(r[13], o + 24);
        for (int k = 26; k < DREC; k++) o[k] = 0.0f;
        return;
    }
    e -= Ns_cap;
    if (e >= Nt) return;
    const double *t = tgt64 + (size_t)e * TREC;
    float *o = tgtdf + (size_t)e * DREC;
    o[0] = (float)t[0];
    o[1] = (float)t[15];
    split2(t[2], o + 2);
    split2(t[11], o + 4);
    split2(t[12], o + 6);
    split2(t[3], o + 8);
    split2(t[6], o + 10);
    split2(t[7], o + 12);
    split2(t[8], o + 14);
    split2(t[9] * ry, o + 16);
    split2(t[10] * ry * ry, o + 18);
    for (int k = 20; k < DREC; k++) o[k] = 0.0f;
}

constexpr int PDF_TPB = 128, PDF_CH = 64;

__global__ void __launch_bounds__(PDF_TPB)
k_pairs_df(const float *__restrict__ src, int per_split, const float *__restrict__ tgt, int Nt,
           double *__restrict__ part, df ry, df ry2)
{
    __shared__ __align__(16) float sh[PDF_CH * DREC];
    const int split = blockIdx.y;
    const float *sb = src + (size_t)split * per_split * DREC;
    const int t = blockIdx.x * PDF_TPB + threadIdx.x;
    const float *tr = tgt + (size_t)min(t, Nt - 1) * DREC;
    const float tx = tr[0], ty = tr[1];
    const df tz = ld2(tr + 2), cTB = ld2(tr + 4), cBT = ld2(tr + 6), tB = ld2(tr + 8);
    const df tf = ld2(tr + 10), tg = ld2(tr + 12), A = ld2(tr + 14), Bry = ld2(tr + 16),
             Cry2 = ld2(tr + 18);
    df aT1 = mk(0, 0), aT2 = mk(0, 0), aS = mk(0, 0), aB1 = mk(0, 0), aB2 = mk(0, 0);

    for (int c0 = 0; c0 < per_split; c0 += PDF_CH) {
        __syncthreads();
        const float4 *g = reinterpret_cast<const float4 *>(sb + (size_t)c0 * DREC);
        float4 *sv = reinterpret_cast<float4 *>(sh);
        for (int e = threadIdx.x; e < PDF_CH * DREC / 4; e += PDF_TPB) sv[e] = g[e];
        __syncthreads();
        for (int s = 0; s < PDF_CH; s++) {
            const float *r = sh + s * DREC;
            const float sx = r[0] - tx;  // exact: half-integer mesh offsets
            const float dj = r[1] - ty;  // exact: integer row offset
            const float sxx = sx * sx, djj = dj * dj, sdj = sx * dj;  // exact
            const df rho2 = df_add_f(df_mulf(ry2, djj), sxx);
            const df zs = ld2(r + 2), bs = ld2(r + 4), zxs = ld2(r + 6), zys = ld2(r + 8);
            const df bxs = ld2(r + 10), bys = ld2(r + 12);
            const df w1f = ld2(r + 14), w2zx = ld2(r + 16), w1g = ld2(r + 18), w2sb = ld2(r + 20);
            const df w1 = ld2(r + 22), w2 = ld2(r + 24);
            // S2 at the top target
            {
                const df q = df_add(df_add(df_mulf(A, sxx), df_mulf(Bry, sdj)), df_mulf(Cry2, djj));
                aS = df_add(aS, df_mul_s(w2, df_rsqrt(q)));
            }
            // top target, top source
            {
                const df d = df_sub(zs, tz);
                const df ri = df_rsqrt(df_add_s(rho2, df_sqr_s(d)));
                const df ri3 = df_mul_s(df_sqr_s(ri), ri);
                const df num = df_sub(df_sub(d, df_mulf(zxs, sx)), df_mulf(zys, dj));
                const df dens = df_sub(w1f, df_mul(tf, w1));
                aT1 = df_add(aT1, df_mul_s(df_mul_s(dens, num), ri3));
                aT2 = df_add(aT2, df_mul_s(w2zx, ri));
            }
            // top target, bottom source
            {
                const df d = df_sub(bs, cTB);
                const df ri = df_rsqrt(df_add_s(rho2, df_sqr_s(d)));
                const df ri3 = df_mul_s(df_sqr_s(ri), ri);
                const df num = df_sub(df_sub(d, df_mulf(bxs, sx)), df_mulf(bys, dj));
                aT1 = df_sub(aT1, df_mul_s(df_mul_s(w1g, num), ri3));
                aT2 = df_add(aT2, df_mul_s(w2sb, ri));
            }
            // bottom target, top source
            {
                const df d = df_sub(zs, cBT);
                const df ri = df_rsqrt(df_add_s(rho2, df_sqr_s(d)));
                const df ri3 = df_mul_s(df_sqr_s(ri), ri);
                const df num = df_sub(df_sub(d, df_mulf(zxs, sx)), df_mulf(zys, dj));
                aB1 = df_add(aB1, df_mul_s(df_mul_s(w1f, num), ri3));
                aB2 = df_add(aB2, df_mul_s(w2zx, ri));
            }
            // bottom target, bottom source
            {
                const df d = df_sub(bs, tB);
                const df ri = df_rsqrt(df_add_s(rho2, df_sqr_s(d)));
                const df ri3 = df_mul_s(df_sqr_s(ri), ri);
                const df num = df_sub(df_sub(d, df_mulf(bxs, sx)), df_mulf(bys, dj));
                const df dens = df_sub(w1g, df_mul(tg, w1));
                aB1 = df_sub(aB1, df_mul_s(df_mul_s(dens, num), ri3));
            }
        }
    }
    if (t >= Nt) return;
    const df acc[NACC] = {aT1, aT2, aS, aB1, aB2};
#pragma unroll
    for (int q = 0; q < NACC; q++)
        part[((size_t)split * NACC + q) * Nt + t] = (double)acc[q].hi + (double)acc[q].lo;
}

PairPlan plan_df(int Nt, int Ns, int splits_req, int sms)
{
    return make_plan(Nt, Ns, PDF_TPB, 1, PDF_CH, splits_req, sms);
}

int pairs_df_launch(bfs_ctx *c, cudaStream_t s)
{
    const int tot = c->Ns_cap + c->Nt;
    k_records_df<<<(tot + 255) / 256, 256, 0, s>>>(c->d_src64, c->d_tgt64, c->d_srcdf, c->d_tgtdf,
                                                   c->Ns_cap, c->Nt, c->dy / c->dx);
    c->launches++;
    const double ryd = c->dy / c->dx, ry2d = ryd * ryd;
    df ry, ry2;
    ry.hi = (float)ryd;
    ry.lo = (float)(ryd - (double)ry.hi);
    ry2.hi = (float)ry2d;
    ry2.lo = (float)(ry2d - (double)ry2.hi);
    const PairPlan &p = c->plandf;
    k_pairs_df<<<dim3(p.tiles, p.splits), PDF_TPB, 0, s>>>(c->d_srcdf, p.per_split, c->d_tgtdf, c->Nt,
                                                          c->d_part, ry, ry2);
    c->launches++;
    BFS_CUDA_TRY(c, cudaGetLastError());
    return BFS_OK;
}

}  // namespace bfs
