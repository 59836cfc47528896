// Block-banded preconditioner P = banded Jacobian of the linearised discrete
// system (Buttle et al., arXiv:1709.08803, Sec. 4.2 and App. A, B).
//
// Layout.  Unknowns and equations are regrouped slice by slice: slice l owns
// the nb = 3(N+1) unknowns [zeta(1), zeta_x(1..N) | phi(1), phi_x | psi(1), psi_x]
// and the nb equations [F5, F6, F1(1..N-1) | F3, F4, F2 | F8, F9, F7].  P is then
// an M x M block matrix of nb x nb blocks; App. A keeps the blocks within
// half_band h of the diagonal, so block row l stores blocks l-h .. l+h at
// d_pc + (l (2h+1) + (m - l + h)) nb^2 (row-major).
//
// Entries (derived by differentiating the linear residual of App. B; every
// kernel there is a function of horizontal distance only, and the linear
// Jacobian does not depend on u, on the topography or on the sign of I4):
//   F1 = phi_x* + zeta*/F^2 - 1, F2 and F7 the linear boundary integral
//   equation with K5 = 1/r, K6 = (r^2+1)^(-3/2), K7 = (r^2+1)^(-1/2), and the
//   radiation rows.  Nodal values follow from q(1) and q_x by the trapezoid
//   rule, T(i, n) being the weight of q_x(n) in q(i); half-point values are
//   means of the two neighbouring nodes, H(k, n) = (T(k,n) + T(k+1,n)) / 2.
//
// Factorisation (no pivoting across blocks; partial pivoting inside the
// diagonal blocks by Gauss-Jordan inversion), one-ended:
//   for k: D_k^-1;  W_kj = D_k^-1 U_kj;  S_ij -= S_ik W_kj;  L_ik = S_ik D_k^-1
// stored in place: diagonal slot D_k^-1, lower slots L, upper slots W, so that
//   forward  y_k = x_k - sum_i L_ki y_i
//   backward z_k = D_k^-1 y_k - sum_j W_kj z_j.
// Two-ended ("twisted", for the FP32 sweeps of apply.cu): the same step for
// slices k = 0..t-1 with the coupled slices above them, and for k = M-1 down to
// t+h with the coupled slices below them (W'_kj = D_k^-1 S_kj in the lower
// slots of row k, U'_ik = S_ik D_k^-1 in the upper slots of column k).  The two
// chains meet only in the h middle slices t..t+h-1, whose Schur complement C
// (h nb square, both chains' updates added) is inverted whole; C^-1 replaces
// the middle-middle blocks.  Both orders are exact block LU of the same banded
// matrix; the second halves the sweeps' chain of dependent steps.
#include <math.h>

#include <algorithm>
#include <memory>
#include <vector>

#include <cooperative_groups.h>

#include "bfs_internal.cuh"

namespace bfs {

__device__ __forceinline__ double trap_T(int i, int n)  // 1-based
{
    if (i == 1) return 0.0;
    if (n == 1) return 0.5;
    if (n < i) return 1.0;
    if (n == i) return 0.5;
    return 0.0;
}

__device__ __forceinline__ double half_H(int k, int n) { return 0.5 * (trap_T(k, n) + trap_T(k + 1, n)); }

__device__ double rect_S2_pc(double s1, double s2, double t1, double t2);

struct PcArgs {
    int N, M, half, h, nb;
    double x1, y1, dx, dy, F, n_rad, xhi, ylo, yhi, tau;
};

__device__ __forceinline__ double trap_w(const PcArgs &a, int i, int j)  // 0-based
{
    double cx = (i == 0 || i == a.N - 1) ? 0.5 : 1.0;
    double cy = a.half ? ((j == a.M - 1) ? 0.5 : 1.0) : ((j == 0 || j == a.M - 1) ? 0.5 : 1.0);
    return a.dx * a.dy * cx * cy;
}

// Closed-form integral of 1/r over the mesh rectangle seen from (xs, ys)
// (the A = C = 1, B = 0 case of the S2 integral of Sec. 3.1).
__device__ double g_K5(double s, double t)
{
    double r = sqrt(s * s + t * t), g = 0.0;
    if (t != 0.0) g += t * ((s >= 0.0) ? log(s + r) : (log(t * t) - log(r - s)));
    if (s != 0.0) g += s * ((t >= 0.0) ? log(t + r) : (log(s * s) - log(r - t)));
    return g;
}

__device__ double rect_S2_pc(double s1, double s2, double t1, double t2)
{
    return g_K5(s2, t2) - g_K5(s1, t2) - g_K5(s2, t1) + g_K5(s1, t1);
}

// Row sums of w K5 over all nodes (and images) minus the closed-form integral:
// the coefficient of zeta_x* in the linear F2.
__global__ void k_rowsum5(PcArgs a, double *out)
{
    int e = blockIdx.x * blockDim.x + threadIdx.x;
    int Nt = (a.N - 1) * a.M;
    if (e >= Nt) return;
    int k = e % (a.N - 1), l = e / (a.N - 1);
    double xs = a.x1 + (k + 0.5) * a.dx, ys = a.y1 + l * a.dy;
    double acc = 0.0;
    for (int img = 0; img < (a.half ? 2 : 1); img++)
        for (int j = (img ? 1 : 0); j < a.M; j++) {
            double t = (img ? -1.0 : 1.0) * (a.y1 + j * a.dy) - ys;
            for (int i = 0; i < a.N; i++) {
                double s = a.x1 + i * a.dx - xs;
                acc += trap_w(a, i, j) * rsqrt(s * s + t * t);
            }
        }
    out[e] = acc - rect_S2_pc(a.x1 - xs, a.xhi - xs, a.ylo - ys, a.yhi - ys);
}

// Dense entries of block (l, m): one CTA per (l, d, k), threads over source nodes n.
__global__ void k_form_dense(PcArgs a, double *pc, const double *rowsum5)
{
    extern __shared__ double sh[];  // W6[N], suffix[N+1]
    const int N = a.N, NB = a.N + 1, nb = a.nb, h = a.h;
    const int k0 = blockIdx.x, d = blockIdx.y, l = blockIdx.z;
    const int m = l + d - h;
    if (m < 0 || m >= a.M) return;
    double *W6 = sh, *suf = sh + N;
    double *blk = pc + ((size_t)l * (2 * h + 1) + d) * nb * nb;
    const double xs = a.x1 + (k0 + 0.5) * a.dx, ys = a.y1 + l * a.dy;
    const double ym = a.y1 + m * a.dy;
    const bool img = a.half && m >= 1;
    const size_t r2 = (size_t)(1 * NB + 2 + k0) * nb, r7 = (size_t)(2 * NB + 2 + k0) * nb;
    for (int i = threadIdx.x; i < N; i += blockDim.x) {
        double s = a.x1 + i * a.dx - xs, w = trap_w(a, i, m);
        double t1 = ym - ys, p1 = s * s + t1 * t1;
        double k5 = rsqrt(p1), k7 = rsqrt(p1 + 1.0), k6 = k7 * k7 * k7;
        if (img) {
            double t2 = -ym - ys, p2 = s * s + t2 * t2;
            double q7 = rsqrt(p2 + 1.0);
            k5 += rsqrt(p2);
            k7 += q7;
            k6 += q7 * q7 * q7;
        }
        double v5 = w * k5;
        if (l == m && (i == k0 || i == k0 + 1)) v5 -= 0.5 * rowsum5[l * (N - 1) + k0];
        blk[r2 + 0 * NB + 1 + i] = v5;     // dF2 / d zeta_x(i)
        blk[r7 + 0 * NB + 1 + i] = w * k7;  // dF7 / d zeta_x(i)
        W6[i] = w * k6;
    }
    __syncthreads();
    if (threadIdx.x == 0) {  // suffix sums of w K6 along the slice
        double acc = 0.0;
        suf[N] = 0.0;
        for (int i = N - 1; i >= 0; i--) { acc += W6[i]; suf[i] = acc; }
    }
    __syncthreads();
    for (int i = threadIdx.x; i <= N; i += blockDim.x) {
        double v;
        if (i == 0) v = suf[0];  // d / d psi(1): every node carries psi(1)
        else {
            int n0 = i - 1;
            if (n0 == 0) v = 0.5 * a.dx * suf[1];
            else if (n0 < N - 1) v = a.dx * (0.5 * W6[n0] + suf[n0 + 1]);
            else v = 0.5 * a.dx * W6[N - 1];
        }
        blk[r2 + 2 * NB + i] = v;  // dF2 / d psi
        blk[r7 + 1 * NB + i] = v;  // dF7 / d phi  (equal blocks, Sec. 4.2)
    }
}

// Sparse entries of the diagonal block of slice l: one thread per row.
__global__ void k_form_sparse(PcArgs a, double *pc)
{
    const int NB = a.N + 1, nb = a.nb, h = a.h;
    int e = blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= a.M * nb) return;
    int l = e / nb, r = e % nb;
    double *row = pc + ((size_t)l * (2 * h + 1) + h) * nb * nb + (size_t)r * nb;
    int grp = r / NB, rr = r % NB;
    const double x1 = a.x1, n = a.n_rad, dx = a.dx, F2 = a.F * a.F;
    const double TWO_PI = 6.283185307179586476925286766559;
    int f = grp;  // radiation rows act on the group's own field
    if (rr == 0) {
        row[f * NB + 0] = n;
        row[f * NB + 1] = x1;
        return;
    }
    if (rr == 1) {
        row[f * NB + 1] = n - x1 / dx;
        row[f * NB + 2] = x1 / dx;
        return;
    }
    int k = rr - 1;  // 1-based collocation index
    if (grp == 0) {  // F1 = phi_x* + zeta*/F^2 - 1
        row[0] = 1.0 / F2;
        for (int p = 1; p <= a.N; p++) row[p] = dx * half_H(k, p) / F2;
        row[NB + k] = 0.5;
        row[NB + k + 1] = 0.5;
    } else {  // F2 (phi) or F7 (psi): -2 pi (q* - x*)
        row[f * NB + 0] = -TWO_PI;
        for (int p = 1; p <= a.N; p++) row[f * NB + p] = -TWO_PI * dx * half_H(k, p);
    }
}

// Surface tension in the F1 rows: -tau (zeta_xx* + zeta_yy*) with zeta_xx* the
// x-difference of zeta_x across the half point and zeta_yy* the mean of the
// nodal second y-differences; the nodal zeta of slice l' is zeta(1) + dx times
// the trapezoid weights of zeta_x, so each stencil row l' adds entries to
// block (l, l') when it lies in the band.  One thread per F1 row.
__global__ void k_form_tension(PcArgs a, double *pc)
{
    const int N = a.N, M = a.M, nb = a.nb, h = a.h;
    const int e = blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= M * (N - 1)) return;
    const int l = e / (N - 1), k = e % (N - 1) + 1;  // k 1-based
    const size_t r = (size_t)(k + 1) * nb;             // row of F1(k) in its slice block
    auto block = [&](int lp) { return pc + ((size_t)l * (2 * h + 1) + (lp - l + h)) * nb * nb; };
    double *d = block(l);
    d[r + k] += a.tau / a.dx;
    d[r + k + 1] -= a.tau / a.dx;
    int js[4];
    double cs[4];
    int ns = 0;
    if (l == 0) {
        if (a.half) { js[0] = 0; cs[0] = -2.0; js[1] = 1; cs[1] = 2.0; ns = 2; }
        else if (M >= 4) { js[0] = 0; cs[0] = 2.0; js[1] = 1; cs[1] = -5.0; js[2] = 2; cs[2] = 4.0; js[3] = 3; cs[3] = -1.0; ns = 4; }
        else { js[0] = 0; cs[0] = 1.0; js[1] = 1; cs[1] = -2.0; js[2] = 2; cs[2] = 1.0; ns = 3; }
    } else if (l == M - 1) {
        if (M >= 4) { js[0] = M - 1; cs[0] = 2.0; js[1] = M - 2; cs[1] = -5.0; js[2] = M - 3; cs[2] = 4.0; js[3] = M - 4; cs[3] = -1.0; ns = 4; }
        else { js[0] = M - 1; cs[0] = 1.0; js[1] = M - 2; cs[1] = -2.0; js[2] = M - 3; cs[2] = 1.0; ns = 3; }
    } else {
        js[0] = l - 1; cs[0] = 1.0; js[1] = l; cs[1] = -2.0; js[2] = l + 1; cs[2] = 1.0; ns = 3;
    }
    const double f = -a.tau / (a.dy * a.dy);
    for (int q = 0; q < ns; q++) {
        const int lp = js[q];
        if (lp - l > h || l - lp > h) continue;  // outside the band (App. A)
        double *row = block(lp) + r;
        const double c = f * cs[q];
        row[0] += c;
        for (int p = 1; p <= N; p++) row[p] += c * a.dx * half_H(k, p);
    }
}

// ---------------------------------------------------------------------------
// Gauss-Jordan inversion with partial pivoting on ping-pong buffers
// X = [D | I] (n x 2n, row-major), one or two matrices in one cooperative
// launch: CTA b works on matrix b % nmat, a bounded grid barrier between pivot
// columns (see grid_sync below).
// ---------------------------------------------------------------------------
struct CoopBar;
__device__ bool grid_sync(CoopBar *b, int *flag, unsigned int spin);

struct GjSet {
    double *X0[2], *X1[2];  // ping-pong buffers [D | I] of each matrix (n x 2n)
    int nmat;
};

__global__ void __launch_bounds__(256) k_gj_coop(GjSet set, int nb, int *pivflag, CoopBar *bar, int *flag,
                                                 unsigned int spin)
{
    __shared__ double bv[8];
    __shared__ int bi[8];
    __shared__ int piv;
    __shared__ double pval;
    const int ld = 2 * nb;
    const int mat = blockIdx.x % set.nmat, lb = blockIdx.x / set.nmat, lg = gridDim.x / set.nmat;
    const double *Xi = set.X0[mat];
    double *Xo = set.X1[mat];
    for (int c = 0; c < nb; c++) {
        double best = -1.0;
        int bidx = c;
        for (int r = c + threadIdx.x; r < nb; r += blockDim.x) {
            double v = fabs(__ldcg(Xi + (size_t)r * ld + c));
            if (v > best) { best = v; bidx = r; }
        }
        for (int o = 16; o > 0; o >>= 1) {
            double ov = __shfl_down_sync(0xffffffffu, best, o);
            int oi = __shfl_down_sync(0xffffffffu, bidx, o);
            if (ov > best || (ov == best && oi < bidx)) { best = ov; bidx = oi; }
        }
        if ((threadIdx.x & 31) == 0) { bv[threadIdx.x >> 5] = best; bi[threadIdx.x >> 5] = bidx; }
        __syncthreads();
        if (threadIdx.x == 0) {
            double b = bv[0];
            int i = bi[0];
            for (int w = 1; w < (int)(blockDim.x >> 5); w++)
                if (bv[w] > b || (bv[w] == b && bi[w] < i)) { b = bv[w]; i = bi[w]; }
            piv = i;
            pval = __ldcg(Xi + (size_t)i * ld + c);
            if (!(b > 0.0) && lb == 0) atomicOr(pivflag, 1);
        }
        __syncthreads();
        const int p = piv;
        const double ip = pval != 0.0 ? 1.0 / pval : 0.0;
        for (int r = lb; r < nb; r += lg) {
            const int src = (r == c) ? p : ((r == p) ? c : r);
            const double *xs = Xi + (size_t)src * ld;
            const double *xp = Xi + (size_t)p * ld;
            double *xo = Xo + (size_t)r * ld;
            if (r == c) {
                for (int q = c + threadIdx.x; q < ld; q += blockDim.x) __stcg(xo + q, __ldcg(xp + q) * ip);
            } else {
                const double f = __ldcg(xs + c) * ip;
                for (int q = c + threadIdx.x; q < ld; q += blockDim.x)
                    __stcg(xo + q, fma(-f, __ldcg(xp + q), __ldcg(xs + q)));
            }
        }
        if (!grid_sync(bar, flag, spin)) return;
        const double *t = Xi;
        Xi = Xo;
        Xo = const_cast<double *>(t);
    }
}

// ---------------------------------------------------------------------------
// In-place Gauss-Jordan inversion with partial pivoting, rows resident in
// shared memory, no grid barrier.  CTA group g of a launch inverts matrix g
// (one or two matrices, n x n row-major, FP64); CTA b of the group keeps a
// contiguous run of rows in shared memory for the whole inversion.  Pivoting
// is implicit (rows are never moved): the pivot of column k is the unused row
// with the largest |S[i][k]|, and the update, applied to every row i != p,
//   S[p][j] /= a (j != k), S[p][k] = 1/a;  S[i][j] -= S[i][k] S[p][j] / a (j != k),
//   S[i][k] = -S[i][k] / a          (a = S[p][k])
// stores in column k the column p of the growing inverse transformation, so
// that at the end A^-1[k][j] = S[perm[k]][pinv[j]] (perm[k]: the pivot row of
// column k) -- the gather k_gj_unperm undoes the permutation.
//
// Instead of a grid barrier per column, every CTA publishes, for the next
// column, its best candidate (|value| and row, then a tag word released after
// the candidate row's data) in a slot of its own; the CTAs of the group poll
// the tags, agree on the largest candidate (ties: the lowest row) and read
// its row from the winner's slot.  Slots alternate between two parities, so a
// CTA may publish column k+1 while slower ones still read column k.  The
// launch is cooperative (all CTAs resident); each poll is bounded, after which
// bit 2 of *flag is raised and the CTA returns.
// ---------------------------------------------------------------------------
constexpr int GJR_TPB = 256;
constexpr int GJR_MAXR = 16;  // rows per CTA

struct GjRowsArgs {
    double *S0, *S1;            // the matrices in; the in-place result out
    int n, nmat, G;             // G: CTAs per matrix
    unsigned long long *slot;   // [2 parities][nmat G][2]: |value| bits, (row << 32) | tag
    double *data;               // [2 parities][nmat G][n]: candidate rows
    int *perm;                  // [nmat][2 n]: perm, then pinv
    int *pivflag, *flag;
    unsigned int spin;
};

__device__ __forceinline__ unsigned long long ld_acq_u64(const unsigned long long *p)
{
    unsigned long long v;
    asm volatile("ld.acquire.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
    return v;
}

__device__ __forceinline__ void st_rel_u64(unsigned long long *p, unsigned long long v)
{
    asm volatile("st.release.gpu.global.u64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}

__global__ void __launch_bounds__(GJR_TPB) k_gj_rows(GjRowsArgs a)
{
    extern __shared__ double gsm[];  // nr rows of n, then the scaled pivot row (n)
    __shared__ double rv[GJR_TPB / 32];
    __shared__ int ri[GJR_TPB / 32], rrow[GJR_TPB / 32];
    __shared__ double fcol[GJR_MAXR];
    __shared__ unsigned char used[GJR_MAXR];
    __shared__ double cand_v;
    __shared__ int cand_sh, win_sh, ok_sh, prow_sh;
    const int n = a.n, tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int mat = blockIdx.x / a.G, lb = blockIdx.x - mat * a.G;
    if (mat >= a.nmat) return;
    const int Geff = min(a.G, n);
    if (lb >= Geff) return;  // no rows here
    const int base = n / Geff, extra = n % Geff;
    const int nr = base + (lb < extra ? 1 : 0), r0 = lb * base + min(lb, extra);
    const int NS = a.nmat * a.G, me = mat * a.G + lb, s0 = mat * a.G;
    double *S = gsm, *pr = gsm + (size_t)nr * n;
    double *Mg = mat ? a.S1 : a.S0;
    for (int e = tid; e < nr * n; e += GJR_TPB) S[e] = Mg[(size_t)r0 * n + e];
    if (tid < GJR_MAXR) used[tid] = 0;
    __syncthreads();

    // candidate of this CTA for column k into the slots of parity par
    auto publish = [&](int k, int par) {
        if (warp == 0) {
            double v = -1.0;
            int i = -1;
            for (int r = lane; r < nr; r += 32)
                if (!used[r]) {
                    const double x = fabs(S[(size_t)r * n + k]);
                    if (x > v || i < 0) { v = x; i = r; }
                }
            for (int o = 16; o > 0; o >>= 1) {
                const double ov = __shfl_down_sync(0xffffffffu, v, o);
                const int oi = __shfl_down_sync(0xffffffffu, i, o);
                if (oi >= 0 && (i < 0 || ov > v || (ov == v && oi < i))) { v = ov; i = oi; }
            }
            if (lane == 0) { cand_sh = i; cand_v = v; }
        }
        __syncthreads();
        const int ci = cand_sh;
        double *d = a.data + ((size_t)par * NS + me) * n;
        if (ci >= 0)
            for (int j = tid; j < n; j += GJR_TPB) __stcg(d + j, S[(size_t)ci * n + j]);
        __syncthreads();
        if (tid == 0) {
            unsigned long long *sl = a.slot + ((size_t)par * NS + me) * 2;
            const unsigned int row = ci >= 0 ? (unsigned int)(r0 + ci) : 0x7fffffffu;
            __threadfence();
            __stcg(reinterpret_cast<double *>(sl), ci >= 0 ? cand_v : -1.0);
            st_rel_u64(sl + 1, ((unsigned long long)row << 32) | (unsigned int)(k + 1));
        }
    };

    publish(0, 0);
    for (int k = 0; k < n; k++) {
        const int par = k & 1;
        // the candidates of every CTA of the group: thread t polls CTA t's slot
        double v = -1.0;
        int row = 0x7fffffff, who = -1;
        bool ok = true;
        for (int t = tid; t < Geff; t += GJR_TPB) {
            const unsigned long long *sl = a.slot + ((size_t)par * NS + s0 + t) * 2;
            unsigned long long w = ld_acq_u64(sl + 1);
            unsigned int spins = 0;
            while ((unsigned int)w != (unsigned int)(k + 1)) {
                if (++spins > a.spin) { ok = false; break; }
                __nanosleep(20);
                w = ld_acq_u64(sl + 1);
            }
            if (!ok) break;
            const double x = __ldcg(reinterpret_cast<const double *>(sl));
            const int r = (int)(w >> 32);
            if (x > v || (x == v && r < row)) { v = x; row = r; who = t; }
        }
        if (!__syncthreads_and(ok)) {
            if (tid == 0) atomicOr(a.flag, 2);
            return;
        }
        for (int o = 16; o > 0; o >>= 1) {
            const double ov = __shfl_down_sync(0xffffffffu, v, o);
            const int orow = __shfl_down_sync(0xffffffffu, row, o), ow = __shfl_down_sync(0xffffffffu, who, o);
            if (ov > v || (ov == v && orow < row)) { v = ov; row = orow; who = ow; }
        }
        if (lane == 0) { rv[warp] = v; ri[warp] = who; rrow[warp] = row; }
        __syncthreads();
        if (tid == 0) {
            double b = -1.0;
            int w = -1, wr = 0x7fffffff;
            for (int q = 0; q < GJR_TPB / 32; q++) {
                if (ri[q] < 0) continue;
                if (w < 0 || rv[q] > b || (rv[q] == b && rrow[q] < wr)) { b = rv[q]; w = ri[q]; wr = rrow[q]; }
            }
            win_sh = w;
            prow_sh = wr;
            ok_sh = (w >= 0 && b > 0.0);
            if (!ok_sh && lb == 0) atomicOr(a.pivflag, 1);
        }
        __syncthreads();
        // the winner's data: its tag was acquired by the polling thread before the
        // barrier above, which orders these reads after it
        const int w = win_sh, p = prow_sh;
        const double *pd = a.data + ((size_t)par * NS + s0 + max(w, 0)) * n;
        const double piv = __ldcg(pd + k);
        const double inv = (ok_sh && piv != 0.0) ? 1.0 / piv : 0.0;
        for (int j = tid; j < n; j += GJR_TPB) pr[j] = __ldcg(pd + j) * inv;
        for (int i = tid; i < nr; i += GJR_TPB) fcol[i] = S[(size_t)i * n + k];
        if (lb == 0 && tid == 0) a.perm[(size_t)mat * 2 * n + k] = p;
        __syncthreads();
        // the update of every row of this CTA
        const int ip = (p >= r0 && p < r0 + nr) ? p - r0 : -1;
        for (int i = 0; i < nr; i++) {
            double *Si = S + (size_t)i * n;
            const double f = fcol[i];
            if (i == ip) {
                for (int j = tid; j < n; j += GJR_TPB) Si[j] = j == k ? inv : pr[j];
            } else {
                for (int j = tid; j < n; j += GJR_TPB) Si[j] = j == k ? -f * inv : fma(-f, pr[j], Si[j]);
            }
        }
        if (ip >= 0 && tid == 0) used[ip] = 1;
        __syncthreads();
        if (k + 1 < n) publish(k + 1, par ^ 1);
    }
    for (int e = tid; e < nr * n; e += GJR_TPB) Mg[(size_t)r0 * n + e] = S[e];
    if (lb == 0) {  // the inverse permutation (perm is complete: this CTA recorded it)
        __syncthreads();
        int *pm = a.perm + (size_t)mat * 2 * n;
        for (int k2 = tid; k2 < n; k2 += GJR_TPB) pm[n + pm[k2]] = k2;
    }
}

// One nb x nb block into (or out of) a row-major matrix of row length ld at block (a, b).
__global__ void k_blk_put(const double *__restrict__ D, double *__restrict__ X, int nb, int ld, int a, int b)
{
    for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < (size_t)nb * nb;
         e += (size_t)gridDim.x * blockDim.x) {
        const int r = (int)(e / nb), c = (int)(e % nb);
        X[(size_t)(a * nb + r) * ld + b * nb + c] = D[e];
    }
}

__global__ void k_blk_get(const double *__restrict__ X, double *__restrict__ D, int nb, int ld, int a, int b)
{
    for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < (size_t)nb * nb;
         e += (size_t)gridDim.x * blockDim.x) {
        const int r = (int)(e / nb), c = (int)(e % nb);
        D[e] = X[(size_t)(a * nb + r) * ld + b * nb + c];
    }
}

// A^-1[k][j] = S[perm[k]][pinv[j]] into the destination (row-major, ld n).
__global__ void k_gj_unperm(const double *__restrict__ S, const int *__restrict__ perm, double *__restrict__ D,
                            int n)
{
    const int *pinv = perm + n;
    for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < (size_t)n * n;
         e += (size_t)gridDim.x * blockDim.x) {
        const int k = (int)(e / n), j = (int)(e % n);
        D[e] = S[(size_t)perm[k] * n + pinv[j]];
    }
}

// One nb x nb block into (or out of) the n x 2n Gauss-Jordan buffer at block
// position (a, b); the identity in the right half.
__global__ void k_gj_put(const double *__restrict__ D, double *__restrict__ X, int nb, int n, int a, int b)
{
    for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < (size_t)nb * nb;
         e += (size_t)gridDim.x * blockDim.x) {
        const int r = (int)(e / nb), c = (int)(e % nb);
        X[(size_t)(a * nb + r) * 2 * n + b * nb + c] = D[e];
    }
}

__global__ void k_gj_eye(double *__restrict__ X, int n)
{
    for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < (size_t)n * n;
         e += (size_t)gridDim.x * blockDim.x) {
        const int r = (int)(e / n), c = (int)(e % n);
        X[(size_t)r * 2 * n + n + c] = r == c ? 1.0 : 0.0;
    }
}

__global__ void k_gj_get(const double *__restrict__ X, double *__restrict__ D, int nb, int n, int a, int b)
{
    for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < (size_t)nb * nb;
         e += (size_t)gridDim.x * blockDim.x) {
        const int r = (int)(e / nb), c = (int)(e % nb);
        D[e] = X[(size_t)(a * nb + r) * 2 * n + n + b * nb + c];
    }
}

// FP64 -> hi + lo FP32 pair by bit manipulation, with no FP64 arithmetic (the
// FP64 pipe of this GPU retires two operations per clock per SM): hi keeps the
// sign, the exponent and the top 23 stored mantissa bits (a truncation), lo
// the remaining 29 bits rounded to FP32, so |v - hi - lo| <= 2^-48 |v| and
// |lo| < 2^-23 |hi|.  |v| < 2^-126 gives 0 (and lo flushes to 0 below about
// 2^-102: the kernels run with flush-to-zero); |v| >= 2^128, infinities and
// NaN give an infinite or NaN hi.
__device__ __forceinline__ float2 df2_split(double v)
{
    const unsigned long long b = (unsigned long long)__double_as_longlong(v);
    const unsigned int hi32 = (unsigned int)(b >> 32), lo32 = (unsigned int)b;
    const int e = (int)((hi32 >> 20) & 0x7ffu);
    const unsigned int sgn = hi32 & 0x80000000u;
    if (e < 897) return make_float2(__uint_as_float(sgn), 0.f);
    if (e > 1150) {
        const bool nan = e == 0x7ff && ((hi32 & 0xfffffu) | lo32);
        return make_float2(__uint_as_float(sgn | 0x7f800000u | (nan ? 0x400000u : 0u)), 0.f);
    }
    const float h = __uint_as_float(sgn | ((unsigned int)(e - 896) << 23) | ((hi32 & 0xfffffu) << 3) | (lo32 >> 29));
    const float r = __uint2float_rn(lo32 & 0x1fffffffu);
    const int sc = e - 1075;  // weight of the last stored mantissa bit
    const float l = sc >= -126 ? __fmul_rn(r, __uint_as_float((unsigned int)(sc + 127) << 23))
                               : __fmul_rn(__fmul_rn(r, __uint_as_float((unsigned int)(sc + 191) << 23)), 0x1p-64f);
    return make_float2(h, sgn ? -l : l);
}

// ---------------------------------------------------------------------------
// Batched FP64 GEMM on nb x nb row-major blocks: C = alpha A B + beta C.
// ---------------------------------------------------------------------------
constexpr int GB_MAX = 64;
struct GemmBatch {
    const double *A[GB_MAX];
    const double *B[GB_MAX];
    double *C[GB_MAX];
};

constexpr int TM = 64, TN = 64, TK = 16;

__global__ void __launch_bounds__(256) k_dgemm(GemmBatch gb, int n, double alpha, double beta)
{
    __shared__ double As[TK][TM + 1];
    __shared__ double Bs[TK][TN + 1];
    const double *A = gb.A[blockIdx.z], *B = gb.B[blockIdx.z];
    double *C = gb.C[blockIdx.z];
    const int tx = threadIdx.x % 16, ty = threadIdx.x / 16;
    const int row0 = blockIdx.y * TM, col0 = blockIdx.x * TN;
    double acc[4][4] = {};
    for (int k0 = 0; k0 < n; k0 += TK) {
        for (int e = threadIdx.x; e < TM * TK; e += 256) {
            int r = e / TK, kk = e % TK;
            int gr = row0 + r, gk = k0 + kk;
            As[kk][r] = (gr < n && gk < n) ? A[(size_t)gr * n + gk] : 0.0;
        }
        for (int e = threadIdx.x; e < TK * TN; e += 256) {
            int kk = e / TN, cc = e % TN;
            int gk = k0 + kk, gc = col0 + cc;
            Bs[kk][cc] = (gk < n && gc < n) ? B[(size_t)gk * n + gc] : 0.0;
        }
        __syncthreads();
#pragma unroll
        for (int kk = 0; kk < TK; kk++) {
            double a[4], b[4];
#pragma unroll
            for (int i = 0; i < 4; i++) a[i] = As[kk][ty * 4 + i];
#pragma unroll
            for (int j = 0; j < 4; j++) b[j] = Bs[kk][tx * 4 + j];
#pragma unroll
            for (int i = 0; i < 4; i++)
#pragma unroll
                for (int j = 0; j < 4; j++) acc[i][j] = fma(a[i], b[j], acc[i][j]);
        }
        __syncthreads();
    }
#pragma unroll
    for (int i = 0; i < 4; i++) {
        int gr = row0 + ty * 4 + i;
        if (gr >= n) continue;
#pragma unroll
        for (int j = 0; j < 4; j++) {
            int gc = col0 + tx * 4 + j;
            if (gc >= n) continue;
            double *cp = C + (size_t)gr * n + gc;
            *cp = beta == 0.0 ? alpha * acc[i][j] : fma(alpha, acc[i][j], beta * *cp);
        }
    }
}

// The same GEMM in double-float arithmetic on the FP32 pipes (about 40 T
// lane-ops/s on GB300 against 0.6 T for FP64 FMA).  Each FP64 operand is split
// as its tile is staged into an FP32 pair (df2_split: 48 significant bits, no
// FP64 arithmetic).  A product is hi*hi exactly -- the FMA returns the
// rounding error of the rounded product (Dekker) -- plus the cross terms
// hi*lo + lo*hi in FP32; lo*lo, below 2^-48 of it, is dropped.  The running
// sum is an unevaluated pair: Knuth's two-sum on the high parts, the errors and
// cross terms added into the low part.  Each step is exact to about 2^-46, so
// the product is FP64-grade for a preconditioner (relative error of order
// K 2^-48).  The explicit _rn intrinsics keep the compiler from contracting
// the product into the two-sum, which would break its exactness.
__global__ void __launch_bounds__(256, 3) k_dfgemm(GemmBatch gb, int n, double alpha, double beta)
{
    // tiles [k][row] with rows padded to 68 floats: 16-byte aligned for the
    // vector loads of the inner loop, and staging stores spread over the banks
    constexpr int LD = TM + 4;
    __shared__ __align__(16) float Ah[TK][LD], Al[TK][LD];
    __shared__ __align__(16) float Bh[TK][LD], Bl[TK][LD];
    const double *A = gb.A[blockIdx.z], *B = gb.B[blockIdx.z];
    double *C = gb.C[blockIdx.z];
    const int tid = threadIdx.x, tx = tid % 16, ty = tid / 16;
    const int row0 = blockIdx.y * TM, col0 = blockIdx.x * TN;
    // staging map: A element (row ar + 16 q, k ak), B element (k bk + 4 q, col bc); q < 4
    const int ak = tid % TK, ar = tid / TK, bc = tid % TN, bk = tid / TN;
    double ra[4], rb[4];
    auto fetch = [&](int k0) {
#pragma unroll
        for (int q = 0; q < 4; q++) {
            const int gr = row0 + ar + 16 * q, gk = k0 + ak;
            ra[q] = (gr < n && gk < n) ? A[(size_t)gr * n + gk] : 0.0;
            const int gk2 = k0 + bk + 4 * q, gc = col0 + bc;
            rb[q] = (gk2 < n && gc < n) ? B[(size_t)gk2 * n + gc] : 0.0;
        }
    };
    auto stage = [&]() {
#pragma unroll
        for (int q = 0; q < 4; q++) {
            const float2 a = df2_split(ra[q]), b = df2_split(rb[q]);
            Ah[ak][ar + 16 * q] = a.x;
            Al[ak][ar + 16 * q] = a.y;
            Bh[bk + 4 * q][bc] = b.x;
            Bl[bk + 4 * q][bc] = b.y;
        }
    };
    float hi[4][4], lo[4][4];
#pragma unroll
    for (int i = 0; i < 4; i++)
#pragma unroll
        for (int j = 0; j < 4; j++) { hi[i][j] = 0.f; lo[i][j] = 0.f; }
    fetch(0);
    for (int k0 = 0; k0 < n; k0 += TK) {
        stage();
        __syncthreads();
        if (k0 + TK < n) fetch(k0 + TK);  // the next tiles' loads overlap this tile's products
#pragma unroll 4
        for (int kk = 0; kk < TK; kk++) {
            const float4 ah4 = *reinterpret_cast<const float4 *>(&Ah[kk][ty * 4]);
            const float4 al4 = *reinterpret_cast<const float4 *>(&Al[kk][ty * 4]);
            const float4 bh4 = *reinterpret_cast<const float4 *>(&Bh[kk][tx * 4]);
            const float4 bl4 = *reinterpret_cast<const float4 *>(&Bl[kk][tx * 4]);
            const float ah[4] = {ah4.x, ah4.y, ah4.z, ah4.w}, al[4] = {al4.x, al4.y, al4.z, al4.w};
            const float bh[4] = {bh4.x, bh4.y, bh4.z, bh4.w}, bl[4] = {bl4.x, bl4.y, bl4.z, bl4.w};
#pragma unroll
            for (int i = 0; i < 4; i++)
#pragma unroll
                for (int j = 0; j < 4; j++) {
                    const float p = __fmul_rn(ah[i], bh[j]);
                    float e = fmaf(ah[i], bh[j], -p);
                    e = fmaf(ah[i], bl[j], e);
                    e = fmaf(al[i], bh[j], e);
                    const float sm = __fadd_rn(hi[i][j], p);
                    const float bp = __fsub_rn(sm, hi[i][j]);
                    const float err = __fadd_rn(__fsub_rn(hi[i][j], __fsub_rn(sm, bp)), __fsub_rn(p, bp));
                    hi[i][j] = sm;
                    lo[i][j] = __fadd_rn(lo[i][j], __fadd_rn(err, e));
                }
        }
        __syncthreads();
    }
#pragma unroll
    for (int i = 0; i < 4; i++) {
        int gr = row0 + ty * 4 + i;
        if (gr >= n) continue;
#pragma unroll
        for (int j = 0; j < 4; j++) {
            int gc = col0 + tx * 4 + j;
            if (gc >= n) continue;
            double *cp = C + (size_t)gr * n + gc;
            const double v = (double)hi[i][j] + (double)lo[i][j];
            *cp = beta == 0.0 ? alpha * v : fma(alpha, v, beta * *cp);
        }
    }
}

// ---------------------------------------------------------------------------
// Blocked Gauss-Jordan inversion in double-float, for the factors of the
// FP32-swept preconditioner (whose own rounding, 2^-24, is far above the
// 2^-46 of the arithmetic here).  Columns are taken in panels of bw: one CTA
// per matrix runs the bw elimination steps on the n x bw panel alone, with the
// rows resident in shared memory as hi/lo float pairs and the same implicit
// partial pivoting as k_gj_rows (pivot of column k: the unused row with the
// largest |S[i][k]|, ties to the lowest row; rows never move).  The steps of a
// panel multiply the matrix from the left by E = I + sum_j (v_j - e_pj) e_pj^T
// (p_j its pivot rows, v_j the scaled elimination column of step j), and the
// in-place storage leaves E[:, p_j] in panel column j.  So, with T the pivot
// rows taken before the update,
//     A[:, c] <- A[:, c] + (E[:, P] - I[:, P]) T[:, c]     (c outside the panel)
// while the panel columns take E[:, P] itself.  The panel kernel writes
// Pm = E[:, P] (n x bw) and Tm = T (bw x n, its panel columns replaced by the
// identity), and zeroes the pivot rows and the panel columns of A; the
// product A += Pm Tm (k_gjp_update) then completes the panel.  Per panel the
// serial part is bw steps inside one CTA (two block barriers each) instead of
// bw grid-wide exchanges; the rest is one rank-bw product over the whole GPU.
// The result is read through perm / pinv as for k_gj_rows.
// ---------------------------------------------------------------------------
constexpr int GJP_TPB = 512, GJP_WARPS = GJP_TPB / 32, GJP_BMAX = 64;
constexpr size_t GJP_SMEM = 225 * 1024;

struct GjPanelArgs {
    float2 *A0, *A1;  // the matrices, n x n row-major hi/lo pairs, inverted in place
    float2 *P0, *P1;  // E[:, P] of the current panel, n x bw
    float2 *T0, *T1;  // its pivot rows, bw x n
    int *perm;        // [nmat][2 n]: pivot row of each column, then the inverse permutation
    int n, k0, bw;
    int *pivflag;
};

// a + b in double-float (Knuth's two-sum of the high parts, then renormalised)
__device__ __forceinline__ float2 df2_add(float2 a, float2 b)
{
    const float t = __fadd_rn(a.x, b.x);
    const float bb = __fsub_rn(t, a.x);
    const float err = __fadd_rn(__fsub_rn(a.x, __fsub_rn(t, bb)), __fsub_rn(b.x, bb));
    const float l = __fadd_rn(err, __fadd_rn(a.y, b.y));
    const float h = __fadd_rn(t, l);
    return make_float2(h, __fsub_rn(l, __fsub_rn(h, t)));
}

__device__ __forceinline__ double df2_join(float2 a) { return (double)a.x + (double)a.y; }

// a b in double-float (two-product by fused multiply-add; lo*lo dropped)
__device__ __forceinline__ float2 df2_mul(float2 a, float2 b)
{
    const float p = __fmul_rn(a.x, b.x);
    float e = fmaf(a.x, b.x, -p);
    e = fmaf(a.x, b.y, e);
    e = fmaf(a.y, b.x, e);
    const float h = __fadd_rn(p, e);
    return make_float2(h, __fsub_rn(e, __fsub_rn(h, p)));
}

// s - a b in double-float: Knuth's two-sum of s.hi and the rounded product,
// the product's error and s.lo into the low part, then renormalised
__device__ __forceinline__ float2 df2_fms(float2 s, float2 a, float2 b)
{
    const float p = __fmul_rn(a.x, b.x);
    float e = fmaf(a.x, b.x, -p);
    e = fmaf(a.x, b.y, e);
    e = fmaf(a.y, b.x, e);
    const float t = __fsub_rn(s.x, p);
    const float bb = __fsub_rn(t, s.x);
    const float err = __fsub_rn(__fsub_rn(s.x, __fsub_rn(t, bb)), __fadd_rn(p, bb));
    const float l = __fadd_rn(__fsub_rn(s.y, e), err);
    const float h = __fadd_rn(t, l);
    return make_float2(h, __fsub_rn(l, __fsub_rn(h, t)));
}

// One panel.  BW: the allocated panel width (16, 32 or 64; the last panel of a
// matrix may use fewer columns, bw <= BW).  Lanes own columns (a lane holds
// columns lane and lane + 32 when BW = 64; half-warps take two rows at once
// when BW = 16), warps own rows.  A step has three phases between block
// barriers: (1) every thread copies its rows' entries of column j to fcol,
// zeroes them in S and offers the largest unused one as a pivot candidate;
// (2) warp 0 picks the pivot p, forms 1/a in double-float from an FP32
// reciprocal and one Newton step, and scales the pivot row into pr;
// (3) every row takes S[i][c] - fcol[i] pr[c], which with S[i][j] = 0 is also
// the elimination column -f_i / a, and the thread that owns row p then
// overwrites it with pr.  Phase 3 keeps the thread's columns of pr in
// registers and updates GJP_U rows at a time, loads first, so that the
// dependent double-float chains of several rows overlap.
constexpr int GJP_U = 4;

// Pivot candidate of row i with high part x as one ordered 32-bit key: the
// bit pattern of |x| (non-negative floats order as unsigned integers) with its
// low 11 bits replaced by 2047 - i, so that one warp-wide unsigned maximum
// picks the largest |x| to 12 mantissa bits, ties to the lowest row.  Key 0:
// no candidate (every row of a panel has a positive key).
constexpr unsigned int GJP_ROWMASK = 2047u;

__device__ __forceinline__ unsigned int gjp_key(float x, int i)
{
    return ((__float_as_uint(fabsf(x)) >> 11) << 11) | (GJP_ROWMASK - (unsigned int)i);
}

// 1 / a in double-float: the FP32 reciprocal y0 and one Newton step,
// y0 + y0 (1 - a y0), the residual formed exactly by df2_fms
__device__ __forceinline__ float2 df2_recip(float2 a)
{
    const float y0 = __frcp_rn(a.x);
    const float2 r = df2_fms(make_float2(1.f, 0.f), a, make_float2(y0, 0.f));
    const float c = __fmul_rn(y0, r.x);
    const float h = __fadd_rn(y0, c);
    return make_float2(h, __fsub_rn(c, __fsub_rn(h, y0)));
}

template <int BW>
__global__ void __launch_bounds__(GJP_TPB, 1) k_gjp_panel(GjPanelArgs a)
{
    constexpr int TPR = BW >= 32 ? 32 : BW;     // threads per row
    constexpr int NC = BW >= 32 ? BW / 32 : 1;  // columns per thread
    constexpr int RPW = 32 / TPR;               // rows per warp and pass
    constexpr int RSTEP = GJP_WARPS * RPW;      // rows per CTA and pass
    extern __shared__ float2 ps[];  // S: n BW, fcol: n, pr: GJP_BMAX; then used: n bytes
    __shared__ unsigned int ck[GJP_WARPS];
    __shared__ int prow[GJP_BMAX];
    const int mat = blockIdx.x, n = a.n, k0 = a.k0, bw = a.bw;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int cl = lane % TPR, r0 = warp * RPW + lane / TPR;
    // this thread's rows: r0, r0 + RSTEP, ...; nfull of them in whole groups of GJP_U
    const int nrow = r0 < n ? (n - r0 + RSTEP - 1) / RSTEP : 0;
    const int nfull = nrow - nrow % GJP_U;
    float2 *A = mat ? a.A1 : a.A0;
    float2 *Pm = mat ? a.P1 : a.P0;
    float2 *Tm = mat ? a.T1 : a.T0;
    // entry (i, c) of the panel sits at i BW + (c ^ (i mod BW)): rows stay
    // contiguous for the row-wise phases and a column read by consecutive rows
    // falls into distinct banks
    auto sx = [](int i, int c) { return (size_t)i * BW + (c ^ (i & (BW - 1))); };
    int *perm = a.perm + (size_t)mat * 2 * n;
    float2 *S = ps, *fcol = ps + (size_t)n * BW, *pr = fcol + n;
    unsigned char *used = reinterpret_cast<unsigned char *>(pr + GJP_BMAX);
    for (int i = tid; i < n; i += GJP_TPB) used[i] = 0;
    __syncthreads();
    for (int q = tid; q < k0; q += GJP_TPB) used[perm[q]] = 1;
    // the panel into shared memory, GJP_U rows of loads in flight per thread
    for (int ib = r0; ib < n; ib += GJP_U * RSTEP) {
        float2 v[GJP_U][NC];
#pragma unroll
        for (int u = 0; u < GJP_U; u++)
#pragma unroll
            for (int c = 0; c < NC; c++) {
                const int i = ib + u * RSTEP, col = cl + c * 32;
                v[u][c] = (i < n && col < bw) ? A[(size_t)i * n + k0 + col] : make_float2(0.f, 0.f);
            }
#pragma unroll
        for (int u = 0; u < GJP_U; u++)
#pragma unroll
            for (int c = 0; c < NC; c++) {
                const int i = ib + u * RSTEP, col = cl + c * 32;
                if (i < n) S[sx(i, col)] = v[u][c];
            }
    }
    __syncthreads();
    for (int j = 0; j < bw; j++) {
        {  // (1) column j out to fcol and zeroed; the pivot candidates
            unsigned int key = 0;
            for (int i = tid; i < n; i += GJP_TPB) {
                const float2 x = S[sx(i, j)];
                fcol[i] = x;
                S[sx(i, j)] = make_float2(0.f, 0.f);
                if (!used[i]) key = max(key, gjp_key(x.x, i));
            }
            key = __reduce_max_sync(0xffffffffu, key);
            if (lane == 0) ck[warp] = key;
        }
        __syncthreads();
        if (warp == 0) {  // (2) the pivot, 1/a and the scaled pivot row
            const unsigned int key = __reduce_max_sync(0xffffffffu, lane < GJP_WARPS ? ck[lane] : 0u);
            const int p = min((int)(GJP_ROWMASK - (key & GJP_ROWMASK)), n - 1);
            const float2 piv = fcol[p];
            const float2 inv = piv.x != 0.f ? df2_recip(piv) : make_float2(0.f, 0.f);
            for (int c = lane; c < bw; c += 32) pr[c] = c == j ? inv : df2_mul(S[sx(p, c)], inv);
            if (lane == 0) {
                if (piv.x == 0.f) atomicOr(a.pivflag, 1);
                used[p] = 1;
                prow[j] = p;
                perm[k0 + j] = p;
            }
        }
        __syncthreads();
        // (3) every row: S[i][c] -= f_i pr[c]; then the pivot row takes pr
        const int p = prow[j];
        float2 prv[NC];
#pragma unroll
        for (int c = 0; c < NC; c++) prv[c] = cl + c * 32 < bw ? pr[cl + c * 32] : make_float2(0.f, 0.f);
        for (int q = 0; q < nfull; q += GJP_U) {
            float2 sv[GJP_U][NC], fv[GJP_U];
#pragma unroll
            for (int u = 0; u < GJP_U; u++) {
                const int i = r0 + (q + u) * RSTEP;
                fv[u] = fcol[i];
#pragma unroll
                for (int c = 0; c < NC; c++) sv[u][c] = S[sx(i, cl + c * 32)];
            }
#pragma unroll
            for (int u = 0; u < GJP_U; u++)
#pragma unroll
                for (int c = 0; c < NC; c++) sv[u][c] = df2_fms(sv[u][c], fv[u], prv[c]);
#pragma unroll
            for (int u = 0; u < GJP_U; u++) {
                const int i = r0 + (q + u) * RSTEP;
#pragma unroll
                for (int c = 0; c < NC; c++) S[sx(i, cl + c * 32)] = sv[u][c];
            }
        }
        for (int q = nfull; q < nrow; q++) {
            const int i = r0 + q * RSTEP;
            const float2 f = fcol[i];
#pragma unroll
            for (int c = 0; c < NC; c++) {
                float2 *e = S + sx(i, cl + c * 32);
                *e = df2_fms(*e, f, prv[c]);
            }
        }
        if (p >= r0 && (p - r0) % RSTEP == 0)
#pragma unroll
            for (int c = 0; c < NC; c++) S[sx(p, cl + c * 32)] = prv[c];
        __syncthreads();
    }
    // E[:, P] out (ld bw); the pivot rows out (panel columns: the identity), then zeroed
    for (int i = r0; i < n; i += RSTEP)
#pragma unroll
        for (int c = 0; c < NC; c++) {
            const int col = cl + c * 32;
            if (col < bw) Pm[(size_t)i * bw + col] = S[sx(i, col)];
        }
    for (int jr = warp; jr < bw; jr += GJP_WARPS) {
        const float2 *src = A + (size_t)prow[jr] * n;
        float2 *dst = Tm + (size_t)jr * n;
        for (int cb = lane; cb < n; cb += 8 * 32) {
            float2 v[8];
#pragma unroll
            for (int q = 0; q < 8; q++) {
                const int col = cb + q * 32;
                v[q] = col < n ? src[col] : make_float2(0.f, 0.f);
            }
#pragma unroll
            for (int q = 0; q < 8; q++) {
                const int col = cb + q * 32, c2 = col - k0;
                if (col < n)
                    dst[col] = (c2 >= 0 && c2 < bw) ? make_float2(c2 == jr ? 1.f : 0.f, 0.f) : v[q];
            }
        }
    }
    __syncthreads();
    for (int jr = warp; jr < bw; jr += GJP_WARPS) {
        float2 *row = A + (size_t)prow[jr] * n;
        for (int col = lane; col < n; col += 32) row[col] = make_float2(0.f, 0.f);
    }
    for (int i = r0; i < n; i += RSTEP)
#pragma unroll
        for (int c = 0; c < NC; c++) {
            const int col = cl + c * 32;
            if (col < bw) A[(size_t)i * n + k0 + col] = make_float2(0.f, 0.f);
        }
    if (k0 + bw == n) {  // last panel: the inverse permutation
        __syncthreads();
        for (int k = tid; k < n; k += GJP_TPB) perm[n + perm[k]] = k;
    }
}

// The same panel over a cluster of GJC_CS CTAs, rows split in contiguous
// ranges, each range resident in its own CTA's shared memory, so that one
// panel column costs 1/GJC_CS of the update in each CTA.  A pivot step has one
// cluster barrier.  Before it, every CTA moves its rows' entries of column j
// to fcol (zeroing them in S), picks its best unused row and copies that row,
// its pivot entry and its key into a candidate slot of its own (two slots, by
// column parity).  After it, every CTA reads the GJC_CS keys and the winner's
// slot through distributed shared memory, forms 1/a and the scaled pivot row
// itself (the same values in every CTA) and updates its rows.  The parity lets
// a CTA publish column j+1 while slower ones still read column j; a final
// cluster barrier keeps every CTA's shared memory alive until all reads end.
constexpr int GJC_CS = 8;

struct GjcSlot {
    float2 row[GJP_BMAX];
    float2 piv;
    unsigned int key;
};

template <int BW>
__global__ void __cluster_dims__(GJC_CS, 1, 1) __launch_bounds__(GJP_TPB, 1) k_gjc_panel(GjPanelArgs a)
{
    constexpr int TPR = BW >= 32 ? 32 : BW;
    constexpr int NC = BW >= 32 ? BW / 32 : 1;
    constexpr int RPW = 32 / TPR;
    constexpr int RSTEP = GJP_WARPS * RPW;
    namespace cg = cooperative_groups;
    cg::cluster_group cluster = cg::this_cluster();
    extern __shared__ float2 ps[];  // S: chunk BW, fcol: chunk, pr: GJP_BMAX; then used: chunk bytes
    __shared__ GjcSlot slot[2];
    __shared__ unsigned int ck[GJP_WARPS];
    __shared__ int prow[GJP_BMAX];
    const int rank = (int)cluster.block_rank(), mat = blockIdx.x / GJC_CS;
    const int n = a.n, k0 = a.k0, bw = a.bw;
    const int chunk = (n + GJC_CS - 1) / GJC_CS;
    const int rlo = min(n, rank * chunk), nr = min(n, rlo + chunk) - rlo;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int cl = lane % TPR, r0 = warp * RPW + lane / TPR;
    const int nrow = r0 < nr ? (nr - r0 + RSTEP - 1) / RSTEP : 0;
    const int nfull = nrow - nrow % GJP_U;
    float2 *A = mat ? a.A1 : a.A0;
    float2 *Pm = mat ? a.P1 : a.P0;
    float2 *Tm = mat ? a.T1 : a.T0;
    int *perm = a.perm + (size_t)mat * 2 * n;
    auto sx = [](int i, int c) { return (size_t)i * BW + (c ^ (i & (BW - 1))); };
    float2 *S = ps, *fcol = ps + (size_t)chunk * BW, *pr = fcol + chunk;
    unsigned char *used = reinterpret_cast<unsigned char *>(pr + GJP_BMAX);
    for (int i = tid; i < nr; i += GJP_TPB) used[i] = 0;
    __syncthreads();
    for (int q = tid; q < k0; q += GJP_TPB) {
        const int p = perm[q] - rlo;
        if (p >= 0 && p < nr) used[p] = 1;
    }
    // this CTA's rows of the panel into shared memory
    for (int ib = r0; ib < nr; ib += GJP_U * RSTEP) {
        float2 v[GJP_U][NC];
#pragma unroll
        for (int u = 0; u < GJP_U; u++)
#pragma unroll
            for (int c = 0; c < NC; c++) {
                const int i = ib + u * RSTEP, col = cl + c * 32;
                v[u][c] = (i < nr && col < bw) ? A[(size_t)(rlo + i) * n + k0 + col] : make_float2(0.f, 0.f);
            }
#pragma unroll
        for (int u = 0; u < GJP_U; u++)
#pragma unroll
            for (int c = 0; c < NC; c++) {
                const int i = ib + u * RSTEP, col = cl + c * 32;
                if (i < nr) S[sx(i, col)] = v[u][c];
            }
    }
    __syncthreads();
    for (int j = 0; j < bw; j++) {
        const int par = j & 1;
        {  // column j out to fcol and zeroed; this CTA's candidate
            unsigned int key = 0;
            for (int i = tid; i < nr; i += GJP_TPB) {
                const float2 x = S[sx(i, j)];
                fcol[i] = x;
                S[sx(i, j)] = make_float2(0.f, 0.f);
                if (!used[i]) key = max(key, gjp_key(x.x, rlo + i));
            }
            key = __reduce_max_sync(0xffffffffu, key);
            if (lane == 0) ck[warp] = key;
        }
        __syncthreads();
        if (warp == 0) {  // the candidate slot: key, pivot entry and row (column j already zeroed)
            const unsigned int key = __reduce_max_sync(0xffffffffu, lane < GJP_WARPS ? ck[lane] : 0u);
            GjcSlot &sl = slot[par];
            if (key) {
                const int li = (int)(GJP_ROWMASK - (key & GJP_ROWMASK)) - rlo;
                for (int c = lane; c < bw; c += 32) sl.row[c] = S[sx(li, c)];
                if (lane == 0) sl.piv = fcol[li];
            }
            if (lane == 0) sl.key = key;
        }
        cluster.sync();
        if (warp == 0) {  // the winner over the cluster, 1/a and the scaled pivot row
            const unsigned int rk = lane < GJC_CS ? cluster.map_shared_rank(&slot[par], lane)->key : 0u;
            const unsigned int wkey = __reduce_max_sync(0xffffffffu, rk);
            const int w = __ffs(__ballot_sync(0xffffffffu, lane < GJC_CS && rk == wkey)) - 1;
            const GjcSlot *ws = cluster.map_shared_rank(&slot[par], max(w, 0));
            const int p = min((int)(GJP_ROWMASK - (wkey & GJP_ROWMASK)), n - 1);
            const float2 piv = ws->piv;
            const float2 inv = piv.x != 0.f ? df2_recip(piv) : make_float2(0.f, 0.f);
            for (int c = lane; c < bw; c += 32) pr[c] = c == j ? inv : df2_mul(ws->row[c], inv);
            if (lane == 0) {
                if (piv.x == 0.f && rank == 0) atomicOr(a.pivflag, 1);
                prow[j] = p;
                if (rank == 0) perm[k0 + j] = p;
                if (p >= rlo && p < rlo + nr) used[p - rlo] = 1;
            }
        }
        __syncthreads();
        // every row of this CTA: S[i][c] -= f_i pr[c]; then the pivot row takes pr
        const int pl = prow[j] - rlo;
        float2 prv[NC];
#pragma unroll
        for (int c = 0; c < NC; c++) prv[c] = cl + c * 32 < bw ? pr[cl + c * 32] : make_float2(0.f, 0.f);
        for (int q = 0; q < nfull; q += GJP_U) {
            float2 sv[GJP_U][NC], fv[GJP_U];
#pragma unroll
            for (int u = 0; u < GJP_U; u++) {
                const int i = r0 + (q + u) * RSTEP;
                fv[u] = fcol[i];
#pragma unroll
                for (int c = 0; c < NC; c++) sv[u][c] = S[sx(i, cl + c * 32)];
            }
#pragma unroll
            for (int u = 0; u < GJP_U; u++)
#pragma unroll
                for (int c = 0; c < NC; c++) sv[u][c] = df2_fms(sv[u][c], fv[u], prv[c]);
#pragma unroll
            for (int u = 0; u < GJP_U; u++) {
                const int i = r0 + (q + u) * RSTEP;
#pragma unroll
                for (int c = 0; c < NC; c++) S[sx(i, cl + c * 32)] = sv[u][c];
            }
        }
        for (int q = nfull; q < nrow; q++) {
            const int i = r0 + q * RSTEP;
            const float2 f = fcol[i];
#pragma unroll
            for (int c = 0; c < NC; c++) {
                float2 *e = S + sx(i, cl + c * 32);
                *e = df2_fms(*e, f, prv[c]);
            }
        }
        if (pl >= r0 && pl < nr && (pl - r0) % RSTEP == 0)
#pragma unroll
            for (int c = 0; c < NC; c++) S[sx(pl, cl + c * 32)] = prv[c];
        __syncthreads();
    }
    cluster.sync();  // no CTA leaves while another may still read its slots
    // E[:, P] out for this CTA's rows; the pivot rows jr = rank (mod GJC_CS) out
    // (panel columns: the identity), then zeroed with this CTA's panel columns
    for (int i = r0; i < nr; i += RSTEP)
#pragma unroll
        for (int c = 0; c < NC; c++) {
            const int col = cl + c * 32;
            if (col < bw) Pm[(size_t)(rlo + i) * bw + col] = S[sx(i, col)];
        }
    for (int jr = rank + GJC_CS * warp; jr < bw; jr += GJC_CS * GJP_WARPS) {
        const float2 *src = A + (size_t)prow[jr] * n;
        float2 *dst = Tm + (size_t)jr * n;
        for (int cb = lane; cb < n; cb += 8 * 32) {
            float2 v[8];
#pragma unroll
            for (int q = 0; q < 8; q++) {
                const int col = cb + q * 32;
                v[q] = col < n ? src[col] : make_float2(0.f, 0.f);
            }
#pragma unroll
            for (int q = 0; q < 8; q++) {
                const int col = cb + q * 32, c2 = col - k0;
                if (col < n)
                    dst[col] = (c2 >= 0 && c2 < bw) ? make_float2(c2 == jr ? 1.f : 0.f, 0.f) : v[q];
            }
        }
    }
    __syncthreads();
    for (int jr = rank + GJC_CS * warp; jr < bw; jr += GJC_CS * GJP_WARPS) {
        float2 *row = A + (size_t)prow[jr] * n;
        for (int col = lane; col < n; col += 32) row[col] = make_float2(0.f, 0.f);
    }
    for (int i = r0; i < nr; i += RSTEP)
#pragma unroll
        for (int c = 0; c < NC; c++) {
            const int col = cl + c * 32;
            if (col < bw) A[(size_t)(rlo + i) * n + k0 + col] = make_float2(0.f, 0.f);
        }
    if (k0 + bw == n && rank == 0) {  // last panel: the inverse permutation
        __syncthreads();
        for (int k = tid; k < n; k += GJP_TPB) perm[n + perm[k]] = k;
    }
}

// A += Pm Tm (n x bw by bw x n) for one or two matrices (blockIdx.z), in
// 32 x 32 tiles (many CTAs per SM: one rank-bw product is a few microseconds
// of work): the whole bw extent of both operands is staged once, then each
// thread forms 2 x 2 entries with the double-float products and sums of
// k_dfgemm and adds each to its entry in double-float.
constexpr int GU_T = 32;

__global__ void __launch_bounds__(256) k_gjp_update(GjPanelArgs a)
{
    __shared__ float Ah[GJP_BMAX][GU_T + 1], Al[GJP_BMAX][GU_T + 1];
    __shared__ float Bh[GJP_BMAX][GU_T], Bl[GJP_BMAX][GU_T];
    const int n = a.n, bw = a.bw;
    float2 *C = blockIdx.z ? a.A1 : a.A0;
    const float2 *P = blockIdx.z ? a.P1 : a.P0;
    const float2 *T = blockIdx.z ? a.T1 : a.T0;
    const int tx = threadIdx.x % 16, ty = threadIdx.x / 16;
    const int row0 = blockIdx.y * GU_T, col0 = blockIdx.x * GU_T;
    for (int e = threadIdx.x; e < GU_T * bw; e += 256) {
        const int r = e / bw, kk = e - r * bw, gr = row0 + r;
        const float2 v = gr < n ? P[(size_t)gr * bw + kk] : make_float2(0.f, 0.f);
        Ah[kk][r] = v.x;
        Al[kk][r] = v.y;
    }
    for (int e = threadIdx.x; e < GU_T * bw; e += 256) {
        const int kk = e / GU_T, cc = e - kk * GU_T, gc = col0 + cc;
        const float2 v = gc < n ? T[(size_t)kk * n + gc] : make_float2(0.f, 0.f);
        Bh[kk][cc] = v.x;
        Bl[kk][cc] = v.y;
    }
    __syncthreads();
    float hi[2][2] = {{0.f, 0.f}, {0.f, 0.f}}, lo[2][2] = {{0.f, 0.f}, {0.f, 0.f}};
    for (int kk = 0; kk < bw; kk++) {
        const float ah[2] = {Ah[kk][ty * 2], Ah[kk][ty * 2 + 1]}, al[2] = {Al[kk][ty * 2], Al[kk][ty * 2 + 1]};
        const float bh[2] = {Bh[kk][tx * 2], Bh[kk][tx * 2 + 1]}, bl[2] = {Bl[kk][tx * 2], Bl[kk][tx * 2 + 1]};
#pragma unroll
        for (int i = 0; i < 2; i++)
#pragma unroll
            for (int j = 0; j < 2; j++) {
                const float p = __fmul_rn(ah[i], bh[j]);
                float e = fmaf(ah[i], bh[j], -p);
                e = fmaf(ah[i], bl[j], e);
                e = fmaf(al[i], bh[j], e);
                const float sm = __fadd_rn(hi[i][j], p);
                const float bp = __fsub_rn(sm, hi[i][j]);
                const float err = __fadd_rn(__fsub_rn(hi[i][j], __fsub_rn(sm, bp)), __fsub_rn(p, bp));
                hi[i][j] = sm;
                lo[i][j] = __fadd_rn(lo[i][j], __fadd_rn(err, e));
            }
    }
#pragma unroll
    for (int i = 0; i < 2; i++) {
        const int gr = row0 + ty * 2 + i;
        if (gr >= n) continue;
#pragma unroll
        for (int j = 0; j < 2; j++) {
            const int gc = col0 + tx * 2 + j;
            if (gc < n) {
                float2 *cp = C + (size_t)gr * n + gc;
                *cp = df2_add(*cp, make_float2(hi[i][j], lo[i][j]));
            }
        }
    }
}

// FP64 matrix -> hi/lo pairs in place (each element's 8 bytes rewritten by
// the thread that read them)
__global__ void k_df2_split_inplace(double *x, size_t cnt)
{
    for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < cnt; e += (size_t)gridDim.x * blockDim.x) {
        const float2 v = df2_split(x[e]);
        reinterpret_cast<float2 *>(x)[e] = v;
    }
}

// A^-1[k][j] = S[perm[k]][pinv[j]], from the hi/lo pairs into FP64
__global__ void k_gjp_unperm(const float2 *__restrict__ S, const int *__restrict__ perm, double *__restrict__ D,
                             int n)
{
    const int *pinv = perm + n;
    for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < (size_t)n * n;
         e += (size_t)gridDim.x * blockDim.x) {
        const int k = (int)(e / n), j = (int)(e % n);
        D[e] = df2_join(S[(size_t)perm[k] * n + pinv[j]]);
    }
}

// Batched block products of the factorisation: FP64 when the sweeps are FP64,
// double-float when they sweep FP32 copies of the factors (whose own rounding
// is 2^-24, so the factors' 2^-46 is far below what the sweeps see).
static int gemm_batch(bfs_ctx *c, std::vector<const double *> &A, std::vector<const double *> &B,
                      std::vector<double *> &C, double alpha, double beta, cudaStream_t s)
{
    const int nb = c->nb;
    const bool df = c->opt.precond_precision == BFS_FP32C && c->opt.surface_tension == 0.0;
    for (size_t o = 0; o < A.size(); o += GB_MAX) {
        GemmBatch gb;
        int cnt = (int)std::min<size_t>(GB_MAX, A.size() - o);
        for (int i = 0; i < cnt; i++) { gb.A[i] = A[o + i]; gb.B[i] = B[o + i]; gb.C[i] = C[o + i]; }
        dim3 grid((nb + TN - 1) / TN, (nb + TM - 1) / TM, cnt);
        if (df) k_dfgemm<<<grid, 256, 0, s>>>(gb, nb, alpha, beta);
        else k_dgemm<<<grid, 256, 0, s>>>(gb, nb, alpha, beta);
        c->launches++;
    }
    BFS_CUDA_TRY(c, cudaGetLastError());
    return BFS_OK;
}

// ---------------------------------------------------------------------------
// One cooperative launch per apply: permutation in, forward sweep, backward
// sweep, permutation out, with a grid barrier between dependent slices.  The
// launch is cooperative, so every block is resident and the barrier always
// completes; its spin is still bounded (about one second), after which the
// kernel raises bit 2 of the context flag and returns.
// ---------------------------------------------------------------------------
struct CoopBar {
    unsigned int count;
    unsigned int gen;
};

// Barrier of the Gauss-Jordan kernel (one per pivot column).
__device__ bool grid_sync(CoopBar *b, int *flag, unsigned int spin)
{
    __shared__ int ok;
    __syncthreads();
    if (threadIdx.x == 0) {
        ok = 1;
        volatile unsigned int *vgen = &b->gen;
        const unsigned int g = *vgen;
        __threadfence();
        const unsigned int arrived = atomicAdd(&b->count, 1u);
        if (arrived == gridDim.x - 1) {
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

// Barrier of the apply kernel: the counter only grows within a launch (it is
// zeroed before each launch); barrier number e completes when the counter
// reaches e * gridDim.x.  Arrival is a release add, the wait an acquire load,
// so no separate fences are needed.  The wait is bounded (about a second);
// on timeout bit 2 of the flag is raised and false is returned.
__device__ __forceinline__ bool grid_sync_epoch(unsigned int *count, unsigned int epoch, int *flag,
                                                unsigned int spin)
{
    __shared__ int ok;
    __syncthreads();
    if (threadIdx.x == 0) {
        ok = 1;
        unsigned int old;
        asm volatile("atom.add.release.gpu.u32 %0, [%1], 1;" : "=r"(old) : "l"(count) : "memory");
        const unsigned int target = epoch * gridDim.x;
        unsigned int v = old + 1, spins = 0;
        while (v < target) {
            asm volatile("ld.acquire.gpu.u32 %0, [%1];" : "=r"(v) : "l"(count) : "memory");
            if (v >= target) break;
            if (++spins > spin) {
                atomicOr(flag, 2);
                ok = 0;
                break;
            }
            __nanosleep(16);
        }
    }
    __syncthreads();
    return ok;
}

struct ApplyArgs {
    const double *pc;
    const double *r;
    double *z, *x, *y;
    int nb, NB, M, h;
    CoopBar *bar;
    int *flag;
    unsigned int spin;
};

constexpr int AP_TPB = 1024;
constexpr int AP_WARPS = AP_TPB / 32;
constexpr int AP_NQ = 4;  // columns per lane and block row (a warp covers <= 128 columns)

// One CTA per SM.  Rows of a slice are dealt out round-robin over the CTAs and
// within a CTA over groups of warps; the warps of a group split the columns
// of the row (at most 128 per warp, 4 per lane), and every lane first issues
// the loads of two blocks at once, so a step costs about two memory latencies
// rather than one per column chunk.  Partial dots meet in shared memory.
__global__ void __launch_bounds__(AP_TPB, 1) k_apply_coop(ApplyArgs a)
{
    __shared__ double red[AP_WARPS];
    const int nb = a.nb, NB = a.NB, M = a.M, h = a.h, nd = 2 * h + 1;
    const size_t bsz = (size_t)nb * nb;
    const int n = 3 * NB * M;
    const int gtid = blockIdx.x * blockDim.x + threadIdx.x, gstride = gridDim.x * blockDim.x;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int rpc = (nb + gridDim.x - 1) / gridDim.x;                   // rows per CTA
    const int wpg = min(AP_WARPS, (nb + 32 * AP_NQ - 1) / (32 * AP_NQ)); // warps per row
    const int groups = AP_WARPS / wpg;                                   // rows per round
    const int grp = warp / wpg, wig = warp - grp * wpg;
    const int cw = (nb + wpg - 1) / wpg;
    const int c0 = wig * cw, c1 = min(nb, c0 + cw);
    unsigned int *cnt = &a.bar->count;
    unsigned int epoch = 0;
    auto prefetch_step = [&](int pass, int k) {
        if (k < 0 || k >= M) return;
        int lo2, hi2;
        if (pass == 0) { lo2 = max(0, k - h); hi2 = k - 1; }
        else { lo2 = k; hi2 = min(M - 1, k + h); }
        for (int rb = 0; rb < rpc; rb += groups) {
            const int rr = rb + grp;
            if (grp >= groups || rr >= rpc) continue;
            const int row = blockIdx.x + rr * gridDim.x;
            if (row >= nb) continue;
            for (int m = lo2; m <= hi2; m++) {
                const double *rp = a.pc + ((size_t)k * nd + (m - k + h)) * bsz + (size_t)row * nb;
                for (int c = c0 + lane * 16; c < c1; c += 32 * 16)  // one 128-byte line per 16 doubles
                    asm volatile("prefetch.global.L2 [%0];" ::"l"(rp + c));
            }
        }
    };
    prefetch_step(0, 0);
    prefetch_step(0, 1);
    for (int e = gtid; e < n; e += gstride) {
        int g = e / (NB * M), rem = e % (NB * M), l = rem / NB, p = rem % NB;
        __stcg(a.x + (size_t)l * nb + g * NB + p, a.r[e]);
    }
    if (!grid_sync_epoch(cnt, ++epoch, a.flag, a.spin)) return;
    for (int pass = 0; pass < 2; pass++) {
        for (int kk = 0; kk < M; kk++) {
            const int k = pass == 0 ? kk : M - 1 - kk;
            {
                const int k2 = pass == 0 ? k + 2 : k - 2;
                if (k2 >= 0 && k2 < M) prefetch_step(pass, k2);
                else if (pass == 0) prefetch_step(1, M - 1 - (k2 - M));
            }
            int lo, hi;
            if (pass == 0) { lo = max(0, k - h); hi = k - 1; }   // L_ki, i < k, against y_i
            else { lo = k; hi = min(M - 1, k + h); }             // D_k^-1 y_k, W_kj x_j
            // same trip count for every thread of the CTA (the body has barriers)
            for (int rb = 0; rb < rpc; rb += groups) {
                const int rr = rb + grp;
                const int row = (grp < groups && rr < rpc) ? blockIdx.x + rr * gridDim.x : nb;
                double acc = 0.0;
                if (row < nb) {
                    for (int m = lo; m <= hi; m += 2) {
                        double fa[2][AP_NQ], va[2][AP_NQ];
#pragma unroll
                        for (int bb = 0; bb < 2; bb++) {
                            const int mm = m + bb;
                            const bool ok = mm <= hi;
                            const double *rp = a.pc + ((size_t)k * nd + (mm - k + h)) * bsz + (size_t)row * nb;
                            const double *v = (pass == 0 || mm == k) ? a.y + (size_t)mm * nb : a.x + (size_t)mm * nb;
#pragma unroll
                            for (int q = 0; q < AP_NQ; q++) {
                                const int c = c0 + lane + 32 * q;
                                const bool in = ok && c < c1;
                                fa[bb][q] = in ? __ldg(rp + c) : 0.0;
                                va[bb][q] = in ? __ldcg(v + c) : 0.0;
                            }
                        }
#pragma unroll
                        for (int bb = 0; bb < 2; bb++) {
                            const double sg = (pass == 1 && m + bb == k) ? 1.0 : -1.0;
                            double t = 0.0;
#pragma unroll
                            for (int q = 0; q < AP_NQ; q++) t = fma(fa[bb][q], va[bb][q], t);
                            acc = fma(sg, t, acc);
                        }
                    }
                }
                for (int o = 16; o > 0; o >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, o);
                if (lane == 0) red[warp] = acc;
                __syncthreads();
                if (wig == 0 && lane == 0 && row < nb) {
                    double s = 0.0;
                    for (int w = 0; w < wpg; w++) s += red[grp * wpg + w];  // grp < groups here
                    if (pass == 0) __stcg(a.y + (size_t)k * nb + row, __ldcg(a.x + (size_t)k * nb + row) + s);
                    else __stcg(a.x + (size_t)k * nb + row, s);
                }
                __syncthreads();
            }
            if (!grid_sync_epoch(cnt, ++epoch, a.flag, a.spin)) return;
        }
    }
    for (int e = gtid; e < n; e += gstride) {
        int g = e / (NB * M), rem = e % (NB * M), l = rem / NB, p = rem % NB;
        a.z[e] = __ldcg(a.x + (size_t)l * nb + g * NB + p);
    }
}

static PcArgs pc_args(const bfs_ctx *c, int h)
{
    PcArgs a;
    a.N = c->N; a.M = c->M; a.half = c->half; a.h = h; a.nb = 3 * (c->N + 1);
    a.x1 = c->x1; a.y1 = c->y1; a.dx = c->dx; a.dy = c->dy; a.F = c->F; a.n_rad = c->opt.n_rad;
    a.xhi = c->x1 + (c->N - 1) * c->dx;
    a.yhi = c->y1 + (c->M - 1) * c->dy;
    a.ylo = c->half ? -a.yhi : c->y1;
    a.tau = c->opt.surface_tension;
    return a;
}

void precond_free(bfs_ctx *c)
{
    gm_graphs_clear(c);  // the graphs captured the factor and sweep buffers
    cudaFree(c->d_pc);
    cudaFree(c->d_pc32);
    cudaFree(c->d_flow);
    cudaFree(c->d_tasks);
    c->d_pc32 = nullptr;
    c->d_flow = nullptr;
    c->d_tasks = nullptr;
    c->h_tasks.clear();
    c->sweep_table = 0;
    c->sweep_ntags = 0;
    c->pc_twist = -1;
    cudaFree(c->d_gj);
    cudaFree(c->d_gjscr);
    cudaFree(c->d_gjdata);
    c->d_gjscr = nullptr;
    c->d_gjdata = nullptr;
    cudaFree(c->d_rowsum5);
    cudaFree(c->d_pivflag);
    cudaFree(c->d_perm_a);
    c->d_pc = c->d_gj = c->d_rowsum5 = c->d_perm_a = c->d_perm_b = nullptr;
    c->d_pivflag = nullptr;
    c->pc_ready = 0;
}

static unsigned int wait_spin(const bfs_ctx *c)
{
    return c->opt.wait_polls > 0 ? (unsigned int)c->opt.wait_polls : (1u << 24);
}

// Gauss-Jordan inversion of one or two n x n matrices already loaded as
// [D | I] into set.X0; returns in *res the buffers holding [. | D^-1].
static int gj_invert(bfs_ctx *c, GjSet set, int n, double **res, cudaStream_t s)
{
    int gj_per_sm = 0;
    BFS_CUDA_TRY(c, cudaOccupancyMaxActiveBlocksPerMultiprocessor(&gj_per_sm, k_gj_coop, 256, 0));
    if (gj_per_sm < 1) {
        c->err = "Gauss-Jordan kernel cannot be resident";
        return BFS_ECUDA;
    }
    int grid = std::min(num_sms(c->device) * std::min(gj_per_sm, 2), n * set.nmat);
    grid -= grid % set.nmat;
    CoopBar *bar = reinterpret_cast<CoopBar *>(c->d_pivflag + 4);
    BFS_CUDA_TRY(c, cudaMemsetAsync(bar, 0, 2 * sizeof(unsigned int), s));
    int nv = n;
    int *pf = c->d_pivflag, *fl = c->d_flag;
    unsigned int spin = wait_spin(c);
    void *args[] = {&set, &nv, &pf, &bar, &fl, &spin};
    BFS_CUDA_TRY(c, cudaLaunchCooperativeKernel((const void *)k_gj_coop, dim3(grid), dim3(256), args, 0, s));
    c->launches++;
    for (int i = 0; i < set.nmat; i++) res[i] = (n % 2 == 0) ? set.X0[i] : set.X1[i];  // after n ping-pong steps
    return BFS_OK;
}

// In-place inversion of one or two n x n matrices (row-major, contiguous) by
// k_gj_rows, results gathered into dst[i] (which may be another buffer).
// Returns 1 if the kernel's tiles do not take n (the caller falls back).
static int gj_rows_invert(bfs_ctx *c, double *const *work, double *const *dst, int nmat, int n, cudaStream_t s)
{
    const int G = num_sms(c->device) / nmat;
    const int Geff = std::min(G, n), rmax = (n + Geff - 1) / Geff;
    const size_t smem = sizeof(double) * (size_t)(rmax + 1) * n;
    if (rmax > GJR_MAXR || smem > 200 * 1024) return 1;
    BFS_CUDA_TRY(c, cudaFuncSetAttribute((const void *)k_gj_rows, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         200 * 1024));
    int per_sm = 0;
    BFS_CUDA_TRY(c, cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_gj_rows, GJR_TPB, smem));
    if (per_sm < 1 || per_sm * num_sms(c->device) < G * nmat) return 1;
    GjRowsArgs a;
    a.S0 = work[0];
    a.S1 = nmat > 1 ? work[1] : work[0];
    a.n = n; a.nmat = nmat; a.G = G;
    const int NS = nmat * G;
    a.slot = reinterpret_cast<unsigned long long *>(c->d_gjscr);
    a.perm = reinterpret_cast<int *>(a.slot + 4 * (size_t)NS);
    a.data = c->d_gjdata;
    a.pivflag = c->d_pivflag;
    a.flag = c->d_flag;
    a.spin = c->opt.wait_polls > 0 ? (unsigned int)c->opt.wait_polls : (1u << 24);
    BFS_CUDA_TRY(c, cudaMemsetAsync(a.slot, 0, sizeof(unsigned long long) * 4 * (size_t)NS, s));
    void *args[] = {&a};
    BFS_CUDA_TRY(c, cudaLaunchCooperativeKernel((const void *)k_gj_rows, dim3(G * nmat), dim3(GJR_TPB), args,
                                                smem, s));
    c->launches++;
    for (int i = 0; i < nmat; i++) {
        k_gj_unperm<<<1024, 256, 0, s>>>(work[i], a.perm + (size_t)i * 2 * n, dst[i], n);
        c->launches++;
    }
    BFS_CUDA_TRY(c, cudaGetLastError());
    return BFS_OK;
}

// In-place inversion of one or two n x n matrices (row-major, contiguous) by
// the blocked double-float kernels, results gathered into dst[i].  Returns 1
// if a panel of 8 columns does not fit in shared memory (the caller falls
// back).  Scratch: the perm / pinv words after the slots of d_gjscr, Pm and Tm
// in d_gjdata.
static int gj_panel_invert(bfs_ctx *c, double *const *work, double *const *dst, int nmat, int n, cudaStream_t s,
                           bool allow_cluster = true)
{
    // widest panel whose rows fit: BW columns of float pairs per row, plus fcol,
    // the pivot row and the used flags
    auto fits = [&](int bwid) {
        return sizeof(float2) * ((size_t)n * bwid + n + GJP_BMAX) + (size_t)n <= GJP_SMEM;
    };
    // the cluster form (panels of 64, rows over GJC_CS CTAs) from 128 rows up,
    // when a cluster with its shared memory can be resident
    const int chunk = (n + GJC_CS - 1) / GJC_CS;
    const size_t csmem = sizeof(float2) * ((size_t)chunk * 64 + chunk + GJP_BMAX) + (size_t)chunk;
    bool clus = allow_cluster && n >= 128 && n <= (int)GJP_ROWMASK + 1 && csmem <= GJP_SMEM;
    if (clus) {
        clus = cudaFuncSetAttribute((const void *)k_gjc_panel<64>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                    (int)GJP_SMEM) == cudaSuccess;
        int ncl = 0;
        if (clus) {
            cudaLaunchConfig_t cfg = {};
            cfg.gridDim = dim3(nmat * GJC_CS);
            cfg.blockDim = dim3(GJP_TPB);
            cfg.dynamicSmemBytes = csmem;
            cudaLaunchAttribute at;
            at.id = cudaLaunchAttributeClusterDimension;
            at.val.clusterDim.x = GJC_CS;
            at.val.clusterDim.y = 1;
            at.val.clusterDim.z = 1;
            cfg.attrs = &at;
            cfg.numAttrs = 1;
            clus = cudaOccupancyMaxActiveClusters(&ncl, (const void *)k_gjc_panel<64>, &cfg) == cudaSuccess &&
                   ncl >= 1;
        }
        cudaGetLastError();
    }
    const int BW = clus ? 64 : fits(64) ? 64 : fits(32) ? 32 : fits(16) ? 16 : 0;
    if (!BW || n > (int)GJP_ROWMASK + 1) return 1;
    const void *fn = BW == 64 ? (const void *)k_gjp_panel<64>
                   : BW == 32 ? (const void *)k_gjp_panel<32> : (const void *)k_gjp_panel<16>;
    if (!clus)
        BFS_CUDA_TRY(c, cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)GJP_SMEM));
    const size_t smem = clus ? csmem : sizeof(float2) * ((size_t)n * BW + n + GJP_BMAX) + (size_t)n;
    GjPanelArgs a;
    // the FP64 inputs become hi/lo pairs in place (same bytes per entry)
    for (int i = 0; i < nmat; i++) {
        k_df2_split_inplace<<<1024, 256, 0, s>>>(work[i], (size_t)n * n);
        c->launches++;
    }
    a.A0 = reinterpret_cast<float2 *>(work[0]);
    a.A1 = reinterpret_cast<float2 *>(nmat > 1 ? work[1] : work[0]);
    float2 *pt = reinterpret_cast<float2 *>(c->d_gjdata);
    a.P0 = pt;
    a.T0 = pt + (size_t)n * BW;
    a.P1 = nmat > 1 ? pt + 2 * (size_t)n * BW : a.P0;
    a.T1 = nmat > 1 ? pt + 3 * (size_t)n * BW : a.T0;
    a.perm = reinterpret_cast<int *>(static_cast<unsigned long long *>(c->d_gjscr) + 4 * (size_t)num_sms(c->device));
    a.n = n;
    a.pivflag = c->d_pivflag;
    const dim3 ug((n + GU_T - 1) / GU_T, (n + GU_T - 1) / GU_T, nmat);
    for (int k0 = 0; k0 < n; k0 += BW) {
        a.k0 = k0;
        a.bw = std::min(BW, n - k0);
        if (clus) k_gjc_panel<64><<<nmat * GJC_CS, GJP_TPB, smem, s>>>(a);
        else if (BW == 64) k_gjp_panel<64><<<nmat, GJP_TPB, smem, s>>>(a);
        else if (BW == 32) k_gjp_panel<32><<<nmat, GJP_TPB, smem, s>>>(a);
        else k_gjp_panel<16><<<nmat, GJP_TPB, smem, s>>>(a);
        k_gjp_update<<<ug, 256, 0, s>>>(a);
        c->launches += 2;
    }
    for (int i = 0; i < nmat; i++) {
        k_gjp_unperm<<<1024, 256, 0, s>>>(reinterpret_cast<const float2 *>(work[i]), a.perm + (size_t)i * 2 * n, dst[i], n);
        c->launches++;
    }
    BFS_CUDA_TRY(c, cudaGetLastError());
    return BFS_OK;
}

// Scratch doubles of d_gjdata for matrices of up to nmax rows: the candidate
// rows of k_gj_rows (2 parities x CTAs) or Pm and Tm of two blocked inversions.
static size_t gj_data_doubles(int sms, int nmax)
{
    return std::max<size_t>(2 * (size_t)sms, 4 * (size_t)GJP_BMAX) * (size_t)nmax;
}

int precond_factor(bfs_ctx *c, int half_band, cudaStream_t s)
{
    int h = half_band >= 0 ? half_band : c->opt.half_band;
    if (h < 0) h = 0;
    if (h > c->M - 1) h = c->M - 1;
    if (h > 16) h = 16;  // the sweep kernel takes at most 17 blocks per row
    precond_free(c);
    const int nb = 3 * (c->N + 1), M = c->M, nd = 2 * h + 1;
    c->nb = nb;
    c->pc_h = h;
    // the two-ended order whenever the FP32 task-table sweeps can run its two chains
    int rc = sweep_twist_ok(c, h);
    if (rc < 0) return rc;
    const int twist = rc == 1 ? (M - h) / 2 : -1;
    const size_t bsz = (size_t)nb * nb;
    if (cudaMalloc(&c->d_pc, sizeof(double) * bsz * M * nd) != cudaSuccess) {
        cudaGetLastError();
        c->err = "preconditioner storage: out of device memory";
        return BFS_ENOMEM;
    }
    // Gauss-Jordan buffers: two matrices of nb x 2nb ping-pong, or the h nb x 2 h nb
    // middle system; then h blocks of GEMM scratch
    const size_t gj_doubles = std::max<size_t>(8 * bsz, twist >= 0 ? 4 * (size_t)h * h * bsz : 0);
    // GEMM scratch: W and L of up to two eliminations at once (4 h blocks)
    BFS_CUDA_TRY(c, cudaMalloc(&c->d_gj, sizeof(double) * (gj_doubles + bsz * 4 * (size_t)(h > 0 ? h : 1))));
    BFS_CUDA_TRY(c, cudaMalloc(&c->d_rowsum5, sizeof(double) * (size_t)c->Nt));
    {  // dataflow Gauss-Jordan: 2 parities x CTAs of slots, 2 x (perm, pinv) of the largest
       // matrix, and 2 parities x CTAs candidate rows
        const int G = num_sms(c->device), nmax = std::max(nb, twist >= 0 ? h * nb : nb);
        BFS_CUDA_TRY(c, cudaMalloc(&c->d_gjscr, sizeof(unsigned long long) * 4 * (size_t)G +
                                                    sizeof(int) * 4 * (size_t)nmax));
        BFS_CUDA_TRY(c, cudaMalloc(&c->d_gjdata, sizeof(double) * gj_data_doubles(G, nmax)));
    }
    BFS_CUDA_TRY(c, cudaMalloc(&c->d_pivflag, sizeof(int) * 8));  // [0] pivot flag, [4..5] grid barrier
    BFS_CUDA_TRY(c, cudaMalloc(&c->d_perm_a, sizeof(double) * 2 * (size_t)c->n));
    c->d_perm_b = c->d_perm_a + c->n;
    BFS_CUDA_TRY(c, cudaMemsetAsync(c->d_pc, 0, sizeof(double) * bsz * M * nd, s));
    BFS_CUDA_TRY(c, cudaMemsetAsync(c->d_pivflag, 0, sizeof(int) * 8, s));

    PcArgs a = pc_args(c, h);
    k_rowsum5<<<(c->Nt + 127) / 128, 128, 0, s>>>(a, c->d_rowsum5);
    c->launches++;
    k_form_dense<<<dim3(c->N - 1, nd, M), 128, sizeof(double) * (2 * c->N + 1), s>>>(a, c->d_pc,
                                                                                  c->d_rowsum5);
    c->launches++;
    k_form_sparse<<<(M * nb + 127) / 128, 128, 0, s>>>(a, c->d_pc);
    c->launches++;
    if (a.tau != 0.0) {
        k_form_tension<<<(M * (c->N - 1) + 127) / 128, 128, 0, s>>>(a, c->d_pc);
        c->launches++;
    }
    BFS_CUDA_TRY(c, cudaGetLastError());

    auto B = [&](int l, int m) { return c->d_pc + ((size_t)l * nd + (m - l + h)) * bsz; };
    double *tmp = c->d_gj + gj_doubles;
    // FP32 sweeps: blocked double-float inversions (FP64 ones otherwise)
    const bool df = c->opt.precond_precision == BFS_FP32C && c->opt.surface_tension == 0.0;
    // D_k^-1 in place for the one or two diagonal blocks listed
    auto invert_diag = [&](const int *ks, int cnt) -> int {
        {  // rows in shared memory, no grid barrier
            double *work[2], *dst[2];
            for (int i = 0; i < cnt; i++) {
                work[i] = c->d_gj + (size_t)i * bsz;
                dst[i] = B(ks[i], ks[i]);
                BFS_CUDA_TRY(c, cudaMemcpyAsync(work[i], dst[i], sizeof(double) * bsz, cudaMemcpyDeviceToDevice, s));
            }
            int r = df ? gj_panel_invert(c, work, dst, cnt, nb, s) : 1;
            if (r == 1) r = gj_rows_invert(c, work, dst, cnt, nb, s);
            if (r <= 0) return r;
        }
        GjSet set;
        set.nmat = cnt;
        for (int i = 0; i < cnt; i++) {
            set.X0[i] = c->d_gj + (size_t)i * 4 * bsz;
            set.X1[i] = set.X0[i] + 2 * bsz;
            k_gj_put<<<512, 256, 0, s>>>(B(ks[i], ks[i]), set.X0[i], nb, nb, 0, 0);
            k_gj_eye<<<512, 256, 0, s>>>(set.X0[i], nb);
            c->launches += 2;
        }
        double *res[2];
        int r = gj_invert(c, set, nb, res, s);
        if (r) return r;
        for (int i = 0; i < cnt; i++) {
            k_gj_get<<<512, 256, 0, s>>>(res[i], B(ks[i], ks[i]), nb, nb, 0, 0);
            c->launches++;
        }
        BFS_CUDA_TRY(c, cudaGetLastError());
        return BFS_OK;
    };
    // eliminate slice k (D_k^-1 in place) from the coupled slices lo..hi
    // eliminate slice k (D_k^-1 in place) from the coupled slices lo..hi, for one
    // or two slices of the two chains at once:
    //   W_kj = D_k^-1 S_kj and L_ik = S_ik D_k^-1 (one launch for every product),
    //   S_ij -= S_ik W_kj (one launch, or one per chain where both would update
    //   the same middle blocks), then W and L into their slots
    struct Elim { int k, lo, hi; };
    auto eliminate = [&](const Elim *es, int cnt) -> int {
        std::vector<const double *> A, Bm;
        std::vector<double *> C;
        std::vector<std::pair<double *, double *>> back;  // (slot, scratch)
        double *t = tmp;
        for (int q = 0; q < cnt; q++) {
            const Elim &e = es[q];
            for (int j = e.lo; j <= e.hi; j++) {
                A.push_back(B(e.k, e.k)); Bm.push_back(B(e.k, j)); C.push_back(t);
                back.push_back({B(e.k, j), t});
                t += bsz;
            }
            for (int i = e.lo; i <= e.hi; i++) {
                A.push_back(B(i, e.k)); Bm.push_back(B(e.k, e.k)); C.push_back(t);
                back.push_back({B(i, e.k), t});
                t += bsz;
            }
        }
        if (A.empty()) return BFS_OK;
        int r = gemm_batch(c, A, Bm, C, 1.0, 0.0, s);
        if (r) return r;
        // S_ij -= S_ik W_kj (S_ik still the unscaled block, W from the scratch)
        const bool overlap = cnt == 2 && es[0].hi >= es[1].lo && es[1].hi >= es[0].lo;
        A.clear(); Bm.clear(); C.clear();
        t = tmp;
        for (int q = 0; q < cnt; q++) {
            const Elim &e = es[q];
            const int w = e.hi - e.lo + 1;
            for (int i = e.lo; i <= e.hi; i++)
                for (int j = e.lo; j <= e.hi; j++) {
                    A.push_back(B(i, e.k)); Bm.push_back(t + (size_t)(j - e.lo) * bsz); C.push_back(B(i, j));
                }
            t += 2 * (size_t)w * bsz;
            if (overlap && q == 0) {
                if ((r = gemm_batch(c, A, Bm, C, -1.0, 1.0, s))) return r;
                A.clear(); Bm.clear(); C.clear();
            }
        }
        if (!A.empty() && (r = gemm_batch(c, A, Bm, C, -1.0, 1.0, s))) return r;
        for (auto &bk : back)
            BFS_CUDA_TRY(c, cudaMemcpyAsync(bk.first, bk.second, sizeof(double) * bsz, cudaMemcpyDeviceToDevice, s));
        return BFS_OK;
    };
    if (twist < 0) {
        for (int k = 0; k < M; k++) {
            if ((rc = invert_diag(&k, 1))) return rc;
            const Elim e{k, k + 1, std::min(M - 1, k + h)};
            if (e.hi >= e.lo && (rc = eliminate(&e, 1))) return rc;
        }
    } else {
        const int t0 = twist, t1 = twist + h;
        for (int i = 0; i < std::max(t0, M - t1); i++) {
            int ks[2], cnt = 0;
            const int kt = i < t0 ? i : -1, kb = M - 1 - i >= t1 ? M - 1 - i : -1;
            if (kt >= 0) ks[cnt++] = kt;
            if (kb >= 0) ks[cnt++] = kb;
            if ((rc = invert_diag(ks, cnt))) return rc;
            Elim es[2];
            int ne = 0;
            if (kt >= 0 && kt + 1 <= std::min(M - 1, kt + h)) es[ne++] = {kt, kt + 1, std::min(M - 1, kt + h)};
            if (kb >= 0 && std::max(0, kb - h) <= kb - 1) es[ne++] = {kb, std::max(0, kb - h), kb - 1};
            if (ne && (rc = eliminate(es, ne))) return rc;
        }
        // the middle system C (slices t0..t1-1, h nb square) inverted whole
        const int hn = h * nb;
        {
            double *work = c->d_gj, *out = c->d_gj + (size_t)hn * hn;
            for (int ia = 0; ia < h; ia++)
                for (int ib = 0; ib < h; ib++) {
                    k_blk_put<<<512, 256, 0, s>>>(B(t0 + ia, t0 + ib), work, nb, hn, ia, ib);
                    c->launches++;
                }
            rc = df ? gj_panel_invert(c, &work, &out, 1, hn, s) : 1;
            if (rc == 1) rc = gj_rows_invert(c, &work, &out, 1, hn, s);
            if (rc < 0) return rc;
            if (rc == 0) {
                for (int ia = 0; ia < h; ia++)
                    for (int ib = 0; ib < h; ib++) {
                        k_blk_get<<<512, 256, 0, s>>>(out, B(t0 + ia, t0 + ib), nb, hn, ia, ib);
                        c->launches++;
                    }
                BFS_CUDA_TRY(c, cudaGetLastError());
            }
        }
        if (rc == 1) {
        GjSet set;
        set.nmat = 1;
        set.X0[0] = c->d_gj;
        set.X1[0] = c->d_gj + 2 * (size_t)hn * hn;
        for (int ia = 0; ia < h; ia++)
            for (int ib = 0; ib < h; ib++) {
                k_gj_put<<<512, 256, 0, s>>>(B(t0 + ia, t0 + ib), set.X0[0], nb, hn, ia, ib);
                c->launches++;
            }
        k_gj_eye<<<1024, 256, 0, s>>>(set.X0[0], hn);
        c->launches++;
        double *res[2];
        if ((rc = gj_invert(c, set, hn, res, s))) return rc;
        for (int ia = 0; ia < h; ia++)
            for (int ib = 0; ib < h; ib++) {
                k_gj_get<<<512, 256, 0, s>>>(res[0], B(t0 + ia, t0 + ib), nb, hn, ia, ib);
                c->launches++;
            }
        BFS_CUDA_TRY(c, cudaGetLastError());
        }
    }
    c->pc_twist = twist;
    int flag = 0;
    BFS_CUDA_TRY(c, cudaMemcpyAsync(&flag, c->d_pivflag, sizeof(int), cudaMemcpyDeviceToHost, s));
    BFS_CUDA_TRY(c, cudaStreamSynchronize(s));
    if (flag) {
        c->err = "zero pivot in a diagonal block of the preconditioner";
        return BFS_ESINGULAR;
    }
    // FP32 sweeps only without surface tension: the capillary term makes the
    // diagonal blocks so ill-conditioned (inverse entries of 1e5-1e7 on small
    // meshes) that FP32 copies of the factors no longer precondition
    if (c->opt.precond_precision == BFS_FP32C && c->opt.surface_tension == 0.0) {
        rc = precond_make_f32(c, s);
        if (rc) return rc;
        BFS_CUDA_TRY(c, cudaStreamSynchronize(s));
    }
    c->flow_checked = 0;
    c->pc_ready = 1;
    return BFS_OK;
}

int precond_apply(bfs_ctx *c, const double *r, double *z, cudaStream_t s)
{
    if (!c->pc_ready) {
        c->err = "preconditioner applied before bfs_precond_factor";
        return BFS_ENOPREC;
    }
    cudaEvent_t ev1 = nullptr;
    if (c->prof_on) {
        cudaEvent_t ev0 = prof_event(c);
        ev1 = prof_event(c);
        c->ev_kind.push_back(3);
        cudaEventRecord(ev0, s);
    }
    const int split = apply_flow_launch(c, r, z, s);
    if (split < 0) return split;
    if (split == 1) {
        if (ev1) cudaEventRecord(ev1, s);
        return BFS_OK;
    }
    if (c->pc_twist >= 0) {
        c->err = "two-ended factors need the FP32 sweep kernel";
        return BFS_ECUDA;
    }
    if (c->apply_grid <= 0) {
        int per_sm = 0;
        BFS_CUDA_TRY(c, cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_apply_coop, AP_TPB, 0));
        if (per_sm < 1) {
            c->err = "apply kernel cannot be resident";
            return BFS_ECUDA;
        }
        c->apply_grid = num_sms(c->device);  // one 1024-thread CTA per SM
    }
    ApplyArgs a;
    a.pc = c->d_pc; a.r = r; a.z = z; a.x = c->d_perm_a; a.y = c->d_perm_b;
    a.nb = c->nb; a.NB = c->N + 1; a.M = c->M; a.h = c->pc_h;
    a.bar = reinterpret_cast<CoopBar *>(c->d_pivflag + 4);
    a.flag = c->d_flag;
    a.spin = wait_spin(c);
    BFS_CUDA_TRY(c, cudaMemsetAsync(a.bar, 0, sizeof(CoopBar), s));
    void *args[] = {&a};
    BFS_CUDA_TRY(c, cudaLaunchCooperativeKernel((const void *)k_apply_coop, dim3(c->apply_grid),
                                                dim3(AP_TPB), args, 0, s));
    c->launches++;
    if (ev1) cudaEventRecord(ev1, s);
    return BFS_OK;
}

}  // namespace bfs

// The Gauss-Jordan kernels on caller matrices, with scratch of its own.
extern "C" int bfs_gj_invert(const double *A, double *Ainv, int n, int nmat, int method, void *stream)
{
    if (!A || !Ainv || n < 1 || n > 16384 || nmat < 1 || nmat > 2 || method < 0 || method > 2)
        return BFS_EINVAL;
    std::unique_ptr<bfs_ctx> c(new bfs_ctx{});
    if (cudaGetDevice(&c->device) != cudaSuccess) return BFS_ECUDA;
    cudaStream_t s = (cudaStream_t)stream;
    const int G = bfs::num_sms(c->device);
    const size_t nn = (size_t)n * n;
    double *work = nullptr;
    auto run = [&]() -> int {
        BFS_CUDA_TRY(c, cudaMalloc(&work, sizeof(double) * nmat * nn));
        BFS_CUDA_TRY(c, cudaMalloc(&c->d_gjscr, sizeof(unsigned long long) * 4 * (size_t)G + sizeof(int) * 4 * (size_t)n));
        BFS_CUDA_TRY(c, cudaMalloc(&c->d_gjdata, sizeof(double) * bfs::gj_data_doubles(G, n)));
        BFS_CUDA_TRY(c, cudaMalloc(&c->d_pivflag, sizeof(int) * 8));
        BFS_CUDA_TRY(c, cudaMalloc(&c->d_flag, sizeof(int)));
        BFS_CUDA_TRY(c, cudaMemsetAsync(c->d_pivflag, 0, sizeof(int) * 8, s));
        BFS_CUDA_TRY(c, cudaMemsetAsync(c->d_flag, 0, sizeof(int), s));
        BFS_CUDA_TRY(c, cudaMemcpyAsync(work, A, sizeof(double) * nmat * nn, cudaMemcpyDeviceToDevice, s));
        double *w[2] = {work, work + (nmat > 1 ? nn : 0)}, *d[2] = {Ainv, Ainv + (nmat > 1 ? nn : 0)};
        int r = method >= 1 ? bfs::gj_panel_invert(c.get(), w, d, nmat, n, s, method == 1)
                            : bfs::gj_rows_invert(c.get(), w, d, nmat, n, s);
        if (r == 1) return BFS_EINVAL;
        if (r) return r;
        int fl[2] = {0, 0};
        BFS_CUDA_TRY(c, cudaMemcpyAsync(&fl[0], c->d_pivflag, sizeof(int), cudaMemcpyDeviceToHost, s));
        BFS_CUDA_TRY(c, cudaMemcpyAsync(&fl[1], c->d_flag, sizeof(int), cudaMemcpyDeviceToHost, s));
        BFS_CUDA_TRY(c, cudaStreamSynchronize(s));
        if (fl[1] & 2) return BFS_ETIMEOUT;
        if (fl[0]) return BFS_ESINGULAR;
        return BFS_OK;
    };
    const int rc = run();
    cudaStreamSynchronize(s);
    cudaFree(work);
    cudaFree(c->d_gjscr);
    cudaFree(c->d_gjdata);
    cudaFree(c->d_pivflag);
    cudaFree(c->d_flag);
    return rc;
}
