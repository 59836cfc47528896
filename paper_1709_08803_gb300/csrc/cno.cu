// Learned initial guess (C ABI in include/bfs_cno.h): a small convolutional
// neural operator on the nodal grid (an addition: the paper starts Newton from
// a flat surface or from a nearby solution).  It maps the bottom B = beta + 1, the Froude number
// and the node coordinates to the nodal fields zeta, phi - x and psi - x; the
// guess is accepted only through Newton to the same residual tolerance.
//
// Network: four dilated 3x3 convolutions (dilations 1, 3, 9, 27; widths
// 16 -> 32 -> 32 -> 32 -> 16, of which 4 inputs and 3 outputs are used), SiLU
// between them, zero padding.  Weights and activations are BF16, every
// contraction runs on the tensor cores through mma.sync m16n8k16 with FP32
// accumulation; master weights and the Adam moments are FP32.
//
// Layouts: activations NHWC (batch, row y, column x, channel); layer weights
// are kept in two BF16 copies, [cout][tap][cin] for the forward pass and
// [cin][tap][cout] for the backward pass on the inputs (the same convolution
// kernel run with negated tap offsets), both filled from one FP32 master
// vector holding, per layer, the weights [cout][tap][cin] then the biases.
#include <cuda_bf16.h>
#include <math.h>
#include <stdint.h>
#include <string.h>

#include <new>
#include <string>
#include <vector>

#include "bfs_cno.h"
#include "bfs_internal.cuh"

namespace {

constexpr int NL = 4;
constexpr int CIN[NL] = {16, 32, 32, 32};
constexpr int COUT[NL] = {32, 32, 32, 16};
constexpr int DIL[NL] = {1, 3, 9, 27};
constexpr int IN_REAL = 4, OUT_REAL = 3;

int n_weights(int l) { return COUT[l] * 9 * CIN[l]; }

int n_params()
{
    int s = 0;
    for (int l = 0; l < NL; l++) s += n_weights(l) + COUT[l];
    return s;
}

__device__ __forceinline__ uint32_t pack2(__nv_bfloat16 lo, __nv_bfloat16 hi)
{
    return (uint32_t)__bfloat16_as_ushort(lo) | ((uint32_t)__bfloat16_as_ushort(hi) << 16);
}

__device__ __forceinline__ void mma16816(float c[4], const uint32_t a[4], const uint32_t b[2])
{
    asm volatile(
        "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, "
        "{%8,%9}, {%0,%1,%2,%3};\n"
        : "+f"(c[0]), "+f"(c[1]), "+f"(c[2]), "+f"(c[3])
        : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b[0]), "r"(b[1]));
}

// Implicit-GEMM dilated 3x3 convolution.  out[p][n] = sum over taps t and
// input channels c of in[p + sgn * off(t) * dil][c] * w[n][t][c] (+ bias[n]),
// zero outside the grid.  in: BF16 NHWC with C channels (C in {16, 32});
// w: BF16 [N][9][C]; out: FP32 [P][N].  One warp per 16 pixels, N / 8 MMA
// column tiles per warp.
template <int C, int N>
__global__ void __launch_bounds__(128)
k_conv(const __nv_bfloat16 *__restrict__ in, const __nv_bfloat16 *__restrict__ w,
       const float *__restrict__ bias, float *__restrict__ out, int Bt, int H, int W, int dil, int sgn)
{
    const int lane = threadIdx.x & 31;
    const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int P = Bt * H * W;
    const int p0 = warp * 16;
    if (p0 >= P) return;
    const int r = lane >> 2, cq = (lane & 3) * 2;
    int pix[2], py[2], px[2], pb[2];
    for (int h = 0; h < 2; h++) {
        int p = p0 + r + 8 * h;
        pix[h] = p;
        int pc = p < P ? p : P - 1;
        pb[h] = pc / (H * W);
        int q = pc - pb[h] * H * W;
        py[h] = q / W;
        px[h] = q - py[h] * W;
    }
    float acc[N / 8][4];
#pragma unroll
    for (int nt = 0; nt < N / 8; nt++)
#pragma unroll
        for (int e = 0; e < 4; e++) acc[nt][e] = 0.f;
    const __nv_bfloat16 zero = __float2bfloat16(0.f);
#pragma unroll 1
    for (int t = 0; t < 9; t++) {
        const int oy = (t / 3 - 1) * dil * sgn, ox = (t % 3 - 1) * dil * sgn;
        const __nv_bfloat16 *src[2];
        bool ok[2];
        for (int h = 0; h < 2; h++) {
            int ys = py[h] + oy, xs = px[h] + ox;
            ok[h] = pix[h] < P && ys >= 0 && ys < H && xs >= 0 && xs < W;
            src[h] = in + ((size_t)(pb[h] * H + (ok[h] ? ys : 0)) * W + (ok[h] ? xs : 0)) * C;
        }
#pragma unroll
        for (int c0 = 0; c0 < C; c0 += 16) {
            uint32_t a[4];
            for (int h = 0; h < 2; h++) {
                __nv_bfloat16 v0 = ok[h] ? src[h][c0 + cq] : zero;
                __nv_bfloat16 v1 = ok[h] ? src[h][c0 + cq + 1] : zero;
                __nv_bfloat16 v2 = ok[h] ? src[h][c0 + cq + 8] : zero;
                __nv_bfloat16 v3 = ok[h] ? src[h][c0 + cq + 9] : zero;
                a[h] = pack2(v0, v1);
                a[2 + h] = pack2(v2, v3);
            }
#pragma unroll
            for (int nt = 0; nt < N / 8; nt++) {
                const __nv_bfloat16 *wr = w + ((size_t)(nt * 8 + r) * 9 + t) * C + c0;
                uint32_t b[2] = {pack2(wr[cq], wr[cq + 1]), pack2(wr[cq + 8], wr[cq + 9])};
                mma16816(acc[nt], a, b);
            }
        }
    }
#pragma unroll
    for (int nt = 0; nt < N / 8; nt++) {
        const int n0 = nt * 8 + cq;
        const float b0 = bias ? bias[n0] : 0.f, b1 = bias ? bias[n0 + 1] : 0.f;
        for (int h = 0; h < 2; h++) {
            if (pix[h] >= P) continue;
            float *o = out + (size_t)pix[h] * N + n0;
            o[0] = acc[nt][2 * h] + b0;
            o[1] = acc[nt][2 * h + 1] + b1;
        }
    }
}

// Weight gradient: dw[n][t][c] += sum over pixels p of in[p + off(t) dil][c] * g[p][n],
// with M = 9 C rows (t, c), N columns, the pixels as the contraction.  One warp
// per 16 rows and a chunk of 16 * KSTEPS pixels; FP32 atomics into dw.
template <int C, int N>
__global__ void __launch_bounds__(128)
k_conv_wgrad(const __nv_bfloat16 *__restrict__ in, const __nv_bfloat16 *__restrict__ g,
             float *__restrict__ dw, int Bt, int H, int W, int dil, int pix_per_warp)
{
    const int lane = threadIdx.x & 31;
    const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int rows = 9 * C, rtiles = rows / 16;
    const int rt = warp % rtiles, chunk = warp / rtiles;
    const int P = Bt * H * W;
    const int pbeg = chunk * pix_per_warp;
    if (pbeg >= P) return;
    const int pend = min(P, pbeg + pix_per_warp);
    const int r = lane >> 2, cq = (lane & 3) * 2;
    // the two A rows of this lane: (tap, channel)
    int tt[2], cc[2];
    for (int h = 0; h < 2; h++) {
        int m = rt * 16 + r + 8 * h;
        tt[h] = m / C;
        cc[h] = m - tt[h] * C;
    }
    float acc[N / 8][4];
#pragma unroll
    for (int nt = 0; nt < N / 8; nt++)
#pragma unroll
        for (int e = 0; e < 4; e++) acc[nt][e] = 0.f;
    const __nv_bfloat16 zero = __float2bfloat16(0.f);
    auto xval = [&](int h, int p) -> __nv_bfloat16 {
        if (p >= pend) return zero;
        int b = p / (H * W), q = p - b * H * W, y = q / W, x = q - y * W;
        int ys = y + (tt[h] / 3 - 1) * dil, xs = x + (tt[h] % 3 - 1) * dil;
        if (ys < 0 || ys >= H || xs < 0 || xs >= W) return zero;
        return in[((size_t)(b * H + ys) * W + xs) * C + cc[h]];
    };
    for (int k0 = pbeg; k0 < pend; k0 += 16) {
        uint32_t a[4];
        for (int h = 0; h < 2; h++) {
            a[h] = pack2(xval(h, k0 + cq), xval(h, k0 + cq + 1));
            a[2 + h] = pack2(xval(h, k0 + cq + 8), xval(h, k0 + cq + 9));
        }
#pragma unroll
        for (int nt = 0; nt < N / 8; nt++) {
            const int n = nt * 8 + r;
            auto gv = [&](int p) -> __nv_bfloat16 { return p < pend ? g[(size_t)p * N + n] : zero; };
            uint32_t b[2] = {pack2(gv(k0 + cq), gv(k0 + cq + 1)), pack2(gv(k0 + cq + 8), gv(k0 + cq + 9))};
            mma16816(acc[nt], a, b);
        }
    }
#pragma unroll
    for (int nt = 0; nt < N / 8; nt++) {
        const int n0 = nt * 8 + cq;
        for (int h = 0; h < 2; h++) {
            int m = rt * 16 + r + 8 * h;
            atomicAdd(dw + ((size_t)n0 * 9 * C) + m, acc[nt][2 * h]);
            atomicAdd(dw + ((size_t)(n0 + 1) * 9 * C) + m, acc[nt][2 * h + 1]);
        }
    }
}

__device__ __forceinline__ float sigm(float z) { return 1.f / (1.f + __expf(-z)); }

// input features (FP32, 4 channels) -> BF16, padded to 16 channels
__global__ void k_in_bf16(const float *__restrict__ x, __nv_bfloat16 *__restrict__ o, int P)
{
    int e = blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= P * 16) return;
    int p = e >> 4, c = e & 15;
    o[e] = __float2bfloat16(c < IN_REAL ? x[(size_t)p * IN_REAL + c] : 0.f);
}

// a = silu(z) in BF16
__global__ void k_silu(const float *__restrict__ z, __nv_bfloat16 *__restrict__ a, int n)
{
    int e = blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= n) return;
    float v = z[e];
    a[e] = __float2bfloat16(v * sigm(v));
}

// gz = ga * silu'(z) in BF16
__global__ void k_silu_bwd(const float *__restrict__ ga, const float *__restrict__ z,
                           __nv_bfloat16 *__restrict__ gz, int n)
{
    int e = blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= n) return;
    float v = z[e], s = sigm(v);
    gz[e] = __float2bfloat16(ga[e] * s * (1.f + v * (1.f - s)));
}

// output (FP32, 16 channels, 3 used) vs target (3 channels): loss partials and
// the BF16 gradient 2 (y - t) / count
__global__ void k_mse(const float *__restrict__ y, const float *__restrict__ t, __nv_bfloat16 *__restrict__ gy,
                      float *__restrict__ loss, int P)
{
    __shared__ float sh[256];
    int e = blockIdx.x * blockDim.x + threadIdx.x;
    float l = 0.f;
    if (e < P * 16) {
        int p = e >> 4, c = e & 15;
        float g = 0.f;
        if (c < OUT_REAL) {
            float d = y[e] - t[(size_t)p * OUT_REAL + c];
            l = d * d;
            g = 2.f * d / (float)(P * OUT_REAL);
        }
        gy[e] = __float2bfloat16(g);
    }
    sh[threadIdx.x] = l;
    __syncthreads();
    for (int o = blockDim.x / 2; o > 0; o >>= 1) {
        if (threadIdx.x < o) sh[threadIdx.x] += sh[threadIdx.x + o];
        __syncthreads();
    }
    if (threadIdx.x == 0) atomicAdd(loss, sh[0] / (float)(P * OUT_REAL));
}

// bias gradient: db[n] += sum_p g[p][n]
__global__ void k_bgrad(const __nv_bfloat16 *__restrict__ g, float *__restrict__ db, int P, int N)
{
    int n = blockIdx.y;
    float s = 0.f;
    for (int p = blockIdx.x * blockDim.x + threadIdx.x; p < P; p += gridDim.x * blockDim.x)
        s += __bfloat162float(g[(size_t)p * N + n]);
    for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
    if ((threadIdx.x & 31) == 0) atomicAdd(db + n, s);
}

// master FP32 parameters -> the BF16 forward and backward weight copies
__global__ void k_cast_weights(const float *__restrict__ wm, __nv_bfloat16 *__restrict__ wf,
                               __nv_bfloat16 *__restrict__ wb, int Cin, int Cout)
{
    int e = blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= Cout * 9 * Cin) return;
    int n = e / (9 * Cin), rem = e % (9 * Cin), t = rem / Cin, c = rem % Cin;
    __nv_bfloat16 v = __float2bfloat16(wm[e]);
    wf[e] = v;
    // backward on the inputs: [c][t][n], used with negated tap offsets
    wb[((size_t)c * 9 + t) * Cout + n] = v;
}

__global__ void k_adam(float *__restrict__ p, const float *__restrict__ g, float *__restrict__ m,
                       float *__restrict__ v, int n, float lr, float b1, float b2, float eps, float c1,
                       float c2)
{
    int e = blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= n) return;
    float gi = g[e];
    float mi = b1 * m[e] + (1.f - b1) * gi;
    float vi = b2 * v[e] + (1.f - b2) * gi * gi;
    m[e] = mi;
    v[e] = vi;
    p[e] -= lr * (mi / c1) / (sqrtf(vi / c2) + eps);
}

// nodal predictions (zeta, phi - x, psi - x; one image) -> unknown vector u:
// q(x1) from the first node, q_x by centred differences (one-sided at the ends)
// plus 1 for phi and psi.
__global__ void k_fields_to_u(const float *__restrict__ y, const float *__restrict__ scale,
                              double *__restrict__ u, int N, int M, double dx, double x1)
{
    int e = blockIdx.x * blockDim.x + threadIdx.x;
    const int NB = N + 1;
    if (e >= 3 * NB * M) return;
    int f = e / (NB * M), rem = e % (NB * M), j = rem / NB, pidx = rem % NB;
    auto val = [&](int i) -> double { return (double)y[((size_t)j * N + i) * 16 + f] * scale[f]; };
    double out;
    if (pidx == 0) {
        out = val(0) + (f > 0 ? x1 : 0.0);
    } else {
        int i = pidx - 1;
        double d;
        if (i == 0) d = (-3.0 * val(0) + 4.0 * val(1) - val(2)) / (2.0 * dx);
        else if (i == N - 1) d = (3.0 * val(N - 1) - 4.0 * val(N - 2) + val(N - 3)) / (2.0 * dx);
        else d = (val(i + 1) - val(i - 1)) / (2.0 * dx);
        out = d + (f > 0 ? 1.0 : 0.0);
    }
    u[e] = out;
}

}  // namespace

struct bfs_cno {
    int H, W, Bmax, np;
    float *p, *g, *m, *v;   // FP32 parameters, gradient, Adam moments
    __nv_bfloat16 *wf[NL], *wb[NL];
    float *bias[NL], *dbias[NL], *dw[NL];
    __nv_bfloat16 *act[NL + 1];  // BF16 inputs of each layer (act[0] = features)
    float *z[NL];                // FP32 pre-activations
    float *ga;                   // FP32 gradient w.r.t. a layer's input activations
    __nv_bfloat16 *gz;           // BF16 gradient w.r.t. pre-activations
    float *loss;
    float *scale;                // output scales (3)
    float *xin;                  // features of one image copied from the host (bfs_cno_solve_host)
    int step;
    std::string err;
};

namespace {
thread_local std::string g_cno_err;

template <int C, int N>
void conv(const __nv_bfloat16 *in, const __nv_bfloat16 *w, const float *b, float *out, int Bt, int H,
          int W, int dil, int sgn, cudaStream_t s)
{
    const int P = Bt * H * W, warps = (P + 15) / 16;
    k_conv<C, N><<<(warps + 3) / 4, 128, 0, s>>>(in, w, b, out, Bt, H, W, dil, sgn);
}

void conv_any(int C, int N, const __nv_bfloat16 *in, const __nv_bfloat16 *w, const float *b, float *out,
              int Bt, int H, int W, int dil, int sgn, cudaStream_t s)
{
    if (C == 16 && N == 32) conv<16, 32>(in, w, b, out, Bt, H, W, dil, sgn, s);
    else if (C == 32 && N == 32) conv<32, 32>(in, w, b, out, Bt, H, W, dil, sgn, s);
    else if (C == 32 && N == 16) conv<32, 16>(in, w, b, out, Bt, H, W, dil, sgn, s);
}

void wgrad_any(int C, int N, const __nv_bfloat16 *in, const __nv_bfloat16 *g, float *dw, int Bt, int H,
               int W, int dil, cudaStream_t s)
{
    const int P = Bt * H * W, ppw = 512;
    const int chunks = (P + ppw - 1) / ppw, warps = chunks * (9 * C / 16);
    const int blocks = (warps + 3) / 4;
    if (C == 16 && N == 32) k_conv_wgrad<16, 32><<<blocks, 128, 0, s>>>(in, g, dw, Bt, H, W, dil, ppw);
    else if (C == 32 && N == 32) k_conv_wgrad<32, 32><<<blocks, 128, 0, s>>>(in, g, dw, Bt, H, W, dil, ppw);
    else if (C == 32 && N == 16) k_conv_wgrad<32, 16><<<blocks, 128, 0, s>>>(in, g, dw, Bt, H, W, dil, ppw);
}

int ferr(bfs_cno *n, int code, const std::string &m)
{
    if (n) n->err = m;
    else g_cno_err = m;
    return code;
}

int forward(bfs_cno *n, const float *x, int Bt, cudaStream_t s)
{
    const int P = Bt * n->H * n->W;
    k_in_bf16<<<(P * 16 + 255) / 256, 256, 0, s>>>(x, n->act[0], P);
    for (int l = 0; l < NL; l++) {
        conv_any(CIN[l], COUT[l], n->act[l], n->wf[l], n->bias[l], n->z[l], Bt, n->H, n->W, DIL[l], 1, s);
        if (l < NL - 1) k_silu<<<(P * COUT[l] + 255) / 256, 256, 0, s>>>(n->z[l], n->act[l + 1], P * COUT[l]);
    }
    return cudaGetLastError() == cudaSuccess ? BFS_OK : ferr(n, BFS_ECUDA, "forward launch failed");
}

// gradient of the mean squared error w.r.t. all parameters into n->g; loss into n->loss
int backward(bfs_cno *n, const float *target, int Bt, cudaStream_t s)
{
    const int P = Bt * n->H * n->W;
    cudaMemsetAsync(n->g, 0, sizeof(float) * n->np, s);
    cudaMemsetAsync(n->loss, 0, sizeof(float), s);
    k_mse<<<(P * 16 + 255) / 256, 256, 0, s>>>(n->z[NL - 1], target, n->gz, n->loss, P);
    for (int l = NL - 1; l >= 0; l--) {
        // gz holds dL/dz_l (BF16, COUT[l] channels)
        wgrad_any(CIN[l], COUT[l], n->act[l], n->gz, n->dw[l], Bt, n->H, n->W, DIL[l], s);
        k_bgrad<<<dim3(64, COUT[l]), 256, 0, s>>>(n->gz, n->dbias[l], P, COUT[l]);
        if (l == 0) break;
        conv_any(COUT[l], CIN[l], n->gz, n->wb[l], nullptr, n->ga, Bt, n->H, n->W, DIL[l], -1, s);
        k_silu_bwd<<<(P * CIN[l] + 255) / 256, 256, 0, s>>>(n->ga, n->z[l - 1], n->gz, P * CIN[l]);
    }
    return cudaGetLastError() == cudaSuccess ? BFS_OK : ferr(n, BFS_ECUDA, "backward launch failed");
}

void cast_all(bfs_cno *n, cudaStream_t s)
{
    size_t off = 0;
    for (int l = 0; l < NL; l++) {
        k_cast_weights<<<(n_weights(l) + 255) / 256, 256, 0, s>>>(n->p + off, n->wf[l], n->wb[l], CIN[l], COUT[l]);
        off += n_weights(l) + COUT[l];
    }
}
}  // namespace

extern "C" {

const char *bfs_cno_last_error(const bfs_cno *n) { return n ? n->err.c_str() : g_cno_err.c_str(); }

int bfs_cno_num_params(void) { return n_params(); }

void bfs_cno_destroy(bfs_cno *n)
{
    if (!n) return;
    cudaFree(n->p);
    for (int l = 0; l < NL; l++) {
        cudaFree(n->wf[l]);
        cudaFree(n->wb[l]);
        cudaFree(n->z[l]);
        cudaFree(n->act[l]);
    }
    cudaFree(n->ga);
    cudaFree(n->gz);  // loss and scale live inside the parameter allocation
    cudaFree(n->xin);
    delete n;
}

int bfs_cno_create(int H, int W, int Bmax, bfs_cno **out)
{
    if (!out) return ferr(nullptr, BFS_EINVAL, "out is NULL");
    *out = nullptr;
    if (H < 3 || W < 3 || Bmax < 1) return ferr(nullptr, BFS_EINVAL, "bad grid or batch size");
    bfs_cno *n = new (std::nothrow) bfs_cno();
    if (!n) return ferr(nullptr, BFS_ENOMEM, "host allocation failed");
    n->H = H; n->W = W; n->Bmax = Bmax; n->np = n_params();
    const size_t P = (size_t)Bmax * H * W;
    bool ok = cudaMalloc(&n->p, sizeof(float) * (4 * (size_t)n->np + 4)) == cudaSuccess;
    if (ok) {
        n->g = n->p + n->np; n->m = n->g + n->np; n->v = n->m + n->np;
        n->loss = n->v + n->np; n->scale = n->loss + 1;
        size_t off = 0;
        for (int l = 0; l < NL; l++) {
            n->dw[l] = n->g + off;
            n->bias[l] = n->p + off + n_weights(l);
            n->dbias[l] = n->g + off + n_weights(l);
            off += n_weights(l) + COUT[l];
            ok = ok && cudaMalloc(&n->wf[l], sizeof(__nv_bfloat16) * n_weights(l)) == cudaSuccess;
            ok = ok && cudaMalloc(&n->wb[l], sizeof(__nv_bfloat16) * n_weights(l)) == cudaSuccess;
            ok = ok && cudaMalloc(&n->z[l], sizeof(float) * P * COUT[l]) == cudaSuccess;
            ok = ok && cudaMalloc(&n->act[l], sizeof(__nv_bfloat16) * P * CIN[l]) == cudaSuccess;
        }
        ok = ok && cudaMalloc(&n->ga, sizeof(float) * P * 32) == cudaSuccess;
        ok = ok && cudaMalloc(&n->xin, sizeof(float) * (size_t)H * W * 4) == cudaSuccess;
        ok = ok && cudaMalloc(&n->gz, sizeof(__nv_bfloat16) * P * 32) == cudaSuccess;
    }
    if (!ok || cudaMemset(n->p, 0, sizeof(float) * (4 * (size_t)n->np + 4)) != cudaSuccess) {
        bfs_cno_destroy(n);
        cudaGetLastError();
        return ferr(nullptr, BFS_ENOMEM, "device allocation failed");
    }
    *out = n;
    return BFS_OK;
}

// params: host FP32 vector of bfs_cno_num_params(); out_scale: 3 output scales
int bfs_cno_set_params(bfs_cno *n, const float *params, const float *out_scale)
{
    if (!n || !params) return BFS_EINVAL;
    if (cudaMemcpy(n->p, params, sizeof(float) * n->np, cudaMemcpyHostToDevice) != cudaSuccess)
        return ferr(n, BFS_ECUDA, "parameter upload failed");
    float sc[3] = {1.f, 1.f, 1.f};
    if (out_scale) memcpy(sc, out_scale, sizeof(sc));
    if (cudaMemcpy(n->scale, sc, sizeof(sc), cudaMemcpyHostToDevice) != cudaSuccess)
        return ferr(n, BFS_ECUDA, "scale upload failed");
    cudaMemset(n->m, 0, sizeof(float) * 2 * n->np);
    n->step = 0;
    cast_all(n, 0);
    return cudaDeviceSynchronize() == cudaSuccess ? BFS_OK : ferr(n, BFS_ECUDA, "cast failed");
}

int bfs_cno_get_params(bfs_cno *n, float *params)
{
    if (!n || !params) return BFS_EINVAL;
    return cudaMemcpy(params, n->p, sizeof(float) * n->np, cudaMemcpyDeviceToHost) == cudaSuccess
               ? BFS_OK : ferr(n, BFS_ECUDA, "parameter download failed");
}

// x: device FP32 [Bt][H][W][4]; y: device FP32 [Bt][H][W][16] (channels 0..2 used)
int bfs_cno_forward(bfs_cno *n, const float *x, int Bt, float *y, void *stream)
{
    if (!n || !x || !y || Bt < 1 || Bt > n->Bmax) return ferr(n, BFS_EINVAL, "bad arguments");
    cudaStream_t s = (cudaStream_t)stream;
    int rc = forward(n, x, Bt, s);
    if (rc) return rc;
    const size_t bytes = sizeof(float) * (size_t)Bt * n->H * n->W * 16;
    return cudaMemcpyAsync(y, n->z[NL - 1], bytes, cudaMemcpyDeviceToDevice, s) == cudaSuccess
               ? BFS_OK : ferr(n, BFS_ECUDA, "output copy failed");
}

// gradient of the mean squared error (target: device FP32 [Bt][H][W][3]) into
// grad_host (bfs_cno_num_params floats); *loss_host receives the loss.  Synchronous.
int bfs_cno_gradient(bfs_cno *n, const float *x, const float *target, int Bt, float *grad_host,
                     float *loss_host, void *stream)
{
    if (!n || !x || !target || Bt < 1 || Bt > n->Bmax) return ferr(n, BFS_EINVAL, "bad arguments");
    cudaStream_t s = (cudaStream_t)stream;
    int rc = forward(n, x, Bt, s);
    if (!rc) rc = backward(n, target, Bt, s);
    if (rc) return rc;
    if (grad_host && cudaMemcpyAsync(grad_host, n->g, sizeof(float) * n->np, cudaMemcpyDeviceToHost, s))
        return ferr(n, BFS_ECUDA, "gradient download failed");
    if (loss_host && cudaMemcpyAsync(loss_host, n->loss, sizeof(float), cudaMemcpyDeviceToHost, s))
        return ferr(n, BFS_ECUDA, "loss download failed");
    return cudaStreamSynchronize(s) == cudaSuccess ? BFS_OK : ferr(n, BFS_ECUDA, "synchronisation failed");
}

// one Adam step on the mean squared error; asynchronous (loss stays on device,
// read it with bfs_cno_read_loss)
int bfs_cno_train_step(bfs_cno *n, const float *x, const float *target, int Bt, float lr, void *stream)
{
    if (!n || !x || !target || Bt < 1 || Bt > n->Bmax) return ferr(n, BFS_EINVAL, "bad arguments");
    cudaStream_t s = (cudaStream_t)stream;
    int rc = forward(n, x, Bt, s);
    if (!rc) rc = backward(n, target, Bt, s);
    if (rc) return rc;
    n->step++;
    const float b1 = 0.9f, b2 = 0.999f;
    const float c1 = 1.f - powf(b1, (float)n->step), c2 = 1.f - powf(b2, (float)n->step);
    k_adam<<<(n->np + 255) / 256, 256, 0, s>>>(n->p, n->g, n->m, n->v, n->np, lr, b1, b2, 1e-8f, c1, c2);
    cast_all(n, s);
    return cudaGetLastError() == cudaSuccess ? BFS_OK : ferr(n, BFS_ECUDA, "train step failed");
}

int bfs_cno_read_loss(bfs_cno *n, float *loss_host, void *stream)
{
    if (!n || !loss_host) return BFS_EINVAL;
    cudaStream_t s = (cudaStream_t)stream;
    if (cudaMemcpyAsync(loss_host, n->loss, sizeof(float), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
        cudaStreamSynchronize(s) != cudaSuccess)
        return ferr(n, BFS_ECUDA, "loss download failed");
    return BFS_OK;
}

// Initial guess for ctx from the network: features x (device FP32 [1][M][N][4])
// -> nodal fields -> unknown vector u (device, length 3(N+1)M).
int bfs_cno_guess(bfs_cno *n, bfs_ctx *c, const float *x, double *u, void *stream)
{
    if (!n || !c || !x || !u) return ferr(n, BFS_EINVAL, "NULL argument");
    if (c->M != n->H || c->N != n->W) return ferr(n, BFS_EINVAL, "mesh does not match the network grid");
    cudaStream_t s = (cudaStream_t)stream;
    int rc = forward(n, x, 1, s);
    if (rc) return rc;
    const int tot = 3 * (c->N + 1) * c->M;
    k_fields_to_u<<<(tot + 255) / 256, 256, 0, s>>>(n->z[NL - 1], n->scale, u, c->N, c->M, c->dx, c->x1);
    return cudaGetLastError() == cudaSuccess ? BFS_OK : ferr(n, BFS_ECUDA, "guess launch failed");
}

int bfs_cno_solve(bfs_cno *n, bfs_ctx *c, const float *x, double *u, bfs_stats *st, int *used_fallback,
                  void *stream)
{
    if (!n || !c || !x || !u) return ferr(n, BFS_EINVAL, "NULL argument");
    if (used_fallback) *used_fallback = 0;
    int rc = bfs_cno_guess(n, c, x, u, stream);
    if (rc) return rc;
    bfs_stats s1{};
    rc = bfs_solve(c, u, &s1, stream);
    if (st) *st = s1;
    // accepted only through Newton: a guess from which the solve fails gives way
    // to the method without the network, the uniform stream
    if (rc == BFS_OK || !(rc == BFS_ENOCONV || rc == BFS_ELINESEARCH || rc == BFS_EBREAKDOWN ||
                          rc == BFS_ENAN || rc == BFS_ETIMEOUT))
        return rc;
    if (used_fallback) *used_fallback = 1;
    bfs_stats s2{};
    if ((rc = bfs_flat_guess(c, u, stream))) return rc;
    rc = bfs_solve(c, u, &s2, stream);
    if (st) {
        s2.newton_its += s1.newton_its;
        s2.krylov_its += s1.krylov_its;
        s2.residual_evals_fp64 += s1.residual_evals_fp64;
        s2.residual_evals_fp32 += s1.residual_evals_fp32;
        s2.precond_applies += s1.precond_applies;
        s2.seconds += s1.seconds;
        *st = s2;
    }
    return rc;
}

int bfs_cno_solve_host(bfs_cno *n, bfs_ctx *c, const float *x_host, double *u_host, bfs_stats *st,
                       int *used_fallback, void *stream)
{
    if (!n || !c || !x_host || !u_host) return ferr(n, BFS_EINVAL, "NULL argument");
    if (c->M != n->H || c->N != n->W) return ferr(n, BFS_EINVAL, "mesh does not match the network grid");
    cudaStream_t s = (cudaStream_t)stream;
    int rc = bfs::alloc_solver(c);
    if (rc) return ferr(n, rc, c->err);
    double *u = c->d_uio;  // the context's own device copy of the iterate
    if (cudaMemcpyAsync(n->xin, x_host, sizeof(float) * (size_t)n->H * n->W * 4, cudaMemcpyHostToDevice, s) !=
        cudaSuccess)
        return ferr(n, BFS_ECUDA, "upload of the features failed");
    rc = bfs_cno_solve(n, c, n->xin, u, st, used_fallback, stream);
    if (cudaMemcpyAsync(u_host, u, sizeof(double) * c->n, cudaMemcpyDeviceToHost, s) != cudaSuccess ||
        cudaStreamSynchronize(s) != cudaSuccess)
        return rc ? rc : ferr(n, BFS_ECUDA, "download of u failed");
    return rc;
}

}  // extern "C"
