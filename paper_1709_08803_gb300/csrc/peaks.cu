// Throughput probes for the roofline denominators of the pair kernels: long
// streams of one instruction kind with no dependence between consecutive
// instructions of a thread (eight independent chains) and a full SM of warps,
// so that the pipe, not latency, limits them.
//   kind 0: FP32 fused multiply-add (the FMA pipe; one warp instruction per
//           clock per SM sub-partition at best, the issue limit)
//   kind 1: FP32 reciprocal square root (rsqrtf, the special-function unit,
//           compiled with flush-to-zero as the pair kernel is)
//   kind 2: FP64 fused multiply-add (the FP64 pipe)
//   kind 3: packed FP32x2 fused multiply-add (two lane operations per
//           instruction; the form the FP32C pair kernel uses)
#include "bfs_internal.cuh"

namespace bfs {

constexpr int PK_CHAINS = 8;
constexpr int PK_TPB = 256;

__global__ void __launch_bounds__(PK_TPB) k_peak_ffma(float *out, int iters, float a, float b)
{
    float x[PK_CHAINS];
#pragma unroll
    for (int j = 0; j < PK_CHAINS; j++) x[j] = 1.0f + 1e-3f * (threadIdx.x + j);
    for (int i = 0; i < iters; i++)
#pragma unroll
        for (int j = 0; j < PK_CHAINS; j++) x[j] = fmaf(x[j], a, b);
    float s = 0.f;
#pragma unroll
    for (int j = 0; j < PK_CHAINS; j++) s += x[j];
    out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

__global__ void __launch_bounds__(PK_TPB) k_peak_rsqrt(float *out, int iters)
{
    float x[PK_CHAINS];
#pragma unroll
    for (int j = 0; j < PK_CHAINS; j++) x[j] = 1.0f + 1e-3f * (threadIdx.x + j);
    for (int i = 0; i < iters; i++)
#pragma unroll
        for (int j = 0; j < PK_CHAINS; j++) x[j] = rsqrtf(x[j]);  // stays near 1
    float s = 0.f;
#pragma unroll
    for (int j = 0; j < PK_CHAINS; j++) s += x[j];
    out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

__global__ void __launch_bounds__(PK_TPB) k_peak_dfma(double *out, int iters, double a, double b)
{
    double x[PK_CHAINS];
#pragma unroll
    for (int j = 0; j < PK_CHAINS; j++) x[j] = 1.0 + 1e-3 * (threadIdx.x + j);
    for (int i = 0; i < iters; i++)
#pragma unroll
        for (int j = 0; j < PK_CHAINS; j++) x[j] = fma(x[j], a, b);
    double s = 0.0;
#pragma unroll
    for (int j = 0; j < PK_CHAINS; j++) s += x[j];
    out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

__global__ void __launch_bounds__(PK_TPB) k_peak_ffma2(float *out, int iters, float a, float b)
{
    unsigned long long x[PK_CHAINS], av, bv;
    asm("mov.b64 %0, {%1, %1};" : "=l"(av) : "f"(a));
    asm("mov.b64 %0, {%1, %1};" : "=l"(bv) : "f"(b));
#pragma unroll
    for (int j = 0; j < PK_CHAINS; j++) {
        const float v = 1.0f + 1e-3f * (threadIdx.x + j);
        asm("mov.b64 %0, {%1, %1};" : "=l"(x[j]) : "f"(v));
    }
    for (int i = 0; i < iters; i++)
#pragma unroll
        for (int j = 0; j < PK_CHAINS; j++)
            asm("fma.rn.ftz.f32x2 %0, %0, %1, %2;" : "+l"(x[j]) : "l"(av), "l"(bv));
    float s = 0.f;
#pragma unroll
    for (int j = 0; j < PK_CHAINS; j++) {
        float lo, hi;
        asm("mov.b64 {%0, %1}, %2;" : "=f"(lo), "=f"(hi) : "l"(x[j]));
        s += lo + hi;
    }
    out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

}  // namespace bfs

extern "C" int bfs_peak_probe(int kind, int iters, void *out, void *stream, double *lane_ops)
{
    if (kind < 0 || kind > 3 || iters < 1 || !out) return BFS_EINVAL;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return BFS_ECUDA;
    const int grid = bfs::num_sms(dev) * (2048 / bfs::PK_TPB);  // a full SM of warps each
    cudaStream_t s = (cudaStream_t)stream;
    if (kind == 0)
        bfs::k_peak_ffma<<<grid, bfs::PK_TPB, 0, s>>>((float *)out, iters, 0.999f, 1e-4f);
    else if (kind == 1)
        bfs::k_peak_rsqrt<<<grid, bfs::PK_TPB, 0, s>>>((float *)out, iters);
    else if (kind == 2)
        bfs::k_peak_dfma<<<grid, bfs::PK_TPB, 0, s>>>((double *)out, iters, 0.999, 1e-4);
    else
        bfs::k_peak_ffma2<<<grid, bfs::PK_TPB, 0, s>>>((float *)out, iters, 0.999f, 1e-4f);
    if (cudaGetLastError() != cudaSuccess) return BFS_ECUDA;
    if (lane_ops) *lane_ops = (double)grid * bfs::PK_TPB * (double)iters * bfs::PK_CHAINS * (kind == 3 ? 2 : 1);
    return BFS_OK;
}

extern "C" int bfs_peak_probe_threads(void)
{
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return 0;
    return bfs::num_sms(dev) * 2048;
}
