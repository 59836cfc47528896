// Pressure on the bottom and the force of the fluid on the topography
// (Buttle et al., arXiv:1709.08803, Sec. 2.1): Bernoulli's equation evaluated
// along the bottom, with the bottom kinematic condition folded in,
//   p = 1/2 - [(1 + bx^2) psi_y^2 + (1 + by^2) psi_x^2 - 2 bx by psi_x psi_y] / (2 (1 + bx^2 + by^2)) - beta / F^2,
// from the bottom potential psi of a solution; the force is the trapezoid sum
// of p (beta_x, beta_y, -1) dx dy (the outward normal of the fluid times dS).
#include <math.h>

#include "bfs_internal.cuh"

namespace bfs {

constexpr int PR_BLOCKS = 128, PR_TPB = 256;

__device__ __forceinline__ double ydiff_p(const double *q, int N, int M, int half, double dy, int i, int j)
{
    if (j == 0) {
        if (half) return 0.0;
        return (-3.0 * q[i] + 4.0 * q[i + N] - q[i + 2 * N]) / (2.0 * dy);
    }
    if (j == M - 1)
        return (3.0 * q[i + (size_t)N * (M - 1)] - 4.0 * q[i + (size_t)N * (M - 2)] +
                q[i + (size_t)N * (M - 3)]) / (2.0 * dy);
    return (q[i + (size_t)N * (j + 1)] - q[i + (size_t)N * (j - 1)]) / (2.0 * dy);
}

__global__ void k_bottom_pressure(const double *__restrict__ nodal, const double *__restrict__ beta,
                                  const double *__restrict__ bx, const double *__restrict__ by,
                                  double *__restrict__ p, double *__restrict__ partial, int N, int M,
                                  int half, double dx, double dy, double F)
{
    __shared__ double sh[3][PR_TPB / 32];
    const size_t NM = (size_t)N * M;
    const double *ps = nodal + 6 * NM, *psx = nodal + 7 * NM;
    double f[3] = {0.0, 0.0, 0.0};
    for (int e = blockIdx.x * PR_TPB + threadIdx.x; e < (int)NM; e += PR_BLOCKS * PR_TPB) {
        const int i = e % N, j = e / N;
        const double a = bx[e], b = by[e], gx = psx[e], gy = ydiff_p(ps, N, M, half, dy, i, j);
        const double kin = 0.5 * ((1.0 + a * a) * gy * gy + (1.0 + b * b) * gx * gx - 2.0 * a * b * gx * gy) /
                           (1.0 + a * a + b * b);
        const double pv = 0.5 - kin - beta[e] / (F * F);
        p[e] = pv;
        const double cx = (i == 0 || i == N - 1) ? 0.5 : 1.0;
        const double cy = half ? ((j == M - 1) ? 0.5 : 1.0) : ((j == 0 || j == M - 1) ? 0.5 : 1.0);
        const double w = dx * dy * cx * cy * ((half && j > 0) ? 2.0 : 1.0);
        f[0] += w * pv * a;
        f[1] += w * pv * b;
        f[2] -= w * pv;
    }
    for (int k = 0; k < 3; k++) {
        double v = f[k];
        for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
        if ((threadIdx.x & 31) == 0) sh[k][threadIdx.x >> 5] = v;
    }
    __syncthreads();
    if (threadIdx.x < 3) {
        double v = 0.0;
        for (int w = 0; w < PR_TPB / 32; w++) v += sh[threadIdx.x][w];
        partial[threadIdx.x * PR_BLOCKS + blockIdx.x] = v;
    }
}

__global__ void k_force_final(const double *__restrict__ partial, double *__restrict__ force, int half)
{
    const int k = threadIdx.x;
    if (k >= 3) return;
    double v = 0.0;
    for (int b = 0; b < PR_BLOCKS; b++) v += partial[k * PR_BLOCKS + b];
    force[k] = (half && k == 1) ? 0.0 : v;
}

}  // namespace bfs

extern "C" int bfs_bottom_pressure(bfs_ctx *c, const double *u, double *p, double *force_host, void *stream)
{
    if (!c || !u || !p) {
        if (c) c->err = "NULL argument";
        return BFS_EINVAL;
    }
    cudaStream_t s = (cudaStream_t)stream;
    int rc = bfs::unpack_launch(c, u, s);
    if (rc) return rc;
    double *part = c->d_red;  // 3 * PR_BLOCKS <= the reduction scratch
    bfs::k_bottom_pressure<<<bfs::PR_BLOCKS, bfs::PR_TPB, 0, s>>>(c->d_nodal, c->d_beta, c->d_bx, c->d_by, p, part,
                                                                  c->N, c->M, c->half, c->dx, c->dy, c->F);
    c->launches++;
    bfs::k_force_final<<<1, 32, 0, s>>>(part, c->d_scal + 16, c->half);
    c->launches++;
    BFS_CUDA_TRY(c, cudaGetLastError());
    if (force_host) {
        BFS_CUDA_TRY(c, cudaMemcpyAsync(force_host, c->d_scal + 16, 3 * sizeof(double), cudaMemcpyDeviceToHost, s));
        BFS_CUDA_TRY(c, cudaStreamSynchronize(s));
    }
    return BFS_OK;
}
