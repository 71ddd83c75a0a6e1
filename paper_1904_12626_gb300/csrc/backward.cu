// backward.cu -- gradient of a weighted sum of MP entries through the argmin pairs.
//
// L = sum_i g_i MP_i with MP_i = d(i, j), j = PI_i held fixed.  With z the
// z-normalised windows (population sigma), rho = (1/m) sum_k z_i[k] z_j[k]
// and d = |z_i - z_j| = sqrt(2m(1 - rho)):
//   d rho / d x_{i+k} = (z_j[k] - rho z_i[k]) / (m sigma_i),   d d / d rho = -m / d,
// so  dMP_i/dx_{i+k} = -(z_j[k] - rho z_i[k]) / (sigma_i d)  and symmetrically
// for the j window.  One warp handles one row: it forms rho and d directly
// from the series (FP64), then scatters both windows' contributions with
// FP64 atomic adds (a window pair can overlap, and many rows can share a
// neighbour, so the scatter needs atomics).
#include <cmath>

#include "internal.cuh"

namespace mpgb {
namespace {

__global__ void backward_kernel(const double *__restrict__ x, long long l, int m,
                                const double *__restrict__ mu, const double *__restrict__ invn,
                                const uint8_t *__restrict__ flat,
                                const int64_t *__restrict__ pi, const double *__restrict__ g,
                                double *grad, Hdr *hdr)
{
    const int lane = threadIdx.x & 31;
    const long long warp = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const long long nwarps = ((long long)gridDim.x * blockDim.x) >> 5;
    const double sm = sqrt((double)m);
    for (long long i = warp; i < l; i += nwarps) {
        const long long j = pi[i];
        const double gi = g[i];
        if (j < 0 || gi == 0.0) continue;
        if (j >= l) {
            if (lane == 0) set_status(hdr, MP_EINVAL);
            continue;
        }
        if (flat[i] || flat[j]) continue;
        const double mi = mu[i], mj = mu[j];
        const double ai = invn[i] * sm, aj = invn[j] * sm;     // z = (x - mu) * a, a = 1/sigma
        double sp = 0.0, sd = 0.0;
        for (int k = lane; k < m; k += 32) {
            const double zi = (x[i + k] - mi) * ai;
            const double zj = (x[j + k] - mj) * aj;
            sp = fma(zi, zj, sp);
            const double df = zi - zj;
            sd = fma(df, df, sd);
        }
        for (int o = 16; o > 0; o >>= 1) {
            sp += __shfl_xor_sync(0xffffffffu, sp, o);
            sd += __shfl_xor_sync(0xffffffffu, sd, o);
        }
        const double rho = sp / (double)m;
        const double d = sqrt(sd);
        if (d < 1e-12) continue;
        const double ci = -gi * ai / d;                        // -g / (sigma_i d)
        const double cj = -gi * aj / d;
        for (int k = lane; k < m; k += 32) {
            const double zi = (x[i + k] - mi) * ai;
            const double zj = (x[j + k] - mj) * aj;
            atomicAdd(grad + i + k, ci * (zj - rho * zi));
            atomicAdd(grad + j + k, cj * (zi - rho * zj));
        }
    }
}

}  // namespace

cudaError_t launch_backward(const double *x64, long long n, int m, const double *mu,
                            const double *invn, const uint8_t *flat, const int64_t *pi,
                            const double *grad_mp, double *grad_x, Hdr *hdr, cudaStream_t st)
{
    const long long l = n - m + 1;
    cudaError_t e = cudaMemsetAsync(grad_x, 0, sizeof(double) * (size_t)n, st);
    if (e != cudaSuccess || l <= 0) return e;
    const int threads = 256;
    long long blocks = (l * 32 + threads - 1) / threads;
    if (blocks > 65536) blocks = 65536;
    backward_kernel<<<(unsigned)blocks, threads, 0, st>>>(x64, l, m, mu, invn, flat, pi, grad_mp,
                                                          grad_x, hdr);
    return cudaGetLastError();
}

}  // namespace mpgb
