// finalize.cu -- keys to (MP, PI), with the exact FP64 distance refine.
//
// A key holds the best correlation found for an index and the lowest
// neighbour index reaching it.  MP = sqrt(2m(1 - rho)) (Sec. 2's z-normalised
// Euclidean distance written through the correlation), clamped to
// [0, 2 sqrt(m)].  With refine on (the default), MP is instead the distance
// of the pair (i, PI[i]) recomputed directly in FP64 from the series,
// sqrt(sum_k (z_i[k] - z_j[k])^2), which removes the error the recurrence
// left in rho while keeping the neighbour the kernel chose.
//
// Flat windows (all values equal) have the closed-form answer of the
// zero-variance convention: distance sqrt(2m) to everything, so PI is the
// lowest admissible index.
#include <cmath>

#include "internal.cuh"

namespace mpgb {
namespace {

__device__ __forceinline__ double exact_distance(const FinDesc &F, long long i, long long j,
                                                 double invR)
{
    const double s2m = sqrt(2.0 * (double)F.m);
    if (F.flatC[j]) return s2m;
    const double invC = F.invC[j];
    const double muR = F.muR[i], muC = F.muC[j];
    const double *xr = F.xR + i, *xc = F.xC + j;
    // Through the correlation first: d^2 = 2m(1 - rho), three FP64 operations per
    // sample (both windows centred: leaving the column's mean out, exact in exact
    // arithmetic, lets the rounding of the row's mean meet the column's offset,
    // which ill-conditioned windows would notice).  The rounding of rho (a few
    // ulps, times 2m) only matters when d is small, so below d^2 = 1 the distance
    // is summed directly from its definition.
    {
        double c0 = 0.0, c1 = 0.0, c2 = 0.0, c3 = 0.0;
        int t = 0;
        for (; t + 3 < F.m; t += 4) {
            c0 = fma(xr[t] - muR, xc[t] - muC, c0);
            c1 = fma(xr[t + 1] - muR, xc[t + 1] - muC, c1);
            c2 = fma(xr[t + 2] - muR, xc[t + 2] - muC, c2);
            c3 = fma(xr[t + 3] - muR, xc[t + 3] - muC, c3);
        }
        for (; t < F.m; ++t) c0 = fma(xr[t] - muR, xc[t] - muC, c0);
        const double rho = ((c0 + c1) + (c2 + c3)) * invR * invC;
        const double d2 = 2.0 * (double)F.m * (1.0 - rho);
        if (d2 >= 1.0) {
            const double d = sqrt(d2);
            const double cap = 2.0 * sqrt((double)F.m);
            return d > cap ? cap : d;
        }
    }
    double a0 = 0.0, a1 = 0.0;                    // two chains: FP64 latency
    int t = 0;
    for (; t + 1 < F.m; t += 2) {
        const double d0 = (xr[t] - muR) * invR - (xc[t] - muC) * invC;
        const double d1 = (xr[t + 1] - muR) * invR - (xc[t + 1] - muC) * invC;
        a0 = fma(d0, d0, a0);
        a1 = fma(d1, d1, a1);
    }
    if (t < F.m) {
        const double d0 = (xr[t] - muR) * invR - (xc[t] - muC) * invC;
        a0 = fma(d0, d0, a0);
    }
    double d = sqrt((double)F.m * (a0 + a1));
    const double cap = 2.0 * sqrt((double)F.m);
    return d > cap ? cap : d;
}

// non-normalised distance ||x_i - x_j|| in FP64 from the series
__device__ __forceinline__ double exact_raw_distance(const FinDesc &F, long long i, long long j)
{
    const double *xr = F.xR + i, *xc = F.xC + j;
    double a0 = 0.0, a1 = 0.0;
    int t = 0;
    for (; t + 1 < F.m; t += 2) {
        const double d0 = xr[t] - xc[t], d1 = xr[t + 1] - xc[t + 1];
        a0 = fma(d0, d0, a0);
        a1 = fma(d1, d1, a1);
    }
    if (t < F.m) {
        const double d0 = xr[t] - xc[t];
        a0 = fma(d0, d0, a0);
    }
    return sqrt(a0 + a1);
}

template <bool FP64KEY>
__device__ __forceinline__ void finalize_one(const FinDesc &F, long long i, long long l, int refine)
{
    const double INF = __longlong_as_double(0x7ff0000000000000ll);
    if (i >= l) {
        F.mp[i] = INF;
        F.pi[i] = -1;
        return;
    }
    const double s2m = sqrt(2.0 * (double)F.m);
    double mpv = INF;
    long long piv = -1;
    if (F.flatR[i]) {
        // lowest admissible index (every candidate ties at distance sqrt(2m))
        if (F.kmin < 0) piv = F.lC > 0 ? 0 : -1;
        else if (F.dir > 0) piv = (i + F.kmin < F.lC) ? i + F.kmin : -1;
        else if (F.dir < 0) piv = (i >= F.kmin) ? 0 : -1;
        else piv = (i >= F.kmin) ? 0 : ((i + F.kmin < F.lC) ? i + F.kmin : -1);
        if (piv >= 0) mpv = s2m;
    } else {
        double rho = 0.0;
        bool have;
        if (FP64KEY) {
            const Key128 k = reinterpret_cast<const Key128 *>(F.key)[i];
            have = (k.hi | k.lo) != 0ull;
            if (have) {
                rho = __longlong_as_double((long long)unord64(k.hi));
                piv = (long long)(~0ull - k.lo);
            }
        } else {
            // FP32-mixed candidate key: hi = (value, ~index), lo = lower bound
            const Key128 k = reinterpret_cast<const Key128 *>(F.key)[i];
            have = k.hi != 0ull;
            if (have) {
                const double v = (double)__uint_as_float(unord32((unsigned)(k.hi >> 32)));
                const double lb = (double)__uint_as_float(unord32((unsigned)(k.lo >> 32)));
                rho = 0.5 * (v + lb);
                piv = (long long)(0xFFFFFFFFu - (unsigned)(k.hi & 0xFFFFFFFFull));
            }
        }
        if (have) {
            if (F.raw) {                         // key value: the score -d^2 / 2
                mpv = refine ? exact_raw_distance(F, i, piv) : sqrt(rho < 0.0 ? -2.0 * rho : 0.0);
            } else if (refine) {
                mpv = exact_distance(F, i, piv, F.invR[i]);
            } else {
                rho = rho > 1.0 ? 1.0 : (rho < -1.0 ? -1.0 : rho);
                mpv = sqrt(2.0 * (double)F.m * (1.0 - rho));
            }
        }
    }
    F.mp[i] = mpv == INF ? INF : mpv * F.scale;
    F.pi[i] = piv;
}

template <bool FP64KEY>
__global__ void finalize_kernel(const FinDesc *__restrict__ fins, int refine)
{
    const FinDesc F = fins[blockIdx.y];
    if (F.mp == nullptr || F.pi == nullptr) return;
    const long long l = F.l > 0 ? F.l : 0;
    const long long end = F.pad_to > l ? F.pad_to : l;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < end;
         i += (long long)gridDim.x * blockDim.x)
        finalize_one<FP64KEY>(F, i, l, refine);
}

}  // namespace

namespace {
// anytime runs write their outputs where the caller says, per run
__global__ void bind_outputs_kernel(FinDesc *fins, double *mp, long long *pi)
{
    fins[0].mp = mp;
    fins[0].pi = pi;
}
}  // namespace

cudaError_t launch_bind_outputs(FinDesc *fins, double *mp, long long *pi, cudaStream_t st)
{
    bind_outputs_kernel<<<1, 1, 0, st>>>(fins, mp, pi);
    return cudaGetLastError();
}

cudaError_t launch_finalize(const FinDesc *fins, int nfin, long long max_len, int fp64,
                            int refine, cudaStream_t st)
{
    if (nfin <= 0 || max_len <= 0) return cudaSuccess;
    const int threads = 256;
    long long per = (max_len + threads - 1) / threads;       // blocks per descriptor
    const long long cap = 65536 / nfin > 0 ? 65536 / nfin : 1;
    if (per > cap) per = cap;
    const dim3 grid((unsigned)per, (unsigned)nfin);
    if (fp64)
        finalize_kernel<true><<<grid, threads, 0, st>>>(fins, refine);
    else
        finalize_kernel<false><<<grid, threads, 0, st>>>(fins, refine);
    return cudaGetLastError();
}

}  // namespace mpgb
