// seed.cu -- a first exact candidate for every window before the tile kernel.
//
// The tile kernel skips a cell whose correlation (FP32 path: its upper
// bound) is below the running threshold of its row or column.  With empty
// keys every threshold starts at -inf, so the first visits of each window
// all pass and every one of them costs a merge into global memory.  On
// smooth series (random walks) it is worse: a column is visited by the
// diagonals of a tile from the farthest to the nearest, so its correlations
// mostly increase from visit to visit and nearly every visit improves the
// key.  Seeding each key with the exact correlation of one nearby admissible
// partner starts the thresholds near their final values:
//   self-join: partners w + kmin and w - kmin (the nearest admissible
//              windows; the higher exact correlation, the lower index on a tie);
//              a left (right) profile takes only w - kmin (w + kmin);
//   AB-join:   partner min(w, l_partner - 1).
// The seed is a genuine candidate of the join (exact, admissible), so the
// answer is unchanged: it only prunes cells that could not win.
#include <cmath>

#include "join_tile.cuh"

namespace mpgb {
namespace {

// exact FP64 centred dot product of window a of series xa (mean mua) with
// window b of series xb (the second mean drops out: the first factor sums to 0)
__device__ __forceinline__ double seed_dot(const double *__restrict__ xa, double mua,
                                           const double *__restrict__ xb, int m)
{
    double a0 = 0.0, a1 = 0.0, a2 = 0.0, a3 = 0.0;     // four chains: FP64 latency
    int t = 0;
    for (; t + 3 < m; t += 4) {
        a0 = fma(xa[t] - mua, xb[t], a0);
        a1 = fma(xa[t + 1] - mua, xb[t + 1], a1);
        a2 = fma(xa[t + 2] - mua, xb[t + 2], a2);
        a3 = fma(xa[t + 3] - mua, xb[t + 3], a3);
    }
    for (; t < m; ++t) a0 = fma(xa[t] - mua, xb[t], a0);
    return (a0 + a1) + (a2 + a3);
}

template <bool FP64>
__global__ void seed_kernel(const StatSet *__restrict__ sets, const double *__restrict__ mu,
                            const double *__restrict__ inv, const uint8_t *__restrict__ flat,
                            float4 *s32, D4 *s64, Key128 *keys)
{
    const int set = blockIdx.y;
    const StatSet S = sets[set];
    if (S.l <= 0) return;
    const StatSet Y = sets[S.partner];
    if (Y.l <= 0) return;
    for (long long w = (long long)blockIdx.x * blockDim.x + threadIdx.x; w < S.l;
         w += (long long)gridDim.x * blockDim.x) {
        const long long q = S.sbase + w;
        if (flat[q]) continue;                     // closed form, never joined
        long long j1, j2;
        if (S.kmin >= 0) {
            j1 = S.dir <= 0 ? w - S.kmin : -1;     // lower index first: wins ties
            j2 = S.dir >= 0 ? w + S.kmin : -1;
            if (j1 < 0) j1 = -1;
            if (j2 >= Y.l) j2 = -1;
        } else {
            j1 = w < Y.l ? w : Y.l - 1;
            j2 = -1;
        }
        const double *xw = S.x + w;
        const double muw = mu[q], invw = inv[q];
        long long best = -1;
        double rb = 0.0;
        float rbf = 0.0f;
        for (int k = 0; k < 2; ++k) {
            const long long j = k == 0 ? j1 : j2;
            if (j < 0 || (k == 1 && j == j1)) continue;
            const double dot = seed_dot(xw, muw, Y.x + j, S.m);
            // correlation, or the non-normalised score q - h_i - h_j (mu = 0, inv = h)
            const double r = S.raw ? (dot - invw) - inv[Y.sbase + j] : dot * invw * inv[Y.sbase + j];
            if (FP64) {
                if (best < 0 || r > rb) { best = j; rb = r; }
            } else {
                const float rf = (float)r;
                if (best < 0 || rf > rbf) { best = j; rbf = rf; }
            }
        }
        if (best < 0) continue;
        if (FP64) {
            keys[q] = TraitsF64::pack(rb, best);
            s64[q].w = rb + 0.0;
        } else {
            Cand c;
            c.V = c.L = rbf;
            c.idx = best;
            keys[q] = cand_key(c);
            s32[q].w = rbf;
        }
    }
}

}  // namespace

cudaError_t launch_seed(const StatSet *sets, int nsets, long long max_l, const double *mu,
                        const double *inv, const uint8_t *flat, float4 *s32, D4 *s64,
                        void *keys, int fp64, cudaStream_t st)
{
    if (nsets <= 0 || max_l <= 0) return cudaSuccess;
    const int threads = 256;
    long long per = (max_l + threads - 1) / threads;
    const long long cap = 65536 / nsets > 0 ? 65536 / nsets : 1;
    if (per > cap) per = cap;
    const dim3 grid((unsigned)per, (unsigned)nsets);
    if (fp64)
        seed_kernel<true><<<grid, threads, 0, st>>>(sets, mu, inv, flat, s32, s64,
                                                     reinterpret_cast<Key128 *>(keys));
    else
        seed_kernel<false><<<grid, threads, 0, st>>>(sets, mu, inv, flat, s32, s64,
                                                      reinterpret_cast<Key128 *>(keys));
    return cudaGetLastError();
}

}  // namespace mpgb
