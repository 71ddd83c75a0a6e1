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
#include "launch_shape.cuh"

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
                            float4 *s32, D4 *s64, Key128 *keys, int skip_self)
{
    const int set = blockIdx.y;
    const StatSet S = sets[set];
    if (S.l <= 0 || (skip_self && S.kmin >= 0)) return;
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

// ---- FP32 path, self-join sets: the same seeds by the diagonal recurrence ----
//
// The pairs (w, w + kmin) all lie on diagonal kmin, so instead of two dot
// products per window a thread walks a run of windows of that diagonal (at
// most kSeedRun; shorter for short series, see launch_shape.cuh): an
// exact FP64 dot product at the run's start, then the FP64 recurrence
// c += df_w dg_j + df_j dg_w.  Window w offers j = w + kmin to its own key (its
// right side) and j receives w (its left side); a key takes the larger value,
// the lower index on a tie, through an integer max on the FP32 keys' high word
// (value, inverted index).  seed_finish_kernel completes the keys (exact: the
// lower bound is the value) and the thresholds.
constexpr int kSeedRun = 128;
constexpr int kMinSeedRun = 16;
constexpr int kSeedThreads = 32;

__device__ __forceinline__ unsigned long long seed_pack(double r, long long idx)
{
    const float v = (float)r + 0.0f;
    return ((unsigned long long)ord32(__float_as_uint(v)) << 32) |
           (unsigned long long)(0xFFFFFFFFu - (unsigned)idx);
}

__global__ void seed_diag_kernel(const StatSet *__restrict__ sets, const double *__restrict__ mu,
                                 const double *__restrict__ inv, const uint8_t *__restrict__ flat,
                                 const D4 *__restrict__ s64, Key128 *keys, int run)
{
    const StatSet S = sets[blockIdx.y];
    if (S.l <= 0 || S.kmin < 0 || S.dir < 0) return;     // AB sets; left roles are filled here
    const StatSet Y = sets[S.partner];
    const long long k = S.kmin;
    const long long w0 = ((long long)blockIdx.x * blockDim.x + threadIdx.x) * run;
    long long wend = w0 + run;
    if (wend > S.l) wend = S.l;
    if (wend > Y.l - k) wend = Y.l - k;                  // j = w + k must be a window
    if (w0 >= wend) return;
    const double *ir = inv + S.sbase, *ic = inv + Y.sbase;
    const D4 *sr = s64 + S.sbase, *sc = s64 + Y.sbase;
    const uint8_t *fr = flat + S.sbase, *fc = flat + Y.sbase;
    const double *xa = S.x + w0, *xb = Y.x + w0 + k;
    const double ma = mu[S.sbase + w0];
    double a0 = 0.0, a1 = 0.0, a2 = 0.0, a3 = 0.0;
    int t = 0;
    for (; t + 3 < S.m; t += 4) {
        a0 = fma(xa[t] - ma, xb[t], a0);
        a1 = fma(xa[t + 1] - ma, xb[t + 1], a1);
        a2 = fma(xa[t + 2] - ma, xb[t + 2], a2);
        a3 = fma(xa[t + 3] - ma, xb[t + 3], a3);
    }
    for (; t < S.m; ++t) a0 = fma(xa[t] - ma, xb[t], a0);
    double c = (a0 + a1) + (a2 + a3);
    Key128 *kr = keys + S.sbase, *kc = keys + Y.sbase;
    for (long long w = w0; w < wend; ++w) {
        const long long j = w + k;
        const double r = S.raw ? (c - ir[w]) - ic[j] : c * ir[w] * ic[j];
        if (!fr[w]) atomicMax(&kr[w].hi, seed_pack(r, j));
        if (!fc[j]) atomicMax(&kc[j].hi, seed_pack(r, w));
        if (w + 1 < wend) {
            const D4 a = sr[w + 1], b = sc[j + 1];
            c = fma(a.x, b.y, c);
            c = fma(b.x, a.y, c);
        }
    }
}

// complete the seeded keys (exact: lower bound = value) and their thresholds
__global__ void seed_finish_kernel(const StatSet *__restrict__ sets,
                                   const uint8_t *__restrict__ flat, float4 *s32, Key128 *keys)
{
    const StatSet S = sets[blockIdx.y];
    if (S.l <= 0 || S.kmin < 0) return;
    for (long long w = (long long)blockIdx.x * blockDim.x + threadIdx.x; w < S.l;
         w += (long long)gridDim.x * blockDim.x) {
        const long long q = S.sbase + w;
        const unsigned long long hi = keys[q].hi;
        if (hi == 0ull || flat[q]) continue;
        keys[q].lo = hi & 0xFFFFFFFF00000000ull;
        s32[q].w = __uint_as_float(unord32((unsigned)(hi >> 32)));
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
    Key128 *k128 = reinterpret_cast<Key128 *>(keys);
    if (fp64) {
        seed_kernel<true><<<grid, threads, 0, st>>>(sets, mu, inv, flat, s32, s64, k128, 0);
        return cudaGetLastError();
    }
    // FP32 path: AB sets from a dot product each, self-join sets along diagonal kmin
    seed_kernel<false><<<grid, threads, 0, st>>>(sets, mu, inv, flat, s32, s64, k128, 1);
    const int run = spread_run(max_l, nsets, kSeedThreads, kSeedRun, kMinSeedRun);
    const long long runs = (max_l + run - 1) / run;
    const dim3 gd((unsigned)((runs + kSeedThreads - 1) / kSeedThreads), (unsigned)nsets);
    seed_diag_kernel<<<gd, kSeedThreads, 0, st>>>(sets, mu, inv, flat, s64, k128, run);
    seed_finish_kernel<<<grid, threads, 0, st>>>(sets, flat, s32, k128);
    return cudaGetLastError();
}

}  // namespace mpgb
