// fragile.cu -- exact handling of ill-conditioned windows.
//
// The FP32 recurrence carries an absolute error that grows with the
// covariances met along a diagonal; a correlation divides it by the two
// windows' centred norms.  For a window whose norm is tiny compared with its
// set (typically a window that is flat except for a few samples, next to a
// constant stretch) that quotient is meaningless, so such "fragile" windows
// are left out of the tile kernel (the inverse norm the tile kernel reads is
// set to NaN, so no comparison involving them is ever true) and every pair
// they take part in is computed here exactly, in FP64.  The same holds, much
// further out, for the FP64 recurrence, so both precisions use this pass.
//
// Cost.  For a window x_f and any candidate window y with centred values
// ~y, the centred dot product is sum_t ~y[t] * (x_f[t] - L) for any constant
// L, because the centred ~y sums to zero.  Taking L = the value most of a
// near-constant window repeats, only the few samples that differ from L
// contribute, so a fragile window costs (candidates) x (samples != L)
// multiply-adds instead of (candidates) x m.
#include <cmath>
#include <type_traits>

#include "join_tile.cuh"

namespace mpgb {
namespace {

constexpr int kFragileThreads = 256;
constexpr int kMaxSparse = 2048;               // samples != L kept in shared memory

// exact FP64 correlation of window a of series (xa, mua, inva) with window b of
// (xb, mub, invb), by one thread
__device__ __forceinline__ double thread_correlation(const double *xa, const double *mua,
                                                     const double *inva, long long a,
                                                     const double *xb, const double *invb,
                                                     long long b, int m)
{
    const double mu = mua[a];
    double acc = 0.0;
    for (int t = 0; t < m; ++t) acc = fma(xa[a + t] - mu, xb[b + t], acc);
    return acc * inva[a] * invb[b];
}

// Merge the exact candidate (e, idx) into the FP32-path key of window own of
// series O; the key's candidates are windows of series K.  When the key holds
// an unverified candidate that the decision needs, its exact value is
// computed here.
__device__ void merge_exact_f32(Key128 *key, float e, long long idx, long long own,
                                const double *xo, const double *muo, const double *invo,
                                const double *xk, const double *muk, const double *invk, int m,
                                Hdr *hdr)
{
    Cand c;
    c.V = c.L = e;
    c.idx = idx;
    float kx = 0.0f;
    long long kx_idx = -1;
    for (int round = 0; round < kMergeRounds; ++round) {
        const Key128 cur = key_peek(key);
        const int dec = classify(c, cur, kx, kx_idx);
        if (dec == kDiscard) return;
        if (dec == kReplace) {
            if (key_same(cas128(key, cur, cand_key(c)), cur)) return;
            continue;
        }
        // only the key's candidate can be unverified here
        kx_idx = key_cand(cur).idx;
        kx = (float)thread_correlation(xk, muk, invk, kx_idx, xo, invo, own, m);
    }
    set_status(hdr, MP_ETIMEOUT);
}

__global__ void fragile_mark_kernel(const StatSet *__restrict__ sets, const double *set_acc,
                                    const double *__restrict__ inv,
                                    const uint8_t *__restrict__ flat, float4 *s32, D4 *s64,
                                    unsigned long long *frag_list, Hdr *hdr)
{
    const int set = blockIdx.y;
    const StatSet S = sets[set];
    const double cnt = set_acc[2 * set + 1];
    if (S.l <= 0 || cnt <= 0.0) return;
    const double s_ref = exp(set_acc[2 * set] / cnt);          // geometric mean norm
    const double cut = kFragileFactor * s_ref;
    for (long long w = (long long)blockIdx.x * blockDim.x + threadIdx.x; w < S.l;
         w += (long long)gridDim.x * blockDim.x) {
        const long long q = S.sbase + w;
        const double invn = inv[q];
        if (flat[q] || !(invn > 0.0)) continue;
        if (1.0 / invn < cut) {
            // out of the tile kernel: no comparison with a NaN norm is true
            if (s32) s32[q].z = __int_as_float(0x7fc00000);
            else s64[q].z = __longlong_as_double(0x7ff8000000000000ll);
            const unsigned long long e = atomicAdd(&hdr->frag_count, 1ull);
            frag_list[e] = ((unsigned long long)set << 40) | (unsigned long long)w;
        }
    }
}

template <class Tr>
__global__ void __launch_bounds__(kFragileThreads)
fragile_pass_kernel(const StatSet *__restrict__ sets, const double *__restrict__ mu,
                    const double *__restrict__ inv, const unsigned long long *__restrict__ frag_list,
                    typename Tr::Key *keys, Hdr *hdr)
{
    using T = typename Tr::T;
    using Key = typename Tr::Key;
    using Packed = typename Tr::Packed;
    __shared__ int s_pos[kMaxSparse];
    __shared__ double s_val[kMaxSparse];
    __shared__ int s_cnt[2];
    __shared__ double s_level;
    __shared__ Packed s_best[kFragileThreads / 32];
    const unsigned long long count = hdr->frag_count;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    for (unsigned long long e = blockIdx.x; e < count; e += gridDim.x) {
        const unsigned long long ent = frag_list[e];
        const int xs = (int)(ent >> 40);
        const long long f = (long long)(ent & ((1ull << 40) - 1));
        const StatSet SX = sets[xs];
        const StatSet SY = sets[SX.partner];
        if (!index_ok(hdr, f, SX.l)) continue;                    // block-uniform: one entry per block
        const int m = SX.m;
        const double *xf = SX.x + f;
        // level L: whichever end value the window repeats more often
        if (tid < 2) s_cnt[tid] = 0;
        __syncthreads();
        const double a0 = xf[0], a1 = xf[m - 1];
        int c0 = 0, c1 = 0;
        for (int t = tid; t < m; t += blockDim.x) {
            c0 += (xf[t] == a0);
            c1 += (xf[t] == a1);
        }
        atomicAdd(&s_cnt[0], c0);
        atomicAdd(&s_cnt[1], c1);
        __syncthreads();
        if (tid == 0) {
            const int best = s_cnt[0] >= s_cnt[1] ? s_cnt[0] : s_cnt[1];
            s_level = best >= 2 ? (s_cnt[0] >= s_cnt[1] ? a0 : a1) : 0.0;
            s_cnt[0] = 0;
        }
        __syncthreads();
        const double L = s_level;
        for (int t = tid; t < m; t += blockDim.x) {
            const double v = xf[t] - L;
            if (v != 0.0) {
                const int k = atomicAdd(&s_cnt[0], 1);
                if (k < kMaxSparse) {
                    s_pos[k] = t;
                    s_val[k] = v;
                }
            }
        }
        __syncthreads();
        const int nnz = s_cnt[0];
        const bool sparse = nnz <= kMaxSparse;
        const double inv_f = inv[SX.sbase + f];
        const double *yx = SY.x;
        const double *ymu = mu + SY.sbase;
        const double *yinv = inv + SY.sbase;
        Key *ykey = keys + SY.sbase;
        Packed best = Tr::pzero();
        for (long long j = tid; j < SY.l; j += blockDim.x) {
            if (SX.kmin >= 0) {                                   // self-join exclusion zone
                const long long dd = SX.dir > 0 ? j - f : (SX.dir < 0 ? f - j : (j > f ? j - f : f - j));
                if (dd < SX.kmin) continue;
            }
            const double muj = ymu[j];
            const double *yj = yx + j;
            double c = 0.0;
            if (sparse) {
                for (int k = 0; k < nnz; ++k) c = fma(yj[s_pos[k]] - muj, s_val[k], c);
            } else {
                for (int t = 0; t < m; ++t) c = fma(yj[t] - muj, xf[t] - L, c);
            }
            const T rho = (T)(c * yinv[j] * inv_f);
            if constexpr (std::is_same<Tr, TraitsF32>::value) {
                const Key128 cur = key_peek(ykey + j);
                const Cand q = key_cand(cur);
                if (key_empty(cur) || rho >= q.L)
                    merge_exact_f32(ykey + j, rho, f, j, yx, ymu, yinv, SX.x, mu + SX.sbase,
                                    inv + SX.sbase, m, hdr);
            } else {
                const Packed kj = Tr::pack(rho, f);
                if (Tr::pgt(kj, Tr::peek(ykey + j))) Tr::merge(ykey, j, kj, hdr);
            }
            const Packed kf = Tr::pack(rho, j);
            if (Tr::pgt(kf, best)) best = kf;
        }
        for (int o = 16; o > 0; o >>= 1) {
            const Packed y = Tr::pshfl(best, o);
            if (Tr::pgt(y, best)) best = y;
        }
        if (lane == 0) s_best[warp] = best;
        __syncthreads();
        if (tid == 0) {
            Packed b = Tr::pzero();
            for (int w = 0; w < (int)(blockDim.x >> 5); ++w)
                if (Tr::pgt(s_best[w], b)) b = s_best[w];
            if (Tr::pgt(b, Tr::pzero())) {
                if constexpr (std::is_same<Tr, TraitsF32>::value)
                    merge_exact_f32(keys + SX.sbase + f, Tr::pval(b), Tr::pidx(b), f, SX.x,
                                    mu + SX.sbase, inv + SX.sbase, yx, ymu, yinv, m, hdr);
                else
                    Tr::merge(keys + SX.sbase, f, b, hdr);
            }
        }
        __syncthreads();
    }
}

}  // namespace

cudaError_t launch_fragile_mark(const StatSet *sets, int nsets, long long max_l,
                                const double *set_acc, const double *inv, const uint8_t *flat,
                                float4 *s32, D4 *s64, unsigned long long *frag_list, Hdr *hdr,
                                cudaStream_t st)
{
    if (nsets <= 0 || max_l <= 0) return cudaSuccess;
    const int threads = 256;
    long long per = (max_l + threads - 1) / threads;
    const long long cap = 65536 / nsets > 0 ? 65536 / nsets : 1;
    if (per > cap) per = cap;
    fragile_mark_kernel<<<dim3((unsigned)per, (unsigned)nsets), threads, 0, st>>>(
        sets, set_acc, inv, flat, s32, s64, frag_list, hdr);
    return cudaGetLastError();
}

cudaError_t launch_fragile_pass(const StatSet *sets, const double *mu, const double *inv,
                                const unsigned long long *frag_list, void *keys, int fp64,
                                Hdr *hdr, int grid, cudaStream_t st)
{
    if (fp64)
        fragile_pass_kernel<TraitsF64><<<grid, kFragileThreads, 0, st>>>(
            sets, mu, inv, frag_list, reinterpret_cast<Key128 *>(keys), hdr);
    else
        fragile_pass_kernel<TraitsF32><<<grid, kFragileThreads, 0, st>>>(
            sets, mu, inv, frag_list, reinterpret_cast<Key128 *>(keys), hdr);
    return cudaGetLastError();
}

}  // namespace mpgb
