// join_tile.cuh -- the persistent diagonal-tile kernel (shared by the FP32-mixed
// and the all-FP64 instantiations).
//
// What one cell does.  For a row window i and a column window j = i + k the
// centred dot product follows the diagonal recurrence
//     c(i,j) = c(i-1,j-1) + df_i dg_j + df_j dg_i          (2 FMA)
// (the reuse of the previous dot product that the paper credits to STOMP,
// Sec. 3.3.2, evaluated diagonal by diagonal in SCRIMP's order, Sec. 3.3.3),
// and the Pearson correlation is rho = c * invn_j * invn_i (2 MUL).  The
// nearest neighbour maximises rho: d = sqrt(2m(1 - rho)) (Sec. 2: the MP is
// the smallest z-normalised Euclidean distance).
//
// Layout of the work.  A tile is `tile_rows` rows of a band of TD = 32 W D
// consecutive diagonals.  Thread t of the CTA owns the D diagonals
// k0 + tD .. k0 + tD + D-1 (its "slots") and walks the tile's rows; at row i
// its slots touch columns i + k0 + tD + d.  Going to row i+1 every slot's
// column is the next slot's previous column, so the column statistics live in
// a register ring that is rotated by unrolling D rows: each row step loads
// one new column (plus the row's statistics, a shared-memory broadcast).
// Row and column statistics of a chunk of rows are staged in shared memory
// as {df, dg, invn, threshold}; column entries are padded one slot in D so
// that the lanes' strided loads fall in distinct banks.
//
// Maxima without per-cell index bookkeeping.  Each row and each column
// carries a threshold: the best correlation already known for that index
// (read from the global keys when the chunk is staged; +inf for flat
// windows, whose answer is closed-form).  The fast path only asks, per cell,
// "is rho >= the row's threshold or the column's threshold?" (2 compares,
// OR-ed into one predicate), so a cell costs 2 FMA + 2 MUL + 2 compares.
// When any lane of the warp saw a hit in a group of D rows, the warp replays
// that group from the saved covariances with the same arithmetic (so the
// correlations are bit-identical) and, for each hit, merges the packed key
// (order-preserving correlation bits, inverted index) into the global key
// array with an atomic max, so ties resolve to the lowest index whatever the
// order tiles run in.  After warm-up almost no group hits.
//
// Anchors.  The first covariance of each diagonal in a tile, and every
// `anchor_every` rows after it, is an exact FP64 dot product of the two
// windows; in the FP32-mixed instantiation only the recurrence runs in FP32.
#pragma once

#include <cmath>

#include "internal.cuh"

namespace mpgb {

// 128-bit compare-and-swap (sm_90+): returns the value found at *a
__device__ __forceinline__ Key128 cas128(Key128 *a, Key128 cmp, Key128 nv)
{
    Key128 old;
    asm volatile(
        "{\n\t.reg .b128 d, b, c;\n\t"
        "mov.b128 b, {%3, %4};\n\t"
        "mov.b128 c, {%5, %6};\n\t"
        "atom.global.cas.b128 d, [%2], b, c;\n\t"
        "mov.b128 {%0, %1}, d;\n\t}"
        : "=l"(old.lo), "=l"(old.hi)
        : "l"(a), "l"(cmp.lo), "l"(cmp.hi), "l"(nv.lo), "l"(nv.hi)
        : "memory");
    return old;
}

struct TraitsF32 {
    using T = float;
    using S4 = float4;
    using Key = unsigned long long;
    using Packed = unsigned long long;
    static __device__ __forceinline__ const S4 *rs(const Prob &P) { return P.rS32; }
    static __device__ __forceinline__ const S4 *cs(const Prob &P) { return P.cS32; }
    static __device__ __forceinline__ T inf() { return __int_as_float(0x7f800000); }
    static __device__ __forceinline__ T fma_(T a, T b, T c) { return fmaf(a, b, c); }
    static __device__ __forceinline__ T thr_of(const Key *k, long long idx)
    {
        const unsigned long long v = __ldcg(k + idx);
        return v == 0ull ? -inf() : __uint_as_float(unord32((unsigned)(v >> 32)));
    }
    static __device__ __forceinline__ Packed pack(T rho, long long idx)
    {
        rho += 0.0f;                              // -0 -> +0: all zero correlations tie
        return ((unsigned long long)ord32(__float_as_uint(rho)) << 32) |
               (unsigned long long)(0xFFFFFFFFu - (unsigned)idx);
    }
    static __device__ __forceinline__ Packed pzero() { return 0ull; }
    static __device__ __forceinline__ bool pgt(Packed a, Packed b) { return a > b; }
    static __device__ __forceinline__ Packed pshfl(Packed a, int o)
    {
        return __shfl_xor_sync(0xffffffffu, a, o);
    }
    static __device__ __forceinline__ T pval(Packed a)
    {
        return __uint_as_float(unord32((unsigned)(a >> 32)));
    }
    static __device__ __forceinline__ void merge(Key *k, long long idx, Packed p, Hdr *)
    {
        atomicMax(k + idx, p);
    }
};

struct TraitsF64 {
    using T = double;
    using S4 = D4;
    using Key = Key128;
    using Packed = Key128;
    static __device__ __forceinline__ const S4 *rs(const Prob &P) { return P.rS64; }
    static __device__ __forceinline__ const S4 *cs(const Prob &P) { return P.cS64; }
    static __device__ __forceinline__ T inf() { return __longlong_as_double(0x7ff0000000000000ll); }
    static __device__ __forceinline__ T fma_(T a, T b, T c) { return fma(a, b, c); }
    static __device__ __forceinline__ T thr_of(const Key *k, long long idx)
    {
        const unsigned long long hi = __ldcg(&k[idx].hi);
        const unsigned long long lo = __ldcg(&k[idx].lo);
        return (hi == 0ull && lo == 0ull) ? -inf() : __longlong_as_double((long long)unord64(hi));
    }
    static __device__ __forceinline__ Packed pack(T rho, long long idx)
    {
        rho += 0.0;
        Packed p;
        p.hi = ord64((unsigned long long)__double_as_longlong(rho));
        p.lo = ~0ull - (unsigned long long)idx;
        return p;
    }
    static __device__ __forceinline__ Packed pzero() { return Packed{0ull, 0ull}; }
    static __device__ __forceinline__ bool pgt(Packed a, Packed b)
    {
        return a.hi > b.hi || (a.hi == b.hi && a.lo > b.lo);
    }
    static __device__ __forceinline__ Packed pshfl(Packed a, int o)
    {
        Packed r;
        r.hi = __shfl_xor_sync(0xffffffffu, a.hi, o);
        r.lo = __shfl_xor_sync(0xffffffffu, a.lo, o);
        return r;
    }
    static __device__ __forceinline__ T pval(Packed a)
    {
        return __longlong_as_double((long long)unord64(a.hi));
    }
    static __device__ __forceinline__ void merge(Key *k, long long idx, Packed p, Hdr *hdr)
    {
        Key128 *a = k + idx;
        Key128 cur;
        cur.hi = __ldcg(&a->hi);
        cur.lo = __ldcg(&a->lo);
        for (unsigned it = 0; it < kCasRetryLimit; ++it) {
            if (!pgt(p, cur)) return;
            const Key128 old = cas128(a, cur, p);
            if (old.lo == cur.lo && old.hi == cur.hi) return;
            cur = old;
        }
        set_status(hdr, MP_ETIMEOUT);
    }
};

template <class Tr>
__device__ __forceinline__ typename Tr::S4 make4(typename Tr::T a, typename Tr::T b,
                                                 typename Tr::T c, typename Tr::T d)
{
    typename Tr::S4 v;
    v.x = a; v.y = b; v.z = c; v.w = d;
    return v;
}

// Exact FP64 covariances c(a, j0 + d), d < D, of the row window a against
// the column windows j0 + d (sum over the centred row window times the raw
// column window: the column mean drops out because the centred row window
// sums to zero).  Slots whose column window does not exist get 0.
template <class Tr, int D>
__device__ __forceinline__ void anchor_covariances(const Prob &P, long long a, long long j0,
                                                   typename Tr::T (&c)[D])
{
    const double *__restrict__ xr = P.rX + a;
    const double *__restrict__ xc = P.cX;
    const double mu = P.rMu[a];
    const long long last = P.nC - 1;
    double acc[D];
#pragma unroll
    for (int d = 0; d < D; ++d) acc[d] = 0.0;
    const int m = P.m;
    for (int t = 0; t < m; ++t) {
        const double xt = __ldg(xr + t) - mu;
#pragma unroll
        for (int d = 0; d < D; ++d) {
            long long q = j0 + d + t;
            q = q < last ? q : last;
            acc[d] = fma(xt, __ldg(xc + q), acc[d]);
        }
    }
#pragma unroll
    for (int d = 0; d < D; ++d) c[d] = (j0 + d < P.lC) ? (typename Tr::T)acc[d] : (typename Tr::T)0;
}

// smem index of staged column q (one padding slot every D entries)
template <int D>
__device__ __forceinline__ int cpos(int q) { return q + q / D; }

template <class Tr, int D, int W, int RC>
struct TileShape {
    static constexpr int NT = W * 32;
    static constexpr int TD = NT * D;
    static constexpr int NCOL = RC + TD;
    static constexpr int NCOLP = NCOL + NCOL / D + 1;
    static constexpr int SMEM = (RC + NCOLP) * (int)sizeof(typename Tr::S4);
};

// MINB: minimum resident CTAs per SM the register allocation must allow
template <class Tr, int D, int W, int RC, int MINB>
__global__ void __launch_bounds__(W * 32, MINB)
join_tile_kernel(const Prob *__restrict__ probs, const Band *__restrict__ bands,
                 const unsigned long long *__restrict__ tile_prefix, Hdr *hdr, int tile_rows,
                 int anchor_every)
{
    using T = typename Tr::T;
    using S4 = typename Tr::S4;
    using Key = typename Tr::Key;
    using Packed = typename Tr::Packed;
    using Sh = TileShape<Tr, D, W, RC>;
    constexpr int NT = Sh::NT;
    constexpr int TD = Sh::TD;
    static_assert(TD <= kMaxTileDiags, "tile wider than the stats padding");

    extern __shared__ __align__(32) unsigned char smem_raw[];
    S4 *sRow = reinterpret_cast<S4 *>(smem_raw);
    S4 *sCol = sRow + RC;
    __shared__ unsigned long long s_tile;

    const int lane = threadIdx.x & 31;
    const int lane_off = threadIdx.x * D;
    const int nb = hdr->nbands;
    const unsigned long long ntiles = tile_prefix[nb];
    const T INF = Tr::inf();

    for (;;) {
        __syncthreads();
        if (threadIdx.x == 0) s_tile = atomicAdd(&hdr->ticket, 1ull);
        __syncthreads();
        const unsigned long long tile = s_tile;
        if (tile >= ntiles) break;
        int lo = 0, hi = nb;                       // tile_prefix[lo] <= tile < tile_prefix[hi]
        while (hi - lo > 1) {
            const int mid = (lo + hi) >> 1;
            if (tile_prefix[mid] <= tile) lo = mid; else hi = mid;
        }
        const Band bd = bands[lo];
        const Prob &P = probs[bd.prob];
        const long long k0 = bd.k0;
        const long long lR = P.lR, lC = P.lC;
        const long long rows_end = min(lR, lC - k0);
        const long long i0 = (long long)(tile - tile_prefix[lo]) * tile_rows;
        const long long i1 = min(i0 + (long long)tile_rows, rows_end);
        const long long kl = k0 + lane_off;        // slot d walks diagonal kl + d
        const S4 *__restrict__ rS = Tr::rs(P);
        const S4 *__restrict__ cS = Tr::cs(P);
        Key *rKey = reinterpret_cast<Key *>(P.rKey);
        Key *cKey = reinterpret_cast<Key *>(P.cKey);

        T c[D];
        for (long long r = i0; r < i1; r += RC) {
            const int nrows = (int)min((long long)RC, i1 - r);
            const int nrr = (nrows + D - 1) / D * D;
            __syncthreads();
            for (int t = threadIdx.x; t < nrr; t += NT) {
                const long long i = r + t;
                const S4 v = rS[i];
                const T thr = (v.w != (T)0 || i >= lR) ? INF : Tr::thr_of(rKey, i);
                sRow[t] = make4<Tr>(v.x, v.y, v.z, thr);
            }
            const long long cb = r + k0;
            const int ncols = nrr + TD;
            for (int t = threadIdx.x; t < ncols; t += NT) {
                const long long j = cb + t;
                const S4 v = cS[j];
                const T thr = (v.w != (T)0 || j >= lC) ? INF : Tr::thr_of(cKey, j);
                sCol[cpos<D>(t)] = make4<Tr>(v.x, v.y, v.z, thr);
            }
            __syncthreads();
            if (r == i0 || (anchor_every > 0 && (r - i0) % anchor_every == 0)) {
                // covariance at row a = r - 1 so that row r applies the update; at
                // r = 0 the update of row 0 adds 0 (df_0 = dg_0 = 0)
                const long long a = r > 0 ? r - 1 : 0;
                anchor_covariances<Tr, D>(P, a, a + kl, c);
            }
            S4 cs[D];
#pragma unroll
            for (int d = 0; d < D; ++d) cs[d] = sCol[cpos<D>(lane_off + d)];

            for (int s = 0; s < nrr; s += D) {
                T c0[D];
#pragma unroll
                for (int d = 0; d < D; ++d) c0[d] = c[d];
                bool hit = false;
#pragma unroll
                for (int u = 0; u < D; ++u) {
                    const S4 rw = sRow[s + u];
#pragma unroll
                    for (int d = 0; d < D; ++d) {
                        const S4 &cc = cs[(d + u) % D];
                        c[d] = Tr::fma_(rw.x, cc.y, c[d]);
                        c[d] = Tr::fma_(cc.x, rw.y, c[d]);
                        const T rho = c[d] * cc.z * rw.z;
                        hit |= (rho >= rw.w);
                        hit |= (rho >= cc.w);
                    }
                    cs[u % D] = sCol[cpos<D>(lane_off + s + u + D)];
                }
                if (__any_sync(0xffffffffu, hit)) {
                    // replay the D rows from c0 with bookkeeping
                    for (int u = 0; u < D; ++u) {
                        const S4 rw = sRow[s + u];
                        const long long i = r + s + u;
                        T rho[D];
                        bool prow = false;
#pragma unroll
                        for (int d = 0; d < D; ++d) {
                            const int q = cpos<D>(lane_off + s + u + d);
                            const S4 cc = sCol[q];
                            c0[d] = Tr::fma_(rw.x, cc.y, c0[d]);
                            c0[d] = Tr::fma_(cc.x, rw.y, c0[d]);
                            rho[d] = c0[d] * cc.z * rw.z;
                            prow |= (rho[d] >= rw.w);
                            if (rho[d] >= cc.w) {
                                Tr::merge(cKey, i + kl + d, Tr::pack(rho[d], i), hdr);
                                sCol[q].w = rho[d];
                            }
                        }
                        if (__any_sync(0xffffffffu, prow)) {
                            Packed best = Tr::pzero();
#pragma unroll
                            for (int d = 0; d < D; ++d) {
                                if (rho[d] >= rw.w) {
                                    const Packed p = Tr::pack(rho[d], i + kl + d);
                                    if (Tr::pgt(p, best)) best = p;
                                }
                            }
#pragma unroll
                            for (int o = 16; o > 0; o >>= 1) {
                                const Packed y = Tr::pshfl(best, o);
                                if (Tr::pgt(y, best)) best = y;
                            }
                            if (lane == 0) {
                                Tr::merge(rKey, i, best, hdr);
                                const T v = Tr::pval(best);
                                if (v > sRow[s + u].w) sRow[s + u].w = v;
                            }
                        }
                        __syncwarp();
                    }
#pragma unroll
                    for (int d = 0; d < D; ++d) cs[d].w = sCol[cpos<D>(lane_off + s + D + d)].w;
                }
            }
        }
    }
}

}  // namespace mpgb
