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
// carries a threshold: a lower bound of the best correlation its key already
// holds (kept in the .w lane of the packed statistics, staged with them; +inf
// for flat windows, whose answer is closed-form; keys start seeded).  The
// fast path (fast_subchunk) only asks, per cell, "is rho >= the row's
// threshold or the column's threshold?" (2 compares OR-ed into one
// predicate), so a cell costs 2 FMA + 2 MUL + 2 compares.  A group of D rows
// in which any lane hit is recorded with its starting covariances; after
// each sub-chunk of kQueue groups the recorded groups are replayed with the
// same arithmetic and bookkeeping: the FP32-mixed instantiation reduces the
// group to certified candidates (replay_group_f32, keys in cand_f32.cuh), the
// FP64 one merges (correlation, inverted index) keys by 128-bit CAS
// (replay_group).  Either way ties resolve to the lowest index whatever the
// order tiles run in.
//
// Non-normalised distance (RAW): the same loop ranks cells by the score
// q - h_i - h_j (2 subtractions instead of the 2 multiplies), see internal.cuh.
//
// Anchors.  The first covariance of each diagonal in a tile, and every
// `anchor_every` rows after it, is a dot product of the two windows: exact
// FP64 in the FP64 instantiation; in the FP32-mixed one an FP32 dot product of
// values centred in FP64 (anchor_covariances_f32), whose rounding enters the
// error bias like m more steps of the recurrence.
#pragma once

#include <cmath>

#include "internal.cuh"
#include "cand_f32.cuh"

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
    // The fast path compares an upper bound of the correlation (the covariance
    // carries a bias equal to a bound on its accumulated rounding error); a
    // candidate reaches its key with its bounds, and is compared exactly only
    // where the bounds cannot decide (see cand_f32.cuh).  Packed is the
    // (value, inverted index) word the replay ranks a row's cells by.
    static constexpr bool kBias = true;
    static constexpr float kEps = 1.1920929e-7f;          // 2^-23
    using T = float;
    using S4 = float4;
    using Key = Key128;                           // candidate keys, see cand_f32.cuh
    using Packed = unsigned long long;
    static __device__ __forceinline__ S4 *rs(const Prob &P) { return P.rS32; }
    static __device__ __forceinline__ S4 *cs(const Prob &P) { return P.cS32; }
    static __device__ __forceinline__ S4 ld(const S4 *p) { return __ldcg(p); }
    static __device__ __forceinline__ T inf() { return __int_as_float(0x7f800000); }
    static __device__ __forceinline__ T fma_(T a, T b, T c) { return fmaf(a, b, c); }
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
    static __device__ __forceinline__ long long pidx(Packed a)
    {
        return (long long)(0xFFFFFFFFu - (unsigned)(a & 0xFFFFFFFFull));
    }
};

struct TraitsF64 {
    static constexpr bool kBias = false;        // FP64 recurrence values go to the keys directly
    static constexpr double kEps = 2.220446049250313e-16;
    using T = double;
    using S4 = D4;
    using Key = Key128;
    using Packed = Key128;
    static __device__ __forceinline__ S4 *rs(const Prob &P) { return P.rS64; }
    static __device__ __forceinline__ S4 *cs(const Prob &P) { return P.cS64; }
    static __device__ __forceinline__ S4 ld(const S4 *p)
    {
        const double2 a = __ldcg(reinterpret_cast<const double2 *>(p));
        const double2 b = __ldcg(reinterpret_cast<const double2 *>(p) + 1);
        return make_d4(a.x, a.y, b.x, b.y);
    }
    static __device__ __forceinline__ T inf() { return __longlong_as_double(0x7ff0000000000000ll); }
    static __device__ __forceinline__ T fma_(T a, T b, T c) { return fma(a, b, c); }
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
    static __device__ __forceinline__ long long pidx(Packed a) { return (long long)(~0ull - a.lo); }
    static __device__ __forceinline__ Packed peek(const Key *k)
    {
        Packed p;
        p.hi = __ldcg(&k->hi);
        p.lo = __ldcg(&k->lo);
        return p;
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

// Exact FP64 correlation of row window i and column window j, computed by
// the whole warp (lanes split the window, then a butterfly sum); every lane
// returns the value.  Column mean omitted for the same reason as in the
// anchors.
static __device__ __noinline__ double exact_correlation(const Prob &P, long long i, long long j,
                                                    int lane)
{
    const double *__restrict__ xr = P.rX + i;
    const double *__restrict__ xc = P.cX + j;
    const double mu = P.rMu[i];
    const int m = P.m;
    double acc0 = 0.0, acc1 = 0.0;
    int t = lane;
    for (; t + 96 < m; t += 128) {           // four loads per operand in flight
        const double a0 = __ldg(xr + t), a1 = __ldg(xr + t + 32), a2 = __ldg(xr + t + 64),
                     a3 = __ldg(xr + t + 96);
        const double b0 = __ldg(xc + t), b1 = __ldg(xc + t + 32), b2 = __ldg(xc + t + 64),
                     b3 = __ldg(xc + t + 96);
        acc0 = fma(a0 - mu, b0, acc0);
        acc1 = fma(a1 - mu, b1, acc1);
        acc0 = fma(a2 - mu, b2, acc0);
        acc1 = fma(a3 - mu, b3, acc1);
    }
    for (; t < m; t += 32) acc0 = fma(__ldg(xr + t) - mu, __ldg(xc + t), acc0);
    double acc = acc0 + acc1;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    if (P.raw) return (acc - P.rInv[i]) - P.cInv[j];      // mu = 0, inv = h: the score
    return acc * P.rInv[i] * P.cInv[j];
}

// The value a cell is ranked by: the correlation c invn_i invn_j, or with
// RAW (non-normalised distance) the score q - h_i - h_j = -d^2 / 2; z is the
// stats lane holding invn (or h).
template <bool RAW, class T>
__device__ __forceinline__ T cell_score(T c, T zc, T zr)
{
    if constexpr (RAW) return (c - zc) - zr;
    else return c * zc * zr;
}

// running sums of a staged window's squared norm (1/invn^2, or 2h with RAW),
// df^2, dg^2 and a count (flat, fragile and padding entries skipped); with
// RAW also the largest h (*hmax)
constexpr float kBiasSigma = 2.0f;

template <bool RAW, class S4>
__device__ __forceinline__ void track_max(float *mx, float *hmax, const S4 &v)
{
    const float z = (float)v.z;
    if (RAW ? (z == z) : (z > 0.f)) {
        mx[0] += RAW ? 2.0f * z : __fdividef(1.0f, z * z);   // an RMS estimate: approximate is fine
        mx[1] += (float)v.x * (float)v.x;
        mx[2] += (float)v.y * (float)v.y;
        mx[3] += 1.0f;
        if (RAW) *hmax = fmaxf(*hmax, z);
    }
}

// Asynchronous 16-byte global -> shared copies (L2 reads: thresholds other CTAs
// raised are seen) of one packed statistics entry; stage_wait() completes this
// thread's copies (other threads' need a barrier after it).
template <class S4>
__device__ __forceinline__ void stage_async(S4 *dst, const S4 *src)
{
    const unsigned d = (unsigned)__cvta_generic_to_shared(dst);
    const char *g = reinterpret_cast<const char *>(src);
#pragma unroll
    for (int h = 0; h < (int)(sizeof(S4) / 16); ++h)
        asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(d + 16u * h), "l"(g + 16 * h)
                     : "memory");
}
__device__ __forceinline__ void stage_wait()
{
    asm volatile("cp.async.commit_group;\ncp.async.wait_group 0;\n" ::: "memory");
}

// smem index of staged column q (one padding slot every D entries)
template <int D>
__device__ __forceinline__ int cpos(int q) { return q + q / D; }

// Terms of an FP32-mixed anchor staged in shared memory per pass.
constexpr int kAnchorTerms = 512;

// FP32-mixed anchors: covariances c(a, j0 + d), j0 = a + k0 + lane_off, for
// the D diagonals of every thread of the CTA (all threads call this together;
// it uses the chunk staging area and ends with a barrier).  The same
// centred-row identity as the FP64 anchors: sum_t (x_{a+t} - mu_a) y_{j+t}
// equals sum_t (x_{a+t} - mu_a)(y_{j+t} - g) for any constant g.  The row
// values a_t = x_{a+t} - mu_a are formed in FP64 and rounded to FP32; the
// column values are formed in FP64 against the CTA's reference g0 (the mean
// of its middle column window) and staged as FP32 hi + lo pairs, and each
// thread shifts them to its own reference g (the mean of its middle window)
// in FP32 (b_j = (hi_j - g_hi) + (lo_j - g_lo)), so that its products are
// those of nearly centred windows and the running sums stay near the size of
// the result.  The dot products then run as FP32 FMA chains.  Their rounding
// is bounded like the recurrence's (each step rounds a partial sum at most
// B = ||a|| ||b|| in size), so the caller adds B sqrt(m + 4) to the error
// bias; returned: B, the largest over the warp (the replay shares one bias per
// warp).  The FP32 pipe runs these 64 times faster than FP64 multiply-adds on
// this GPU, which matters where m is large against the tile height.
template <int D, int NT>
static __device__ __noinline__ float anchor_covariances_f32(const Prob &P, long long a, long long k0,
                                                            float *c_out)
{
    constexpr int TD = NT * D;
    constexpr int MT = kAnchorTerms;
    extern __shared__ __align__(32) unsigned char smem_raw[];
    float *sA = reinterpret_cast<float *>(smem_raw);
    float *sHi = sA + MT;
    float *sLo = sHi + cpos<D>(TD + MT);
    const int tid = threadIdx.x;
    const int lane_off = tid * D;
    const int m = P.m;
    const long long last = P.nC - 1;
    const long long lastw = P.lC - 1;
    const long long cb = a + k0;                 // column of diagonal k0 at row a
    const double mu = P.rMu[a];
    const long long wr = cb + TD / 2;
    const double g0 = P.cMu[wr < lastw ? wr : lastw];
    const long long wt = cb + lane_off + D / 2;
    const double dg = (wt <= lastw ? P.cMu[wt] : g0) - g0;
    const float g_hi = (float)dg, g_lo = (float)(dg - (double)g_hi);
    float acc[D];
#pragma unroll
    for (int d = 0; d < D; ++d) acc[d] = 0.0f;
    float sa = 0.0f, sb = 0.0f;
    for (int tb = 0; tb < m; tb += MT) {
        const int mt = min(MT, m - tb);
        const int mtp = (mt + D - 1) / D * D;    // padded with a_t = 0
        for (int q = tid; q < mtp; q += NT)
            sA[q] = q < mt ? (float)(P.rX[a + tb + q] - mu) : 0.0f;
        const int nb = TD + mtp - 1;             // column values lane_off + t + d
        for (int q = tid; q < nb; q += NT) {
            long long j = cb + tb + q;
            j = j < last ? j : last;
            const double v = P.cX[j] - g0;
            const float h = (float)v;
            sHi[cpos<D>(q)] = h;
            sLo[cpos<D>(q)] = (float)(v - (double)h);
        }
        __syncthreads();
        // ring of column values: diagonal d at step t reads slot (t + d) mod D
        float b[D];
#pragma unroll
        for (int v = 0; v < D - 1; ++v) {
            const int q = cpos<D>(lane_off + v);
            b[v] = (sHi[q] - g_hi) + (sLo[q] - g_lo);
            sb = fmaf(b[v], b[v], sb);
        }
        for (int t = 0; t < mtp; t += D) {
#pragma unroll
            for (int u = 0; u < D; ++u) {
                const int q = cpos<D>(lane_off + t + u + D - 1);
                const float bn = (sHi[q] - g_hi) + (sLo[q] - g_lo);
                b[(u + D - 1) % D] = bn;
                sb = fmaf(bn, bn, sb);
                const float at = sA[t + u];
                sa = fmaf(at, at, sa);
#pragma unroll
                for (int d = 0; d < D; ++d) acc[d] = fmaf(at, b[(u + d) % D], acc[d]);
            }
        }
        __syncthreads();
    }
#pragma unroll
    for (int d = 0; d < D; ++d) c_out[d] = (cb + lane_off + d < P.lC) ? acc[d] : 0.0f;
    float bnd = sqrtf(sa) * sqrtf(sb);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) bnd = fmaxf(bnd, __shfl_xor_sync(0xffffffffu, bnd, o));
    return bnd;
}


template <class T, int D>
struct CovArr {
    T v[D];
};

// Replay one group of D rows of a thread's D diagonals from the covariances
// saved at the group's start, with the same arithmetic as the fast path (so
// the correlations are bit-identical), and merge every candidate that reaches
// a row's or a column's threshold into the keys (FP64 path: the recurrence's
// values are exact enough to go to the keys directly).
template <class Tr, int D, bool RAW>
__device__ __noinline__ void replay_group(const Prob &P, typename Tr::S4 *sRow,
                                          typename Tr::S4 *sCol, typename Tr::S4 *rS,
                                          typename Tr::S4 *cS, typename Tr::Key *rKey,
                                          typename Tr::Key *cKey, Hdr *hdr,
                                          CovArr<typename Tr::T, D> c0, long long r, int s,
                                          long long kl, int lane_off, int lane)
{
    using T = typename Tr::T;
    using S4 = typename Tr::S4;
    using Packed = typename Tr::Packed;
    for (int u = 0; u < D; ++u) {
        const S4 rw = sRow[s + u];
        const long long i = r + s + u;
        T rho[D];
        bool rowc[D], colc[D];
        bool any = false;
#pragma unroll
        for (int d = 0; d < D; ++d) {
            const S4 cc = sCol[cpos<D>(lane_off + s + u + d)];
            c0.v[d] = Tr::fma_(rw.x, cc.y, c0.v[d]);
            c0.v[d] = Tr::fma_(cc.x, rw.y, c0.v[d]);
            rho[d] = cell_score<RAW>(c0.v[d], cc.z, rw.z);
            rowc[d] = rho[d] >= rw.w;
            colc[d] = rho[d] >= cc.w;
            any |= rowc[d] | colc[d];
        }
        if (!__any_sync(0xffffffffu, any)) continue;
        Packed best = Tr::pzero();
#pragma unroll
        for (int d = 0; d < D; ++d) {
            if (colc[d] && index_ok(hdr, i + kl + d, P.lC)) {
                const long long j = i + kl + d;
                const int q = cpos<D>(lane_off + s + u + d);
                Tr::merge(cKey, j, Tr::pack(rho[d], i), hdr);
                if (rho[d] > sCol[q].w) {
                    sCol[q].w = rho[d];
                    cS[j].w = rho[d];
                }
            }
            if (rowc[d]) {
                const Packed p = Tr::pack(rho[d], i + kl + d);
                if (Tr::pgt(p, best)) best = p;
            }
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            const Packed y = Tr::pshfl(best, o);
            if (Tr::pgt(y, best)) best = y;
        }
        if (lane == 0 && Tr::pgt(best, Tr::pzero()) && index_ok(hdr, i, P.lR)) {
            Tr::merge(rKey, i, best, hdr);
            const T v = Tr::pval(best);
            if (v > sRow[s + u].w) {
                sRow[s + u].w = v;
                rS[i].w = v;
            }
        }
        __syncwarp();
    }
}

// Merge candidate c (pending on this lane) into *key.  The whole warp calls
// this together; exact correlations that a decision needs are computed by
// the warp, one at a time.  For a row key (row_side) the candidate index is
// a column and the exact pair is (own, idx); for a column key it is a row and
// the pair is (idx, own).
static __device__ __noinline__ void warp_merge(const Prob &P, bool pending, Cand c, Key128 *key,
                                           bool row_side, long long own, float4 *gthr,
                                           float4 *sthr, int lane, Hdr *hdr)
{
    float kx = 0.0f;
    long long kx_idx = -1;
    for (int round = 0; round < kMergeRounds; ++round) {
        bool need_c = false, need_k = false;
        long long kpair = -1;
        if (pending) {
            const Key128 cur = key_peek(key);
            const int dec = classify(c, cur, kx, kx_idx);
            if (dec == kDiscard) {
                pending = false;
                Cand q = key_cand(cur);
                if (kx_idx >= 0 && q.idx == kx_idx && q.L != q.V) {   // keep what was learnt
                    q.V = q.L = kx;
                    if (key_same(cas128(key, cur, cand_key(q)), cur)) raise_thr(gthr, sthr, kx);
                }
                // the staged threshold may predate the key's candidate (committed by
                // another tile): lift it to the key's lower bound, so this tile stops
                // proposing candidates the key already beats
                if (sthr && q.L > sthr->w) sthr->w = q.L;
            } else if (dec == kReplace) {
                if (key_same(cas128(key, cur, cand_key(c)), cur)) {
                    pending = false;
                    raise_thr(gthr, sthr, c.L);
                }
            } else {
                need_c = (dec & kNeedCand) != 0;
                need_k = (dec & kNeedKey) != 0;
                if (need_k) kpair = key_cand(cur).idx;
            }
        }
        if (!__any_sync(0xffffffffu, pending)) return;
        unsigned mask = __ballot_sync(0xffffffffu, need_c);
        while (mask) {
            const int src = __ffs(mask) - 1;
            mask &= mask - 1;
            const long long a = __shfl_sync(0xffffffffu, row_side ? own : c.idx, src);
            const long long b = __shfl_sync(0xffffffffu, row_side ? c.idx : own, src);
            const bool ok = index_ok(hdr, a, P.lR) & index_ok(hdr, b, P.lC);   // warp-uniform
            const float e = ok ? (float)exact_correlation(P, a, b, lane) : 0.0f;
            if (lane == src) c.V = c.L = e;
        }
        mask = __ballot_sync(0xffffffffu, need_k);
        while (mask) {
            const int src = __ffs(mask) - 1;
            mask &= mask - 1;
            const long long a = __shfl_sync(0xffffffffu, row_side ? own : kpair, src);
            const long long b = __shfl_sync(0xffffffffu, row_side ? kpair : own, src);
            const bool ok = index_ok(hdr, a, P.lR) & index_ok(hdr, b, P.lC);   // warp-uniform
            const float e = ok ? (float)exact_correlation(P, a, b, lane) : 0.0f;
            if (lane == src) {
                kx = e;
                kx_idx = kpair;
            }
        }
    }
    if (pending) set_status(hdr, MP_ETIMEOUT);
}

// A column candidate of one replayed group, staged in shared memory so the
// warp's lanes can merge the group's candidates together.
struct MergeItem {
    float V, L;
    int meta;                                   // source lane | slot o << 5 | row u << 10
    int pad;
};
constexpr int kItemsPerWarp = 32;

// FP32-mixed replay of one group of D rows (see cand_f32.cuh for the keys).
// U = upper bound of a cell's correlation from the biased recurrence; its
// lower bound is U - W, W = 2 ebias invn_i invn_j.
//  * Rows: the row's top cell by U is its candidate; cells whose U reaches the
//    top's lower bound are compared exactly and the best exact one is taken.
//    Lane u keeps row u's candidate; the D row keys are merged together.
//  * Columns: a lane meets each of its 2D-1 columns (offset o = u + d) in up
//    to D cells; every cell at or above the column's threshold competes for
//    the column's slot.  The slot keeps its top cell by U (lower row on a tie);
//    if another cell reaches the top's lower bound, the slot's overlapping
//    cells are compared exactly.  At row u the open slots are u..u+D-1, kept
//    in a register window that shifts by one per row; a closed slot with a
//    candidate goes to a short per-lane list.
// Exact comparisons take a second pass (rare).  The warp's column candidates
// are then compacted through shared memory and merged one per lane, so a
// group costs a few global round trips, not one per cell.
template <int D, bool RAW>
__device__ __forceinline__ void replay_group_f32(const Prob &P, float4 *sRow, float4 *sCol,
                                                 float4 *rS, float4 *cS, Key128 *rKey,
                                                 Key128 *cKey, Hdr *hdr, CovArr<float, D> c0,
                                                 long long r, int s, long long kl, int lane_off,
                                                 int lane, float ebias, MergeItem *items)
{
    constexpr int NS = 2 * D - 1;
    const long long k0 = kl - lane_off;         // first diagonal of the tile
    const CovArr<float, D> cstart = c0;
    // open slots: a?[d] is slot u + d at row u
    float aU[D], aW[D], a2[D];
    int au[D];
#pragma unroll
    for (int d = 0; d < D; ++d) {
        aU[d] = -INFINITY;
        a2[d] = -INFINITY;
        aW[d] = 0.0f;
        au[d] = -1;
    }
    // closed slots with a candidate: V, L, meta = o | u << 5 | verify << 10
    float lV[NS], lL[NS];
    int lmeta[NS];
    int ln = 0;
    unsigned long long rtop = 0ull;             // lane u: row u's top (U, column)
    float rlt = 0.0f;                           // lane u: the top's lower bound
    unsigned bandrows = 0u;                     // rows whose top needs exact comparison

    // pass 1: bounds only.  A row no lane hits (no cell at its row's or its
    // column's threshold) only advances the recurrence; the window of open
    // column slots shifts only while some lane holds one.
    bool open = false;                          // this lane holds an open slot
#pragma unroll 1
    for (int u = 0; u < D; ++u) {
        const float4 rw = sRow[s + u];
        const long long i = r + s + u;
        float U[D];
        bool hit = false;
#pragma unroll
        for (int d = 0; d < D; ++d) {
            const float4 cc = sCol[cpos<D>(lane_off + s + u + d)];
            c0.v[d] = fmaf(rw.x, cc.y, c0.v[d]);
            c0.v[d] = fmaf(cc.x, rw.y, c0.v[d]);
            U[d] = cell_score<RAW>(c0.v[d], cc.z, rw.z);
            hit |= (U[d] >= cc.w) | (U[d] >= rw.w);
        }
        if (__any_sync(0xffffffffu, hit)) {
            float M = -INFINITY;                // the lane's largest cell (lowest column on
            int dm = 0;                         // ties; NaN never wins)
#pragma unroll
            for (int d = 0; d < D; ++d) {
                const float4 cc = sCol[cpos<D>(lane_off + s + u + d)];
                if (U[d] >= cc.w) {
                    open = true;
                    if (U[d] > aU[d]) {
                        a2[d] = aU[d];
                        aU[d] = U[d];
                        aW[d] = RAW ? 2.0f * ebias : 2.0f * ebias * cc.z * rw.z;
                        au[d] = u;
                    } else if (U[d] > a2[d]) {
                        a2[d] = U[d];
                    }
                }
                if (U[d] > M) {
                    M = U[d];
                    dm = d;
                }
            }
            unsigned long long top = M >= rw.w ? TraitsF32::pack(M, i + kl + dm) : 0ull;
            // rows hit only through columns skip the row reduction
            if (__any_sync(0xffffffffu, top != 0ull)) {
#pragma unroll
                for (int o = 16; o > 0; o >>= 1) {
                    const unsigned long long y = __shfl_xor_sync(0xffffffffu, top, o);
                    if (y > top) top = y;
                }
                const long long jt = TraitsF32::pidx(top);     // warp-uniform
                const float czt = sCol[cpos<D>((int)(jt - r - k0))].z;
                const float lt = TraitsF32::pval(top) - (RAW ? 2.0f * ebias : 2.0f * ebias * czt * rw.z);
                bool band = false;
#pragma unroll
                for (int d = 0; d < D; ++d)
                    band |= (U[d] >= rw.w) && (i + kl + d != jt) && (U[d] >= lt);
                if (__any_sync(0xffffffffu, band)) bandrows |= 1u << u;
                if (lane == u) {
                    rtop = top;
                    rlt = lt;
                }
            }
        }
        if (__any_sync(0xffffffffu, open)) {
            // slot u is closed: list it, shift the window
            if (au[0] >= 0) {
                lV[ln] = aU[0];
                lL[ln] = aU[0] - aW[0];
                lmeta[ln] = u | (au[0] << 5) | ((a2[0] >= aU[0] - aW[0]) ? 1 << 10 : 0);
                ++ln;
            }
#pragma unroll
            for (int d = 0; d + 1 < D; ++d) {
                aU[d] = aU[d + 1];
                aW[d] = aW[d + 1];
                a2[d] = a2[d + 1];
                au[d] = au[d + 1];
            }
            aU[D - 1] = -INFINITY;
            a2[D - 1] = -INFINITY;
            aW[D - 1] = 0.0f;
            au[D - 1] = -1;
            open = false;
#pragma unroll
            for (int d = 0; d + 1 < D; ++d) open |= au[d] >= 0;
        }
    }
#pragma unroll
    for (int d = 0; d + 1 < D; ++d)             // slots D .. 2D-2
        if (au[d] >= 0) {
            lV[ln] = aU[d];
            lL[ln] = aU[d] - aW[d];
            lmeta[ln] = (D + d) | (au[d] << 5) | ((a2[d] >= aU[d] - aW[d]) ? 1 << 10 : 0);
            ++ln;
        }

    // pass 2 (rare): exact comparisons for overlapping slot cells and row bands
    bool anyv = false;
    for (int k = 0; k < ln; ++k) anyv |= (lmeta[k] >> 10) & 1;
    unsigned long long rex = 0ull;               // lane u: row u's best exact (value, column)
    if (__any_sync(0xffffffffu, anyv) || bandrows != 0u) {
        float lo_l[NS];                          // slot o: lower bound of its top, or +inf
        unsigned long long ex_l[NS];             // slot o: best exact (value, row)
        for (int o = 0; o < NS; ++o) {
            lo_l[o] = INFINITY;
            ex_l[o] = 0ull;
        }
        for (int k = 0; k < ln; ++k)
            if ((lmeta[k] >> 10) & 1) lo_l[lmeta[k] & 31] = lL[k];
        c0 = cstart;
#pragma unroll 1
        for (int u = 0; u < D; ++u) {
            const float4 rw = sRow[s + u];
            const long long i = r + s + u;
            const bool rb = (bandrows >> u) & 1u;
            const float ltu = __shfl_sync(0xffffffffu, rlt, u);
            unsigned ms = 0u, mr = 0u;          // this lane's cells (bit d) needing an exact value
#pragma unroll
            for (int d = 0; d < D; ++d) {
                const float4 cc = sCol[cpos<D>(lane_off + s + u + d)];
                c0.v[d] = fmaf(rw.x, cc.y, c0.v[d]);
                c0.v[d] = fmaf(cc.x, rw.y, c0.v[d]);
                const float Uc = cell_score<RAW>(c0.v[d], cc.z, rw.z);
                if (Uc >= lo_l[u + d]) ms |= 1u << d;
                if (rb && Uc >= ltu) mr |= 1u << d;
            }
            // the warp's pending cells, one at a time (lowest lane, then lowest d)
            unsigned long long rbest = 0ull;
            unsigned pend = ms | mr;
#pragma unroll 1
            for (;;) {
                const unsigned has = __ballot_sync(0xffffffffu, pend != 0u);
                if (!has) break;
                const int src = __ffs(has) - 1;
                const int d = __shfl_sync(0xffffffffu, __ffs(pend) - 1, src);
                const unsigned bit = 1u << d;
                const long long j = __shfl_sync(0xffffffffu, kl, src) + i + d;
                const bool ns = (__shfl_sync(0xffffffffu, ms, src) & bit) != 0u;
                const bool nr = (__shfl_sync(0xffffffffu, mr, src) & bit) != 0u;
                if (lane == src) pend &= ~bit;
                const bool ok = index_ok(hdr, i, P.lR) & index_ok(hdr, j, P.lC);
                const float e = ok ? (float)exact_correlation(P, i, j, lane) : 0.0f;
                if (ns && lane == src) {
                    const unsigned long long p = TraitsF32::pack(e, i);
                    if (p > ex_l[u + d]) ex_l[u + d] = p;
                }
                if (nr) {
                    const unsigned long long p = TraitsF32::pack(e, j);
                    if (p > rbest) rbest = p;
                }
            }
            if (lane == u && rb) rex = rbest;
        }
        for (int k = 0; k < ln; ++k)
            if ((lmeta[k] >> 10) & 1) {
                const unsigned long long e = ex_l[lmeta[k] & 31];
                lV[k] = lL[k] = TraitsF32::pval(e);
                lmeta[k] = (lmeta[k] & 31) | ((int)(TraitsF32::pidx(e) - (r + s)) << 5);
            }
    }

    // column candidates: compact the warp's lists through shared memory and
    // merge one per lane per step
    int incl = ln;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int y = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += y;
    }
    const int excl = incl - ln;
    const int total = __shfl_sync(0xffffffffu, incl, 31);
    for (int base = 0; base < total; base += kItemsPerWarp) {
        for (int k = 0; k < ln; ++k) {
            const int g = excl + k;
            if (g >= base && g < base + kItemsPerWarp) {
                MergeItem it;
                it.V = lV[k];
                it.L = lL[k];
                it.meta = lane | ((lmeta[k] & 31) << 5) | (((lmeta[k] >> 5) & 31) << 10);
                it.pad = 0;
                items[g - base] = it;
            }
        }
        __syncwarp();
        const bool has = base + lane < total;
        Cand c;
        c.V = c.L = 0.0f;
        c.idx = -1;
        long long j = 0;
        int q = 0;
        if (has) {
            const MergeItem it = items[lane];
            const int sl = it.meta & 31, o = (it.meta >> 5) & 31, u = it.meta >> 10;
            // the source lane's first diagonal: lane_off is threadIdx.x * D
            const int src_off = lane_off + (sl - lane) * D;
            c.V = it.V;
            c.L = it.L;
            c.idx = r + s + u;
            j = r + s + k0 + src_off + o;
            q = src_off + s + o;
        }
        const bool in = has && index_ok(hdr, j, P.lC);
        warp_merge(P, in, c, cKey + (in ? j : 0), false, j, cS + (in ? j : 0), sCol + cpos<D>(q), lane,
                   hdr);
        __syncwarp();
    }

    // row candidates: lane u merges row u's
    Cand rc;
    rc.V = rc.L = 0.0f;
    rc.idx = -1;
    if (lane < D && rtop != 0ull) {
        if ((bandrows >> lane) & 1u) {
            rc.V = rc.L = TraitsF32::pval(rex);
            rc.idx = TraitsF32::pidx(rex);
        } else {
            rc.V = TraitsF32::pval(rtop);
            rc.L = rlt;
            rc.idx = TraitsF32::pidx(rtop);
        }
    }
    const long long ir = r + s + (lane < D ? lane : 0);
    const bool rin = rc.idx >= 0 && index_ok(hdr, ir, P.lR);
    warp_merge(P, rin, rc, rKey + ir, true, ir, rS + ir, sRow + s + (lane < D ? lane : 0), lane, hdr);
    __syncwarp();
}

// groups the fast path records before their replays run: a whole 512-row
// chunk, so a chunk is one pass of the fast path and then its replays in one
// burst (the replay code runs warm, and the fast path is called once per chunk;
// tile kernel ms at 16 / 32 / 64 groups, variant 7: self-join 2^20 102.7 /
// 101.9 / 100.7, AB 263 / 260 / 258, 4096 ragged walks 1297 / 1287 / 1274, pan
// 68.9 / 67.9 / 66.6).  The FP64 path keeps 16 (its covariances are twice the
// size, and the recorded groups live in local memory).
template <class Tr>
__host__ __device__ constexpr int queue_len() { return Tr::kBias ? 64 : 16; }

// The two halves of a cell's score: the part that depends on the column,
// t = c invn_j (RAW: c - h_j), and the row's factor applied to it,
// t invn_i (RAW: t - h_i).  The second half is non-decreasing in t (invn_i >= 0;
// NaN for an ill-conditioned row makes every comparison false), and rounding is
// monotone, so the largest score of a row's cells is finish(max_d t_d) exactly.
template <bool RAW, class T>
__device__ __forceinline__ T score_part(T c, T zc)
{
    if constexpr (RAW) return c - zc;
    else return c * zc;
}
template <bool RAW, class T>
__device__ __forceinline__ T score_finish(T t, T zr)
{
    if constexpr (RAW) return t - zr;
    else return t * zr;
}
// max / min that ignore a NaN operand (a NaN score never reaches a threshold)
__device__ __forceinline__ float vmax(float a, float b) { return fmaxf(a, b); }
__device__ __forceinline__ double vmax(double a, double b) { return fmax(a, b); }
__device__ __forceinline__ float vmin(float a, float b) { return fminf(a, b); }
__device__ __forceinline__ double vmin(double a, double b) { return fmin(a, b); }
// three-input max (one instruction in FP32; NaN operands are ignored like fmaxf's)
__device__ __forceinline__ float vmax3(float a, float b, float c)
{
    float d;
    asm("max.f32 %0, %1, %2, %3;" : "=f"(d) : "f"(a), "f"(b), "f"(c));
    return d;
}
__device__ __forceinline__ double vmax3(double a, double b, double c) { return fmax(fmax(a, b), c); }

// Parts of a group's rows the column test takes separately (see fast_subchunk)
template <class Tr, int D>
__host__ __device__ constexpr int col_quarters()
{
    return Tr::kBias ? (D >= 4 ? 4 : D) : 1;
}

// The largest of a row's D partial scores (three-input maxima where D = 8)
template <int D, class T>
__device__ __forceinline__ T row_max(const T (&tv)[D])
{
    if constexpr (D == 8) {
        T m = vmax3(tv[0], tv[1], tv[2]);
        m = vmax3(m, tv[3], tv[4]);
        m = vmax3(m, tv[5], tv[6]);
        return vmax(m, tv[7]);
    } else {
        T m = tv[0];
#pragma unroll
        for (int d = 1; d < D; ++d) m = vmax(m, tv[d]);
        return m;
    }
}

// The per-cell column test of one group of D rows, re-walked from the
// group's starting covariances c0 (row stats at pr[u], column lane_off + s + v
// at pc[v + v / D]): does any lane's cell reach its column's threshold?  Out of
// line: it runs only for groups the fast path's group-level column test flags,
// and keeps the fast path's registers for the hot loop.
template <class Tr, int D, bool RAW>
static __device__ __noinline__ bool column_recheck(const typename Tr::T *c0,
                                                   const typename Tr::S4 *pr,
                                                   const typename Tr::S4 *pc)
{
    using T = typename Tr::T;
    using S4 = typename Tr::S4;
    T c[D];
#pragma unroll
    for (int d = 0; d < D; ++d) c[d] = c0[d];
    bool colhit = false;
#pragma unroll
    for (int u = 0; u < D; ++u) {
        const S4 rw = pr[u];
#pragma unroll
        for (int d = 0; d < D; ++d) {
            const S4 cc = pc[(u + d) + (u + d) / D];
            c[d] = Tr::fma_(rw.x, cc.y, c[d]);
            c[d] = Tr::fma_(cc.x, rw.y, c[d]);
            colhit |= (cell_score<RAW>(c[d], cc.z, rw.z) >= cc.w);
        }
    }
    return __any_sync(0xffffffffu, colhit);
}

// The hot loop: rows s0 .. s1-1 of the staged chunk (whole groups of D rows)
// for this thread's D diagonals.  It only decides which groups of D rows hold
// a cell whose score reaches its row's or its column's threshold; those groups
// are recorded (their starting covariances) and replayed exactly afterwards.
// Per cell: two FMAs (the covariance update), one multiply (c invn_j) and one
// max (three-input maxima: 4 per row of 8); per row, one multiply by invn_i and
// one compare give the exact row test (the row's largest score against the
// row's threshold).  The column test is first taken for the whole group at
// once: the group's largest score against the smallest threshold of the 2D-1
// columns it touches (tabled when the chunk is staged).  That can
// only flag more groups than the per-cell test, so a group it flags (and the
// row test did not) is re-walked from its starting covariances with the
// per-cell column test before it is recorded.  The column stats walk through a
// D-entry register ring; the row stats are a shared-memory broadcast.  Returns
// the number of groups recorded in q_c0 / q_s.
template <class Tr, int D, int RC, bool RAW>
static __device__ __noinline__ int fast_subchunk(typename Tr::T *c_io, int s0, int s1,
                                                 int lane_off, CovArr<typename Tr::T, D> *q_c0,
                                                 int *q_s)
{
    using T = typename Tr::T;
    using S4 = typename Tr::S4;
    extern __shared__ __align__(32) unsigned char smem_raw[];
    const S4 *sRow = reinterpret_cast<const S4 *>(smem_raw);
    const S4 *sCol = sRow + RC;
    T c[D];
#pragma unroll
    for (int d = 0; d < D; ++d) c[d] = c_io[d];
    // padded column position of lane_off + s + v (s a multiple of D, v <= D):
    // q + q / D = (t + s / D) (D + 1) + v with t = lane_off / D, so each group's
    // column stats sit at constant offsets from one pointer that advances by
    // D + 1 per group
    const int t = lane_off / D;
    const S4 *pc = sCol + (t + s0 / D) * (D + 1);
    const S4 *pr = sRow + s0;
    S4 cs[D];
#pragma unroll
    for (int d = 0; d < D; ++d) cs[d] = pc[d];
    int qn = 0;
    for (int s = s0; s < s1; s += D, pc += D + 1, pr += D) {
        T c0[D];
#pragma unroll
        for (int d = 0; d < D; ++d) c0[d] = c[d];
        S4 rws[D];                              // the group's row stats
#pragma unroll
        for (int u = 0; u < D; ++u) rws[u] = pr[u];
        bool rowhit = false;
        // the largest score of each quarter of the group's rows (a quarter's
        // cells touch D/4 + D - 1 of the group's columns); FP64 compares run on
        // the slow FP64 pipe, so the FP64 kernel takes the group whole
        constexpr int NQ = col_quarters<Tr, D>();
        T gq[NQ];
#pragma unroll
        for (int k = 0; k < NQ; ++k) gq[k] = -Tr::inf();
#pragma unroll
        for (int u = 0; u < D; ++u) {
            const S4 &rw = rws[u];
            T tv[D];
#pragma unroll
            for (int d = 0; d < D; ++d) {
                const S4 &cc = cs[(d + u) % D];
                c[d] = Tr::fma_(rw.x, cc.y, c[d]);
                c[d] = Tr::fma_(cc.x, rw.y, c[d]);
                tv[d] = score_part<RAW>(c[d], cc.z);
            }
            const T M = score_finish<RAW>(row_max<D>(tv), rw.z);
            rowhit |= (M >= rw.w);
            gq[u / (D / NQ)] = vmax(gq[u / (D / NQ)], M);
            cs[u % D] = pc[(D + 1) + u];        // column lane_off + s + u + D
        }
        // each quarter's largest score against the smallest threshold of the
        // columns its cells touch, tabled at staging in the padding slot after
        // the group's first D columns (x, y, z, w: quarters 0..3)
        const S4 tq = pc[D];
        bool colmaybe = gq[0] >= tq.x;
        if constexpr (NQ > 1) colmaybe |= gq[1] >= tq.y;
        if constexpr (NQ > 2) colmaybe |= gq[2] >= tq.z;
        if constexpr (NQ > 3) colmaybe |= gq[3] >= tq.w;
        const bool rec = __any_sync(0xffffffffu, rowhit);
        const bool maybe = !rec && __any_sync(0xffffffffu, colmaybe);
        if (rec || maybe) {
            // record the group; a group the column test only may have flagged is
            // kept after the per-cell column test confirms it
#pragma unroll
            for (int d = 0; d < D; ++d) q_c0[qn].v[d] = c0[d];
            q_s[qn] = s;
            bool keep = rec;
            if (maybe) keep = column_recheck<Tr, D, RAW>(q_c0[qn].v, pr, pc);
            if (keep) ++qn;
        }
    }
#pragma unroll
    for (int d = 0; d < D; ++d) c_io[d] = c[d];
    return qn;
}

template <class Tr, int D, int W, int RC>
struct TileShape {
    static constexpr int NT = W * 32;
    static constexpr int TD = NT * D;
    static constexpr int NCOL = RC + TD;
    static constexpr int NCOLP = NCOL + NCOL / D + 1;
    static constexpr int SMEM_STATS = (RC + NCOLP) * (int)sizeof(typename Tr::S4);
    static constexpr int SMEM = SMEM_STATS + (Tr::kBias ? W * kItemsPerWarp * (int)sizeof(MergeItem) : 0);
};

// MINB: minimum resident CTAs per SM the register allocation must allow
template <class Tr, int D, int W, int RC, int MINB, bool RAW>
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
    MergeItem *sItems = reinterpret_cast<MergeItem *>(smem_raw + Sh::SMEM_STATS) +
                        (threadIdx.x >> 5) * kItemsPerWarp;
    __shared__ unsigned long long s_tile;
    // per-chunk sums of {norm^2, df^2, dg^2, count} over the staged rows and
    // columns, and (RAW) the largest h of each (two parity sets of 12): they
    // size the error bias
    __shared__ float s_mx[24];

    (void)tile_rows;                           // each band carries its own tile height
    const int lane = threadIdx.x & 31;
    const int lane_off = threadIdx.x * D;
    const int nb = hdr->nbands;
    const unsigned long long ntiles = tile_prefix[nb];
    const T INF = Tr::inf();
    constexpr int kQueue = queue_len<Tr>();
    CovArr<T, D> q_c0[kQueue];                 // recorded groups of the current sub-chunk
    int q_s[kQueue];

    for (;;) {
        __syncthreads();
        if (threadIdx.x == 0) s_tile = atomicAdd(&hdr->ticket, 1ull);
        if (threadIdx.x < 24) s_mx[threadIdx.x] = 0.0f;
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
        const long long i0 = (long long)(tile - tile_prefix[lo]) * bd.tile_rows;
        const long long i1 = min(i0 + (long long)bd.tile_rows, rows_end);
        const long long kl = k0 + lane_off;        // slot d walks diagonal kl + d
        S4 *rS = Tr::rs(P);
        S4 *cS = Tr::cs(P);
        Key *rKey = reinterpret_cast<Key *>(P.rKey);
        Key *cKey = reinterpret_cast<Key *>(P.cKey);

        T c[D];
        // error bias of the FP32 recurrence: an estimate E of the accumulated
        // rounding of each covariance since its anchor is kept added to it, so
        // the fast path compares (statistical) upper bounds of the correlations.
        // Rounding errors of N steps behave like a random walk: their standard
        // deviation is about 0.41 eps sqrt(N) |c|, with |c| <= s_i s_j.  E uses
        // the chunks' RMS norms and update terms (largest RMS since the anchor)
        // and about five standard deviations, combined in quadrature with the
        // FP32 anchor's rounding (m FMA steps on partial sums of at most B):
        //   E = kBiasSigma eps hypot(C sqrt(N + 16), B sqrt(m + 4)),
        //   C = s_R s_C + 2 (df_R dg_C + df_C dg_R).
        float e_c = 0.0f, e_applied = 0.0f;
        float e_anchor = 0.0f;                   // FP32 anchors: B sqrt(m + 4)
        int e_steps = 0;
        int chunk = 0;
        for (long long r = i0; r < i1; r += RC, ++chunk) {
            const int nrows = (int)min((long long)RC, i1 - r);
            const int nrr = (nrows + D - 1) / D * D;
            const int par = (chunk & 1) * 12;
            __syncthreads();
            const bool anchor_here = r == i0 || (anchor_every > 0 && (r - i0) % anchor_every == 0);
            if constexpr (Tr::kBias) {
                // covariance at row a = r - 1 so that row r applies the update; at
                // r = 0 the update of row 0 adds 0 (df_0 = dg_0 = 0).  The FP32
                // anchors use the staging area, so they run before the staging.
                if (anchor_here) {
                    const long long a = r > 0 ? r - 1 : 0;
                    float bnd = 0.0f;
                    if (index_ok(hdr, a, lR)) {
                        static_assert(kAnchorTerms + 2 * (TD + kAnchorTerms + kAnchorTerms / D + TD / D) <=
                                          Sh::SMEM_STATS / 4,
                                      "anchor staging larger than the chunk staging area");
                        bnd = anchor_covariances_f32<D, NT>(P, a, k0, c);
                    }
                    e_c = 0.0f;
                    e_applied = 0.0f;
                    e_steps = 0;
                    e_anchor = bnd * sqrtf((float)(P.m + 4));
                }
            }
            // stage {df, dg, invn, thr} of the chunk's rows and columns: copies
            // from L2 (so thresholds raised by other CTAs are seen), all of a
            // thread's issued at once as asynchronous copies (one round trip)
            {
                float mx[8] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
                float hm[2] = {0.f, 0.f};
                const long long cb = r + k0;
                const int ncols = nrr + TD;
                // (loops kept rolled: this code runs once per chunk, and its
                // instructions are mostly fetched cold)
#pragma unroll 1
                for (int t = threadIdx.x; t < nrr; t += NT)
                    if (index_ok(hdr, r + t, lR + kPad)) stage_async(sRow + t, rS + r + t);
#pragma unroll 1
                for (int t = threadIdx.x; t < ncols; t += NT)
                    if (index_ok(hdr, cb + t, lC + kPad)) stage_async(sCol + cpos<D>(t), cS + cb + t);
                stage_wait();
                if (Tr::kBias) {                       // this thread's own entries
#pragma unroll 1
                    for (int t = threadIdx.x; t < nrr; t += NT) track_max<RAW>(mx, hm, sRow[t]);
#pragma unroll 1
                    for (int t = threadIdx.x; t < ncols; t += NT) track_max<RAW>(mx + 4, hm + 1, sCol[cpos<D>(t)]);
                }
                if (Tr::kBias) {
                    // warp sums of the 8 quantities by a transposing butterfly:
                    // each exchange halves the values a lane carries, so lane L
                    // ends with the sum of quantity 4 b4 + 2 b3 + b2 (b = bits of L)
                    const bool h4 = lane & 16, h3 = lane & 8, h2 = lane & 4;
                    float w4[4], w2[2];
#pragma unroll
                    for (int j = 0; j < 4; ++j) {
                        const float keep = h4 ? mx[j + 4] : mx[j], send = h4 ? mx[j] : mx[j + 4];
                        w4[j] = keep + __shfl_xor_sync(0xffffffffu, send, 16);
                    }
#pragma unroll
                    for (int j = 0; j < 2; ++j) {
                        const float keep = h3 ? w4[j + 2] : w4[j], send = h3 ? w4[j] : w4[j + 2];
                        w2[j] = keep + __shfl_xor_sync(0xffffffffu, send, 8);
                    }
                    float v = (h2 ? w2[1] : w2[0]) + __shfl_xor_sync(0xffffffffu, h2 ? w2[0] : w2[1], 4);
                    v += __shfl_xor_sync(0xffffffffu, v, 2);
                    v += __shfl_xor_sync(0xffffffffu, v, 1);
                    if ((lane & 3) == 0 && v > 0.f) atomicAdd(&s_mx[par + (lane >> 2)], v);
                    if (RAW) {                         // h >= 0: integer max on the bits
#pragma unroll
                        for (int k = 0; k < 2; ++k) {
                            float v = hm[k];
#pragma unroll
                            for (int o = 16; o > 0; o >>= 1)
                                v = fmaxf(v, __shfl_xor_sync(0xffffffffu, v, o));
                            if (lane == 0 && v > 0.f)
                                atomicMax(reinterpret_cast<int *>(&s_mx[par + 8 + k]),
                                          __float_as_int(v));
                        }
                    }
                }
            }
            __syncthreads();
            // for every D-aligned window of columns, the smallest threshold of the
            // columns each quarter of a group's rows touches (D/4 + D - 1 columns
            // from offset k D/4), into the padding slot after the window's first D
            // columns (the fast path's column test)
            {
                constexpr int NQ = col_quarters<Tr, D>(), RQ = D / NQ;
#pragma unroll 1
                for (int q8 = threadIdx.x; q8 * D < nrr + TD; q8 += NT) {
                    T mn[4] = {Tr::inf(), Tr::inf(), Tr::inf(), Tr::inf()};
#pragma unroll
                    for (int v = 0; v < 2 * D - 1; ++v) {
                        const int q = q8 * D + v;
                        const T w = q < nrr + TD ? (T)sCol[cpos<D>(q)].w : Tr::inf();
#pragma unroll
                        for (int k = 0; k < NQ; ++k)
                            if (v >= k * RQ && v < k * RQ + RQ + D - 1) mn[k] = vmin(mn[k], w);
                    }
                    S4 &slot = sCol[q8 * (D + 1) + D];
                    slot.x = mn[0];
                    slot.y = mn[1];
                    slot.z = mn[2];
                    slot.w = mn[3];
                }
            }
            __syncthreads();
            if (!Tr::kBias && anchor_here) {
                // as above, exact FP64
                const long long a = r > 0 ? r - 1 : 0;
                if (index_ok(hdr, a, lR)) anchor_covariances<Tr, D>(P, a, a + kl, c);
                e_c = 0.0f;
                e_applied = 0.0f;
                e_steps = 0;
            }
            if (Tr::kBias) {
                const float nr = fmaxf(s_mx[par + 3], 1.0f), nc = fmaxf(s_mx[par + 7], 1.0f);
                const float sr = sqrtf(s_mx[par] / nr), fr = sqrtf(s_mx[par + 1] / nr),
                            gr = sqrtf(s_mx[par + 2] / nr), sc = sqrtf(s_mx[par + 4] / nc),
                            fc = sqrtf(s_mx[par + 5] / nc), gc = sqrtf(s_mx[par + 6] / nc);
                const float hsum = RAW ? s_mx[par + 8] + s_mx[par + 9] : 0.0f;
                if (threadIdx.x < 12) s_mx[12 - par + threadIdx.x] = 0.0f;  // the next chunk's set
                e_c = fmaxf(e_c, sr * sc + 2.0f * (fr * gc + fc * gr));
                e_steps += nrr;
                // RAW adds a bound on this chunk's FP32 rounding of h_i, h_j and of
                // the score's two subtractions: about 3 eps (h_i + h_j) / 2 at most,
                // covered by 2 kBiasSigma eps (largest h of the rows + of the columns)
                // the anchor's rounding adds in quadrature (independent of the
                // recurrence's); hypot form, so no square overflows
                const float er = e_c * sqrtf((float)(e_steps + 16));
                const float eh = fmaxf(er, e_anchor), el = fminf(er, e_anchor);
                const float q = eh > 0.0f ? el / eh : 0.0f;
                const float e = kBiasSigma * (float)Tr::kEps * (eh * sqrtf(1.0f + q * q) + 2.0f * hsum);
                const T inc = (T)(e - e_applied);
                e_applied = e;
#pragma unroll
                for (int d = 0; d < D; ++d) c[d] += inc;
            }
            // the fast path runs over sub-chunks of kQueue groups in a function of
            // its own (its registers are allocated for the hot loop alone); a group
            // with a possible candidate only records its starting covariances, and
            // the recorded groups are replayed after the sub-chunk
            for (int s0 = 0; s0 < nrr; s0 += kQueue * D) {
                const int s1 = min(nrr, s0 + kQueue * D);
                const int qn = fast_subchunk<Tr, D, RC, RAW>(c, s0, s1, lane_off, q_c0, q_s);
                for (int e = 0; e < qn; ++e) {
                    // replay a recorded group from its starting covariances, with
                    // bookkeeping (out of line: it is rare)
                    if constexpr (Tr::kBias)
                        replay_group_f32<D, RAW>(P, sRow, sCol, rS, cS, rKey, cKey, hdr, q_c0[e], r,
                                            q_s[e], kl, lane_off, lane, e_applied, sItems);
                    else
                        replay_group<Tr, D, RAW>(P, sRow, sCol, rS, cS, rKey, cKey, hdr, q_c0[e], r,
                                            q_s[e], kl, lane_off, lane);
                }
            }
        }
    }
}

}  // namespace mpgb
