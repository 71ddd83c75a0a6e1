// plan.cu -- problem descriptors and the tile work-queue.
//
// The distance matrix of every problem is cut into bands of `tile_diags`
// consecutive diagonals (the paper's SCRIMP evaluates the matrix diagonal by
// diagonal in any order, Sec. 3.3.3) and each band into tiles of `tile_rows`
// rows.  The planner writes one Band per band and an exclusive prefix sum of
// tiles per band; the persistent tile kernels turn a ticket into
// (band, row tile) with a binary search over that prefix.  Everything is
// computed on the device from device-resident descriptors, so a whole join
// (including batches whose sizes live only on the device) can be recorded in
// a CUDA graph.
#include <cmath>

#include "internal.cuh"

namespace mpgb {
namespace {

// Exclusive scan of a[0..n) in place by one block; a[n] receives the total.
template <typename T>
__device__ void block_exclusive_scan(T *a, long long n)
{
    __shared__ T warp_tot[32];
    __shared__ T carry;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int nwarps = (blockDim.x + 31) >> 5;
    if (tid == 0) carry = 0;
    __syncthreads();
    for (long long base = 0; base < n; base += blockDim.x) {
        const long long idx = base + tid;
        const T v = idx < n ? a[idx] : (T)0;
        T x = v;
        for (int o = 1; o < 32; o <<= 1) {
            const T y = __shfl_up_sync(0xffffffffu, x, o);
            if (lane >= o) x += y;
        }
        if (lane == 31) warp_tot[warp] = x;
        __syncthreads();
        if (warp == 0) {
            T s = lane < nwarps ? warp_tot[lane] : (T)0;
            for (int o = 1; o < 32; o <<= 1) {
                const T y = __shfl_up_sync(0xffffffffu, s, o);
                if (lane >= o) s += y;
            }
            warp_tot[lane] = s;
        }
        __syncthreads();
        const T pre = carry + (warp > 0 ? warp_tot[warp - 1] : (T)0);
        if (idx < n) a[idx] = pre + x - v;
        __syncthreads();
        if (tid == blockDim.x - 1) carry = pre + x;
        __syncthreads();
    }
    if (tid == 0) a[n] = carry;
    __syncthreads();
}

constexpr int kEarlyBands = 16;            // bands of each problem planned in short tiles
constexpr int kEarlyTileRows = 1024;

// Band order: round b holds band b of every problem that has one, problems in
// order.  The tile queue hands out tickets in this order, so the CTAs in flight
// at any time work on neighbouring bands of many problems, and each problem's
// bands start roughly nearest first: a band then compares against keys its
// problem's earlier bands have already improved.  (In problem-major order all
// the bands of a small problem would run at once against the seeds alone and
// most of their candidates would lose at the keys.)
__global__ void plan_kernel(const Prob *__restrict__ probs, int nprob, int TD, int TR,
                            long long *band_off, Band *bands, unsigned long long *tile_prefix,
                            long long max_bands, long long *scratch, Hdr *hdr)
{
    __shared__ long long s_max[32];
    long long my_max = 0;
    for (int p = threadIdx.x; p < nprob; p += blockDim.x) {
        const Prob P = probs[p];
        long long nb = 0;
        if (P.lR > 0 && P.lC > 0 && P.kmax >= P.kmin) nb = (P.kmax - P.kmin) / TD + 1;
        band_off[p] = nb;
        my_max = nb > my_max ? nb : my_max;
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        const long long y = __shfl_xor_sync(0xffffffffu, my_max, o);
        my_max = y > my_max ? y : my_max;
    }
    if ((threadIdx.x & 31) == 0) s_max[threadIdx.x >> 5] = my_max;
    __syncthreads();
    long long max_nb = 0;
    for (int w = 0; w < (int)((blockDim.x + 31) >> 5); ++w) max_nb = s_max[w] > max_nb ? s_max[w] : max_nb;
    block_exclusive_scan<long long>(band_off, nprob);
    long long total = band_off[nprob];
    if (total > max_bands) {                   // workspace sized too small: plan nothing
        if (threadIdx.x == 0) set_status(hdr, MP_ENOMEM);
        total = 0;
        max_nb = 0;
    }
    // slots of round b start at the number of bands of the earlier rounds
    for (long long b = threadIdx.x; b < max_nb; b += blockDim.x) {
        long long c = 0;
        for (int p = 0; p < nprob; ++p) c += (band_off[p + 1] - band_off[p]) > b;
        scratch[b] = c;
    }
    __syncthreads();
    block_exclusive_scan<long long>(scratch, max_nb);
    for (long long b = threadIdx.x; b < max_nb; b += blockDim.x) {
        long long slot = scratch[b];
        // the first bands go in short tiles: with tiles of TR rows about
        // (CTAs / tiles per band) bands would run at once, all against the
        // seeds' thresholds; short tiles let them finish nearly in order,
        // so each starts from the keys its predecessors improved
        const int tr = b < kEarlyBands ? (TR < kEarlyTileRows ? TR : kEarlyTileRows) : TR;
        for (int p = 0; p < nprob; ++p) {
            if (band_off[p + 1] - band_off[p] <= b) continue;
            const Prob P = probs[p];
            const long long k0 = P.kmin + b * TD;
            const long long rows = min(P.lR, P.lC - k0);
            Band bd;
            bd.prob = p;
            bd.tile_rows = tr;
            bd.k0 = k0;
            bands[slot] = bd;
            tile_prefix[slot] = rows > 0 ? (unsigned long long)((rows + tr - 1) / tr) : 0ull;
            ++slot;
        }
    }
    __syncthreads();
    block_exclusive_scan<unsigned long long>(tile_prefix, total);
    if (threadIdx.x == 0) {
        hdr->nbands = (int)total;
        hdr->tile_diags = TD;
        hdr->ntiles = tile_prefix[total];
        hdr->ticket = 0ull;
    }
}

// splitmix64 (Steele, Lea and Flood, 2014): the state advances by the golden
// ratio constant and each output is a bijective mix of the state
__device__ __forceinline__ unsigned long long splitmix64(unsigned long long &state)
{
    state += 0x9E3779B97F4A7C15ull;
    unsigned long long z = state;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

// Reorder the planned bands: slot s takes band perm[s], perm a Fisher-Yates
// shuffle of 0..nb-1 (for i = nb-1 .. 1: swap perm[i] and perm[r % (i+1)],
// r the next splitmix64 output), then rebuild the tile prefix in slot order.
__global__ void permute_bands_kernel(unsigned long long seed, Band *bands,
                                     unsigned long long *tile_prefix, long long *scratch,
                                     long long max_bands, Hdr *hdr)
{
    const long long nb = hdr->nbands;
    long long *perm = scratch;                             // [0, nb)
    Band *old = reinterpret_cast<Band *>(scratch + max_bands);   // [0, nb)
    unsigned long long *cnt = reinterpret_cast<unsigned long long *>(old + max_bands);
    if (threadIdx.x == 0) {
        for (long long s = 0; s < nb; ++s) perm[s] = s;
        unsigned long long st = seed;
        for (long long i = nb - 1; i >= 1; --i) {
            const long long j = (long long)(splitmix64(st) % (unsigned long long)(i + 1));
            const long long t = perm[i];
            perm[i] = perm[j];
            perm[j] = t;
        }
    }
    __syncthreads();
    for (long long s = threadIdx.x; s < nb; s += blockDim.x) {
        old[s] = bands[s];
        cnt[s] = tile_prefix[s + 1] - tile_prefix[s];
    }
    __syncthreads();
    for (long long s = threadIdx.x; s < nb; s += blockDim.x) {
        bands[s] = old[perm[s]];
        tile_prefix[s] = cnt[perm[s]];
    }
    __syncthreads();
    block_exclusive_scan<unsigned long long>(tile_prefix, nb);
    if (threadIdx.x == 0) {
        hdr->band_total = nb;
        hdr->band_done = 0;
        hdr->nbands = 0;                                   // nothing open yet
        hdr->ticket = 0ull;
        hdr->ntiles = 0ull;
    }
}

__global__ void anytime_window_kernel(double fraction, const unsigned long long *tile_prefix,
                                      Hdr *hdr)
{
    const long long total = hdr->band_total;
    const long long s0 = hdr->band_done;
    long long s1 = (long long)ceil(fraction * (double)total);
    if (s1 > total) s1 = total;
    if (s1 < s0) s1 = s0;
    hdr->ticket = tile_prefix[s0];
    hdr->nbands = (int)s1;
    hdr->ntiles = tile_prefix[s1];
    hdr->band_done = s1;
}

}  // namespace

cudaError_t launch_plan(const Prob *probs, int nprob, int tile_diags, int tile_rows,
                        long long *band_off, Band *bands, unsigned long long *tile_prefix,
                        long long *scratch,
                        long long max_bands, Hdr *hdr, cudaStream_t st)
{
    plan_kernel<<<1, 1024, 0, st>>>(probs, nprob, tile_diags, tile_rows, band_off, bands,
                                    tile_prefix, max_bands, scratch, hdr);
    return cudaGetLastError();
}

// ---- descriptors of a self-join, an AB-join or a pan profile ----

namespace {

__device__ __forceinline__ long long first_diag(int m, double ez, unsigned flags)
{
    long long e = (long long)ceil(ez * (double)m);
    if (flags & MP_FLAG_EXCL_INCLUSIVE) e += 1;
    return e;
}

__global__ void family_descs_kernel(FamilyParams F)
{
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    const int RAW = (F.flags & MP_FLAG_RAW) ? 1 : 0;
    const size_t ksz = sizeof(Key128);
    if (F.kind == 0 || F.kind == 2) {          // self-join / pan: one set, problem, output per m
        const int nset = F.kind == 0 ? 1 : F.nm;
        if (k >= nset) return;
        const int m = F.kind == 0 ? F.m : F.ms[k];
        const long long l = F.n - m + 1;
        const long long sb = (long long)k * (F.n + kPad);
        StatSet S;
        S.x = F.x64; S.n = F.n; S.l = l; S.sbase = sb; S.m = m; S.partner = k;
        S.kmin = first_diag(m, F.ez, F.flags);
        S.dir = 0; S.raw = RAW;
        F.sets[k] = S;
        Prob P;
        P.rS32 = P.cS32 = F.s32 ? F.s32 + sb : nullptr;
        P.rS64 = P.cS64 = F.s64 + sb;
        P.rX = P.cX = F.x64;
        P.rMu = P.cMu = F.mu + sb;
        P.rInv = P.cInv = F.inv + sb;
        P.rKey = P.cKey = F.keys + (size_t)sb * ksz;
        P.lR = P.lC = l;
        P.nC = F.n;
        P.kmin = first_diag(m, F.ez, F.flags);
        P.kmax = l - 1;
        P.m = m;
        P.raw = RAW;
        F.probs[k] = P;
        FinDesc D;
        D.key = P.rKey;
        D.xR = D.xC = F.x64;
        D.muR = D.muC = P.rMu;
        D.invR = D.invC = P.rInv;
        D.flatR = D.flatC = F.flat + sb;
        D.l = l; D.lC = l;
        D.kmin = P.kmin;
        D.pad_to = F.kind == 0 ? l : F.out_stride;
        D.mp = F.mp_a + (long long)k * F.out_stride;
        D.pi = F.pi_a + (long long)k * F.out_stride;
        D.scale = (F.flags & MP_FLAG_PAN_NORMALIZE) && F.kind == 2 ? 1.0 / sqrt(2.0 * m) : 1.0;
        D.m = m;
        D.dir = 0; D.raw = RAW; D.pad = 0;
        F.fins[k] = D;
        return;
    }
    if (F.kind == 3) {
        // left/right self-join: the series enters twice, as set 0 (right role:
        // its keys collect j > i) and set 1 (left role: keys collect j < i);
        // one problem, rows = set 0, columns = set 1, diagonals E .. l-1, so a
        // cell (i, i+k) offers j = i+k to i's right key and i to j's left key.
        if (k >= 2) return;
        const int m = F.m;
        const long long l = F.n - m + 1;
        const long long E = first_diag(m, F.ez, F.flags);
        const long long sb0 = 0, sb1 = F.n + kPad;
        const long long sb = k == 0 ? sb0 : sb1;
        StatSet S;
        S.x = F.x64; S.n = F.n; S.l = l; S.sbase = sb; S.m = m; S.partner = 1 - k;
        S.kmin = E;
        S.dir = k == 0 ? 1 : -1; S.raw = RAW;
        F.sets[k] = S;
        if (k == 0) {
            Prob P;
            P.rS32 = F.s32 ? F.s32 + sb0 : nullptr;
            P.cS32 = F.s32 ? F.s32 + sb1 : nullptr;
            P.rS64 = F.s64 + sb0;
            P.cS64 = F.s64 + sb1;
            P.rX = P.cX = F.x64;
            P.rMu = F.mu + sb0;
            P.cMu = F.mu + sb1;
            P.rInv = F.inv + sb0;
            P.cInv = F.inv + sb1;
            P.rKey = F.keys + (size_t)sb0 * ksz;
            P.cKey = F.keys + (size_t)sb1 * ksz;
            P.lR = P.lC = l;
            P.nC = F.n;
            P.kmin = E;
            P.kmax = l - 1;
            P.m = m;
            P.raw = RAW;
            F.probs[0] = P;
        }
        FinDesc D;
        D.key = F.keys + (size_t)sb * ksz;
        D.xR = D.xC = F.x64;
        D.muR = F.mu + sb;
        D.muC = F.mu + (k == 0 ? sb1 : sb0);
        D.invR = F.inv + sb;
        D.invC = F.inv + (k == 0 ? sb1 : sb0);
        D.flatR = F.flat + sb;
        D.flatC = F.flat + (k == 0 ? sb1 : sb0);
        D.l = l; D.lC = l;
        D.kmin = E;
        D.pad_to = l;
        D.mp = k == 0 ? F.mp_a : F.mp_b;
        D.pi = k == 0 ? F.pi_a : F.pi_b;
        D.scale = 1.0;
        D.m = m;
        D.dir = S.dir; D.raw = RAW; D.pad = 0;
        F.fins[k] = D;
        return;
    }
    // AB-join: sets 0 (A) and 1 (B); problem 0 = A rows x B columns (k >= 0),
    // problem 1 = B rows x A columns (k >= 1); outputs A side then B side.
    if (k >= 2) return;
    const int m = F.m;
    const long long la = F.na - m + 1, lb = F.nb - m + 1;
    const long long sbA = 0, sbB = F.na + kPad;
    const double *xa = F.x64, *xb = F.x64 + F.na;
    StatSet S;
    S.m = m; S.partner = 1 - k; S.kmin = -1; S.dir = 0; S.raw = RAW;
    if (k == 0) { S.x = xa; S.n = F.na; S.l = la; S.sbase = sbA; }
    else { S.x = xb; S.n = F.nb; S.l = lb; S.sbase = sbB; }
    F.sets[k] = S;
    const bool rowA = (k == 0);
    const long long sbR = rowA ? sbA : sbB, sbC = rowA ? sbB : sbA;
    Prob P;
    P.rS32 = F.s32 ? F.s32 + sbR : nullptr;
    P.cS32 = F.s32 ? F.s32 + sbC : nullptr;
    P.rS64 = F.s64 + sbR;
    P.cS64 = F.s64 + sbC;
    P.rX = rowA ? xa : xb;
    P.cX = rowA ? xb : xa;
    P.rMu = F.mu + sbR;
    P.cMu = F.mu + sbC;
    P.rInv = F.inv + sbR;
    P.cInv = F.inv + sbC;
    P.rKey = F.keys + (size_t)sbR * ksz;
    P.cKey = F.keys + (size_t)sbC * ksz;
    P.lR = rowA ? la : lb;
    P.lC = rowA ? lb : la;
    P.nC = rowA ? F.nb : F.na;
    P.kmin = rowA ? 0 : 1;
    P.kmax = P.lC - 1;
    P.m = m;
    P.raw = RAW;
    F.probs[k] = P;
    FinDesc D;
    D.key = P.rKey;
    D.xR = P.rX; D.muR = P.rMu; D.invR = P.rInv; D.flatR = F.flat + sbR;
    D.xC = P.cX; D.muC = P.cMu; D.invC = P.cInv; D.flatC = F.flat + sbC;
    D.l = P.lR; D.lC = P.lC;
    D.kmin = -1;
    D.pad_to = P.lR;
    D.mp = rowA ? F.mp_a : F.mp_b;
    D.pi = rowA ? F.pi_a : F.pi_b;
    D.scale = 1.0;
    D.m = m;
    D.dir = 0; D.raw = RAW; D.pad = 0;
    F.fins[k] = D;
}

__global__ void batched_descs_kernel(const int64_t *__restrict__ offsets,
                                     const int32_t *__restrict__ ms, int B, double ez,
                                     unsigned flags, int fp64, const double *x64, double *mu,
                                     double *inv, float4 *s32, D4 *s64, uint8_t *flat, char *keys,
                                     double *mp,
                                     int64_t *pi, const int64_t *__restrict__ out_offsets,
                                     StatSet *sets, Prob *probs, FinDesc *fins, Hdr *hdr)
{
    const int RAW = (flags & MP_FLAG_RAW) ? 1 : 0;
    const int b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= B) return;
    const size_t ksz = sizeof(Key128);
    const long long o0 = offsets[0];
    const long long off = offsets[b] - o0;
    const long long n = offsets[b + 1] - offsets[b];
    const int m = ms[b];
    long long l = n - m + 1;
    if (m < 4 || n < 0) {
        set_status(hdr, MP_EINVAL);
        l = 0;
    }
    if (l < 0) l = 0;
    const long long cap = out_offsets[b + 1] - out_offsets[b];
    if (l > cap) {
        set_status(hdr, MP_EINVAL);
        l = 0;
    }
    const long long sb = off + (long long)b * kPad;
    StatSet S;
    S.x = x64 + off; S.n = n; S.l = l; S.sbase = sb; S.m = m; S.partner = b;
    S.kmin = first_diag(m, ez, flags);
    S.dir = 0; S.raw = RAW;
    sets[b] = S;
    Prob P;
    P.rS32 = P.cS32 = s32 ? s32 + sb : nullptr;
    P.rS64 = P.cS64 = s64 + sb;
    P.rX = P.cX = x64 + off;
    P.rMu = P.cMu = mu + sb;
    P.rInv = P.cInv = inv + sb;
    P.rKey = P.cKey = keys + (size_t)sb * ksz;
    P.lR = P.lC = l;
    P.nC = n;
    P.kmin = first_diag(m, ez, flags);
    P.kmax = l - 1;
    P.m = m;
    P.raw = RAW;
    probs[b] = P;
    FinDesc D;
    D.key = P.rKey;
    D.xR = D.xC = P.rX;
    D.muR = D.muC = P.rMu;
    D.invR = D.invC = P.rInv;
    D.flatR = D.flatC = flat + sb;
    D.l = l; D.lC = l;
    D.kmin = P.kmin;
    D.pad_to = l;
    D.mp = mp + out_offsets[b];
    D.pi = (long long *)pi + out_offsets[b];
    D.scale = 1.0;
    D.m = m;
    D.dir = 0; D.raw = RAW; D.pad = 0;
    fins[b] = D;
}

}  // namespace

cudaError_t launch_family_descs(const FamilyParams &F, cudaStream_t st)
{
    family_descs_kernel<<<1, 256, 0, st>>>(F);
    return cudaGetLastError();
}

cudaError_t launch_batched_descs(const int64_t *offsets, const int32_t *ms, int B, double ez,
                                 unsigned flags, int fp64, const double *x64, double *mu,
                                 double *inv, float4 *s32, D4 *s64, uint8_t *flat, void *keys,
                                 double *mp, int64_t *pi,
                                 const int64_t *out_offsets, StatSet *sets, Prob *probs,
                                 FinDesc *fins, Hdr *hdr, cudaStream_t st)
{
    const int threads = 256;
    batched_descs_kernel<<<(B + threads - 1) / threads, threads, 0, st>>>(
        offsets, ms, B, ez, flags, fp64, x64, mu, inv, s32, s64, flat, (char *)keys, mp, pi,
        out_offsets,
        sets, probs, fins, hdr);
    return cudaGetLastError();
}

}  // namespace mpgb

namespace mpgb {

cudaError_t launch_permute_bands(unsigned long long seed, Band *bands,
                                 unsigned long long *tile_prefix, long long *scratch,
                                 long long max_bands, Hdr *hdr, cudaStream_t st)
{
    permute_bands_kernel<<<1, 1024, 0, st>>>(seed, bands, tile_prefix, scratch, max_bands, hdr);
    return cudaGetLastError();
}

cudaError_t launch_anytime_window(double fraction, const unsigned long long *tile_prefix,
                                  Hdr *hdr, cudaStream_t st)
{
    anytime_window_kernel<<<1, 1, 0, st>>>(fraction, tile_prefix, hdr);
    return cudaGetLastError();
}

}  // namespace mpgb
