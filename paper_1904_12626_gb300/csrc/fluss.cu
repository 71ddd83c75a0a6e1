// fluss.cu -- semantic segmentation from a profile index (FLUSS, the paper's
// Sec. 3.4.2 "Semantic segmentation", after Gharghabi et al. 2017).
//
// Every window i with a neighbour PI[i] >= 0 draws an arc between i and
// PI[i].  A regime change is a place few arcs cross: windows of one regime
// find their neighbours inside it.  With a = min(i, PI[i]), b = max(i, PI[i]):
//   AC[k]  = #{ i : a_i <= k < b_i }                       (arc count)
//   IAC[k] = 2 k (l - k) / l                               (expected count when
//            neighbours are uniformly random: a parabola peaking at l/2)
//   CAC[k] = min(AC[k] / IAC[k], 1), and 1 where IAC[k] = 0 or within `edge`
//            positions of either end (too few arcs can cross there)
// Segment boundaries: the lowest CAC (lowest index on ties), then the lowest
// outside +-seg_excl of every boundary found so far, num_segments times.
//
// AC is a difference array (+1 at a, -1 at b, integer atomics) and a prefix
// sum; all integer, so it is exact and independent of the order of the adds.
#include <cmath>

#include "internal.cuh"

namespace mpgb {
namespace {

constexpr int kScanThreads = 1024;
constexpr int kScanItems = 8;                       // per thread
constexpr int kScanTile = kScanThreads * kScanItems;
constexpr int kSegBlocks = 1216;                   // boundary search: partial minima

__global__ void arc_marks_kernel(const int64_t *__restrict__ pi, long long l, int *marks,
                                 unsigned *status)
{
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < l;
         i += (long long)gridDim.x * blockDim.x) {
        const long long p = pi[i];
        if (p < 0) continue;                        // no neighbour: no arc
        if (p >= l) {
            atomicCAS(status, 0u, (unsigned)MP_EINVAL);
            continue;
        }
        const long long a = p < i ? p : i, b = p < i ? i : p;
        if (a == b) continue;
        atomicAdd(marks + a, 1);
        atomicAdd(marks + b, -1);
    }
}

// block-wide inclusive scan of one value per thread (int)
__device__ __forceinline__ int block_inclusive_scan(int v, int *warp_tot)
{
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    int x = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) warp_tot[warp] = x;
    __syncthreads();
    if (warp == 0) {
        int s = warp_tot[lane];
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int y = __shfl_up_sync(0xffffffffu, s, o);
            if (lane >= o) s += y;
        }
        warp_tot[lane] = s;
    }
    __syncthreads();
    const int r = x + (warp > 0 ? warp_tot[warp - 1] : 0);
    __syncthreads();
    return r;
}

// per-tile sums of the marks
__global__ void __launch_bounds__(kScanThreads) tile_sums_kernel(const int *__restrict__ marks,
                                                                 long long l, int *tile_sum)
{
    __shared__ int warp_tot[32];
    const long long base = (long long)blockIdx.x * kScanTile + (long long)threadIdx.x * kScanItems;
    int s = 0;
#pragma unroll
    for (int k = 0; k < kScanItems; ++k)
        if (base + k < l) s += marks[base + k];
    const int tot = block_inclusive_scan(s, warp_tot);
    if (threadIdx.x == kScanThreads - 1) tile_sum[blockIdx.x] = tot;
}

// exclusive scan of the tile sums, by one block
__global__ void __launch_bounds__(kScanThreads) tile_offsets_kernel(int *tile_sum, int ntiles)
{
    __shared__ int warp_tot[32];
    __shared__ int carry;
    if (threadIdx.x == 0) carry = 0;
    __syncthreads();
    for (int b0 = 0; b0 < ntiles; b0 += kScanThreads) {
        const int idx = b0 + threadIdx.x;
        const int v = idx < ntiles ? tile_sum[idx] : 0;
        const int inc = block_inclusive_scan(v, warp_tot);
        const int c = carry;
        if (idx < ntiles) tile_sum[idx] = c + inc - v;
        __syncthreads();
        if (threadIdx.x == kScanThreads - 1) carry = c + inc;
        __syncthreads();
    }
}

// AC by a scan of the tile with its offset, then CAC
__global__ void __launch_bounds__(kScanThreads) cac_kernel(const int *__restrict__ marks,
                                                           const int *__restrict__ tile_off,
                                                           long long l, long long edge,
                                                           double *cac)
{
    __shared__ int warp_tot[32];
    const long long base = (long long)blockIdx.x * kScanTile + (long long)threadIdx.x * kScanItems;
    int v[kScanItems];
    int s = 0;
#pragma unroll
    for (int k = 0; k < kScanItems; ++k) {
        v[k] = base + k < l ? marks[base + k] : 0;
        s += v[k];
    }
    int run = block_inclusive_scan(s, warp_tot) - s + tile_off[blockIdx.x];
    const double dl = (double)l;
#pragma unroll
    for (int k = 0; k < kScanItems; ++k) {
        const long long q = base + k;
        run += v[k];                                 // AC[q] = sum of marks[0..q]
        if (q >= l) continue;
        double c = 1.0;
        const double iac = 2.0 * (double)q * (double)(l - q) / dl;
        if (q >= edge && q < l - edge && iac > 0.0) {
            const double r = (double)run / iac;
            c = r < 1.0 ? r : 1.0;
        }
        cac[q] = c;
    }
}

constexpr int kSegThreads = 256;

// lowest index wins a tie; -1 (no candidate) loses to anything
__device__ __forceinline__ bool seg_better(double v, long long i, double bv, long long bi)
{
    return i >= 0 && (bi < 0 || v < bv || (v == bv && i < bi));
}

// one boundary search, pass 1: per-block minimum of cac over the positions
// not within seg_excl of an earlier boundary (each element checks them all:
// there are few)
__global__ void __launch_bounds__(kSegThreads) seg_partial_kernel(const double *__restrict__ cac,
                                                                  long long l, const int64_t *segments,
                                                                  int s, long long seg_excl,
                                                                  double *pv, long long *pidx)
{
    __shared__ double s_v[kSegThreads / 32];
    __shared__ long long s_i[kSegThreads / 32];
    double bv = INFINITY;
    long long bi = -1;
    for (long long q = (long long)blockIdx.x * blockDim.x + threadIdx.x; q < l;
         q += (long long)gridDim.x * blockDim.x) {
        bool masked = false;
        for (int t = 0; t < s; ++t) {
            const long long b = segments[t];
            if (b < 0) continue;
            const long long d = q > b ? q - b : b - q;
            masked |= (d < seg_excl) || (d == 0);
        }
        if (masked) continue;
        const double v = cac[q];
        if (seg_better(v, q, bv, bi)) {
            bv = v;
            bi = q;
        }
    }
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        const double ov = __shfl_xor_sync(0xffffffffu, bv, o);
        const long long oi = __shfl_xor_sync(0xffffffffu, bi, o);
        if (seg_better(ov, oi, bv, bi)) {
            bv = ov;
            bi = oi;
        }
    }
    if (lane == 0) {
        s_v[warp] = bv;
        s_i[warp] = bi;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        for (int w = 1; w < kSegThreads / 32; ++w)
            if (seg_better(s_v[w], s_i[w], bv, bi)) {
                bv = s_v[w];
                bi = s_i[w];
            }
        pv[blockIdx.x] = bv;
        pidx[blockIdx.x] = bi;
    }
}

// pass 2: the minimum over the blocks' minima is boundary s (one block)
__global__ void __launch_bounds__(kSegThreads) seg_pick_kernel(const double *pv,
                                                               const long long *pidx,
                                                               int nblocks, int64_t *segments,
                                                               int s)
{
    __shared__ double s_v[kSegThreads / 32];
    __shared__ long long s_i[kSegThreads / 32];
    double bv = INFINITY;
    long long bi = -1;
    for (int b = threadIdx.x; b < nblocks; b += blockDim.x)
        if (seg_better(pv[b], pidx[b], bv, bi)) {
            bv = pv[b];
            bi = pidx[b];
        }
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        const double ov = __shfl_xor_sync(0xffffffffu, bv, o);
        const long long oi = __shfl_xor_sync(0xffffffffu, bi, o);
        if (seg_better(ov, oi, bv, bi)) {
            bv = ov;
            bi = oi;
        }
    }
    if (lane == 0) {
        s_v[warp] = bv;
        s_i[warp] = bi;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        for (int w = 1; w < kSegThreads / 32; ++w)
            if (seg_better(s_v[w], s_i[w], bv, bi)) {
                bv = s_v[w];
                bi = s_i[w];
            }
        segments[s] = bi;
    }
}

}  // namespace

size_t fluss_workspace_bytes(long long l)
{
    const long long ntiles = (l + kScanTile - 1) / kScanTile;
    auto up = [](size_t b) { return (b + 255) & ~(size_t)255; };
    return up(256) + up(sizeof(int) * (size_t)(l + 1)) + up(sizeof(int) * (size_t)(ntiles + 1)) +
           up(16 * (size_t)kSegBlocks);
}

cudaError_t launch_fluss(const int64_t *pi, long long l, long long edge, int num_segments,
                         long long seg_excl, double *cac, int64_t *segments, void *ws,
                         cudaStream_t st)
{
    auto up = [](size_t b) { return (b + 255) & ~(size_t)255; };
    const long long ntiles = (l + kScanTile - 1) / kScanTile;
    char *p = (char *)ws;
    unsigned *status = (unsigned *)p;
    p += up(256);
    int *marks = (int *)p;
    p += up(sizeof(int) * (size_t)(l + 1));
    int *tile = (int *)p;
    p += up(sizeof(int) * (size_t)(ntiles + 1));
    double *work = (double *)p;
    cudaError_t e = cudaMemsetAsync(ws, 0, up(256) + sizeof(int) * (size_t)(l + 1), st);
    if (e != cudaSuccess) return e;
    const int threads = 256;
    long long blocks = (l + threads - 1) / threads;
    if (blocks > 4096) blocks = 4096;
    arc_marks_kernel<<<(unsigned)blocks, threads, 0, st>>>(pi, l, marks, status);
    tile_sums_kernel<<<(unsigned)ntiles, kScanThreads, 0, st>>>(marks, l, tile);
    tile_offsets_kernel<<<1, kScanThreads, 0, st>>>(tile, (int)ntiles);
    cac_kernel<<<(unsigned)ntiles, kScanThreads, 0, st>>>(marks, tile, l, edge, cac);
    if (num_segments > 0 && segments) {
        long long nblk = (l + kSegThreads - 1) / kSegThreads;
        if (nblk > kSegBlocks) nblk = kSegBlocks;
        double *pv = work;
        long long *pidx = reinterpret_cast<long long *>(work + kSegBlocks);
        for (int sg = 0; sg < num_segments; ++sg) {
            seg_partial_kernel<<<(unsigned)nblk, kSegThreads, 0, st>>>(cac, l, segments, sg,
                                                                     seg_excl, pv, pidx);
            seg_pick_kernel<<<1, kSegThreads, 0, st>>>(pv, pidx, (int)nblk, segments, sg);
        }
    }
    return cudaGetLastError();
}

}  // namespace mpgb
