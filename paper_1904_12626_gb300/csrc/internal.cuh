// internal.cuh -- shared definitions of the CUDA path of libmpgb (not installed).
//
// Index space.  Every join works on "stats sets": one series seen through one
// window length m.  A set with l windows owns the stats-index range
// [sbase, sbase + l + kPad) of the workspace arrays (per-window statistics,
// packed FP32/FP64 recurrence inputs, keys); the kPad tail entries are
// padding the tile kernels may read past the last window (their inverse norm
// is NaN, so every comparison against them is false).
//
// Problems.  A "problem" is one trapezoid of the distance matrix walked by
// diagonals: cells (i, i+k) for row windows i of one set (R) and column
// windows j = i+k of another (C), k in [kmin, kmax], 0 <= i < l_R,
// 0 <= j < l_C.  A self-join is one problem (R = C, kmin = E); an AB-join is
// two (A rows x B columns for k >= 0, B rows x A columns for k >= 1); a batch
// or a pan profile is one problem per series or per window length.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

#include "mp.h"

namespace mpgb {

// padding entries after each stats set: >= the widest tile (diagonals) plus
// one register-rotation group, see the tile kernels
constexpr int kMaxTileDiags = 1024;
constexpr int kMaxSlots = 16;
constexpr int kPad = kMaxTileDiags + kMaxSlots + 16;

constexpr int kWindowsPerThread = 32;     // stats kernel: windows per thread run
// Bounded device loops: a 128-bit compare-and-swap is retried at most
// kCasRetryLimit times, and a candidate merge takes at most kMergeRounds
// rounds (each round settles every decision that needs no exact value, and
// computes the exact values the next round needs); a loop that runs out
// records MP_ETIMEOUT in the workspace status word and returns.  Both can be
// lowered at compile time (-DMPGB_CAS_RETRY_LIMIT=..., -DMPGB_MERGE_ROUNDS=...)
// so that a test can make them run out.
#ifndef MPGB_CAS_RETRY_LIMIT
#define MPGB_CAS_RETRY_LIMIT (1u << 20)
#endif
#ifndef MPGB_MERGE_ROUNDS
#define MPGB_MERGE_ROUNDS 64
#endif
constexpr unsigned kCasRetryLimit = MPGB_CAS_RETRY_LIMIT;
constexpr int kMergeRounds = MPGB_MERGE_ROUNDS;

// four doubles, 32-byte aligned (two 16-byte vector loads)
struct alignas(32) D4 {
    double x, y, z, w;
};
__host__ __device__ __forceinline__ D4 make_d4(double x, double y, double z, double w)
{
    D4 v;
    v.x = x; v.y = y; v.z = z; v.w = w;
    return v;
}

struct alignas(16) Key128 {               // FP64 path: (ord64(rho), ~index)
    unsigned long long lo, hi;
};

// Workspace header (first 256 bytes of every workspace)
struct Hdr {
    unsigned int status;                  // first device-side mp_status != MP_OK
    unsigned int pad0;
    unsigned long long ticket;            // tile ticket counter of the persistent kernel
    int nbands;                           // bands the tile kernel may take (a prefix of the
                                          // band order; all of them unless anytime)
    int tile_diags;                       // diagonals per band of the planned tile shape
    unsigned long long ntiles;            // number of tiles (same as tile_prefix[nbands])
    unsigned long long frag_count;        // fragile windows found (FP32-mixed path)
    long long band_total;                 // anytime: bands planned
    long long band_done;                  // anytime: bands processed so far
};

// Non-normalised distance (raw = 1; SiMPle's distance, Sec. 3.3.4: no
// z-normalisation): d(i,j)^2 = ||x_i - x_j||^2 = 2 h_i + 2 h_j - 2 q(i,j)
// with q the raw dot product and h_i = ||x_i||^2 / 2.  The joins maximise the
// score s(i,j) = q(i,j) - h_i - h_j = -d^2 / 2 instead of the correlation.
// q follows the same recurrence as the centred product, q(i,j) = q(i-1,j-1)
// + df_i dg_j + df_j dg_i, with df_i = (x_{i+m-1} - x_{i-1}) / 2 and
// dg_i = x_{i+m-1} + x_{i-1}; the per-window arrays hold mu = 0 and h in the
// slot of the inverse norm, and no window is flat or ill-conditioned.
struct StatSet {
    const double *x;                      // FP64 series of this set
    long long n;                          // series length
    long long l;                          // windows (<= 0: empty set)
    long long sbase;                      // first stats index of this set
    long long kmin;                       // self-join: first admissible |i-j|; -1: AB pair
    int m;
    int partner;                          // set whose windows are this set's candidates
    int dir;                              // self-join candidates: 0 both sides, +1 only
                                          // j > i (right profile), -1 only j < i (left)
    int raw;                              // 1: non-normalised distance (see below)
};

// A window is "fragile" when its centred norm is below kFragileFactor times
// the geometric mean norm of its set: the FP32 recurrence's absolute error,
// divided by so small a norm, would swamp its correlations, so the FP32-mixed
// path leaves it out of the tile kernel and handles its pairs exactly.
constexpr double kFragileFactor = 1.0 / 32;

// Packed per-window inputs of the tile kernels, stats-indexed:
// {df, dg, invn, thr} where thr is the running threshold of the index (the
// best correlation merged into its key so far; +inf for flat windows).
struct Prob {
    float4 *rS32, *cS32;                  // FP32 copies (FP32-mixed path)
    D4 *rS64, *cS64;                      // FP64 (FP64 path, anchors, refine)
    const double *rX, *cX;                // FP64 series
    const double *rMu, *cMu;              // window means
    const double *rInv, *cInv;            // exact inverse norms (never masked)
    void *rKey, *cKey;                    // u64 (FP32 path) or Key128 (FP64 path)
    long long lR, lC;                     // windows of the row / column set
    long long nC;                         // column series length
    long long kmin, kmax;                 // inclusive diagonal range
    int m;
    int raw;                              // 1: non-normalised distance
};

struct Band {
    int prob;
    int tile_rows;                        // rows per tile of this band
    long long k0;                         // first diagonal of the band
};

// Finalize descriptor: one output side of one problem family
struct FinDesc {
    const void *key;                      // keys of this side (stats-indexed, own base)
    const double *xR, *muR, *invR;        // own side
    const uint8_t *flatR;
    const double *xC, *muC, *invC;        // candidate side
    const uint8_t *flatC;
    long long l;                          // windows on this side
    long long lC;                         // windows on the candidate side
    long long kmin;                       // self-join: first admissible |i-j|; -1: AB
    long long pad_to;                     // write +inf / -1 for [l, pad_to)
    double *mp;
    long long *pi;
    double scale;                         // multiply MP by this (pan normalisation)
    int m;
    int dir;                              // as StatSet::dir (flat rows' closed-form PI)
    int raw;                              // 1: non-normalised distance
    int pad;
};

// Parameters of the descriptor kernel of a self-join (kind 0), an AB-join
// (kind 1), a pan profile (kind 2) or a left/right self-join (kind 3); passed
// by value so that building the descriptors needs no host-to-device copy
// (capture-safe).
constexpr int kMaxPan = 256;
struct FamilyParams {
    int kind;
    int nm;
    int m;
    int fp64;
    int ms[kMaxPan];
    const double *x64;
    long long n, na, nb;
    double ez;
    unsigned flags;
    unsigned pad;
    double *mu;
    double *inv;
    float4 *s32;
    D4 *s64;
    uint8_t *flat;
    char *keys;
    double *mp_a;
    long long *pi_a;
    double *mp_b;
    long long *pi_b;
    long long out_stride;
    StatSet *sets;
    Prob *probs;
    FinDesc *fins;
};

// ---- small device helpers ----

__device__ __forceinline__ void set_status(Hdr *h, unsigned st)
{
    atomicCAS(&h->status, 0u, st);
}

// Debug builds (-DMP_DEBUG): is index i inside [0, lim)?  If not, record
// MP_EBOUNDS and let the caller skip the access.  Release builds: always true,
// so the check compiles to nothing.
__device__ __forceinline__ bool index_ok(Hdr *h, long long i, long long lim)
{
#ifdef MP_DEBUG
    if (i >= 0 && i < lim) return true;
    set_status(h, MP_EBOUNDS);
    return false;
#else
    (void)h;
    (void)i;
    (void)lim;
    return true;
#endif
}

// order-preserving map of a float's bits to an unsigned integer
__host__ __device__ __forceinline__ unsigned ord32(unsigned u)
{
    return (u & 0x80000000u) ? ~u : (u | 0x80000000u);
}
__host__ __device__ __forceinline__ unsigned unord32(unsigned o)
{
    return (o & 0x80000000u) ? (o & 0x7fffffffu) : ~o;
}
__host__ __device__ __forceinline__ unsigned long long ord64(unsigned long long u)
{
    return (u & 0x8000000000000000ull) ? ~u : (u | 0x8000000000000000ull);
}
__host__ __device__ __forceinline__ unsigned long long unord64(unsigned long long o)
{
    return (o & 0x8000000000000000ull) ? (o & 0x7fffffffffffffffull) : ~o;
}

// ---- launchers (one translation unit each) ----

// stats.cu
cudaError_t launch_convert(const void *x, int dtype, long long n, double *x64, Hdr *hdr,
                           cudaStream_t st);
cudaError_t launch_stats_sets(const StatSet *sets, int nsets, long long total_index,
                              double *mu, double *inv, float4 *s32, D4 *s64, uint8_t *flat,
                              double *set_acc, cudaStream_t st);

// fragile.cu
cudaError_t launch_fragile_mark(const StatSet *sets, int nsets, long long max_l,
                                const double *set_acc, const double *inv, const uint8_t *flat,
                                float4 *s32, D4 *s64, unsigned long long *frag_list, Hdr *hdr,
                                cudaStream_t st);
cudaError_t launch_fragile_pass(const StatSet *sets, const double *mu, const double *inv,
                                const unsigned long long *frag_list, void *keys, int fp64,
                                Hdr *hdr, int grid, cudaStream_t st);
// fluss.cu
size_t fluss_workspace_bytes(long long l);
cudaError_t launch_fluss(const int64_t *pi, long long l, long long edge, int num_segments,
                         long long seg_excl, double *cac, int64_t *segments, void *ws,
                         cudaStream_t st);

// seed.cu
cudaError_t launch_seed(const StatSet *sets, int nsets, long long max_l, const double *mu,
                        const double *inv, const uint8_t *flat, float4 *s32, D4 *s64,
                        void *keys, int fp64, cudaStream_t st);
cudaError_t launch_stats_public(const void *x, int dtype, long long n, int m, double *mu,
                                double *invn, double *df, double *dg, uint8_t *flat,
                                cudaStream_t st);

// plan.cu
// scratch: at least max_bands + 1 long longs
cudaError_t launch_plan(const Prob *probs, int nprob, int tile_diags, int tile_rows,
                        long long *band_off, Band *bands, unsigned long long *tile_prefix,
                        long long *scratch, long long max_bands, Hdr *hdr, cudaStream_t st);
// anytime self-join: put the bands in a seeded random order (splitmix64,
// Fisher-Yates) and open the window of bands [done, ceil(fraction * total))
cudaError_t launch_permute_bands(unsigned long long seed, Band *bands,
                                 unsigned long long *tile_prefix, long long *scratch,
                                 long long max_bands, Hdr *hdr, cudaStream_t st);
cudaError_t launch_anytime_window(double fraction, const unsigned long long *tile_prefix,
                                  Hdr *hdr, cudaStream_t st);
cudaError_t launch_family_descs(const FamilyParams &F, cudaStream_t st);
cudaError_t launch_batched_descs(const int64_t *offsets, const int32_t *ms, int B, double ez,
                                 unsigned flags, int fp64, const double *x64, double *mu,
                                 double *inv, float4 *s32, D4 *s64, uint8_t *flat, void *keys,
                                 double *mp, int64_t *pi, const int64_t *out_offsets,
                                 StatSet *sets, Prob *probs, FinDesc *fins, Hdr *hdr,
                                 cudaStream_t st);

// join_fp32.cu / join_fp64.cu
int f32_variant_count();
bool f32_variant_info(int v, int *tile_diags, int *chunk_rows, int *threads, int *smem);
cudaError_t launch_join_f32(int v, const Prob *probs, const Band *bands,
                            const unsigned long long *tile_prefix, Hdr *hdr, int tile_rows,
                            int anchor_every, int grid, cudaStream_t st);
int f32_blocks_per_sm(int v);
int f32_raw_blocks_per_sm();
cudaError_t launch_join_f32_raw(const Prob *probs, const Band *bands,
                                const unsigned long long *tile_prefix, Hdr *hdr, int tile_rows,
                                int anchor_every, int grid, cudaStream_t st);
int f64_variant_count();
bool f64_variant_info(int v, int *tile_diags, int *chunk_rows, int *threads, int *smem);
cudaError_t launch_join_f64(int v, const Prob *probs, const Band *bands,
                            const unsigned long long *tile_prefix, Hdr *hdr, int tile_rows,
                            int anchor_every, int grid, cudaStream_t st);
int f64_blocks_per_sm(int v);
int f64_raw_blocks_per_sm();
cudaError_t launch_join_f64_raw(const Prob *probs, const Band *bands,
                                const unsigned long long *tile_prefix, Hdr *hdr, int tile_rows,
                                int anchor_every, int grid, cudaStream_t st);

// finalize.cu
cudaError_t launch_bind_outputs(FinDesc *fins, double *mp, long long *pi, cudaStream_t st);
cudaError_t launch_finalize(const FinDesc *fins, int nfin, long long max_len, int fp64,
                            int refine, cudaStream_t st);

// backward.cu
cudaError_t launch_backward(const double *x64, long long n, int m, const double *mu,
                            const double *invn, const uint8_t *flat, const int64_t *pi,
                            const double *grad_mp, double *grad_x, Hdr *hdr, cudaStream_t st);

}  // namespace mpgb
