/*
 * mp.h -- C ABI of libmpgb, a matrix profile library for one NVIDIA GB300.
 *
 * The matrix profile (MP) of a series is, for every length-m subsequence, the
 * Euclidean distance between z-normalised subsequences to its nearest
 * neighbour in the join set; the profile index (PI) is that neighbour's
 * position (tsmp paper, Sec. 2 "The matrix profile").  A self-join takes one
 * series and skips trivial matches inside an exclusion zone; an AB-join takes
 * two series (Sec. 3.2 "Input arguments and example").  The library computes
 * both exactly, in the diagonal order the paper credits to SCRIMP
 * (Sec. 3.3.3) with the dot-product reuse it credits to STOMP (Sec. 3.3.2).
 *
 * Conventions shared by every entry point:
 *   - window i is x[i .. i+m-1] (0-based); l = n - m + 1 windows
 *     (Sec. 3.4.1 and 3.4.3 print l for two inputs);
 *   - z-normalisation uses the population standard deviation;
 *   - exclusion zone E = ceil(ez * m) (Sec. 3.2); j is excluded from row i
 *     iff |i - j| < E (MP_FLAG_EXCL_INCLUSIVE: iff |i - j| <= E);
 *   - a window whose m values are all equal is "flat": every pair involving
 *     it has correlation 0, i.e. distance sqrt(2m);
 *   - ties go to the lowest index; a row without an admissible neighbour
 *     gets MP = +inf and PI = -1;
 *   - MP is FP64, PI is int64.
 *
 * Memory and streams: every array argument is a DEVICE pointer owned by the
 * caller unless its comment says host.  `stream` is a cudaStream_t passed as
 * void* (NULL = legacy default stream).  Every compute call only enqueues
 * work on `stream`: it never synchronises, never allocates device memory and
 * never throws.  Host-side argument checks return an error before anything
 * is enqueued.  Errors found on the device (non-finite input, a retry limit
 * reached) are recorded in a status word inside the caller's workspace and
 * read back by mp_get_device_status().  All entry points are capture-safe
 * (they may be recorded into a CUDA graph) once mp_init() has run.
 *
 * Workspace: each join needs scratch device memory of at least the size its
 * *_workspace_bytes() query returns; the buffer must be 256-byte aligned and
 * must not be used by two calls in flight at the same time.
 */
#ifndef MPGB_MP_H
#define MPGB_MP_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    MP_OK = 0,
    MP_EINVAL = 1,         /* bad argument (null pointer, m < 4, m > n, ...) */
    MP_EINVAL_DATA = 2,    /* the input holds NaN or Inf (device-detected) */
    MP_ENOMEM = 3,         /* workspace smaller than the size query says */
    MP_ECUDA = 4,          /* a CUDA runtime call failed */
    MP_ETIMEOUT = 5,       /* a bounded device retry loop gave up */
    MP_EUNSUPPORTED = 6,   /* no GPU of the compiled architecture, or an
                              unsupported tile configuration */
    MP_EBOUNDS = 7         /* debug builds (-DMP_DEBUG) only: a device index
                              outside its buffer was caught and the access
                              skipped (device-detected) */
} mp_status;

typedef enum { MP_F32 = 0, MP_F64 = 1 } mp_dtype;                  /* input element type */
typedef enum { MP_PREC_FP64 = 0, MP_PREC_FP32_MIXED = 1 } mp_precision;

/* mp_config.flags */
#define MP_FLAG_EXCL_INCLUSIVE 0x1u   /* exclude |i-j| <= E instead of < E */
#define MP_FLAG_NO_REFINE      0x2u   /* MP from the kernel's correlation instead of
                                         the exact FP64 distance of (i, PI[i]) */
#define MP_FLAG_PAN_NORMALIZE  0x4u   /* mp_pan: divide each row by sqrt(2m) */
#define MP_FLAG_RAW            0x8u   /* non-normalised Euclidean distance (SiMPle,
                                         Sec. 3.3.4): d = ||x_i - x_j||, no
                                         z-normalisation, no flat-window rule;
                                         mp_selfjoin, mp_selfjoin_lr, mp_abjoin */

/*
 * Join parameters.  m: window length (>= 4).  ez: exclusion-zone fraction
 * (>= 0; the paper's default is 1/2, Sec. 3.2).  prec: arithmetic of the
 * diagonal recurrence (MP_PREC_FP32_MIXED keeps stats, anchors and the
 * final distances in FP64).  anchor_every (K): rows between exact FP64
 * re-anchors of each diagonal's covariance; 0 = once per tile.  tile_rows
 * (TR): rows per tile; 0 = the library's choice (16384 FP32-mixed, 4096
 * FP64, halved down to 1024 for joins too small to keep every CTA of the
 * persistent grid busy with that many; mp_batched keeps the default).
 * Both are rounded up to whole chunks of the variant (the FP32-mixed AB-join
 * and the pan profile default to 2048 rows).  variant: compiled tile
 * shape (mp_variant_count/mp_variant_info), or MP_VARIANT_AUTO for the
 * library's choice: variant 7 (four warps per CTA, 5 CTAs per SM) for
 * FP32-mixed joins, variant 3 (four warps, 256-row chunks) for FP32-mixed
 * self-joins, left/right and anytime runs of fewer than about 4e9 cells
 * ((n - m + 1)^2 / 2), variant 0 for the FP64 path and the
 * non-normalised distance.  These
 * three set the speed: the FP32-mixed path returns the same neighbours under
 * every setting, the FP64 path may break ties closer than its rounding
 * differently.  flags: MP_FLAG_*.
 */
typedef struct {
    int32_t m;
    double ez;
    int32_t prec;
    int32_t anchor_every;
    int32_t tile_rows;
    int32_t variant;
    uint32_t flags;
} mp_config;

#define MP_VARIANT_AUTO (-1)

/* Fill `cfg` with the defaults for window m (ez 1/2, FP32-mixed, refine on,
 * tile shape and height left to the library). */
void mp_config_default(mp_config *cfg, int32_t m);

/* Host helpers, no GPU needed.  l = n - m + 1 (0 if m > n or m < 1), per the
 * sizes printed in Sec. 3.4.1/3.4.3; E = ceil(ez * m), per Sec. 3.2 (the
 * worked value 50 * 1/4 -> 13 in Sec. 3.4.3 fixes the rounding). */
int64_t mp_profile_length(int64_t n, int32_t m);
int64_t mp_exclusion_zone(int32_t m, double ez);

/* Library version string and the tile-shape variants compiled in.  Host only. */
const char *mp_version(void);
int32_t mp_variant_count(int32_t prec);
/* For variant v of precision prec: diagonals per tile (TD) and rows per
 * shared-memory chunk (RC).  Returns MP_EINVAL for an unknown variant. */
mp_status mp_variant_info(int32_t prec, int32_t v, int32_t *tile_diags, int32_t *chunk_rows);

/* Human-readable name of a status code (static storage). */
const char *mp_status_string(mp_status st);

/*
 * Check that a GPU of the compiled architecture (sm_103) is present, select
 * it as current if `device` >= 0, and cache per-device launch limits.  Calls
 * on a device run this themselves on first use; call it once before
 * recording any entry point into a CUDA graph.
 */
mp_status mp_init(int32_t device);

/*
 * Per-window statistics (the quantities the z-normalised distance and the
 * diagonal recurrence are built from; the paper's brute-force definition is
 * Sec. 2, the reuse of dot products Sec. 3.3.2):
 *   mu[i]   mean of window i;
 *   invn[i] 1 / ||x_i - mu_i||_2 (0 for a flat window);
 *   df[i]   (x[i+m-1] - x[i-1]) / 2, df[0] = 0;
 *   dg[i]   (x[i+m-1] - mu_i) + (x[i-1] - mu_{i-1}), dg[0] = 0;
 *   flat[i] 1 iff the m values of window i are all equal.
 * With c(i,j) the centred dot product of windows i and j,
 * c(i,j) = c(i-1,j-1) + df[i]*dg[j] + df[j]*dg[i].
 * x: n elements of `dtype`.  All outputs have l entries; any output pointer
 * may be NULL to skip it.  Sums are compensated (double-double).
 */
mp_status mp_stats(const void *x, int32_t dtype, int64_t n, int32_t m,
                   double *mu, double *invn, double *df, double *dg, uint8_t *flat,
                   void *stream);

/*
 * Self-join (Sec. 3.2, one series).  x: n elements of `dtype`.
 * mp: l doubles, pi: l int64 (outputs, overwritten).  ws/ws_bytes: scratch
 * of at least mp_selfjoin_workspace_bytes(n, cfg) bytes.
 */
size_t mp_selfjoin_workspace_bytes(int64_t n, const mp_config *cfg);
mp_status mp_selfjoin(const void *x, int32_t dtype, int64_t n, const mp_config *cfg,
                      double *mp, int64_t *pi, void *ws, size_t ws_bytes, void *stream);

/*
 * Left and right self-join profiles (used by time series chains, Sec. 3.4.3):
 * for window i, mp_left[i] / pi_left[i] is its nearest neighbour among the
 * windows j before it (i - j >= E, E the exclusion zone of cfg), and
 * mp_right[i] / pi_right[i] among the windows after it (j - i >= E).  With
 * MP_FLAG_EXCL_INCLUSIVE both bounds become > E.  The elementwise minimum of
 * the two is the self-join profile (ties: the lower index, i.e. the left
 * side).  A window with no admissible neighbour on a side gets +inf / -1
 * there; a flat window gets sqrt(2m) and the lowest admissible index of that
 * side.  All four outputs have l entries (device, overwritten).  ws/ws_bytes:
 * scratch of at least mp_selfjoin_lr_workspace_bytes(n, cfg) bytes.
 */
size_t mp_selfjoin_lr_workspace_bytes(int64_t n, const mp_config *cfg);
mp_status mp_selfjoin_lr(const void *x, int32_t dtype, int64_t n, const mp_config *cfg,
                         double *mp_left, int64_t *pi_left, double *mp_right, int64_t *pi_right,
                         void *ws, size_t ws_bytes, void *stream);

/*
 * Anytime self-join (SCRIMP's random diagonal order, Sec. 3.3.3, and the
 * partial runs the paper's s_size argument controls, Sec. 3.2): the bands of
 * tile_diags consecutive diagonals (mp_variant_info) are put in a random
 * order and processed a prefix at a time, so a partial run returns a profile
 * that is exact over the diagonals done so far (plus the diagonal E every
 * key is seeded from; pairs of ill-conditioned windows are always done in
 * full) and converges to the self-join.
 *   mp_anytime_begin: statistics, seeding, plan and the band order.  The
 *     order is a Fisher-Yates shuffle of 0..nb-1 driven by splitmix64 from
 *     `seed`: for i = nb-1 down to 1, swap slots i and r % (i+1), r the next
 *     splitmix64 output.
 *   mp_anytime_run: processes the bands up to slot ceil(fraction * nb)
 *     (fraction in [0, 1], cumulative; a smaller value than before processes
 *     nothing new) and writes the best-so-far mp / pi (l entries, device).
 *     fraction = 1 gives the mp_selfjoin result.
 * Both calls take the same n and cfg and the same workspace of at least
 * mp_anytime_workspace_bytes(n, cfg) bytes, which holds the state between
 * runs; runs on one workspace must be serialised.
 */
size_t mp_anytime_workspace_bytes(int64_t n, const mp_config *cfg);
mp_status mp_anytime_begin(const void *x, int32_t dtype, int64_t n, const mp_config *cfg,
                           uint64_t seed, void *ws, size_t ws_bytes, void *stream);
mp_status mp_anytime_run(int64_t n, const mp_config *cfg, double fraction, double *mp,
                         int64_t *pi, void *ws, size_t ws_bytes, void *stream);

/*
 * Semantic segmentation from a self-join profile index (FLUSS, Sec. 3.4.2).
 * pi: l int64 (device; entries < 0 mean "no neighbour"; entries >= l are
 * skipped and set MP_EINVAL in the workspace status, read it with
 * mp_get_device_status).  Every window i with pi[i] >= 0 is an arc between
 * a = min(i, pi[i]) and b = max(i, pi[i]).
 *   cac[k] (l doubles, device, overwritten) = min(AC[k] / IAC[k], 1), with
 *   AC[k] = #{i : a_i <= k < b_i} and IAC[k] = 2 k (l - k) / l; cac[k] = 1
 *   where IAC[k] = 0 and for k < edge or k >= l - edge.
 *   segments (num_segments int64, device; may be NULL when num_segments = 0):
 *   the position of the lowest cac (lowest index on ties), then the lowest
 *   outside |k - s| < seg_excl of every earlier one; -1 once none is left.
 * The paper (Sec. 3.4.2) shows only the number of segments being chosen; both
 * margins are left to the caller (the Python binding defaults both to 5m).
 * ws/ws_bytes: scratch of at least mp_fluss_workspace_bytes(l) bytes.
 */
size_t mp_fluss_workspace_bytes(int64_t l);
mp_status mp_fluss(const int64_t *pi, int64_t l, int64_t edge, int32_t num_segments,
                   int64_t seg_excl, double *cac, int64_t *segments, void *ws, size_t ws_bytes,
                   void *stream);

/*
 * Self-join without a caller workspace (the paper has no counterpart: this
 * is a convenience of the library).  For callers that cannot allocate device
 * memory -- code running inside another framework's CUDA-graph capture, under
 * an allocator that owns all device memory, or in a plugin that only receives
 * its input and output buffers.  Same arguments and results as mp_selfjoin
 * (the same neighbours and distances, bit for bit, for the same cfg), but the
 * scratch is a 64 MiB array the library keeps on every GPU that loads it,
 * until the process exits; nothing is allocated by any call.
 * Size limit: the series' mp_selfjoin workspace must fit in the 64 MiB, about
 * 97 bytes per sample with the FP32-mixed precision and 81 with FP64 (plus the
 * tile plan): n up to 690,456 (FP32-mixed) or 826,400 (FP64) with the
 * default tile shapes; mp_selfjoin_noalloc_max_n(cfg) returns the exact
 * largest n for a configuration (0 for an invalid one).  A larger n returns MP_ENOMEM before
 * any work is enqueued.
 * Each call looks up the array's device address in the current device's
 * context (an address kept from an earlier call would be stale after
 * cudaDeviceReset or in another context); the first call on a device also
 * loads the library's device code there, so make it before any stream
 * capture.  All calls on a device share the array, which keeps the last call's
 * contents (every call clears what must start at zero): calls whose GPU work
 * may overlap race and must be serialised by the caller.
 * Device-side errors (non-finite input, MP_EINVAL_DATA; a bounded retry loop
 * that gave up, MP_ETIMEOUT) land in the array's status word:
 * mp_selfjoin_noalloc_device_status(stream) synchronises `stream`, reads and
 * clears it, like mp_get_device_status does for a caller workspace (the same
 * race caveat applies).
 */
int64_t mp_selfjoin_noalloc_max_n(const mp_config *cfg);
mp_status mp_selfjoin_noalloc(const void *x, int32_t dtype, int64_t n, const mp_config *cfg,
                              double *mp, int64_t *pi, void *stream);
mp_status mp_selfjoin_noalloc_device_status(void *stream);

/*
 * AB-join (Sec. 3.2, two series; no exclusion zone).  For every window of a:
 * the nearest window of b (mp_a, pi_a: la entries).  For every window of b:
 * the nearest window of a (mp_b, pi_b: lb entries; both may be NULL to skip
 * that side).  a and b share `dtype`.
 */
size_t mp_abjoin_workspace_bytes(int64_t na, int64_t nb, const mp_config *cfg);
mp_status mp_abjoin(const void *a, int64_t na, const void *b, int64_t nb, int32_t dtype,
                    const mp_config *cfg, double *mp_a, int64_t *pi_a,
                    double *mp_b, int64_t *pi_b, void *ws, size_t ws_bytes, void *stream);

/*
 * Batched ragged self-joins in one persistent launch: series b is
 * values[offsets[b] .. offsets[b+1]) with window ms[b] (cfg->m is ignored;
 * cfg->ez, prec and flags apply to all).  offsets: B+1 int64 (device),
 * ms: B int32 (device), out_offsets: B+1 int64 (device) with
 * out_offsets[b+1] - out_offsets[b] >= l_b; series b's MP/PI go to
 * mp/pi[out_offsets[b] ..).  A series with l_b <= 0 writes nothing.
 * total_values = offsets[B] and max_m bound the workspace (host values).
 */
size_t mp_batched_workspace_bytes(int64_t total_values, int32_t B, int32_t max_m,
                                  const mp_config *cfg);
mp_status mp_batched(const void *values, int32_t dtype, int64_t total_values,
                     const int64_t *offsets, const int32_t *ms, int32_t B, int32_t max_m,
                     const mp_config *cfg, double *mp, int64_t *pi, const int64_t *out_offsets,
                     void *ws, size_t ws_bytes, void *stream);

/*
 * Pan matrix profile: the self-join of one series at every window size in
 * ms (host array of nm sizes, each >= 4 and <= n), in one persistent launch.
 * pan and pi are row-major [nm x (n - min(ms) + 1)]; row k holds the MP/PI
 * for window ms[k] in its first n - ms[k] + 1 entries and +inf / -1 after.
 * MP_FLAG_PAN_NORMALIZE divides each MP row by sqrt(2 ms[k]).
 */
size_t mp_pan_workspace_bytes(int64_t n, const int32_t *ms, int32_t nm, const mp_config *cfg);
mp_status mp_pan(const void *x, int32_t dtype, int64_t n, const int32_t *ms, int32_t nm,
                 const mp_config *cfg, double *pan, int64_t *pi, void *ws, size_t ws_bytes,
                 void *stream);

/*
 * Gradient of L = sum_i grad_mp[i] * MP[i] with respect to x, holding each
 * argmin pair (i, pi[i]) fixed.  With z_i, z_j the z-normalised windows,
 * rho their correlation, d their distance and sigma the population standard
 * deviations:
 *   dMP_i/dx[i+k] = -(z_j[k] - rho z_i[k]) / (sigma_i d)
 *   dMP_i/dx[j+k] = -(z_i[k] - rho z_j[k]) / (sigma_j d)
 * A row contributes nothing when pi[i] < 0, either window is flat, or
 * d < 1e-12.  (The paper has no gradient; this is the derivative of the
 * Sec. 2 distance.)  x: n of dtype; pi: l int64; grad_mp: l doubles;
 * grad_x: n doubles, overwritten.
 */
size_t mp_backward_workspace_bytes(int64_t n, int32_t m);
mp_status mp_backward(const void *x, int32_t dtype, int64_t n, int32_t m, const int64_t *pi,
                      const double *grad_mp, double *grad_x, void *ws, size_t ws_bytes,
                      void *stream);

/*
 * Diagnostics.  While enabled (process-wide, off by default), every join
 * records a pair of CUDA events on the caller's stream around its tile
 * kernel (the persistent diagonal-tile launch), on the current device;
 * mp_timing_last_ms() waits for the most recent pair and returns the
 * kernel's elapsed milliseconds.  Leave it disabled while recording a join
 * into a CUDA graph.
 */
mp_status mp_timing_enable(int32_t on);
mp_status mp_timing_last_ms(float *ms);

/*
 * Diagnostics: the FP64 pipe's throughput on the current device, in FP64
 * lane-operations per second (fused multiply-adds from eight independent
 * chains per thread, 32 warps per SM, three timed launches after a warm-up;
 * synchronises the device).  The all-FP64 kernel's roofline is reported
 * against it.  Allocates nothing.
 */
mp_status mp_probe_fp64_rate(double *lane_ops_per_s);

/*
 * Synchronise `stream`, read the status word of workspace `ws` (the one the
 * preceding calls used), clear it, and return it (MP_OK if no device-side
 * error was recorded).
 */
mp_status mp_get_device_status(void *ws, void *stream);

#ifdef __cplusplus
}
#endif

#endif /* MPGB_MP_H */
