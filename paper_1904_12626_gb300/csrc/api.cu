// api.cu -- the C ABI (include/mp.h): argument checks, workspace layout and the
// launch sequence of every join.  Host code only; the kernels live in the
// other translation units.
#include <cmath>
#include <cstring>
#include <mutex>

#include "internal.cuh"

using namespace mpgb;

namespace {

constexpr int kMaxDevices = 64;
constexpr int kMaxVariants = 16;          // compiled tile shapes per precision, at most
constexpr int kDefaultTileRowsF32 = 16384;
constexpr int kDefaultTileRowsF64 = 4096;
// FP32-mixed AB-joins: shorter row tiles by default.  Both series' keys improve
// as bands complete, and short tiles let the bands of a problem finish nearly in
// the order they start, so each band starts from thresholds its predecessors
// raised (2^21 x 2^19 walk / white-noise mix, m = 512, tile kernel ms at 1024 /
// 2048 / 4096 / 8192 rows: variant 0 358 / 347 / 355 / 476, variant 7 333 / 323
// / 331 / 445).
constexpr int kDefaultTileRowsAbF32 = 2048;

// The tile shape MP_VARIANT_AUTO stands for in FP32-mixed joins: four warps per
// CTA at 5 CTAs per SM (variant 7; 1024 diagonals per band).  Tile kernel ms,
// variant 0 / 7 at the default heights: self-join 2^20 (m = 256) 106.6 / 102.9,
// AB 2^21 x 2^19 (m = 512) 295 / 264, 4096 ragged walks 1335 / 1300, gradient
// input 2^16 (m = 128) 1.40 / 1.36; pan profiles (64 window sizes of a 2^16
// walk) at 2048-row tiles 64.1 ms.
constexpr int kAutoVariantF32 = 7;
constexpr int kAutoVariantPan = 7;
// Small self-joins (and left/right and anytime runs) take variant 3 (four
// warps, 256-row chunks, 4 CTAs per SM): a persistent grid of 760 CTAs has few
// tiles to share there.  Tile kernel ms, variant 3 / 7, random walks, m = 64,
// 128, 256: 2^14 windows 0.80 / 0.99, 0.73 / 0.84, 0.99 / 1.07; 2^15 0.71 /
// 0.96, 0.74 / 0.94, 1.07 / 1.20; 2^16 1.20 / 1.37, 1.22 / 1.36, 1.48 / 1.71;
// 2^17 3.03 / 2.98, 2.99 / 2.95, 3.27 / 3.31; 2^18 9.50 / 8.75, 9.22 / 8.44,
// 9.77 / 9.08.  The two cross near 2^17 windows, about 8e9 cells.
constexpr int kAutoVariantSmall = 3;
constexpr double kSmallJoinCells = 4.0e9;
// FP32-mixed pan profiles: 2048-row tiles by default, for the AB-join's reason
// (64 window sizes of a 2^16 walk, tile kernel: variant 7 at 2048 rows 64.1 ms,
// the autotuner's choice, against 66.8 ms for variant 1 at 4096 rows)
constexpr int kDefaultTileRowsPanF32 = 2048;
constexpr long long kMaxN = 2147483647ll;

struct DeviceInfo {
    bool ready = false;
    cudaEvent_t ev[2] = {nullptr, nullptr};     // timing diagnostics
    bool ev_used = false;
    bool ok = false;
    int sms = 0;
    int f32_bps[kMaxVariants] = {0};
    int f64_bps[kMaxVariants] = {0};
    int f32_raw_bps = 0, f64_raw_bps = 0;       // MP_FLAG_RAW kernels (variant 0 shape)
};
DeviceInfo g_dev[kMaxDevices];
std::mutex g_mu;
bool g_timing = false;
int g_timing_dev = -1;

mp_status device_info(int dev, const DeviceInfo **out)
{
    if (dev < 0 || dev >= kMaxDevices) return MP_EUNSUPPORTED;
    std::lock_guard<std::mutex> lk(g_mu);
    DeviceInfo &d = g_dev[dev];
    if (!d.ready) {
        cudaDeviceProp p;
        if (cudaGetDeviceProperties(&p, dev) != cudaSuccess) return MP_ECUDA;
        d.ok = (p.major == 10 && p.minor == 3);
        d.sms = p.multiProcessorCount;
        if (d.ok) {
            int cur = -1;
            cudaGetDevice(&cur);
            if (cur != dev) cudaSetDevice(dev);
            for (int v = 0; v < f32_variant_count() && v < kMaxVariants; ++v) d.f32_bps[v] = f32_blocks_per_sm(v);
            for (int v = 0; v < f64_variant_count() && v < kMaxVariants; ++v) d.f64_bps[v] = f64_blocks_per_sm(v);
            d.f32_raw_bps = f32_raw_blocks_per_sm();
            d.f64_raw_bps = f64_raw_blocks_per_sm();
            if (cur != dev && cur >= 0) cudaSetDevice(cur);
        }
        d.ready = true;
    }
    *out = &d;
    return d.ok ? MP_OK : MP_EUNSUPPORTED;
}

mp_status current_device(const DeviceInfo **out)
{
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return MP_ECUDA;
    return device_info(dev, out);
}

inline long long ceil_div(long long a, long long b) { return (a + b - 1) / b; }

// resolved tile configuration of a call
struct TileCfg {
    int fp64;
    int variant;
    int tile_diags;
    int chunk_rows;
    int tile_rows;
    int anchor_every;
    bool refine;
    bool raw;                // MP_FLAG_RAW: non-normalised distance (variant 0 only)
};

// auto_variant: the tile shape MP_VARIANT_AUTO stands for in this family
// (FP32-mixed only; the FP64 path and the non-normalised distance take 0)
mp_status resolve(const mp_config *cfg, TileCfg *t, int auto_variant = kAutoVariantF32)
{
    if (!cfg) return MP_EINVAL;
    if (cfg->prec != MP_PREC_FP64 && cfg->prec != MP_PREC_FP32_MIXED) return MP_EINVAL;
    if (!(cfg->ez >= 0.0) || !std::isfinite(cfg->ez)) return MP_EINVAL;
    if (cfg->anchor_every < 0 || cfg->tile_rows < 0) return MP_EINVAL;
    t->fp64 = cfg->prec == MP_PREC_FP64;
    const bool raw_flag = (cfg->flags & MP_FLAG_RAW) != 0;
    t->variant = cfg->variant >= 0 ? cfg->variant
                                   : ((t->fp64 || raw_flag) ? 0 : auto_variant);
    if (t->variant >= kMaxVariants) return MP_EUNSUPPORTED;
    int threads = 0, smem = 0;
    const bool ok = t->fp64 ? f64_variant_info(t->variant, &t->tile_diags, &t->chunk_rows, &threads, &smem)
                            : f32_variant_info(t->variant, &t->tile_diags, &t->chunk_rows, &threads, &smem);
    if (!ok) return MP_EUNSUPPORTED;
    const int rc = t->chunk_rows;
    int tr = cfg->tile_rows > 0 ? cfg->tile_rows : (t->fp64 ? kDefaultTileRowsF64 : kDefaultTileRowsF32);
    tr = (int)(ceil_div(tr, rc) * rc);
    t->tile_rows = tr;
    t->anchor_every = cfg->anchor_every > 0 ? (int)(ceil_div(cfg->anchor_every, rc) * rc) : 0;
    if (t->anchor_every >= tr) t->anchor_every = 0;
    t->refine = (cfg->flags & MP_FLAG_NO_REFINE) == 0;
    t->raw = (cfg->flags & MP_FLAG_RAW) != 0;
    if (t->raw && t->variant != 0) return MP_EUNSUPPORTED;
    return MP_OK;
}

// The tile shape MP_VARIANT_AUTO stands for in a self-join of n samples.
int self_auto_variant(int64_t n, const mp_config *cfg)
{
    if (!cfg) return kAutoVariantF32;
    const double l = (double)(n - cfg->m + 1);
    return (l > 0.0 && 0.5 * l * l < kSmallJoinCells) ? kAutoVariantSmall : kAutoVariantF32;
}

// Row-tile height of a join whose caller left it to the library.  The tile
// kernel is persistent: every CTA takes tickets until none is left, so a join
// ends when its busiest CTA does, up to one tile after the average.  The
// default height has the fewest FP64 anchors (m multiply-adds per diagonal
// per tile); a join so small that one such tile exceeds a quarter of a CTA's
// share of the cells gets the height halved, down to kMinFitRows.  Only the
// speed changes: every height gives the same neighbours.
constexpr int kFitTilesPerCta = 4;
constexpr int kMinFitRows = 1024;

void fit_tile_rows(const mp_config *cfg, TileCfg *t, double cells, const DeviceInfo *d)
{
    if (cfg->tile_rows > 0 || !(cells > 0.0) || d == nullptr) return;
    const int bps = t->raw ? (t->fp64 ? d->f64_raw_bps : d->f32_raw_bps)
                           : (t->fp64 ? d->f64_bps[t->variant] : d->f32_bps[t->variant]);
    if (bps <= 0 || d->sms <= 0) return;
    const double share = cells / ((double)d->sms * (double)bps);
    long long tr = t->tile_rows;
    while (tr > kMinFitRows && (double)tr * t->tile_diags * kFitTilesPerCta > share) tr >>= 1;
    tr = ceil_div(tr, t->chunk_rows) * t->chunk_rows;
    t->tile_rows = (int)tr;
    if (t->anchor_every >= t->tile_rows) t->anchor_every = 0;
}

// admissible pairs of a self-join (an estimate for the inclusive zone)
double self_cells(int64_t n, int32_t m, double ez)
{
    const double l = (double)(n - m + 1), e = std::ceil(ez * (double)m);
    return l > e ? (l - e) * (l - e + 1.0) / 2.0 : 0.0;
}

// Workspace layout shared by every join.
struct LayoutReq {
    long long nx = 0;        // FP64 copy of the input values
    long long S = 0;         // stats-index space
    int nsets = 0, nprob = 0, nfin = 0;
    long long max_bands = 0;
    int fp64 = 0;
};

struct Layout {
    Hdr *hdr;
    double *x64, *mu, *inv;
    float4 *s32;
    D4 *s64;
    uint8_t *flat;
    char *keys;
    double *set_acc;
    unsigned long long *frag_list;
    StatSet *sets;
    Prob *probs;
    FinDesc *fins;
    long long *band_off;
    Band *bands;
    unsigned long long *tile_prefix;
    long long *scratch;      // band reordering (anytime): 32 bytes per band
    size_t bytes;
};

Layout carve(void *base, const LayoutReq &r)
{
    Layout L;
    size_t off = 0;
    auto take = [&](size_t bytes) -> void * {
        const size_t o = (off + 255) & ~(size_t)255;
        off = o + bytes;
        return base ? (void *)((char *)base + o) : nullptr;
    };
    const size_t ksz = sizeof(Key128);
    L.hdr = (Hdr *)take(256);
    L.x64 = (double *)take(sizeof(double) * (size_t)r.nx);
    L.mu = (double *)take(sizeof(double) * (size_t)r.S);
    L.inv = (double *)take(sizeof(double) * (size_t)r.S);
    L.s32 = r.fp64 ? nullptr : (float4 *)take(sizeof(float4) * (size_t)r.S);
    L.s64 = (D4 *)take(sizeof(D4) * (size_t)r.S);
    L.flat = (uint8_t *)take((size_t)r.S);
    L.keys = (char *)take(ksz * (size_t)r.S);
    L.set_acc = (double *)take(sizeof(double) * 2 * (size_t)r.nsets);
    L.frag_list = (unsigned long long *)take(sizeof(unsigned long long) * (size_t)r.S);
    L.sets = (StatSet *)take(sizeof(StatSet) * (size_t)r.nsets);
    L.probs = (Prob *)take(sizeof(Prob) * (size_t)r.nprob);
    L.fins = (FinDesc *)take(sizeof(FinDesc) * (size_t)r.nfin);
    L.band_off = (long long *)take(sizeof(long long) * (size_t)(r.nprob + 1));
    L.bands = (Band *)take(sizeof(Band) * (size_t)(r.max_bands > 0 ? r.max_bands : 1));
    L.tile_prefix = (unsigned long long *)take(sizeof(unsigned long long) * (size_t)(r.max_bands + 1));
    L.scratch = (long long *)take(32 * (size_t)(r.max_bands > 0 ? r.max_bands : 1));
    L.bytes = (off + 255) & ~(size_t)255;
    return L;
}

bool aligned256(const void *p) { return ((uintptr_t)p & 255u) == 0; }

#define MP_CU(call)                                   \
    do {                                              \
        if ((call) != cudaSuccess) return MP_ECUDA;   \
    } while (0)

// stats -> keys reset -> [fragile windows marked] -> keys seeded -> plan
mp_status prepare_join(const Layout &L, const LayoutReq &r, const TileCfg &t, long long max_fin_len,
                       cudaStream_t st)
{
    MP_CU(cudaMemsetAsync(L.set_acc, 0, sizeof(double) * 2 * (size_t)r.nsets, st));
    MP_CU(launch_stats_sets(L.sets, r.nsets, r.S, L.mu, L.inv, L.s32, L.s64, L.flat, L.set_acc,
                            st));
    const size_t ksz = sizeof(Key128);
    MP_CU(cudaMemsetAsync(L.keys, 0, ksz * (size_t)r.S, st));
    MP_CU(launch_fragile_mark(L.sets, r.nsets, max_fin_len, L.set_acc, L.inv, L.flat, L.s32,
                              L.s64, L.frag_list, L.hdr, st));
    MP_CU(launch_seed(L.sets, r.nsets, max_fin_len, L.mu, L.inv, L.flat, L.s32, L.s64, L.keys,
                      t.fp64, st));
    MP_CU(launch_plan(L.probs, r.nprob, t.tile_diags, t.tile_rows, L.band_off, L.bands,
                      L.tile_prefix, L.scratch, r.max_bands, L.hdr, st));
    return MP_OK;
}

// persistent join over the open bands -> [fragile pairs exactly] -> finalize
mp_status execute_join(const Layout &L, const LayoutReq &r, const TileCfg &t, long long max_fin_len,
                       const DeviceInfo *dev, cudaStream_t st)
{
    const int bps = t.raw ? (t.fp64 ? dev->f64_raw_bps : dev->f32_raw_bps)
                          : (t.fp64 ? dev->f64_bps[t.variant] : dev->f32_bps[t.variant]);
    if (bps <= 0) return MP_EUNSUPPORTED;
    const int grid = dev->sms * bps;
    DeviceInfo *dm = const_cast<DeviceInfo *>(dev);
    const bool timing = g_timing && dm->ev[0] != nullptr;
    if (timing) MP_CU(cudaEventRecord(dm->ev[0], st));
    if (t.raw && t.fp64)
        MP_CU(launch_join_f64_raw(L.probs, L.bands, L.tile_prefix, L.hdr, t.tile_rows,
                                  t.anchor_every, grid, st));
    else if (t.raw)
        MP_CU(launch_join_f32_raw(L.probs, L.bands, L.tile_prefix, L.hdr, t.tile_rows,
                                  t.anchor_every, grid, st));
    else if (t.fp64)
        MP_CU(launch_join_f64(t.variant, L.probs, L.bands, L.tile_prefix, L.hdr, t.tile_rows,
                              t.anchor_every, grid, st));
    else
        MP_CU(launch_join_f32(t.variant, L.probs, L.bands, L.tile_prefix, L.hdr, t.tile_rows,
                              t.anchor_every, grid, st));
    if (timing) {
        MP_CU(cudaEventRecord(dm->ev[1], st));
        dm->ev_used = true;
    }
    MP_CU(launch_fragile_pass(L.sets, L.mu, L.inv, L.frag_list, L.keys, t.fp64, L.hdr,
                              dev->sms * 8, st));
    MP_CU(launch_finalize(L.fins, r.nfin, max_fin_len, t.fp64, t.refine ? 1 : 0, st));
    return MP_OK;
}

mp_status run_join(const Layout &L, const LayoutReq &r, const TileCfg &t, long long max_fin_len,
                   const DeviceInfo *dev, cudaStream_t st)
{
    const mp_status s = prepare_join(L, r, t, max_fin_len, st);
    if (s != MP_OK) return s;
    return execute_join(L, r, t, max_fin_len, dev, st);
}

bool valid_dtype(int32_t dtype) { return dtype == MP_F32 || dtype == MP_F64; }

LayoutReq self_req(int64_t n, int32_t m, const TileCfg &t)
{
    LayoutReq r;
    const long long l = n - m + 1;
    r.nx = n;
    r.S = n + kPad;
    r.nsets = r.nprob = r.nfin = 1;
    r.max_bands = ceil_div(l > 0 ? l : 0, t.tile_diags) + 1;
    r.fp64 = t.fp64;
    return r;
}

// left/right self-join: the series' windows twice (right role, left role)
LayoutReq lr_req(int64_t n, int32_t m, const TileCfg &t)
{
    LayoutReq r;
    const long long l = n - m + 1;
    r.nx = n;
    r.S = 2 * (n + kPad);
    r.nsets = 2;
    r.nprob = 1;
    r.nfin = 2;
    r.max_bands = ceil_div(l > 0 ? l : 0, t.tile_diags) + 1;
    r.fp64 = t.fp64;
    return r;
}

LayoutReq ab_req(int64_t na, int64_t nb, int32_t m, const TileCfg &t)
{
    LayoutReq r;
    r.nx = na + nb;
    r.S = na + nb + 2 * (long long)kPad;
    r.nsets = r.nprob = r.nfin = 2;
    r.max_bands = ceil_div(na, t.tile_diags) + ceil_div(nb, t.tile_diags) + 2;
    r.fp64 = t.fp64;
    (void)m;
    return r;
}

LayoutReq pan_req(int64_t n, const int32_t *ms, int32_t nm, const TileCfg &t)
{
    LayoutReq r;
    r.nx = n;
    r.S = (long long)nm * (n + kPad);
    r.nsets = r.nprob = r.nfin = nm;
    long long b = 0;
    for (int k = 0; k < nm; ++k) b += ceil_div(n - ms[k] + 1, t.tile_diags) + 1;
    r.max_bands = b;
    r.fp64 = t.fp64;
    return r;
}

LayoutReq batched_req(int64_t total, int32_t B, const TileCfg &t)
{
    LayoutReq r;
    r.nx = total;
    r.S = total + (long long)B * kPad;
    r.nsets = r.nprob = r.nfin = B;
    r.max_bands = ceil_div(total, t.tile_diags) + B;
    r.fp64 = t.fp64;
    return r;
}

}  // namespace

extern "C" {

void mp_config_default(mp_config *cfg, int32_t m)
{
    if (!cfg) return;
    std::memset(cfg, 0, sizeof(*cfg));
    cfg->m = m;
    cfg->ez = 0.5;
    cfg->prec = MP_PREC_FP32_MIXED;
    cfg->anchor_every = 0;
    cfg->tile_rows = 0;
    cfg->variant = MP_VARIANT_AUTO;
    cfg->flags = 0;
}

int64_t mp_profile_length(int64_t n, int32_t m)
{
    if (m < 1 || (int64_t)m > n) return 0;
    return n - (int64_t)m + 1;
}

int64_t mp_exclusion_zone(int32_t m, double ez) { return (int64_t)std::ceil(ez * (double)m); }

const char *mp_version(void) { return "mpgb 0.1 (sm_103a)"; }

int32_t mp_variant_count(int32_t prec)
{
    return prec == MP_PREC_FP64 ? f64_variant_count() : f32_variant_count();
}

mp_status mp_variant_info(int32_t prec, int32_t v, int32_t *tile_diags, int32_t *chunk_rows)
{
    int td = 0, rc = 0, th = 0, sm = 0;
    const bool ok = prec == MP_PREC_FP64 ? f64_variant_info(v, &td, &rc, &th, &sm)
                                         : f32_variant_info(v, &td, &rc, &th, &sm);
    if (!ok) return MP_EINVAL;
    if (tile_diags) *tile_diags = td;
    if (chunk_rows) *chunk_rows = rc;
    return MP_OK;
}

const char *mp_status_string(mp_status st)
{
    switch (st) {
    case MP_OK: return "ok";
    case MP_EINVAL: return "invalid argument";
    case MP_EINVAL_DATA: return "input holds NaN or Inf";
    case MP_ENOMEM: return "workspace too small";
    case MP_ECUDA: return "CUDA runtime error";
    case MP_ETIMEOUT: return "device retry limit reached";
    case MP_EUNSUPPORTED: return "unsupported device or configuration";
    case MP_EBOUNDS: return "device index out of bounds (debug build)";
    }
    return "unknown status";
}

mp_status mp_init(int32_t device)
{
    if (device >= 0 && cudaSetDevice(device) != cudaSuccess) return MP_ECUDA;
    const DeviceInfo *d = nullptr;
    return current_device(&d);
}

mp_status mp_stats(const void *x, int32_t dtype, int64_t n, int32_t m, double *mu, double *invn,
                   double *df, double *dg, uint8_t *flat, void *stream)
{
    if (!x || !valid_dtype(dtype) || m < 4 || (int64_t)m > n || n > kMaxN) return MP_EINVAL;
    const DeviceInfo *d = nullptr;
    const mp_status s = current_device(&d);
    if (s != MP_OK) return s;
    MP_CU(launch_stats_public(x, dtype, n, m, mu, invn, df, dg, flat, (cudaStream_t)stream));
    return MP_OK;
}

size_t mp_selfjoin_workspace_bytes(int64_t n, const mp_config *cfg)
{
    TileCfg t;
    if (resolve(cfg, &t, self_auto_variant(n, cfg)) != MP_OK || n < 1) return 0;
    return carve(nullptr, self_req(n, cfg->m, t)).bytes;
}

mp_status mp_selfjoin(const void *x, int32_t dtype, int64_t n, const mp_config *cfg, double *mp,
                      int64_t *pi, void *ws, size_t ws_bytes, void *stream)
{
    TileCfg t;
    if (!x || !mp || !pi || !ws || !valid_dtype(dtype) || !aligned256(ws)) return MP_EINVAL;
    mp_status s = resolve(cfg, &t, self_auto_variant(n, cfg));
    if (s != MP_OK) return s;
    const int32_t m = cfg->m;
    if (m < 4 || (int64_t)m > n || n > kMaxN) return MP_EINVAL;
    const LayoutReq r = self_req(n, m, t);
    const Layout L = carve(ws, r);
    if (ws_bytes < L.bytes) return MP_ENOMEM;
    const DeviceInfo *d = nullptr;
    if ((s = current_device(&d)) != MP_OK) return s;
    cudaStream_t st = (cudaStream_t)stream;
    MP_CU(cudaMemsetAsync(L.hdr, 0, 256, st));
    MP_CU(launch_convert(x, dtype, n, L.x64, L.hdr, st));
    FamilyParams F;
    std::memset(&F, 0, sizeof(F));
    F.kind = 0; F.m = m; F.fp64 = t.fp64; F.x64 = L.x64; F.n = n; F.ez = cfg->ez; F.flags = cfg->flags;
    F.mu = L.mu; F.inv = L.inv; F.s32 = L.s32; F.s64 = L.s64; F.flat = L.flat; F.keys = L.keys;
    F.mp_a = mp; F.pi_a = (long long *)pi; F.out_stride = 0;
    F.sets = L.sets; F.probs = L.probs; F.fins = L.fins;
    MP_CU(launch_family_descs(F, st));
    fit_tile_rows(cfg, &t, self_cells(n, m, cfg->ez), d);
    return run_join(L, r, t, n - m + 1, d, st);
}

size_t mp_anytime_workspace_bytes(int64_t n, const mp_config *cfg)
{
    return mp_selfjoin_workspace_bytes(n, cfg);
}

mp_status mp_anytime_begin(const void *x, int32_t dtype, int64_t n, const mp_config *cfg,
                           uint64_t seed, void *ws, size_t ws_bytes, void *stream)
{
    TileCfg t;
    if (!x || !ws || !valid_dtype(dtype) || !aligned256(ws)) return MP_EINVAL;
    mp_status s = resolve(cfg, &t, self_auto_variant(n, cfg));
    if (s != MP_OK) return s;
    const int32_t m = cfg->m;
    if (m < 4 || (int64_t)m > n || n > kMaxN) return MP_EINVAL;
    const LayoutReq r = self_req(n, m, t);
    const Layout L = carve(ws, r);
    if (ws_bytes < L.bytes) return MP_ENOMEM;
    const DeviceInfo *d = nullptr;
    if ((s = current_device(&d)) != MP_OK) return s;
    cudaStream_t st = (cudaStream_t)stream;
    MP_CU(cudaMemsetAsync(L.hdr, 0, 256, st));
    MP_CU(launch_convert(x, dtype, n, L.x64, L.hdr, st));
    FamilyParams F;
    std::memset(&F, 0, sizeof(F));
    F.kind = 0; F.m = m; F.fp64 = t.fp64; F.x64 = L.x64; F.n = n; F.ez = cfg->ez; F.flags = cfg->flags;
    F.mu = L.mu; F.inv = L.inv; F.s32 = L.s32; F.s64 = L.s64; F.flat = L.flat; F.keys = L.keys;
    F.mp_a = nullptr; F.pi_a = nullptr; F.out_stride = 0;   // outputs bound per run
    F.sets = L.sets; F.probs = L.probs; F.fins = L.fins;
    MP_CU(launch_family_descs(F, st));
    fit_tile_rows(cfg, &t, self_cells(n, m, cfg->ez), d);
    if ((s = prepare_join(L, r, t, n - m + 1, st)) != MP_OK) return s;
    MP_CU(launch_permute_bands(seed, L.bands, L.tile_prefix, L.scratch, r.max_bands, L.hdr, st));
    return MP_OK;
}

mp_status mp_anytime_run(int64_t n, const mp_config *cfg, double fraction, double *mp,
                         int64_t *pi, void *ws, size_t ws_bytes, void *stream)
{
    TileCfg t;
    if (!mp || !pi || !ws || !aligned256(ws) || !(fraction >= 0.0 && fraction <= 1.0))
        return MP_EINVAL;
    mp_status s = resolve(cfg, &t, self_auto_variant(n, cfg));
    if (s != MP_OK) return s;
    const int32_t m = cfg->m;
    if (m < 4 || (int64_t)m > n || n > kMaxN) return MP_EINVAL;
    const LayoutReq r = self_req(n, m, t);
    const Layout L = carve(ws, r);
    if (ws_bytes < L.bytes) return MP_ENOMEM;
    const DeviceInfo *d = nullptr;
    if ((s = current_device(&d)) != MP_OK) return s;
    cudaStream_t st = (cudaStream_t)stream;
    MP_CU(launch_bind_outputs(L.fins, mp, (long long *)pi, st));
    MP_CU(launch_anytime_window(fraction, L.tile_prefix, L.hdr, st));
    fit_tile_rows(cfg, &t, self_cells(n, m, cfg->ez), d);      // as planned by the begin call
    return execute_join(L, r, t, n - m + 1, d, st);
}

size_t mp_fluss_workspace_bytes(int64_t l)
{
    if (l < 1 || l > kMaxN) return 0;
    return fluss_workspace_bytes(l);
}

mp_status mp_fluss(const int64_t *pi, int64_t l, int64_t edge, int32_t num_segments,
                   int64_t seg_excl, double *cac, int64_t *segments, void *ws, size_t ws_bytes,
                   void *stream)
{
    if (!pi || !cac || !ws || l < 1 || l > kMaxN || edge < 0 || seg_excl < 0 ||
        num_segments < 0 || (num_segments > 0 && !segments) || !aligned256(ws))
        return MP_EINVAL;
    if (ws_bytes < fluss_workspace_bytes(l)) return MP_ENOMEM;
    const DeviceInfo *d = nullptr;
    const mp_status s = current_device(&d);
    if (s != MP_OK) return s;
    MP_CU(launch_fluss(pi, l, edge, num_segments, seg_excl, cac, segments, ws,
                       (cudaStream_t)stream));
    return MP_OK;
}

size_t mp_selfjoin_lr_workspace_bytes(int64_t n, const mp_config *cfg)
{
    TileCfg t;
    if (resolve(cfg, &t, self_auto_variant(n, cfg)) != MP_OK || n < 1) return 0;
    return carve(nullptr, lr_req(n, cfg->m, t)).bytes;
}

mp_status mp_selfjoin_lr(const void *x, int32_t dtype, int64_t n, const mp_config *cfg,
                         double *mp_left, int64_t *pi_left, double *mp_right, int64_t *pi_right,
                         void *ws, size_t ws_bytes, void *stream)
{
    TileCfg t;
    if (!x || !mp_left || !pi_left || !mp_right || !pi_right || !ws || !valid_dtype(dtype) ||
        !aligned256(ws))
        return MP_EINVAL;
    mp_status s = resolve(cfg, &t, self_auto_variant(n, cfg));
    if (s != MP_OK) return s;
    const int32_t m = cfg->m;
    if (m < 4 || (int64_t)m > n || n > kMaxN) return MP_EINVAL;
    const LayoutReq r = lr_req(n, m, t);
    const Layout L = carve(ws, r);
    if (ws_bytes < L.bytes) return MP_ENOMEM;
    const DeviceInfo *d = nullptr;
    if ((s = current_device(&d)) != MP_OK) return s;
    cudaStream_t st = (cudaStream_t)stream;
    MP_CU(cudaMemsetAsync(L.hdr, 0, 256, st));
    MP_CU(launch_convert(x, dtype, n, L.x64, L.hdr, st));
    FamilyParams F;
    std::memset(&F, 0, sizeof(F));
    F.kind = 3; F.m = m; F.fp64 = t.fp64; F.x64 = L.x64; F.n = n; F.ez = cfg->ez; F.flags = cfg->flags;
    F.mu = L.mu; F.inv = L.inv; F.s32 = L.s32; F.s64 = L.s64; F.flat = L.flat; F.keys = L.keys;
    F.mp_a = mp_right; F.pi_a = (long long *)pi_right;
    F.mp_b = mp_left; F.pi_b = (long long *)pi_left;
    F.sets = L.sets; F.probs = L.probs; F.fins = L.fins;
    MP_CU(launch_family_descs(F, st));
    fit_tile_rows(cfg, &t, self_cells(n, m, cfg->ez), d);
    return run_join(L, r, t, n - m + 1, d, st);
}

size_t mp_abjoin_workspace_bytes(int64_t na, int64_t nb, const mp_config *cfg)
{
    TileCfg t;
    if (resolve(cfg, &t) != MP_OK || na < 1 || nb < 1) return 0;
    return carve(nullptr, ab_req(na, nb, cfg->m, t)).bytes;
}

mp_status mp_abjoin(const void *a, int64_t na, const void *b, int64_t nb, int32_t dtype,
                    const mp_config *cfg, double *mp_a, int64_t *pi_a, double *mp_b, int64_t *pi_b,
                    void *ws, size_t ws_bytes, void *stream)
{
    TileCfg t;
    if (!a || !b || !mp_a || !pi_a || !ws || !valid_dtype(dtype) || !aligned256(ws)) return MP_EINVAL;
    if ((mp_b == nullptr) != (pi_b == nullptr)) return MP_EINVAL;
    mp_status s = resolve(cfg, &t);
    if (s != MP_OK) return s;
    const int32_t m = cfg->m;
    if (m < 4 || (int64_t)m > na || (int64_t)m > nb || na > kMaxN || nb > kMaxN) return MP_EINVAL;
    const LayoutReq r = ab_req(na, nb, m, t);
    const Layout L = carve(ws, r);
    if (ws_bytes < L.bytes) return MP_ENOMEM;
    const DeviceInfo *d = nullptr;
    if ((s = current_device(&d)) != MP_OK) return s;
    cudaStream_t st = (cudaStream_t)stream;
    MP_CU(cudaMemsetAsync(L.hdr, 0, 256, st));
    MP_CU(launch_convert(a, dtype, na, L.x64, L.hdr, st));
    MP_CU(launch_convert(b, dtype, nb, L.x64 + na, L.hdr, st));
    FamilyParams F;
    std::memset(&F, 0, sizeof(F));
    F.kind = 1; F.m = m; F.fp64 = t.fp64; F.x64 = L.x64; F.na = na; F.nb = nb; F.ez = cfg->ez;
    F.flags = cfg->flags;
    F.mu = L.mu; F.inv = L.inv; F.s32 = L.s32; F.s64 = L.s64; F.flat = L.flat; F.keys = L.keys;
    F.mp_a = mp_a; F.pi_a = (long long *)pi_a; F.mp_b = mp_b; F.pi_b = (long long *)pi_b;
    F.sets = L.sets; F.probs = L.probs; F.fins = L.fins;
    MP_CU(launch_family_descs(F, st));
    const long long la = na - m + 1, lb = nb - m + 1;
    if (cfg->tile_rows <= 0 && !t.fp64) {
        t.tile_rows = (int)(ceil_div(kDefaultTileRowsAbF32, t.chunk_rows) * t.chunk_rows);
        if (t.anchor_every >= t.tile_rows) t.anchor_every = 0;
    }
    fit_tile_rows(cfg, &t, (double)la * (double)lb, d);
    return run_join(L, r, t, la > lb ? la : lb, d, st);
}

size_t mp_pan_workspace_bytes(int64_t n, const int32_t *ms, int32_t nm, const mp_config *cfg)
{
    TileCfg t;
    if (resolve(cfg, &t, kAutoVariantPan) != MP_OK || !ms || nm < 1 || nm > kMaxPan || n < 1) return 0;
    for (int k = 0; k < nm; ++k)
        if (ms[k] < 4 || ms[k] > n) return 0;
    return carve(nullptr, pan_req(n, ms, nm, t)).bytes;
}

mp_status mp_pan(const void *x, int32_t dtype, int64_t n, const int32_t *ms, int32_t nm,
                 const mp_config *cfg, double *pan, int64_t *pi, void *ws, size_t ws_bytes,
                 void *stream)
{
    TileCfg t;
    if (!x || !ms || !pan || !pi || !ws || !valid_dtype(dtype) || !aligned256(ws)) return MP_EINVAL;
    if (nm < 1 || nm > kMaxPan || n > kMaxN) return MP_EINVAL;
    int32_t mmin = ms[0];
    for (int k = 0; k < nm; ++k) {
        if (ms[k] < 4 || (int64_t)ms[k] > n) return MP_EINVAL;
        if (ms[k] < mmin) mmin = ms[k];
    }
    mp_status s = resolve(cfg, &t, kAutoVariantPan);
    if (s != MP_OK) return s;
    const LayoutReq r = pan_req(n, ms, nm, t);
    const Layout L = carve(ws, r);
    if (ws_bytes < L.bytes) return MP_ENOMEM;
    const DeviceInfo *d = nullptr;
    if ((s = current_device(&d)) != MP_OK) return s;
    cudaStream_t st = (cudaStream_t)stream;
    MP_CU(cudaMemsetAsync(L.hdr, 0, 256, st));
    MP_CU(launch_convert(x, dtype, n, L.x64, L.hdr, st));
    FamilyParams F;
    std::memset(&F, 0, sizeof(F));
    F.kind = 2; F.nm = nm; F.fp64 = t.fp64; F.x64 = L.x64; F.n = n; F.ez = cfg->ez;
    F.flags = cfg->flags;
    for (int k = 0; k < nm; ++k) F.ms[k] = ms[k];
    F.mu = L.mu; F.inv = L.inv; F.s32 = L.s32; F.s64 = L.s64; F.flat = L.flat; F.keys = L.keys;
    F.mp_a = pan; F.pi_a = (long long *)pi; F.out_stride = n - mmin + 1;
    F.sets = L.sets; F.probs = L.probs; F.fins = L.fins;
    MP_CU(launch_family_descs(F, st));
    double cells = 0.0;
    for (int k = 0; k < nm; ++k) cells += self_cells(n, ms[k], cfg->ez);
    if (cfg->tile_rows <= 0 && !t.fp64) {
        t.tile_rows = (int)(ceil_div(kDefaultTileRowsPanF32, t.chunk_rows) * t.chunk_rows);
        if (t.anchor_every >= t.tile_rows) t.anchor_every = 0;
    }
    fit_tile_rows(cfg, &t, cells, d);
    return run_join(L, r, t, n - mmin + 1, d, st);
}

size_t mp_batched_workspace_bytes(int64_t total_values, int32_t B, int32_t max_m,
                                  const mp_config *cfg)
{
    TileCfg t;
    (void)max_m;
    if (resolve(cfg, &t) != MP_OK || B < 1 || total_values < 0) return 0;
    return carve(nullptr, batched_req(total_values, B, t)).bytes;
}

mp_status mp_batched(const void *values, int32_t dtype, int64_t total_values,
                     const int64_t *offsets, const int32_t *ms, int32_t B, int32_t max_m,
                     const mp_config *cfg, double *mp, int64_t *pi, const int64_t *out_offsets,
                     void *ws, size_t ws_bytes, void *stream)
{
    TileCfg t;
    if (!values || !offsets || !ms || !mp || !pi || !out_offsets || !ws || !valid_dtype(dtype) ||
        !aligned256(ws))
        return MP_EINVAL;
    if (B < 1 || B > 65535 || total_values < 1 || total_values > kMaxN || max_m < 4) return MP_EINVAL;
    mp_status s = resolve(cfg, &t);
    if (s != MP_OK) return s;
    const LayoutReq r = batched_req(total_values, B, t);
    const Layout L = carve(ws, r);
    if (ws_bytes < L.bytes) return MP_ENOMEM;
    const DeviceInfo *d = nullptr;
    if ((s = current_device(&d)) != MP_OK) return s;
    cudaStream_t st = (cudaStream_t)stream;
    MP_CU(cudaMemsetAsync(L.hdr, 0, 256, st));
    MP_CU(launch_convert(values, dtype, total_values, L.x64, L.hdr, st));
    MP_CU(launch_batched_descs(offsets, ms, B, cfg->ez, cfg->flags, t.fp64, L.x64, L.mu, L.inv,
                               L.s32, L.s64, L.flat, L.keys, mp, pi, out_offsets, L.sets, L.probs,
                               L.fins, L.hdr, st));
    // every series is at most total_values long: finalize covers that bound
    return run_join(L, r, t, total_values, d, st);
}

size_t mp_backward_workspace_bytes(int64_t n, int32_t m)
{
    if (m < 4 || (int64_t)m > n) return 0;
    const long long l = n - m + 1;
    size_t off = 256;
    auto take = [&](size_t b) { off = ((off + 255) & ~(size_t)255) + b; };
    take(sizeof(double) * (size_t)n);
    take(sizeof(double) * (size_t)l);
    take(sizeof(double) * (size_t)l);
    take((size_t)l);
    return (off + 255) & ~(size_t)255;
}

mp_status mp_backward(const void *x, int32_t dtype, int64_t n, int32_t m, const int64_t *pi,
                      const double *grad_mp, double *grad_x, void *ws, size_t ws_bytes, void *stream)
{
    if (!x || !pi || !grad_mp || !grad_x || !ws || !valid_dtype(dtype) || !aligned256(ws))
        return MP_EINVAL;
    if (m < 4 || (int64_t)m > n || n > kMaxN) return MP_EINVAL;
    if (ws_bytes < mp_backward_workspace_bytes(n, m)) return MP_ENOMEM;
    const DeviceInfo *d = nullptr;
    mp_status s = current_device(&d);
    if (s != MP_OK) return s;
    const long long l = n - m + 1;
    size_t off = 0;
    auto take = [&](size_t b) -> char * {
        const size_t o = (off + 255) & ~(size_t)255;
        off = o + b;
        return (char *)ws + o;
    };
    Hdr *hdr = (Hdr *)take(256);
    double *x64 = (double *)take(sizeof(double) * (size_t)n);
    double *mu = (double *)take(sizeof(double) * (size_t)l);
    double *invn = (double *)take(sizeof(double) * (size_t)l);
    uint8_t *flat = (uint8_t *)take((size_t)l);
    cudaStream_t st = (cudaStream_t)stream;
    MP_CU(cudaMemsetAsync(hdr, 0, 256, st));
    MP_CU(launch_convert(x, dtype, n, x64, hdr, st));
    MP_CU(launch_stats_public(x64, MP_F64, n, m, mu, invn, nullptr, nullptr, flat, st));
    MP_CU(launch_backward(x64, n, m, mu, invn, flat, pi, grad_mp, grad_x, hdr, st));
    return MP_OK;
}

mp_status mp_timing_enable(int32_t on)
{
    const DeviceInfo *d = nullptr;
    mp_status s = current_device(&d);
    if (s != MP_OK) return s;
    int dev = 0;
    cudaGetDevice(&dev);
    std::lock_guard<std::mutex> lk(g_mu);
    DeviceInfo &dm = g_dev[dev];
    if (on && dm.ev[0] == nullptr) {
        if (cudaEventCreate(&dm.ev[0]) != cudaSuccess || cudaEventCreate(&dm.ev[1]) != cudaSuccess)
            return MP_ECUDA;
    }
    g_timing = on != 0;
    g_timing_dev = dev;
    return MP_OK;
}

mp_status mp_timing_last_ms(float *ms)
{
    if (!ms || g_timing_dev < 0) return MP_EINVAL;
    DeviceInfo &dm = g_dev[g_timing_dev];
    if (!dm.ev_used) return MP_EINVAL;
    if (cudaEventSynchronize(dm.ev[1]) != cudaSuccess) return MP_ECUDA;
    if (cudaEventElapsedTime(ms, dm.ev[0], dm.ev[1]) != cudaSuccess) return MP_ECUDA;
    return MP_OK;
}

mp_status mp_get_device_status(void *ws, void *stream)
{
    if (!ws) return MP_EINVAL;
    cudaStream_t st = (cudaStream_t)stream;
    if (cudaStreamSynchronize(st) != cudaSuccess) return MP_ECUDA;
    unsigned v = 0;
    if (cudaMemcpy(&v, ws, sizeof(v), cudaMemcpyDeviceToHost) != cudaSuccess) return MP_ECUDA;
    if (v != 0 && cudaMemset(ws, 0, sizeof(v)) != cudaSuccess) return MP_ECUDA;
    return (mp_status)v;
}

}  // extern "C"
