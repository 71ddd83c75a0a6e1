// stats.cu -- input conversion and per-window statistics (FP64, compensated).
//
// For window i of length m: mean mu_i, inverse centred norm
// invn_i = 1 / ||x_i - mu_i||_2 (0 when the window is flat), and the update
// terms of the diagonal recurrence
//     df_i = (x_{i+m-1} - x_{i-1}) / 2,
//     dg_i = (x_{i+m-1} - mu_i) + (x_{i-1} - mu_{i-1}),      df_0 = dg_0 = 0,
// which satisfy c(i,j) = c(i-1,j-1) + df_i dg_j + df_j dg_i for the centred
// dot product c (this is the dot-product reuse the paper credits to STOMP,
// Sec. 3.3.2, written in covariance form).
//
// Each thread owns a run of consecutive windows (at most kWindowsPerThread;
// shorter when a series is short, so that the blocks of kStatsThreads
// threads still reach every SM: the work is FP64-bound, and the FP64 pipes
// of idle SMs are lost).  It seeds the window sums
// sum(x) and sum(x^2) of the run's first window with a direct double-double
// (106-bit) summation and then slides them window to window, adding the
// entering sample and subtracting the leaving one in double-double, so the
// windowed sums are compensated prefix differences that never lose the
// low-order bits a plain FP64 running sum would.  The centred sum of
// squares is sum(x^2) - mean * sum(x), also in double-double, which stays
// exact to FP64 even when the series sits far from zero.
//
// Flatness (all m values equal) is decided exactly by counting, with the same
// sliding scheme, the positions t in the window where x[t] != x[t+1].
#include <cmath>

#include "internal.cuh"
#include "launch_shape.cuh"

namespace mpgb {
namespace {

constexpr int kStatsThreads = 32;      // one warp per block: short series spread over more SMs
constexpr int kMinStatsRun = 4;

struct dd {
    double hi, lo;
};

__device__ __forceinline__ dd two_sum(double a, double b)
{
    const double s = a + b;
    const double bb = s - a;
    const double e = (a - (s - bb)) + (b - bb);
    return {s, e};
}
__device__ __forceinline__ dd quick_two_sum(double a, double b)
{
    const double s = a + b;
    return {s, b - (s - a)};
}
__device__ __forceinline__ dd dd_add(dd a, double b)
{
    dd s = two_sum(a.hi, b);
    s.lo += a.lo;
    return quick_two_sum(s.hi, s.lo);
}
__device__ __forceinline__ dd dd_add(dd a, dd b)
{
    dd s = two_sum(a.hi, b.hi);
    s.lo += a.lo + b.lo;
    return quick_two_sum(s.hi, s.lo);
}
__device__ __forceinline__ dd two_prod(double a, double b)
{
    const double p = a * b;
    return {p, fma(a, b, -p)};
}
__device__ __forceinline__ dd dd_neg(dd a) { return {-a.hi, -a.lo}; }
__device__ __forceinline__ dd dd_mul(dd a, dd b)
{
    dd p = two_prod(a.hi, b.hi);
    p.lo = fma(a.hi, b.lo, fma(a.lo, b.hi, p.lo));
    return quick_two_sum(p.hi, p.lo);
}
__device__ __forceinline__ dd dd_div(dd a, double b)
{
    const double q1 = a.hi / b;
    const dd r = dd_add(a, dd_neg(two_prod(q1, b)));
    return quick_two_sum(q1, r.hi / b);
}

struct WindowOut {
    double mu, invn, df, dg;
    double h;                                // ||x_i||^2 / 2 (non-normalised distance)
    double dgr;                              // x_{i+m-1} + x_{i-1} (non-normalised recurrence)
    bool flat;
};

// Walk windows [i, iend) of series x (length-m windows, l of them), calling
// emit(w, WindowOut) for each.  T is the input element type.
template <typename T, typename Emit>
__device__ __forceinline__ void walk_windows(const T *__restrict__ x, int m, long long i,
                                             long long iend, Emit emit)
{
    const long long w0 = i > 0 ? i - 1 : 0;
    dd s1 = {0.0, 0.0}, s2 = {0.0, 0.0};
    int changes = 0;
    for (int t = 0; t < m; ++t) {
        const double v = (double)x[w0 + t];
        s1 = dd_add(s1, v);
        s2 = dd_add(s2, two_prod(v, v));
        if (t > 0 && x[w0 + t] != x[w0 + t - 1]) ++changes;
    }
    double mu_prev = 0.0;
    for (long long w = w0; w < iend; ++w) {
        if (w > w0) {
            const double vin = (double)x[w + m - 1];
            const double vout = (double)x[w - 1];
            s1 = dd_add(dd_add(s1, vin), -vout);
            s2 = dd_add(dd_add(s2, two_prod(vin, vin)), dd_neg(two_prod(vout, vout)));
            changes += (x[w + m - 1] != x[w + m - 2]) ? 1 : 0;
            changes -= (x[w] != x[w - 1]) ? 1 : 0;
        }
        const dd mean = dd_div(s1, (double)m);
        const double mu = mean.hi;
        if (w >= i) {
            const dd var = dd_add(s2, dd_neg(dd_mul(mean, s1)));
            WindowOut o;
            o.mu = mu;
            o.flat = (changes == 0);
            o.invn = (o.flat || !(var.hi > 0.0)) ? 0.0 : 1.0 / sqrt(var.hi);
            o.h = 0.5 * (s2.hi + s2.lo);
            if (w > 0) {
                const double a = (double)x[w + m - 1];
                const double b = (double)x[w - 1];
                o.df = 0.5 * (a - b);
                o.dg = (a - mu) + (b - mu_prev);
                o.dgr = a + b;
            } else {
                o.df = 0.0;
                o.dg = 0.0;
                o.dgr = 0.0;
            }
            emit(w, o);
        }
        mu_prev = mu;
    }
}

template <typename T>
__global__ void convert_kernel(const T *__restrict__ x, long long n, double *__restrict__ y,
                               Hdr *hdr)
{
    bool bad = false;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x) {
        const double v = (double)x[i];
        bad |= !isfinite(v);
        y[i] = v;
    }
    if (__any_sync(0xffffffffu, bad) && (threadIdx.x & 31) == 0) set_status(hdr, MP_EINVAL_DATA);
}

__global__ void stats_sets_kernel(const StatSet *__restrict__ sets, int nsets, long long total,
                                  int run, double *__restrict__ mu, double *__restrict__ inv,
                                  float4 *__restrict__ s32,
                                  D4 *__restrict__ s64, uint8_t *__restrict__ flat,
                                  double *__restrict__ set_acc)
{
    long long g = ((long long)blockIdx.x * blockDim.x + threadIdx.x) * run;
    if (g >= total) return;
    const long long gend = min(g + (long long)run, total);
    int lo = 0, hi = nsets;                       // sets[lo].sbase <= g < sets[hi].sbase
    while (hi - lo > 1) {
        const int mid = (lo + hi) >> 1;
        if (sets[mid].sbase <= g) lo = mid; else hi = mid;
    }
    int s = lo;
    while (g < gend && s < nsets) {
        const StatSet S = sets[s];
        if (g < S.sbase) g = S.sbase;
        if (g >= gend) break;
        const long long l = S.l > 0 ? S.l : 0;
        const long long ext = l + kPad;
        const long long i = g - S.sbase;
        if (i >= ext) {                           // in the gap after this set
            ++s;
            continue;
        }
        const long long iend = min(ext, i + (gend - g));
        const long long vend = min(iend, l);
        if (i < vend) {
            const long long base = S.sbase;
            double logsum = 0.0, cnt = 0.0;
            walk_windows<double>(S.x, S.m, i, vend, [&](long long w, const WindowOut &o) {
                const long long q = base + w;
                if (S.raw) {                            // non-normalised: q-recurrence terms
                    const float ninf = __int_as_float(0xff800000);
                    if (mu) mu[q] = 0.0;
                    if (inv) inv[q] = o.h;
                    if (flat) flat[q] = 0;
                    if (s32) s32[q] = make_float4((float)o.df, (float)o.dgr, (float)o.h, ninf);
                    if (s64) s64[q] = make_d4(o.df, o.dgr, o.h,
                                              __longlong_as_double((long long)0xfff0000000000000ull));
                    return;
                }
                if (o.invn > 0.0) {                     // norm statistics of the set
                    logsum -= log(o.invn);
                    cnt += 1.0;
                }
                if (mu) mu[q] = o.mu;
                if (inv) inv[q] = o.invn;
                if (flat) flat[q] = o.flat ? 1 : 0;
                // .w starts as the running threshold of this index: +inf for a flat
                // window (its answer is closed-form, the tile kernel never updates
                // it), -inf otherwise (no candidate seen yet)
                const float t32 = o.flat ? __int_as_float(0x7f800000) : __int_as_float(0xff800000);
                const double t64 = o.flat ? __longlong_as_double(0x7ff0000000000000ll)
                                          : __longlong_as_double((long long)0xfff0000000000000ull);
                if (s32) s32[q] = make_float4((float)o.df, (float)o.dg, (float)o.invn, t32);
                if (s64) s64[q] = make_d4(o.df, o.dg, o.invn, t64);
            });
            if (set_acc && cnt > 0.0) {
                atomicAdd(set_acc + 2 * s, logsum);
                atomicAdd(set_acc + 2 * s + 1, cnt);
            }
        }
        for (long long w = (i > l ? i : l); w < iend; ++w) {      // padding entries
            const long long q = S.sbase + w;
            if (mu) mu[q] = 0.0;
            if (inv) inv[q] = 0.0;
            if (flat) flat[q] = 0;
            if (s32) s32[q] = make_float4(0.0f, 0.0f, __int_as_float(0x7fc00000), __int_as_float(0x7f800000));
            if (s64) s64[q] = make_d4(0.0, 0.0, __longlong_as_double(0x7ff8000000000000ll),
                                      __longlong_as_double(0x7ff0000000000000ll));
        }
        g += iend - i;
        if (iend == ext) ++s;
    }
}

template <typename T>
__global__ void stats_public_kernel(const T *__restrict__ x, long long l, int m, int run,
                                    double *mu, double *invn, double *df, double *dg,
                                    uint8_t *flat)
{
    const long long i = ((long long)blockIdx.x * blockDim.x + threadIdx.x) * run;
    if (i >= l) return;
    const long long iend = min(i + (long long)run, l);
    walk_windows<T>(x, m, i, iend, [&](long long w, const WindowOut &o) {
        if (mu) mu[w] = o.mu;
        if (invn) invn[w] = o.invn;
        if (df) df[w] = o.df;
        if (dg) dg[w] = o.dg;
        if (flat) flat[w] = o.flat ? 1 : 0;
    });
}

}  // namespace

int sm_count()
{
    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || sms < 1)
        return 1;
    return sms;
}

int spread_run(long long items, long long groups, int threads, int run, int min_run)
{
    const long long sms = sm_count();
    auto blocks = [&](int r) { return groups * (((items + r - 1) / r + threads - 1) / threads); };
    while (run > min_run && blocks(run / 2) <= sms) run /= 2;
    return run;
}

cudaError_t launch_convert(const void *x, int dtype, long long n, double *x64, Hdr *hdr,
                           cudaStream_t st)
{
    if (n <= 0) return cudaSuccess;
    const int threads = 256;
    long long blocks = (n + threads - 1) / threads;
    if (blocks > 8192) blocks = 8192;
    if (dtype == MP_F32)
        convert_kernel<float><<<(int)blocks, threads, 0, st>>>((const float *)x, n, x64, hdr);
    else
        convert_kernel<double><<<(int)blocks, threads, 0, st>>>((const double *)x, n, x64, hdr);
    return cudaGetLastError();
}

cudaError_t launch_stats_sets(const StatSet *sets, int nsets, long long total_index, double *mu,
                              double *inv, float4 *s32, D4 *s64, uint8_t *flat, double *set_acc,
                              cudaStream_t st)
{
    if (total_index <= 0 || nsets <= 0) return cudaSuccess;
    const int run = spread_run(total_index, 1, kStatsThreads, kWindowsPerThread, kMinStatsRun);
    const long long runs = (total_index + run - 1) / run;
    const long long blocks = (runs + kStatsThreads - 1) / kStatsThreads;
    stats_sets_kernel<<<(unsigned)blocks, kStatsThreads, 0, st>>>(sets, nsets, total_index, run, mu,
                                                                   inv, s32, s64, flat, set_acc);
    return cudaGetLastError();
}

cudaError_t launch_stats_public(const void *x, int dtype, long long n, int m, double *mu,
                                double *invn, double *df, double *dg, uint8_t *flat,
                                cudaStream_t st)
{
    const long long l = n - m + 1;
    if (l <= 0) return cudaSuccess;
    const int run = spread_run(l, 1, kStatsThreads, kWindowsPerThread, kMinStatsRun);
    const long long runs = (l + run - 1) / run;
    const long long blocks = (runs + kStatsThreads - 1) / kStatsThreads;
    if (dtype == MP_F32)
        stats_public_kernel<float><<<(unsigned)blocks, kStatsThreads, 0, st>>>(
            (const float *)x, l, m, run, mu, invn, df, dg, flat);
    else
        stats_public_kernel<double><<<(unsigned)blocks, kStatsThreads, 0, st>>>(
            (const double *)x, l, m, run, mu, invn, df, dg, flat);
    return cudaGetLastError();
}

}  // namespace mpgb
