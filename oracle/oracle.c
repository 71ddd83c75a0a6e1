/*
 * oracle.c -- plain, slow, FP64 brute-force matrix profile.
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the checker the CUDA library is
 * compared against.  Only the test-suite, the package smoke check and the
 * benchmark's CPU-baseline leg may load it.  It shares no code, header,
 * table or helper with the CUDA path.
 *
 * What it computes is the definition the paper gives (Sec. 2 "The matrix
 * profile"): for every length-m subsequence, the smallest Euclidean distance
 * between z-normalised subsequences to any other subsequence of the join set,
 * with the position of that nearest neighbour (the profile index).  The paper
 * names the brute force, a full distance matrix reduced row by row, as the
 * O(n^2 m) method (Sec. 3.3 "Computational methods"); that is literally what
 * the loops below do, one row at a time so memory stays O(n).
 *
 * Conventions (the paper is silent on these; the readings are fixed here and
 * shared with the library):
 *   - window i is x[i .. i+m-1], 0-based; profile length l = n - m + 1
 *     (Sec. 3.4.1 and 3.4.3 print l for two inputs);
 *   - z-normalisation uses the population standard deviation (divide by m);
 *   - exclusion zone E = ceil(ez * m) (Sec. 3.2, the exclusion_zone argument);
 *     j is excluded from row i iff |i - j| < E, or |i - j| <= E when
 *     `inclusive` is set;
 *   - a window is flat iff all m values are equal; any pair involving a flat
 *     window has correlation 0, hence distance sqrt(2m);
 *   - distances are clamped to [0, 2 sqrt(m)];
 *   - ties go to the lowest index (strict "<" while scanning j upwards);
 *   - a row with no admissible neighbour gets MP = +inf and PI = -1.
 *
 * Parity: every function is pinned by tests that do not use this file's
 * formulas (closed forms, library routines, worked values from the paper);
 * see the test-suite's oracle pin module.
 */
#define _GNU_SOURCE
#include <math.h>
#include <pthread.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#include <unistd.h>

/* ---- sizes (Sec. 3.2 arguments, Sec. 3.4 printed summaries) ---- */

int64_t oracle_profile_length(int64_t n, int32_t m)
{
    if (m < 1 || (int64_t)m > n) return 0;
    return n - (int64_t)m + 1;
}

int64_t oracle_exclusion_zone(int32_t m, double ez)
{
    return (int64_t)ceil(ez * (double)m);
}

/* ---- per-window statistics, two-pass, straight from the definition ---- */

static void window_stats(const double *x, int32_t m, int64_t i,
                         double *mu, double *sigma, int *flat)
{
    const double *w = x + i;
    double s = 0.0;
    double lo = w[0], hi = w[0];
    for (int32_t k = 0; k < m; ++k) {
        s += w[k];
        if (w[k] < lo) lo = w[k];
        if (w[k] > hi) hi = w[k];
    }
    double mean = s / (double)m;
    double v = 0.0;
    for (int32_t k = 0; k < m; ++k) {
        double d = w[k] - mean;
        v += d * d;
    }
    *mu = mean;
    *sigma = sqrt(v / (double)m);
    *flat = (lo == hi);
}

int oracle_window_stats(const double *x, int64_t n, int32_t m,
                        double *mu, double *sigma, uint8_t *flat)
{
    int64_t l = oracle_profile_length(n, m);
    for (int64_t i = 0; i < l; ++i) {
        int f;
        window_stats(x, m, i, &mu[i], &sigma[i], &f);
        flat[i] = (uint8_t)f;
    }
    return 0;
}

/* z-normalised copy of window i (unused by callers when the window is flat) */
static void znorm(const double *x, int32_t m, int64_t i, double mu, double sigma,
                  double *z)
{
    for (int32_t k = 0; k < m; ++k) z[k] = (x[i + k] - mu) / sigma;
}

/* d(zi, zj) = sqrt(sum_k (zi[k] - zj[k])^2), clamped to [0, 2 sqrt(m)] */
static double zdist(const double *zi, const double *zj, int32_t m)
{
    double acc = 0.0;
    for (int32_t k = 0; k < m; ++k) {
        double d = zi[k] - zj[k];
        acc += d * d;
    }
    double d = sqrt(acc);
    double cap = 2.0 * sqrt((double)m);
    return d > cap ? cap : d;
}

/* distance between window i of xa and window j of xb */
static double pair_distance(const double *xa, int64_t i, const double *xb, int64_t j,
                            int32_t m, double *zi, double *zj)
{
    double mui, si, muj, sj;
    int fi, fj;
    window_stats(xa, m, i, &mui, &si, &fi);
    window_stats(xb, m, j, &muj, &sj, &fj);
    if (fi || fj) return sqrt(2.0 * (double)m);
    znorm(xa, m, i, mui, si, zi);
    znorm(xb, m, j, muj, sj, zj);
    return zdist(zi, zj, m);
}

double oracle_distance(const double *x, int64_t n, int32_t m, int64_t i, int64_t j)
{
    int64_t l = oracle_profile_length(n, m);
    if (i < 0 || j < 0 || i >= l || j >= l) return NAN;
    double *buf = malloc(sizeof(double) * 2 * (size_t)m);
    double d = pair_distance(x, i, x, j, m, buf, buf + m);
    free(buf);
    return d;
}

double oracle_distance_ab(const double *a, int64_t na, const double *b, int64_t nb,
                          int32_t m, int64_t i, int64_t j)
{
    if (i < 0 || j < 0 || i >= oracle_profile_length(na, m) ||
        j >= oracle_profile_length(nb, m)) return NAN;
    double *buf = malloc(sizeof(double) * 2 * (size_t)m);
    double d = pair_distance(a, i, b, j, m, buf, buf + m);
    free(buf);
    return d;
}

/* centred dot product c(i,j) = sum_k (x_{i+k} - mu_i)(y_{j+k} - mu_j) */
double oracle_cov(const double *xa, const double *xb, int32_t m, int64_t i, int64_t j)
{
    double mui, si, muj, sj;
    int fi, fj;
    window_stats(xa, m, i, &mui, &si, &fi);
    window_stats(xb, m, j, &muj, &sj, &fj);
    double acc = 0.0;
    for (int32_t k = 0; k < m; ++k) acc += (xa[i + k] - mui) * (xb[j + k] - muj);
    return acc;
}

/*
 * The update terms of the diagonal recurrence, from their definitions:
 *   df_i = (x_{i+m-1} - x_{i-1}) / 2
 *   dg_i = (x_{i+m-1} - mu_i) + (x_{i-1} - mu_{i-1})
 * for i >= 1, and df_0 = dg_0 = 0.  With them,
 *   c(i,j) - c(i-1,j-1) = df_i dg_j + df_j dg_i
 * (cross-series form: df/dg of the row series times those of the column one).
 */
int oracle_mpx_terms(const double *x, int64_t n, int32_t m, double *df, double *dg)
{
    int64_t l = oracle_profile_length(n, m);
    if (l <= 0) return -1;
    df[0] = 0.0;
    dg[0] = 0.0;
    double prev_mu, s;
    int f;
    window_stats(x, m, 0, &prev_mu, &s, &f);
    for (int64_t i = 1; i < l; ++i) {
        double mu;
        window_stats(x, m, i, &mu, &s, &f);
        df[i] = (x[i + m - 1] - x[i - 1]) / 2.0;
        dg[i] = (x[i + m - 1] - mu) + (x[i - 1] - prev_mu);
        prev_mu = mu;
    }
    return 0;
}

/* ---- the joins ---- */

typedef struct {
    const double *xr;      /* row series */
    const double *xc;      /* candidate (column) series */
    int64_t lr, lc;
    int32_t m;
    int self;              /* 1: self-join, apply the exclusion zone */
    int side;              /* self-join: 0 any j, -1 only j < i, +1 only j > i */
    const uint8_t *diag_ok; /* self-join: nullable; j allowed only if diag_ok[|i - j|] */
    int raw;               /* 1: non-normalised distance ||x_i - x_j|| (no z-norm, no flat rule) */
    int64_t excl;
    int inclusive;
    const int64_t *rows;
    int64_t nrows;
    double *mp;
    int64_t *pi;
    double *second;
    /* precomputed per-window stats of the candidate series */
    const double *cmu, *csig;
    const uint8_t *cflat;
    int64_t r0, r1;        /* this worker's slice of `rows` */
} job_t;

static int admissible(const job_t *J, int64_t i, int64_t j)
{
    if (!J->self) return 1;
    if ((J->side < 0 && j >= i) || (J->side > 0 && j <= i)) return 0;
    int64_t d = i > j ? i - j : j - i;
    if (J->diag_ok && !J->diag_ok[d]) return 0;
    return J->inclusive ? (d > J->excl) : (d >= J->excl);
}

static void *join_worker(void *arg)
{
    job_t *J = (job_t *)arg;
    int32_t m = J->m;
    double *zi = malloc(sizeof(double) * (size_t)m);
    double *zj = malloc(sizeof(double) * (size_t)m);
    const double flatd = sqrt(2.0 * (double)m);
    for (int64_t r = J->r0; r < J->r1; ++r) {
        int64_t i = J->rows[r];
        double mui, si;
        int fi;
        window_stats(J->xr, m, i, &mui, &si, &fi);
        if (!fi) znorm(J->xr, m, i, mui, si, zi);
        double best = INFINITY, second = INFINITY;
        int64_t arg_best = -1;
        for (int64_t j = 0; j < J->lc; ++j) {
            if (!admissible(J, i, j)) continue;
            double d;
            if (J->raw) {
                double acc = 0.0;
                for (int32_t k = 0; k < m; ++k) {
                    double e = J->xr[i + k] - J->xc[j + k];
                    acc += e * e;
                }
                d = sqrt(acc);
            } else if (fi || J->cflat[j]) {
                d = flatd;
            } else {
                znorm(J->xc, m, j, J->cmu[j], J->csig[j], zj);
                d = zdist(zi, zj, m);
            }
            if (d < best) {
                second = best;
                best = d;
                arg_best = j;
            } else if (d < second) {
                second = d;
            }
        }
        J->mp[r] = best;
        J->pi[r] = arg_best;
        if (J->second) J->second[r] = second;
    }
    free(zi);
    free(zj);
    return NULL;
}

static int run_join(job_t *tmpl, int nthreads)
{
    int64_t lc = tmpl->lc;
    double *cmu = malloc(sizeof(double) * (size_t)lc);
    double *csig = malloc(sizeof(double) * (size_t)lc);
    uint8_t *cflat = malloc((size_t)lc);
    if (!cmu || !csig || !cflat) {
        free(cmu); free(csig); free(cflat);
        return -2;
    }
    for (int64_t j = 0; j < lc; ++j) {
        int f;
        window_stats(tmpl->xc, tmpl->m, j, &cmu[j], &csig[j], &f);
        cflat[j] = (uint8_t)f;
    }
    tmpl->cmu = cmu;
    tmpl->csig = csig;
    tmpl->cflat = cflat;
    if (nthreads <= 0) nthreads = (int)sysconf(_SC_NPROCESSORS_ONLN);
    if (nthreads < 1) nthreads = 1;
    if ((int64_t)nthreads > tmpl->nrows) nthreads = (int)(tmpl->nrows > 0 ? tmpl->nrows : 1);
    job_t *jobs = malloc(sizeof(job_t) * (size_t)nthreads);
    pthread_t *th = malloc(sizeof(pthread_t) * (size_t)nthreads);
    for (int t = 0; t < nthreads; ++t) {
        jobs[t] = *tmpl;
        jobs[t].r0 = tmpl->nrows * t / nthreads;
        jobs[t].r1 = tmpl->nrows * (t + 1) / nthreads;
        pthread_create(&th[t], NULL, join_worker, &jobs[t]);
    }
    for (int t = 0; t < nthreads; ++t) pthread_join(th[t], NULL);
    free(jobs);
    free(th);
    free(cmu);
    free(csig);
    free(cflat);
    return 0;
}

/*
 * Self-join over the requested rows: mp[r], pi[r] (and the second-smallest
 * distance second[r], nullable) for row i = rows[r].
 */
int oracle_selfjoin(const double *x, int64_t n, int32_t m, int64_t excl, int inclusive,
                    const int64_t *rows, int64_t nrows, double *mp, int64_t *pi,
                    double *second, int nthreads)
{
    int64_t l = oracle_profile_length(n, m);
    if (l <= 0 || m < 2) return -1;
    for (int64_t r = 0; r < nrows; ++r)
        if (rows[r] < 0 || rows[r] >= l) return -1;
    job_t J = {0};
    J.xr = x; J.xc = x; J.lr = l; J.lc = l; J.m = m; J.self = 1;
    J.excl = excl; J.inclusive = inclusive;
    J.rows = rows; J.nrows = nrows; J.mp = mp; J.pi = pi; J.second = second;
    return run_join(&J, nthreads);
}

/*
 * Left (side = -1) or right (side = +1) self-join profile: as oracle_selfjoin,
 * with the candidates restricted to the windows before (after) row i.  The
 * paper's time series chains (Sec. 3.4.3) are built on these two profiles; the
 * paper gives no formula, so this is the self-join definition above with the
 * candidate set cut in two.
 */
int oracle_selfjoin_side(const double *x, int64_t n, int32_t m, int64_t excl, int inclusive,
                         int side, const int64_t *rows, int64_t nrows, double *mp, int64_t *pi,
                         double *second, int nthreads)
{
    int64_t l = oracle_profile_length(n, m);
    if (l <= 0 || m < 2 || (side != -1 && side != 1)) return -1;
    for (int64_t r = 0; r < nrows; ++r)
        if (rows[r] < 0 || rows[r] >= l) return -1;
    job_t J = {0};
    J.xr = x; J.xc = x; J.lr = l; J.lc = l; J.m = m; J.self = 1; J.side = side;
    J.excl = excl; J.inclusive = inclusive;
    J.rows = rows; J.nrows = nrows; J.mp = mp; J.pi = pi; J.second = second;
    return run_join(&J, nthreads);
}

/*
 * Self-join restricted to a set of diagonals: j is a candidate of row i only
 * if diag_ok[|i - j|] (l entries) besides the exclusion zone.  This is what an
 * anytime run (Sec. 3.3.1, 3.3.3: the best-so-far profile over the distance
 * profiles / diagonals computed so far) has seen after a given set of
 * diagonals.
 */
int oracle_selfjoin_diags(const double *x, int64_t n, int32_t m, int64_t excl, int inclusive,
                          const uint8_t *diag_ok, const int64_t *rows, int64_t nrows, double *mp,
                          int64_t *pi, double *second, int nthreads)
{
    int64_t l = oracle_profile_length(n, m);
    if (l <= 0 || m < 2 || !diag_ok) return -1;
    for (int64_t r = 0; r < nrows; ++r)
        if (rows[r] < 0 || rows[r] >= l) return -1;
    job_t J = {0};
    J.xr = x; J.xc = x; J.lr = l; J.lc = l; J.m = m; J.self = 1; J.diag_ok = diag_ok;
    J.excl = excl; J.inclusive = inclusive;
    J.rows = rows; J.nrows = nrows; J.mp = mp; J.pi = pi; J.second = second;
    return run_join(&J, nthreads);
}

/*
 * Non-normalised distance (SiMPle, Sec. 3.3.4: no z-normalisation):
 * d(i,j) = ||x_i - x_j||, the plain Euclidean distance of the raw windows.
 * Self-join with the exclusion zone (raw_ab = 0) or AB-join (raw_ab = 1, b
 * the candidate series).  No flat-window rule applies.
 */
int oracle_join_raw(const double *a, int64_t na, const double *b, int64_t nb, int32_t m,
                    int raw_ab, int64_t excl, int inclusive, const int64_t *rows, int64_t nrows,
                    double *mp, int64_t *pi, double *second, int nthreads)
{
    int64_t la = oracle_profile_length(na, m);
    int64_t lb = raw_ab ? oracle_profile_length(nb, m) : la;
    if (la <= 0 || lb <= 0 || m < 2) return -1;
    for (int64_t r = 0; r < nrows; ++r)
        if (rows[r] < 0 || rows[r] >= la) return -1;
    job_t J = {0};
    J.xr = a; J.xc = raw_ab ? b : a; J.lr = la; J.lc = lb; J.m = m; J.self = !raw_ab;
    J.raw = 1; J.excl = excl; J.inclusive = inclusive;
    J.rows = rows; J.nrows = nrows; J.mp = mp; J.pi = pi; J.second = second;
    return run_join(&J, nthreads);
}

/*
 * AB-join (Sec. 3.2: two series in, no exclusion zone): for window rows[r] of
 * `a`, the nearest window of `b`.
 */
int oracle_abjoin(const double *a, int64_t na, const double *b, int64_t nb, int32_t m,
                  const int64_t *rows, int64_t nrows, double *mp, int64_t *pi,
                  double *second, int nthreads)
{
    int64_t la = oracle_profile_length(na, m), lb = oracle_profile_length(nb, m);
    if (la <= 0 || lb <= 0 || m < 2) return -1;
    for (int64_t r = 0; r < nrows; ++r)
        if (rows[r] < 0 || rows[r] >= la) return -1;
    job_t J = {0};
    J.xr = a; J.xc = b; J.lr = la; J.lc = lb; J.m = m; J.self = 0;
    J.rows = rows; J.nrows = nrows; J.mp = mp; J.pi = pi; J.second = second;
    return run_join(&J, nthreads);
}

/*
 * ---- semantic segmentation (Sec. 3.4.2, FLUSS after Gharghabi et al.) ----
 *
 * The paper cites the method without formulas; these follow its published
 * description.  Each window i with a neighbour pi[i] >= 0 is an arc between
 * a = min(i, pi[i]) and b = max(i, pi[i]); the arc count at position k is the
 * number of arcs with a <= k < b.  The idealised count for neighbours drawn
 * uniformly at random is IAC[k] = 2 k (l - k) / l, and the corrected curve is
 * CAC[k] = min(AC[k] / IAC[k], 1), set to 1 where IAC[k] = 0 and within `edge`
 * positions of either end.
 */

/* arc count at one position, straight from the definition: O(l) */
int64_t oracle_arc_count_at(const int64_t *pi, int64_t l, int64_t k)
{
    int64_t c = 0;
    for (int64_t i = 0; i < l; ++i) {
        if (pi[i] < 0 || pi[i] >= l) continue;
        int64_t a = pi[i] < i ? pi[i] : i, b = pi[i] < i ? i : pi[i];
        if (a <= k && k < b) ++c;
    }
    return c;
}

/* every position by the definition: O(l^2), for small l */
int oracle_arc_counts(const int64_t *pi, int64_t l, int64_t *ac)
{
    if (l < 1) return -1;
    for (int64_t k = 0; k < l; ++k) ac[k] = oracle_arc_count_at(pi, l, k);
    return 0;
}

/* the same counts in O(l): +1 where an arc starts, -1 where it ends, running sum */
int oracle_arc_counts_fast(const int64_t *pi, int64_t l, int64_t *ac)
{
    if (l < 1) return -1;
    for (int64_t k = 0; k < l; ++k) ac[k] = 0;
    for (int64_t i = 0; i < l; ++i) {
        if (pi[i] < 0 || pi[i] >= l) continue;
        int64_t a = pi[i] < i ? pi[i] : i, b = pi[i] < i ? i : pi[i];
        if (a == b) continue;
        ac[a] += 1;
        ac[b] -= 1;
    }
    for (int64_t k = 1; k < l; ++k) ac[k] += ac[k - 1];
    return 0;
}

int oracle_cac(const int64_t *ac, int64_t l, int64_t edge, double *cac)
{
    if (l < 1 || edge < 0) return -1;
    for (int64_t k = 0; k < l; ++k) {
        double iac = 2.0 * (double)k * (double)(l - k) / (double)l;
        double c = 1.0;
        if (k >= edge && k < l - edge && iac > 0.0) {
            double r = (double)ac[k] / iac;
            c = r < 1.0 ? r : 1.0;
        }
        cac[k] = c;
    }
    return 0;
}

/* boundaries: the lowest cac (lowest index on ties), then the lowest outside
   |k - s| < seg_excl of every earlier pick; -1 once nothing is left */
int oracle_segments(const double *cac, int64_t l, int32_t num_segments, int64_t seg_excl,
                    int64_t *segments)
{
    if (l < 1 || num_segments < 0 || seg_excl < 0) return -1;
    for (int32_t s = 0; s < num_segments; ++s) {
        int64_t best = -1;
        for (int64_t k = 0; k < l; ++k) {
            int masked = 0;
            for (int32_t t = 0; t < s; ++t) {
                if (segments[t] < 0) continue;
                int64_t d = k > segments[t] ? k - segments[t] : segments[t] - k;
                if (d < seg_excl || d == 0) masked = 1;
            }
            if (masked) continue;
            if (best < 0 || cac[k] < cac[best]) best = k;
        }
        segments[s] = best;
    }
    return 0;
}

/*
 * Gradient of L = sum_i g_i * MP_i with respect to x, holding each argmin
 * pair (i, pi[i]) fixed.  With zi, zj the z-normalised windows, rho their
 * correlation (1/m) sum zi zj, d = |zi - zj| and sigma the population
 * standard deviations:
 *   dMP_i/dx_{i+k} = -(zj[k] - rho zi[k]) / (sigma_i d)
 *   dMP_i/dx_{j+k} = -(zi[k] - rho zj[k]) / (sigma_j d)
 * A pair contributes nothing when pi[i] < 0, either window is flat, or
 * d < 1e-12.  grad_x (length n) is overwritten.
 */
int oracle_grad(const double *x, int64_t n, int32_t m, const int64_t *pi,
                const double *g, double *grad_x)
{
    int64_t l = oracle_profile_length(n, m);
    if (l <= 0) return -1;
    memset(grad_x, 0, sizeof(double) * (size_t)n);
    double *zi = malloc(sizeof(double) * (size_t)m);
    double *zj = malloc(sizeof(double) * (size_t)m);
    for (int64_t i = 0; i < l; ++i) {
        int64_t j = pi[i];
        if (j < 0 || j >= l || g[i] == 0.0) continue;
        double mui, si, muj, sj;
        int fi, fj;
        window_stats(x, m, i, &mui, &si, &fi);
        window_stats(x, m, j, &muj, &sj, &fj);
        if (fi || fj) continue;
        znorm(x, m, i, mui, si, zi);
        znorm(x, m, j, muj, sj, zj);
        double rho = 0.0;
        for (int32_t k = 0; k < m; ++k) rho += zi[k] * zj[k];
        rho /= (double)m;
        double d = zdist(zi, zj, m);
        if (d < 1e-12) continue;
        for (int32_t k = 0; k < m; ++k) {
            grad_x[i + k] += -g[i] * (zj[k] - rho * zi[k]) / (si * d);
            grad_x[j + k] += -g[i] * (zi[k] - rho * zj[k]) / (sj * d);
        }
    }
    free(zi);
    free(zj);
    return 0;
}
