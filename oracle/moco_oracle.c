/*
 * moco oracle: a plain, slow, obviously correct CPU statement of the
 * translation search of "moco: Fast Motion Correction for Calcium Imaging"
 * (Dubbs, Guevara, Peterka, Yuste; arXiv 1506.06039).
 *
 * TEST INFRASTRUCTURE ONLY. Nothing in the product library links, loads or
 * calls this file; only the tests, the package's smoke check and the
 * benchmark's CPU-baseline leg do. It shares no code, header, table or helper
 * with the CUDA path.
 *
 * Everything here follows the definitions of Section 2 literally:
 *   - f_{s,t} = (1 / Area(D_{s,t})) * sum_{(i,j) in D_{s,t}} (a[i+s][j+t] - b[i][j])^2,
 *     D_{s,t} = {(i,j) : 0 <= i < m, 0 <= j < n, 0 <= i+s < m, 0 <= j+t < n}
 *     (the paper's 1-based set, written 0-based), for every max(|s|,|t|) < w.
 *     The sum is formed in exact int64 by brute force over D: no summed-area
 *     tables, no FFT (those are the paper's speed-ups; they compute the same f).
 *   - Downsampling (Section 2, "downsampled if larger than 256x256"; Section 3,
 *     "we downsample once"): one level when max(m, n) > 256, a 2x2 box. The
 *     oracle carries the exact integer 4-sum; costs are reported in box-mean
 *     units (4-sum cost / 16).
 *   - Upsampling (Section 2): the coarse optimum (s,t) is doubled and f is
 *     evaluated at full resolution for (2s+u, 2t+v), u, v in {-1, 0, 1}; the
 *     minimum is kept.
 *   - More levels (Section 2 says the resolution is "multiplied by two
 *     multiple times"; Section 3 reports that three or four downsamplings
 *     cause severe errors): with L levels, level l is the 2x2 sum of level
 *     l - 1 (floor sizes; level 0 is the image), the exhaustive search runs
 *     on level L, and for l = L-1 down to 0 the doubled optimum is refined by
 *     the 3x3 search on level l's images (exact sums, the same tie-break).
 *     Costs on level L are reported per pixel of the full image (/ 16^L).
 *   - Ties (the paper is silent): among equal f the shift with the smallest
 *     |s| + |t| wins, then the smallest s, then the smallest t. Costs are
 *     compared as exact rationals S1 * A2 vs S2 * A1 in 128-bit integers.
 *   - Correction (Section 2: the found shifts "motion correct" the video; the
 *     paper gives no formula, so the definition below is this project's
 *     reading): corrected[f][i][j] = a_f[i + s_f][j + t_f] where that pixel
 *     lies in the frame, else a fill value; the corrected mean image averages,
 *     per pixel, the frames whose source pixel lies in the frame (exact integer
 *     sum / count in FP64; the fill value where no frame covers the pixel).
 *   - Soft-min and its gradient (not in the paper; the differentiable form):
 *     L_f = -tau_f log sum_{s,t} exp(-f_{s,t} / tau_f), tau_f given, in FP64;
 *     the gradient is the chain rule through Section 2's f.
 *
 * Build: gcc -O2 -fopenmp -shared -fPIC moco_oracle.c -o liboracle.so
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

typedef __int128 i128;

/* ---- Section 2: D_{s,t} and Area(D_{s,t}) --------------------------------- */

/* Number of pairs in D_{s,t}: rows i with 0 <= i, i+s < m, times columns. */
int64_t oracle_area(int m, int n, int s, int t) {
    int64_t rows = 0, cols = 0;
    for (int i = 0; i < m; ++i)
        if (i + s >= 0 && i + s < m) ++rows;
    for (int j = 0; j < n; ++j)
        if (j + t >= 0 && j + t < n) ++cols;
    return rows * cols;
}

/* Area(D_{s,t}) * f_{s,t} for one shift, exact, by brute force over D. */
int64_t oracle_ssd_one(const int32_t *a, const int32_t *b, int m, int n, int s, int t) {
    int64_t S = 0;
    for (int i = 0; i < m; ++i) {
        if (i + s < 0 || i + s >= m) continue;
        for (int j = 0; j < n; ++j) {
            if (j + t < 0 || j + t >= n) continue;
            int64_t d = (int64_t)a[(int64_t)(i + s) * n + (j + t)] - (int64_t)b[(int64_t)i * n + j];
            S += d * d;
        }
    }
    return S;
}

/* All (2w-1)^2 shifts; S[(s+w-1)*(2w-1) + (t+w-1)]. */
void oracle_ssd_all(const int32_t *a, const int32_t *b, int m, int n, int w, int64_t *S) {
    int W = 2 * w - 1;
    for (int s = -(w - 1); s <= w - 1; ++s)
        for (int t = -(w - 1); t <= w - 1; ++t)
            S[(s + w - 1) * W + (t + w - 1)] = oracle_ssd_one(a, b, m, n, s, t);
}

/* ---- Downsampling: one 2x2 box level (exact integer 4-sum) ---------------- */

void oracle_downsample(const uint16_t *a, int m, int n, int32_t *out) {
    int mc = m / 2, nc = n / 2;
    for (int i = 0; i < mc; ++i)
        for (int j = 0; j < nc; ++j)
            out[(int64_t)i * nc + j] = (int32_t)a[(int64_t)(2 * i) * n + 2 * j] +
                                       (int32_t)a[(int64_t)(2 * i + 1) * n + 2 * j] +
                                       (int32_t)a[(int64_t)(2 * i) * n + 2 * j + 1] +
                                       (int32_t)a[(int64_t)(2 * i + 1) * n + 2 * j + 1];
}

static void widen(const uint16_t *a, int64_t count, int32_t *out) {
    for (int64_t k = 0; k < count; ++k) out[k] = (int32_t)a[k];
}

/* 2x2 sums of an int32 image (m x n -> m/2 x n/2, floor). */
static void downsample32(const int32_t *a, int m, int n, int32_t *out) {
    int mc = m / 2, nc = n / 2;
    for (int i = 0; i < mc; ++i)
        for (int j = 0; j < nc; ++j)
            out[(int64_t)i * nc + j] = a[(int64_t)(2 * i) * n + 2 * j] + a[(int64_t)(2 * i + 1) * n + 2 * j] +
                                       a[(int64_t)(2 * i) * n + 2 * j + 1] + a[(int64_t)(2 * i + 1) * n + 2 * j + 1];
}

#define ORACLE_MAX_LEVELS 4

/* The level images of a (lev[0] = a widened, lev[l] = 2x2 sums of lev[l-1])
 * into one buffer; off[l] is level l's start, ml[l] x nl[l] its size. */
static void pyramid(const uint16_t *a, int m, int n, int L, int32_t *buf, int64_t *off, int *ml, int *nl) {
    ml[0] = m; nl[0] = n; off[0] = 0;
    widen(a, (int64_t)m * n, buf);
    for (int l = 1; l <= L; ++l) {
        ml[l] = ml[l - 1] / 2; nl[l] = nl[l - 1] / 2;
        off[l] = off[l - 1] + (int64_t)ml[l - 1] * nl[l - 1];
        downsample32(buf + off[l - 1], ml[l - 1], nl[l - 1], buf + off[l]);
    }
}

/* Elements of a pyramid buffer of L levels. */
static int64_t pyramid_size(int m, int n, int L) {
    int64_t total = 0;
    for (int l = 0; l <= L; ++l) { total += (int64_t)m * n; m /= 2; n /= 2; }
    return total;
}

/* Paper rule for the number of levels: one iff the image is larger than 256x256. */
int oracle_levels(int m, int n) { return (m > 256 || n > 256) ? 1 : 0; }

/* ---- Comparison with the tie-break --------------------------------------- */

/* Returns 1 when candidate 1 beats candidate 2: smaller S/A, then smaller
 * |s|+|t|, then smaller s, then smaller t. */
static int better(int64_t S1, int64_t A1, int s1, int t1, int64_t S2, int64_t A2, int s2, int t2) {
    i128 l = (i128)S1 * (i128)A2, r = (i128)S2 * (i128)A1;
    if (l != r) return l < r;
    int k1 = abs(s1) + abs(t1), k2 = abs(s2) + abs(t2);
    if (k1 != k2) return k1 < k2;
    if (s1 != s2) return s1 < s2;
    return t1 < t2;
}

/* ---- Align one frame ------------------------------------------------------ */

typedef struct {
    int32_t s, t;        /* final shift */
    int32_t sc, tc;      /* optimum on the searched (coarse) grid */
    double fbest;        /* coarse f at the optimum, box-mean units */
    double margin;       /* (f2 - f1) / f1 on the searched grid */
    double ffinal;       /* full-resolution f at the final shift (= fbest w/o levels) */
} oracle_result;

/* a is the frame; bp the template's pyramid (offsets boff, sizes ml x nl). */
static void align_one(const uint16_t *a, const int32_t *bp, const int64_t *boff, int m, int n, int w, int L,
                      int32_t *ap, int64_t *Sbuf, oracle_result *res) {
    int64_t off[ORACLE_MAX_LEVELS + 1];
    int ml[ORACLE_MAX_LEVELS + 1], nl[ORACLE_MAX_LEVELS + 1];
    pyramid(a, m, n, L, ap, off, ml, nl);
    const int32_t *A = ap + off[L], *B = bp + boff[L];
    const int mc = ml[L], nc = nl[L];
    double unit = 1.0;
    for (int l = 0; l < L; ++l) unit *= 16.0;
    int W = 2 * w - 1;
    /* Exhaustive search over max(|s|,|t|) < w on the searched level. */
    oracle_ssd_all(A, B, mc, nc, w, Sbuf);
    int bs = 0, bt = 0;
    int64_t bS = -1, bA = 1;
    for (int s = -(w - 1); s <= w - 1; ++s)
        for (int t = -(w - 1); t <= w - 1; ++t) {
            int64_t S = Sbuf[(s + w - 1) * W + (t + w - 1)];
            int64_t Ar = oracle_area(mc, nc, s, t);
            if (bS < 0 || better(S, Ar, s, t, bS, bA, bs, bt)) {
                bS = S; bA = Ar; bs = s; bt = t;
            }
        }
    /* Second-best value over every other shift, for the margin. */
    double f1 = (double)bS / (double)bA / unit, f2 = INFINITY;
    for (int s = -(w - 1); s <= w - 1; ++s)
        for (int t = -(w - 1); t <= w - 1; ++t) {
            if (s == bs && t == bt) continue;
            double f = (double)Sbuf[(s + w - 1) * W + (t + w - 1)] / (double)oracle_area(mc, nc, s, t) / unit;
            if (f < f2) f2 = f;
        }
    res->sc = bs; res->tc = bt;
    res->fbest = f1;
    if (f1 > 0) res->margin = (f2 - f1) / f1;
    else res->margin = (f2 > 0) ? INFINITY : 0.0;
    res->ffinal = f1;
    /* Upsampling, one level at a time: double, then the 3x3 search. */
    int64_t fS = bS, fA = bA;
    for (int l = L - 1; l >= 0; --l) {
        int ps = bs, pt = bt;
        int first = 1;
        for (int u = -1; u <= 1; ++u)
            for (int v = -1; v <= 1; ++v) {
                int s = 2 * ps + u, t = 2 * pt + v;
                int64_t S = oracle_ssd_one(ap + off[l], bp + boff[l], ml[l], nl[l], s, t);
                int64_t Ar = oracle_area(ml[l], nl[l], s, t);
                if (first || better(S, Ar, s, t, fS, fA, bs, bt)) {
                    fS = S; fA = Ar; bs = s; bt = t; first = 0;
                }
            }
    }
    res->s = bs; res->t = bt;
    if (L > 0) res->ffinal = (double)fS / (double)fA;
}

/* Align T frames (uint16, T x m x n) against the template (uint16, m x n).
 * levels: -1 = the paper's rule, else 0 or 1. Outputs (each nullable except
 * shifts): shifts[T][2] final, coarse[T][2], fbest[T], margin[T], ffinal[T].
 * nthreads <= 0 uses the OpenMP default. Returns 0, or -1 on bad arguments. */
int oracle_align(const uint16_t *frames, int64_t T, const uint16_t *tmpl, int m, int n, int w,
                 int levels, int32_t *shifts, int32_t *coarse, double *fbest, double *margin,
                 double *ffinal, int nthreads) {
    if (levels < 0) levels = oracle_levels(m, n);
    if (levels > ORACLE_MAX_LEVELS) return -1;
    int mc = m >> levels, nc = n >> levels;
    if (w < 1 || 2 * w - 1 > mc || 2 * w - 1 > nc) return -1;
    int64_t boff[ORACLE_MAX_LEVELS + 1];
    int bml[ORACLE_MAX_LEVELS + 1], bnl[ORACLE_MAX_LEVELS + 1];
    int32_t *bp = (int32_t *)malloc(sizeof(int32_t) * (size_t)pyramid_size(m, n, levels));
    pyramid(tmpl, m, n, levels, bp, boff, bml, bnl);
#ifdef _OPENMP
    if (nthreads > 0) omp_set_num_threads(nthreads);
#endif
    int failed = 0;
#pragma omp parallel
    {
        int32_t *ap = (int32_t *)malloc(sizeof(int32_t) * (size_t)pyramid_size(m, n, levels));
        int64_t *Sb = (int64_t *)malloc(sizeof(int64_t) * (size_t)(2 * w - 1) * (2 * w - 1));
        if (!ap || !Sb) {
#pragma omp atomic write
            failed = 1;
        } else {
#pragma omp for schedule(dynamic, 1)
            for (int64_t f = 0; f < T; ++f) {
                oracle_result r;
                align_one(frames + f * (int64_t)m * n, bp, boff, m, n, w, levels, ap, Sb, &r);
                shifts[2 * f] = r.s; shifts[2 * f + 1] = r.t;
                if (coarse) { coarse[2 * f] = r.sc; coarse[2 * f + 1] = r.tc; }
                if (fbest) fbest[f] = r.fbest;
                if (margin) margin[f] = r.margin;
                if (ffinal) ffinal[f] = r.ffinal;
            }
        }
        free(ap); free(Sb);
    }
    free(bp);
    return failed ? -2 : 0;
}

/* The upsampling step of Section 2 on its own, at full resolution: for each
 * frame and its given optimum (sc, tc) on the 2x2-box grid, the best of the
 * nine shifts (2 sc + u, 2 tc + v), u, v in {-1, 0, 1}, by exact sums over D
 * and the same tie-break as the search. Every candidate needs a non-empty D
 * (|2 sc| + 1 < m and |2 tc| + 1 < n); a frame whose coarse shift breaks that
 * gets (INT32_MIN, INT32_MIN) and ffinal NaN (the library's contract for
 * caller-given coarse shifts). Returns 0, or -2 when out of memory. */
int oracle_refine(const uint16_t *frames, int64_t T, const uint16_t *tmpl, int m, int n, const int32_t *coarse,
                  int32_t *shifts, double *ffinal, int nthreads) {
    int32_t *b = (int32_t *)malloc(sizeof(int32_t) * (size_t)m * n);
    if (!b) return -2;
    widen(tmpl, (int64_t)m * n, b);
#ifdef _OPENMP
    if (nthreads > 0) omp_set_num_threads(nthreads);
#endif
    int failed = 0;
#pragma omp parallel
    {
        int32_t *a = (int32_t *)malloc(sizeof(int32_t) * (size_t)m * n);
        if (!a) {
#pragma omp atomic write
            failed = 1;
        } else {
#pragma omp for schedule(dynamic, 1)
            for (int64_t f = 0; f < T; ++f) {
                const int64_t sc = coarse[2 * f], tc = coarse[2 * f + 1];
                const int64_t as = sc < 0 ? -sc : sc, at = tc < 0 ? -tc : tc;
                if (2 * as + 1 >= m || 2 * at + 1 >= n) {
                    shifts[2 * f] = INT32_MIN; shifts[2 * f + 1] = INT32_MIN;
                    if (ffinal) ffinal[f] = NAN;
                    continue;
                }
                widen(frames + f * (int64_t)m * n, (int64_t)m * n, a);
                int bs = 0, bt = 0, first = 1;
                int64_t bS = 0, bA = 1;
                for (int u = -1; u <= 1; ++u)
                    for (int v = -1; v <= 1; ++v) {
                        const int s = (int)(2 * sc + u), t = (int)(2 * tc + v);
                        const int64_t S = oracle_ssd_one(a, b, m, n, s, t);
                        const int64_t Ar = oracle_area(m, n, s, t);
                        if (first || better(S, Ar, s, t, bS, bA, bs, bt)) {
                            bS = S; bA = Ar; bs = s; bt = t; first = 0;
                        }
                    }
                shifts[2 * f] = bs; shifts[2 * f + 1] = bt;
                if (ffinal) ffinal[f] = (double)bS / (double)bA;
            }
        }
        free(a);
    }
    free(b);
    return failed ? -2 : 0;
}

/* The searched-grid cost surface of T frames in FP64, box-mean units:
 * cost[f][(s+w-1)*(2w-1) + (t+w-1)] = f_{s,t}. Optional exact sums S (int64). */
int oracle_cost_surface(const uint16_t *frames, int64_t T, const uint16_t *tmpl, int m, int n,
                        int w, int levels, double *cost, int64_t *S_out, int nthreads) {
    if (levels < 0) levels = oracle_levels(m, n);
    if (levels > ORACLE_MAX_LEVELS) return -1;
    int mc = m >> levels, nc = n >> levels;
    if (w < 1 || 2 * w - 1 > mc || 2 * w - 1 > nc) return -1;
    int W = 2 * w - 1;
    double unit = 1.0;
    for (int l = 0; l < levels; ++l) unit *= 16.0;
    int64_t boff[ORACLE_MAX_LEVELS + 1];
    int bml[ORACLE_MAX_LEVELS + 1], bnl[ORACLE_MAX_LEVELS + 1];
    int32_t *bp = (int32_t *)malloc(sizeof(int32_t) * (size_t)pyramid_size(m, n, levels));
    pyramid(tmpl, m, n, levels, bp, boff, bml, bnl);
    const int32_t *bc = bp + boff[levels];
#ifdef _OPENMP
    if (nthreads > 0) omp_set_num_threads(nthreads);
#endif
#pragma omp parallel
    {
        int32_t *ap = (int32_t *)malloc(sizeof(int32_t) * (size_t)pyramid_size(m, n, levels));
        int64_t *S = (int64_t *)malloc(sizeof(int64_t) * (size_t)W * W);
#pragma omp for schedule(dynamic, 1)
        for (int64_t f = 0; f < T; ++f) {
            const uint16_t *a = frames + f * (int64_t)m * n;
            int64_t off[ORACLE_MAX_LEVELS + 1];
            int ml[ORACLE_MAX_LEVELS + 1], nl[ORACLE_MAX_LEVELS + 1];
            pyramid(a, m, n, levels, ap, off, ml, nl);
            const int32_t *ac = ap + off[levels];
            oracle_ssd_all(ac, bc, mc, nc, w, S);
            for (int s = -(w - 1); s <= w - 1; ++s)
                for (int t = -(w - 1); t <= w - 1; ++t) {
                    int k = (s + w - 1) * W + (t + w - 1);
                    if (cost) cost[f * (int64_t)W * W + k] = (double)S[k] / (double)oracle_area(mc, nc, s, t) / unit;
                    if (S_out) S_out[f * (int64_t)W * W + k] = S[k];
                }
        }
        free(ap); free(S);
    }
    free(bp);
    return 0;
}

/* ---- Real-valued form (FP64): cost, soft-min loss and its gradient -------- */

/* f_{s,t} in FP64 for real images a, b (m x n), all (2w-1)^2 shifts. */
void oracle_cost_f64(const double *a, const double *b, int m, int n, int w, double *cost) {
    int W = 2 * w - 1;
    for (int s = -(w - 1); s <= w - 1; ++s)
        for (int t = -(w - 1); t <= w - 1; ++t) {
            double S = 0.0;
            for (int i = 0; i < m; ++i) {
                if (i + s < 0 || i + s >= m) continue;
                for (int j = 0; j < n; ++j) {
                    if (j + t < 0 || j + t >= n) continue;
                    double d = a[(int64_t)(i + s) * n + (j + t)] - b[(int64_t)i * n + j];
                    S += d * d;
                }
            }
            cost[(s + w - 1) * W + (t + w - 1)] = S / (double)oracle_area(m, n, s, t);
        }
}

static int cmp_double(const void *x, const void *y) {
    double a = *(const double *)x, b = *(const double *)y;
    return (a > b) - (a < b);
}

/* Temperature of one frame: scale * the median of its (2w-1)^2 costs (an odd
 * count, so the exact middle element). */
double oracle_median(const double *cost, int count) {
    double *tmp = (double *)malloc(sizeof(double) * (size_t)count);
    memcpy(tmp, cost, sizeof(double) * (size_t)count);
    qsort(tmp, (size_t)count, sizeof(double), cmp_double);
    double med = tmp[count / 2];
    free(tmp);
    return med;
}

/* Soft-min loss over frames: L = sum_f -tau_f log sum_{s,t} exp(-f_{s,t}/tau_f).
 * frames: T x m x n (FP64), tmpl: m x n (FP64), tau[T] given (held constant).
 * If grad_tmpl (m x n) / grad_frames (T x m x n) are non-null they receive
 * dL/db and dL/da (overwritten). Per-frame losses go to loss_f if non-null. */
double oracle_softmin_loss(const double *frames, int64_t T, const double *tmpl, int m, int n,
                           int w, const double *tau, double *loss_f, double *grad_tmpl,
                           double *grad_frames, int nthreads) {
    int W = 2 * w - 1, K = W * W;
    double total = 0.0;
    if (grad_tmpl) memset(grad_tmpl, 0, sizeof(double) * (size_t)m * n);
#ifdef _OPENMP
    if (nthreads > 0) omp_set_num_threads(nthreads);
#endif
#pragma omp parallel
    {
        double *cost = (double *)malloc(sizeof(double) * (size_t)K);
        double *gb = grad_tmpl ? (double *)calloc((size_t)m * n, sizeof(double)) : NULL;
        double local = 0.0;
#pragma omp for schedule(dynamic, 1)
        for (int64_t f = 0; f < T; ++f) {
            const double *a = frames + f * (int64_t)m * n;
            oracle_cost_f64(a, tmpl, m, n, w, cost);
            double tf = tau[f];
            /* Stable log-sum-exp around the minimum cost. With tau = 0 (a
             * median of zero) the soft-min is the min and the weight is shared
             * equally by the minimisers. */
            double fmin = cost[0];
            for (int k = 1; k < K; ++k) if (cost[k] < fmin) fmin = cost[k];
            int nmin = 0;
            for (int k = 0; k < K; ++k) nmin += (cost[k] == fmin);
            double Z = 0.0;
            if (tf > 0)
                for (int k = 0; k < K; ++k) Z += exp(-(cost[k] - fmin) / tf);
            double L = tf > 0 ? fmin - tf * log(Z) : fmin;
            local += L;
            if (loss_f) loss_f[f] = L;
            if (!gb && !grad_frames) continue;
            double *ga = grad_frames ? grad_frames + f * (int64_t)m * n : NULL;
            if (ga) memset(ga, 0, sizeof(double) * (size_t)m * n);
            /* dL/df_{s,t} = softmax weight; df/db and df/da from Section 2's f. */
            for (int s = -(w - 1); s <= w - 1; ++s)
                for (int t = -(w - 1); t <= w - 1; ++t) {
                    int k = (s + w - 1) * W + (t + w - 1);
                    double g = tf > 0 ? exp(-(cost[k] - fmin) / tf) / Z : (cost[k] == fmin ? 1.0 / nmin : 0.0);
                    double q = g / (double)oracle_area(m, n, s, t);
                    for (int i = 0; i < m; ++i) {
                        if (i + s < 0 || i + s >= m) continue;
                        for (int j = 0; j < n; ++j) {
                            if (j + t < 0 || j + t >= n) continue;
                            int64_t ia = (int64_t)(i + s) * n + (j + t), ib = (int64_t)i * n + j;
                            double d = a[ia] - tmpl[ib];
                            if (gb) gb[ib] += -2.0 * q * d;
                            if (ga) ga[ia] += 2.0 * q * d;
                        }
                    }
                }
        }
#pragma omp critical
        {
            total += local;
            if (gb)
                for (int64_t p = 0; p < (int64_t)m * n; ++p) grad_tmpl[p] += gb[p];
        }
        free(cost);
        free(gb);
    }
    return total;
}

/* ---- Correction: apply the found shifts (Section 2, "motion corrected") ---- */

/* corrected[f][i][j] = frames[f][i+s_f][j+t_f] when 0 <= i+s_f < m and
 * 0 <= j+t_f < n, else fill. mean[i][j] = (sum of the in-frame source pixels
 * over f) / (their count), in FP64 from the exact integer sum; fill where the
 * count is 0. Either output may be NULL. */
void oracle_apply_shifts(const uint16_t *frames, int64_t T, int m, int n, const int32_t *shifts,
                         uint16_t fill, uint16_t *corrected, double *mean) {
    uint64_t *sum = mean ? (uint64_t *)calloc((size_t)m * n, sizeof(uint64_t)) : NULL;
    int64_t *cnt = mean ? (int64_t *)calloc((size_t)m * n, sizeof(int64_t)) : NULL;
    for (int64_t f = 0; f < T; ++f) {
        const int s = shifts[2 * f], t = shifts[2 * f + 1];
        const uint16_t *a = frames + f * (int64_t)m * n;
        for (int i = 0; i < m; ++i)
            for (int j = 0; j < n; ++j) {
                const int si = i + s, sj = j + t;
                const int inside = si >= 0 && si < m && sj >= 0 && sj < n;
                const uint16_t v = inside ? a[(int64_t)si * n + sj] : fill;
                if (corrected) corrected[(f * m + i) * (int64_t)n + j] = v;
                if (mean && inside) {
                    sum[(int64_t)i * n + j] += v;
                    cnt[(int64_t)i * n + j] += 1;
                }
            }
    }
    if (mean)
        for (int64_t p = 0; p < (int64_t)m * n; ++p)
            mean[p] = cnt[p] ? (double)sum[p] / (double)cnt[p] : (double)fill;
    free(sum);
    free(cnt);
}
