/*
 * FP64 CPU oracle for the SPIIR hot path.  TEST INFRASTRUCTURE ONLY.
 *
 * Only tests/, __graft_entry__.smoke() and the CPU-baseline leg of bench.py
 * may load this file's library.  It shares no code, header, table or helper
 * with the CUDA path; it is the plain definition of what that path computes,
 * written as nested loops in double precision so that a reader can check it
 * against the paper by eye.
 *
 * The method (paper, section "GPU accelerated SPIIR method", subsection
 * "SPIIR method"): the matched-filter SNR of one chirp template is
 * approximated by a parallel bank of single-pole IIR filters whose outputs
 * are summed.  Written out, for filter l of a template, detector stream x:
 *
 *     y_l[k] = a_l * y_l[k-1] + b_l * x[k - d_l]        (complex a_l, b_l)
 *     z[k]   = sum over the template's filters of y_l[k]
 *
 * with y_l[-1] = 0 and x[k] = 0 for k < 0.  The summation over a template's
 * filters is the step the paper's GPU design performs with warp shuffles and
 * atomics (subsection "Optimized GPU implementation of SPIIR").  The peak
 * (largest |z|, first index on ties) is the quantity the paper uses to
 * identify a signal in the SNR series.
 *
 * Inputs arrive in double.  The Python wrapper promotes the canonical
 * complex64/float32 values exactly, so the oracle sees exactly the numbers
 * the GPU sees; finite-difference tests may pass other doubles.
 *
 * Compile with -O2 -ffp-contract=off (no fused multiply-add, no fast-math),
 * so every product and sum is one IEEE double operation in source order.
 *
 * `mutation` plants one deliberate mistake (0 = none).  It exists only so the
 * tests can show that the pins catch plausible slips; see spiir_ref_filter.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

/* Planted mistakes, for the mutation tests only. */
enum {
    MUT_NONE = 0,
    MUT_CONJ_POLE = 1,     /* uses conj(a) in the recurrence            */
    MUT_DELAY_OFF1 = 2,    /* reads x[k - d - 1]                         */
    MUT_DROP_GAIN_IM = 3,  /* drops the imaginary part of b              */
    MUT_SKIP_LAST = 4,     /* sums all but the template's last filter     */
    MUT_PEAK_LAST_TIE = 5, /* peak keeps the last index on ties           */
    MUT_SWAP_REIM_OUT = 6  /* writes (im, re) instead of (re, im)         */
};

int spiir_ref_max_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

/*
 * One template on one detector stream: z[k] for k in [0, n).
 * zt is [n][2] (re, im), zeroed here.
 */
static void template_response(int64_t l0, int64_t l1, const double *a,
                              const double *b, const int32_t *d,
                              const double *x, int64_t n, double *zt,
                              int mutation)
{
    memset(zt, 0, sizeof(double) * 2 * (size_t)n);
    if (mutation == MUT_SKIP_LAST && l1 > l0) l1 -= 1;
    for (int64_t l = l0; l < l1; ++l) {
        double ar = a[2 * l], ai = a[2 * l + 1];
        double br = b[2 * l], bi = b[2 * l + 1];
        int64_t dl = d[l];
        if (mutation == MUT_CONJ_POLE) ai = -ai;
        if (mutation == MUT_DELAY_OFF1) dl += 1;
        if (mutation == MUT_DROP_GAIN_IM) bi = 0.0;
        double yr = 0.0, yi = 0.0; /* y_l[-1] = 0 */
        for (int64_t k = 0; k < n; ++k) {
            double xk = (k - dl >= 0) ? x[k - dl] : 0.0;
            /* y <- a*y + b*x, complex product written out */
            double nr = ar * yr - ai * yi + br * xk;
            double ni = ar * yi + ai * yr + bi * xk;
            yr = nr;
            yi = ni;
            zt[2 * k] += yr;
            zt[2 * k + 1] += yi;
        }
    }
}

/* Largest |z|^2 and its first index (ties keep the earlier sample). */
static void peak_of(const double *zt, int64_t n, double *best, int64_t *at,
                    int mutation)
{
    double bv = -1.0;
    int64_t bk = -1;
    for (int64_t k = 0; k < n; ++k) {
        double p = zt[2 * k] * zt[2 * k] + zt[2 * k + 1] * zt[2 * k + 1];
        if (p > bv || (mutation == MUT_PEAK_LAST_TIE && p == bv)) {
            bv = p;
            bk = k;
        }
    }
    *best = bv;
    *at = bk;
}

/*
 * Filter every (detector, template) pair.
 *   off[n_templates+1]      CSR offsets of each template's filters
 *   a, b [Ltot][2]          complex pole and gain (re, im)
 *   d [Ltot]                delay in samples
 *   x [n_det][n]            detector streams
 *   z [n_det][n_templates][n][2]   output, or NULL
 *   peak_abs2, peak_idx [n_det][n_templates]   largest |z|^2, first index,
 *                                  or NULL
 * Returns 0, or -1 on allocation failure.
 */
int spiir_ref_filter(int64_t n_templates, int64_t n_det, const int64_t *off,
                     const double *a, const double *b, const int32_t *d,
                     const double *x, int64_t n, double *z, double *peak_abs2,
                     int64_t *peak_idx, int n_threads, int mutation)
{
    int64_t jobs = n_templates * n_det;
    int failed = 0;
    if (n_threads < 1) n_threads = 1;
#pragma omp parallel num_threads(n_threads)
    {
        double *zt = (double *)malloc(sizeof(double) * 2 * (size_t)(n > 0 ? n : 1));
        if (!zt) {
#pragma omp atomic write
            failed = 1;
        }
#pragma omp for schedule(dynamic, 1)
        for (int64_t job = 0; job < jobs; ++job) {
            if (!zt) continue;
            int64_t det = job / n_templates, t = job % n_templates;
            template_response(off[t], off[t + 1], a, b, d, x + det * n, n, zt,
                              mutation);
            if (z) {
                double *dst = z + (det * n_templates + t) * 2 * n;
                if (mutation == MUT_SWAP_REIM_OUT) {
                    for (int64_t k = 0; k < n; ++k) {
                        dst[2 * k] = zt[2 * k + 1];
                        dst[2 * k + 1] = zt[2 * k];
                    }
                } else {
                    memcpy(dst, zt, sizeof(double) * 2 * (size_t)n);
                }
            }
            if (peak_abs2 && peak_idx)
                peak_of(zt, n, peak_abs2 + job, peak_idx + job, mutation);
        }
        free(zt);
    }
    return failed ? -1 : 0;
}

/*
 * Multirate bank.  Filter l runs at the rate of its band:
 *   x_band[k] = x[R * k]   (plain subsampling, R = decim[band_of[l]]),
 * its delay is in band samples.  Each band's summed output z_band is brought
 * to the top rate by linear interpolation,
 *   z_up[m] = (1 - f) z_band[i] + f z_band[min(i + 1, n_band - 1)],
 *   i = floor(m / R), f = (m mod R) / R,
 * and the bands are added.  n_band = ceil(n / R).
 * Arguments as spiir_ref_filter plus band_of[Ltot], decim[n_bands].
 */
int spiir_ref_filter_multirate(int64_t n_templates, int64_t n_det,
                               const int64_t *off, const double *a,
                               const double *b, const int32_t *d,
                               const int32_t *band_of, int32_t n_bands,
                               const int32_t *decim, const double *x, int64_t n,
                               double *z, double *peak_abs2, int64_t *peak_idx,
                               int n_threads)
{
    int64_t jobs = n_templates * n_det;
    int failed = 0;
    if (n_threads < 1) n_threads = 1;
#pragma omp parallel num_threads(n_threads)
    {
        double *zsum = (double *)malloc(sizeof(double) * 2 * (size_t)(n > 0 ? n : 1));
        double *zb = (double *)malloc(sizeof(double) * 2 * (size_t)(n > 0 ? n : 1));
        double *xb = (double *)malloc(sizeof(double) * (size_t)(n > 0 ? n : 1));
        int32_t *sel = NULL;
        if (!zsum || !zb || !xb) {
#pragma omp atomic write
            failed = 1;
        }
#pragma omp for schedule(dynamic, 1)
        for (int64_t job = 0; job < jobs; ++job) {
            if (!zsum || !zb || !xb) continue;
            int64_t det = job / n_templates, t = job % n_templates;
            const double *xd = x + det * n;
            memset(zsum, 0, sizeof(double) * 2 * (size_t)n);
            for (int32_t band = 0; band < n_bands; ++band) {
                int64_t R = decim[band];
                int64_t nb = (n + R - 1) / R;
                for (int64_t k = 0; k < nb; ++k) xb[k] = xd[R * k];
                /* the band's filters: the template's filters with band_of == band */
                memset(zb, 0, sizeof(double) * 2 * (size_t)nb);
                for (int64_t l = off[t]; l < off[t + 1]; ++l) {
                    if (band_of[l] != band) continue;
                    double ar = a[2 * l], ai = a[2 * l + 1];
                    double br = b[2 * l], bi = b[2 * l + 1];
                    int64_t dl = d[l];
                    double yr = 0.0, yi = 0.0;
                    for (int64_t k = 0; k < nb; ++k) {
                        double xk = (k - dl >= 0) ? xb[k - dl] : 0.0;
                        double nr = ar * yr - ai * yi + br * xk;
                        double ni = ar * yi + ai * yr + bi * xk;
                        yr = nr;
                        yi = ni;
                        zb[2 * k] += yr;
                        zb[2 * k + 1] += yi;
                    }
                }
                for (int64_t m = 0; m < n; ++m) {
                    int64_t i = m / R;
                    int64_t i1 = (i + 1 < nb) ? i + 1 : nb - 1;
                    double f = (double)(m % R) / (double)R;
                    zsum[2 * m] += (1.0 - f) * zb[2 * i] + f * zb[2 * i1];
                    zsum[2 * m + 1] += (1.0 - f) * zb[2 * i + 1] + f * zb[2 * i1 + 1];
                }
            }
            if (z) memcpy(z + (det * n_templates + t) * 2 * n, zsum,
                          sizeof(double) * 2 * (size_t)n);
            if (peak_abs2 && peak_idx)
                peak_of(zsum, n, peak_abs2 + job, peak_idx + job, MUT_NONE);
        }
        free(zsum);
        free(zb);
        free(xb);
        (void)sel;
    }
    return failed ? -1 : 0;
}

/*
 * Adjoint (vector-Jacobian product) of the single-rate bank.
 *
 * Given the gradient of a real loss with respect to z in the PyTorch
 * convention, g_z[k] = dL/dRe z[k] + i dL/dIm z[k], the adjoint state of
 * filter l runs backwards in time,
 *   mu_l[k] = g_z[k] + conj(a_l) * mu_l[k+1],   mu_l[n] = 0,
 * and the gradients, in the same convention, are
 *   g_a_l  = sum_k mu_l[k] * conj(y_l[k-1])           (y_l[-1] = 0)
 *   g_b_l  = sum_k mu_l[k] * x[k - d_l]
 *   g_x[m] = sum_l Re( conj(mu_l[m + d_l]) * b_l )    (m + d_l < n)
 * g_a and g_b are summed over detectors (the bank is shared).
 *   gz [n_det][n_templates][n][2]
 *   ga, gb [Ltot][2]       overwritten
 *   gx [n_det][n] or NULL  overwritten
 * The forward y_l is stored in full (fine for the sizes the tests use).
 */
int spiir_ref_adjoint(int64_t n_templates, int64_t n_det, const int64_t *off,
                      const double *a, const double *b, const int32_t *d,
                      const double *x, int64_t n, const double *gz, double *ga,
                      double *gb, double *gx, int n_threads)
{
    int64_t ltot = off[n_templates];
    int failed = 0;
    if (n_threads < 1) n_threads = 1;
    memset(ga, 0, sizeof(double) * 2 * (size_t)ltot);
    memset(gb, 0, sizeof(double) * 2 * (size_t)ltot);
    double *gx_part = NULL;
    if (gx) {
        gx_part = (double *)calloc((size_t)n_threads * (size_t)(n_det * n) + 1,
                                   sizeof(double));
        if (!gx_part) return -1;
    }
#pragma omp parallel num_threads(n_threads)
    {
        int tid = 0;
#ifdef _OPENMP
        tid = omp_get_thread_num();
#endif
        double *y = (double *)malloc(sizeof(double) * 2 * (size_t)(n > 0 ? n : 1));
        if (!y) {
#pragma omp atomic write
            failed = 1;
        }
        /* template of each filter, by scanning the offsets */
#pragma omp for schedule(dynamic, 16)
        for (int64_t l = 0; l < ltot; ++l) {
            if (!y) continue;
            int64_t lo = 0, hi = n_templates; /* find t with off[t] <= l < off[t+1] */
            while (hi - lo > 1) {
                int64_t mid = (lo + hi) / 2;
                if (off[mid] <= l) lo = mid; else hi = mid;
            }
            int64_t t = lo;
            double ar = a[2 * l], ai = a[2 * l + 1];
            double br = b[2 * l], bi = b[2 * l + 1];
            int64_t dl = d[l];
            double sar = 0, sai = 0, sbr = 0, sbi = 0;
            for (int64_t det = 0; det < n_det; ++det) {
                const double *xd = x + det * n;
                const double *g = gz + (det * n_templates + t) * 2 * n;
                double yr = 0.0, yi = 0.0;
                for (int64_t k = 0; k < n; ++k) {
                    double xk = (k - dl >= 0) ? xd[k - dl] : 0.0;
                    double nr = ar * yr - ai * yi + br * xk;
                    double ni = ar * yi + ai * yr + bi * xk;
                    yr = nr;
                    yi = ni;
                    y[2 * k] = yr;
                    y[2 * k + 1] = yi;
                }
                double mr = 0.0, mi = 0.0; /* mu[n] = 0 */
                for (int64_t k = n - 1; k >= 0; --k) {
                    /* mu <- g[k] + conj(a) * mu */
                    double nr = g[2 * k] + (ar * mr + ai * mi);
                    double ni = g[2 * k + 1] + (ar * mi - ai * mr);
                    mr = nr;
                    mi = ni;
                    double ypr = (k >= 1) ? y[2 * (k - 1)] : 0.0;
                    double ypi = (k >= 1) ? y[2 * (k - 1) + 1] : 0.0;
                    /* mu * conj(y[k-1]) */
                    sar += mr * ypr + mi * ypi;
                    sai += mi * ypr - mr * ypi;
                    double xk = (k - dl >= 0) ? xd[k - dl] : 0.0;
                    sbr += mr * xk;
                    sbi += mi * xk;
                    if (gx_part && k - dl >= 0)
                        gx_part[(size_t)tid * (size_t)(n_det * n) + det * n + (k - dl)] +=
                            mr * br + mi * bi;
                }
            }
            ga[2 * l] = sar;
            ga[2 * l + 1] = sai;
            gb[2 * l] = sbr;
            gb[2 * l + 1] = sbi;
        }
        free(y);
    }
    if (gx) {
        for (int64_t i = 0; i < n_det * n; ++i) {
            double s = 0.0;
            for (int th = 0; th < n_threads; ++th)
                s += gx_part[(size_t)th * (size_t)(n_det * n) + i];
            gx[i] = s;
        }
        free(gx_part);
    }
    return failed ? -1 : 0;
}
