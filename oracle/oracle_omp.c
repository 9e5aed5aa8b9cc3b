/*
 * oracle_omp.c -- the oracle's LSQR with its loops split over the host cores.
 *
 * TEST INFRASTRUCTURE (see oracle.h): the all-cores CPU baseline of the
 * benchmark, pinned against the single-threaded oracle by the tests. Shares no
 * code with the GPU library.
 *
 * The paper's OpenMP version of the products (Alg. 2/3, Sec. 3.1) splits the
 * observation rows among threads. Here the rows go to threads star by star
 * (contiguous star ranges, static schedule): aprod 1 writes each row once, so
 * it needs nothing else; in aprod 2 a star's astrometric columns belong to the
 * one thread that owns the star, while the attitude, instrumental and global
 * columns, which any row may touch, go to thread-private accumulators summed
 * into x at the end in thread order. The driver is the oracle's own
 * (oracle_lsqr_core) with these steps and the vector loops split over the
 * threads; sums of the norms and of the column accumulators therefore run in
 * another order than in the single-threaded oracle.
 *
 * Without OpenMP at build time every loop runs on one thread and
 * oracle_omp_threads() says so.
 */
#include <math.h>
#include <stdlib.h>

#include "oracle.h"

#ifdef _OPENMP
#include <omp.h>
#endif

#define ORACLE_API __attribute__((visibility("default")))

enum { N_AXES = 3, N_PAR_AXIS = 4 };

static int n_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

static int thread_id(void)
{
#ifdef _OPENMP
    return omp_get_thread_num();
#else
    return 0;
#endif
}

/* aprod 1 (Eq. 2), the rows of each star on one thread */
static void aprod1_omp(const oracle_sys *s, const double *x, double *y)
{
    const int na = s->n_astro, ni = s->n_ipr;
    const int64_t att0 = (int64_t)na * s->n_stars;
    const int64_t instr0 = att0 + (int64_t)N_AXES * s->n_dfa;
    const int64_t glob0 = instr0 + s->n_instr;
#pragma omp parallel for schedule(static)
    for (int64_t star = 0; star < s->n_stars; ++star) {
        const int64_t offset_astro = (int64_t)na * star;
        for (int64_t i = s->star_ptr[star]; i < s->star_ptr[star + 1]; ++i) {
            const double *a = s->A + i * s->npar;
            double sum = 0.0;
            int k = 0;
            for (int j = 0; j < na; ++j, ++k) sum = sum + a[k] * x[offset_astro + j];
            for (int ax = 0; ax < N_AXES; ++ax) {
                const int64_t k2 = att0 + (int64_t)ax * s->n_dfa + s->knot[i];
                for (int j2 = 0; j2 < N_PAR_AXIS; ++j2, ++k) sum = sum + a[k] * x[k2 + j2];
            }
            for (int j = 0; j < ni; ++j, ++k) sum = sum + a[k] * x[instr0 + s->instr[i * ni + j]];
            for (int j = 0; j < s->n_glob; ++j) sum = sum + a[k + j] * x[glob0 + j];
            y[i] = y[i] + sum;
        }
    }
}

/* aprod 2 (Eq. 3): astrometric columns by the star's thread, the shared columns through
 * thread-private accumulators reduced in thread order */
static void aprod2_omp(const oracle_sys *s, const double *y, double *x)
{
    const int na = s->n_astro, ni = s->n_ipr;
    const int64_t att0 = (int64_t)na * s->n_stars;
    const int64_t nrest = (int64_t)N_AXES * s->n_dfa + s->n_instr + s->n_glob;
    const int64_t ins = (int64_t)N_AXES * s->n_dfa, gl = ins + s->n_instr;
    const int T = n_threads();
    double *priv = (double *)calloc((size_t)T * (size_t)(nrest > 0 ? nrest : 1), sizeof(double));
    if (!priv) abort();
#pragma omp parallel
    {
        double *xp = priv + (int64_t)thread_id() * nrest;
#pragma omp for schedule(static)
        for (int64_t star = 0; star < s->n_stars; ++star) {
            const int64_t offset_astro = (int64_t)na * star;
            for (int64_t i = s->star_ptr[star]; i < s->star_ptr[star + 1]; ++i) {
                const double *a = s->A + i * s->npar;
                const double yi = y[i];
                int k = 0;
                for (int j = 0; j < na; ++j, ++k) x[offset_astro + j] = x[offset_astro + j] + a[k] * yi;
                for (int ax = 0; ax < N_AXES; ++ax) {
                    const int64_t k2 = (int64_t)ax * s->n_dfa + s->knot[i];
                    for (int j2 = 0; j2 < N_PAR_AXIS; ++j2, ++k) xp[k2 + j2] = xp[k2 + j2] + a[k] * yi;
                }
                for (int j = 0; j < ni; ++j, ++k) {
                    const int64_t c = ins + s->instr[i * ni + j];
                    xp[c] = xp[c] + a[k] * yi;
                }
                for (int j = 0; j < s->n_glob; ++j) xp[gl + j] = xp[gl + j] + a[k + j] * yi;
            }
        }
    }
#pragma omp parallel for schedule(static)
    for (int64_t c = 0; c < nrest; ++c) {
        double sum = x[att0 + c];
        for (int t = 0; t < T; ++t) sum = sum + priv[(int64_t)t * nrest + c];
        x[att0 + c] = sum;
    }
    free(priv);
}

/* Alg. 1's p_j = 1/|A_:,j| with the threaded aprod 2 on the squared coefficients */
static void precond_omp(const oracle_sys *s, double *p)
{
    const int64_t nc = oracle_ncols(s);
    const int64_t nv = s->n_rows * s->npar;
    oracle_sys sq = *s;
    double *A2 = (double *)malloc(sizeof(double) * (size_t)(nv > 0 ? nv : 1));
    double *ones = (double *)malloc(sizeof(double) * (size_t)(s->n_rows > 0 ? s->n_rows : 1));
    if (!A2 || !ones) abort();
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < nv; ++i) A2[i] = s->A[i] * s->A[i];
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < s->n_rows; ++i) ones[i] = 1.0;
    sq.A = A2;
    for (int64_t j = 0; j < nc; ++j) p[j] = 0.0;
    aprod2_omp(&sq, ones, p);
    for (int64_t j = 0; j < nc; ++j) p[j] = (p[j] > 0.0) ? 1.0 / sqrt(p[j]) : 1.0;
    free(A2);
    free(ones);
}

static void scale_columns_omp(const oracle_sys *s, const double *p, double *A_out)
{
    const int na = s->n_astro, ni = s->n_ipr;
    const int64_t att0 = (int64_t)na * s->n_stars;
    const int64_t instr0 = att0 + (int64_t)N_AXES * s->n_dfa;
    const int64_t glob0 = instr0 + s->n_instr;
#pragma omp parallel for schedule(static)
    for (int64_t star = 0; star < s->n_stars; ++star) {
        for (int64_t i = s->star_ptr[star]; i < s->star_ptr[star + 1]; ++i) {
            const double *a = s->A + i * s->npar;
            double *o = A_out + i * s->npar;
            int k = 0;
            for (int j = 0; j < na; ++j, ++k) o[k] = a[k] * p[(int64_t)na * star + j];
            for (int ax = 0; ax < N_AXES; ++ax) {
                const int64_t k2 = att0 + (int64_t)ax * s->n_dfa + s->knot[i];
                for (int j2 = 0; j2 < N_PAR_AXIS; ++j2, ++k) o[k] = a[k] * p[k2 + j2];
            }
            for (int j = 0; j < ni; ++j, ++k) o[k] = a[k] * p[instr0 + s->instr[i * ni + j]];
            for (int j = 0; j < s->n_glob; ++j, ++k) o[k] = a[k] * p[glob0 + j];
            for (; k < s->npar; ++k) o[k] = 0.0;
        }
    }
}

/* Eq. 4 with the maximum and the scaled sum of squares reduced over the threads */
static double norm2_omp(int64_t n, const double *a)
{
    double m = 0.0;
#pragma omp parallel for schedule(static) reduction(max : m)
    for (int64_t i = 0; i < n; ++i) {
        const double v = fabs(a[i]);
        if (v > m) m = v;
    }
    if (m == 0.0) return 0.0;
    double ssq = 0.0;
#pragma omp parallel for schedule(static) reduction(+ : ssq)
    for (int64_t i = 0; i < n; ++i) {
        const double q = a[i] / m;
        ssq = ssq + q * q;
    }
    return m * sqrt(ssq);
}

static void scale_omp(int64_t n, double a, const double *x, double *y)
{
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < n; ++i) y[i] = a * x[i];
}

static void copy_omp(int64_t n, const double *x, double *y)
{
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < n; ++i) y[i] = x[i];
}

static void div_omp(int64_t n, double *x, double d)
{
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < n; ++i) x[i] = x[i] / d;
}

static double xw_update_omp(int64_t n, double rho, double t1, double t2, const double *v, double *w, double *x,
                            double *var)
{
    double dknorm = 0.0;
#pragma omp parallel for schedule(static) reduction(+ : dknorm)
    for (int64_t j = 0; j < n; ++j) {
        const double dk = w[j] / rho;
        dknorm = dknorm + dk * dk;
        if (var) var[j] = var[j] + dk * dk;
        x[j] = x[j] + t1 * w[j];
        w[j] = v[j] + t2 * w[j];
    }
    return dknorm;
}

static const oracle_ops omp_ops = {aprod1_omp, aprod2_omp, precond_omp, scale_columns_omp, norm2_omp,
                                   scale_omp, copy_omp, div_omp, xw_update_omp};

ORACLE_API int32_t oracle_omp_threads(void) { return n_threads(); }

ORACLE_API int oracle_lsqr_omp(const oracle_sys *s, const double *b, const oracle_lsqr_params *prm, double *x,
                               double *var, oracle_lsqr_info *info, int32_t threads)
{
#ifdef _OPENMP
    if (threads > 0) omp_set_num_threads(threads);
#else
    (void)threads;
#endif
    return oracle_lsqr_core(s, b, prm, x, var, info, &omp_ops);
}

ORACLE_API void oracle_aprod1_omp(const oracle_sys *s, const double *x, double *y) { aprod1_omp(s, x, y); }

ORACLE_API void oracle_aprod2_omp(const oracle_sys *s, const double *y, double *x) { aprod2_omp(s, y, x); }
