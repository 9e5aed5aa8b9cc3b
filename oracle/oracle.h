/*
 * oracle.h -- plain, slow, obviously correct FP64 CPU reference for the LSQR
 * hot path of the Gaia AVU-GSR solver (arXiv 2308.00778).
 *
 * TEST INFRASTRUCTURE. Only the test suite, the smoke check and the CPU
 * baseline leg of the benchmark may load this library. The GPU library never
 * links, includes or calls it, and it shares no code with the GPU path.
 *
 * Every routine is single-threaded, uses binary64 with round-to-nearest and no
 * FMA contraction (built with -ffp-contract=off), and follows the paper's data
 * layout: the dense-per-row coefficient matrix A_d (Sec. 2) holds npar values
 * per row, row-major (row i, slot j at A[i*npar + j]), section by section:
 * n_astro astrometric, 12 attitude (3 axes x 4 knots), n_ipr instrumental,
 * n_glob global. The paper's standard row is npar = 24: slots [0,5)
 * astrometric, [5,17) attitude, [17,23) instrumental, [23] global (ignored
 * when n_glob = 0). Sec. 2 allows 0 <= n_astro <= 5 and 0 <= n_ipr <= 6
 * coefficients per row; other section choices use the compact row,
 * npar = n_astro + 12 + n_ipr + n_glob.
 */
#ifndef GSR_ORACLE_H
#define GSR_ORACLE_H

#include <stdint.h>

#define ORACLE_NPAR 24 /* the paper's standard row */

typedef struct {
    int64_t n_rows;
    int64_t n_stars;
    const int64_t *star_ptr; /* [n_stars+1], rows of star s are [star_ptr[s], star_ptr[s+1]) */
    int32_t n_dfa;           /* attitude degrees of freedom per axis                       */
    int32_t n_instr;         /* instrumental unknowns                                        */
    int32_t n_glob;          /* global unknowns (and global coefficients per row), 0..5      */
    const double *A;         /* A_d, n_rows x npar, row-major                                */
    const int32_t *knot;     /* first attitude knot of each row (same for the 3 axes)        */
    const int32_t *instr;    /* n_rows x n_ipr instrumental column indices in [0, n_instr)   */
    int32_t n_astro;         /* astrometric unknowns per star = coefficients per row, 0..5   */
    int32_t n_ipr;           /* instrumental coefficients per row, 0..6                      */
    int32_t npar;            /* coefficients per row of A: 24, or n_astro+12+n_ipr+n_glob     */
} oracle_sys;

typedef struct {
    int32_t itnlim;
    double atol, btol, conlim, damp;
    int32_t precond; /* 1: column-norm preconditioning (Alg. 1), 0: none */
} oracle_lsqr_params;

typedef struct {
    int32_t istop, itn;
    double anorm, acond, rnorm, r1norm, r2norm, arnorm, xnorm, bnorm;
} oracle_lsqr_info;

int64_t oracle_ncols(const oracle_sys *s);
void oracle_aprod1(const oracle_sys *s, const double *x, double *y);
void oracle_aprod2(const oracle_sys *s, const double *y, double *x);
double oracle_norm2(int64_t n, const double *a);
void oracle_precond(const oracle_sys *s, double *p);
void oracle_scale_columns(const oracle_sys *s, const double *p, double *A_out);
int oracle_lsqr(const oracle_sys *s, const double *b, const oracle_lsqr_params *prm, double *x, double *var,
                oracle_lsqr_info *info);

/*
 * The steps the LSQR driver delegates: the two products, the preconditioner,
 * the column scaling, the Eq. 4 norm and the elementary vector loops. The
 * plain oracle passes its single-threaded loops; oracle_omp.c passes the same
 * loops with the rows (and vector elements) split over threads.
 */
typedef struct {
    void (*aprod1)(const oracle_sys *s, const double *x, double *y);
    void (*aprod2)(const oracle_sys *s, const double *y, double *x);
    void (*precond)(const oracle_sys *s, double *p);
    void (*scale_columns)(const oracle_sys *s, const double *p, double *A_out);
    double (*norm2)(int64_t n, const double *a);
    void (*scale)(int64_t n, double a, const double *x, double *y);   /* y = a x            */
    void (*copy)(int64_t n, const double *x, double *y);              /* y = x              */
    void (*div)(int64_t n, double *x, double d);                      /* x = x / d          */
    double (*xw_update)(int64_t n, double rho, double t1, double t2, const double *v, double *w, double *x,
                        double *var);  /* dk = w/rho, var += dk^2, x += t1 w, w = v + t2 w; returns sum dk^2 */
} oracle_ops;

/* the LSQR driver of oracle_lsqr with its steps taken from ops */
int oracle_lsqr_core(const oracle_sys *s, const double *b, const oracle_lsqr_params *prm, double *x, double *var,
                     oracle_lsqr_info *info, const oracle_ops *ops);

/* oracle_omp.c: the same LSQR with the steps split over `threads` threads (0: all); the threads the
 * library was built to use (1 when it was built without OpenMP) */
int oracle_lsqr_omp(const oracle_sys *s, const double *b, const oracle_lsqr_params *prm, double *x, double *var,
                    oracle_lsqr_info *info, int32_t threads);
int32_t oracle_omp_threads(void);
void oracle_aprod1_omp(const oracle_sys *s, const double *x, double *y);
void oracle_aprod2_omp(const oracle_sys *s, const double *y, double *x);

#endif
