/*
 * oracle.c -- plain FP64 CPU reference of the LSQR hot path (arXiv 2308.00778).
 *
 * TEST INFRASTRUCTURE (see oracle.h): loaded only by the tests, the smoke
 * check and the benchmark's CPU baseline. Shares no code with the GPU path.
 *
 * Column layout of x (Sec. 2): [astro n_astro*n_stars | attitude axis 0, 1, 2
 * (n_dfa each) | instrumental n_instr | global n_glob].
 */
#include "oracle.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>

#define ORACLE_API __attribute__((visibility("default")))

enum { N_AXES = 3, N_PAR_AXIS = 4 };

ORACLE_API int64_t oracle_ncols(const oracle_sys *s)
{
    return (int64_t)s->n_astro * s->n_stars + (int64_t)N_AXES * s->n_dfa + s->n_instr + s->n_glob;
}

/*
 * aprod 1, Eq. 2: y += A x. The row loop of Alg. 2 (OpenMP column): one sum
 * per observation over its astrometric, attitude, instrumental and global
 * sections, then added to y[i]. The astrometric offset of a row is n_astro *
 * (its star); the attitude offset of axis a is a*n_dfa + knot[i]; the
 * instrumental map F(i,j) is the stored column instr[i*n_ipr+j].
 */
static void aprod1_impl(const oracle_sys *s, const double *x, double *y)
{
    const int na = s->n_astro, ni = s->n_ipr;
    const int64_t att0 = (int64_t)na * s->n_stars;
    const int64_t instr0 = att0 + (int64_t)N_AXES * s->n_dfa;
    const int64_t glob0 = instr0 + s->n_instr;
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

/*
 * aprod 2, Eq. 3: x += A^T y. The row loop of Alg. 3 (OpenMP column): each
 * observation adds A_d[i,j] * y[i] into the column that slot j maps to.
 */
static void aprod2_impl(const oracle_sys *s, const double *y, double *x)
{
    const int na = s->n_astro, ni = s->n_ipr;
    const int64_t att0 = (int64_t)na * s->n_stars;
    const int64_t instr0 = att0 + (int64_t)N_AXES * s->n_dfa;
    const int64_t glob0 = instr0 + s->n_instr;
    for (int64_t star = 0; star < s->n_stars; ++star) {
        const int64_t offset_astro = (int64_t)na * star;
        for (int64_t i = s->star_ptr[star]; i < s->star_ptr[star + 1]; ++i) {
            const double *a = s->A + i * s->npar;
            const double yi = y[i];
            int k = 0;
            for (int j = 0; j < na; ++j, ++k) x[offset_astro + j] = x[offset_astro + j] + a[k] * yi;
            for (int ax = 0; ax < N_AXES; ++ax) {
                const int64_t k2 = att0 + (int64_t)ax * s->n_dfa + s->knot[i];
                for (int j2 = 0; j2 < N_PAR_AXIS; ++j2, ++k) x[k2 + j2] = x[k2 + j2] + a[k] * yi;
            }
            for (int j = 0; j < ni; ++j, ++k) {
                const int64_t c = instr0 + s->instr[i * ni + j];
                x[c] = x[c] + a[k] * yi;
            }
            for (int j = 0; j < s->n_glob; ++j) x[glob0 + j] = x[glob0 + j] + a[k + j] * yi;
        }
    }
}

ORACLE_API void oracle_aprod1(const oracle_sys *s, const double *x, double *y)
{
    aprod1_impl(s, x, y);
}

ORACLE_API void oracle_aprod2(const oracle_sys *s, const double *y, double *x)
{
    aprod2_impl(s, y, x);
}

/*
 * Eq. 4: |a| = max|a_i| * sqrt(sum (a_i / max|a_i|)^2), the scaled form the
 * paper uses instead of cblas_dnrm2 so that squaring neither overflows nor
 * underflows.
 */
ORACLE_API double oracle_norm2(int64_t n, const double *a)
{
    double m = 0.0;
    for (int64_t i = 0; i < n; ++i) {
        const double v = fabs(a[i]);
        if (v > m) m = v;
    }
    if (m == 0.0) return 0.0;
    double ssq = 0.0;
    for (int64_t i = 0; i < n; ++i) {
        const double q = a[i] / m;
        ssq = ssq + q * q;
    }
    return m * sqrt(ssq);
}

/*
 * Preconditioning array p of Alg. 1: p_j = 1 / |A_{:,j}|_2, each column
 * normalised by its own norm (Sec. 2). A column with no nonzero gets p_j = 1.
 * The column norms are accumulated with the aprod 2 row loop applied to the
 * squared coefficients.
 */
ORACLE_API void oracle_precond(const oracle_sys *s, double *p)
{
    const int64_t nc = oracle_ncols(s);
    oracle_sys sq = *s;
    const int64_t nv = s->n_rows * s->npar;
    double *A2 = (double *)malloc(sizeof(double) * (size_t)(nv > 0 ? nv : 1));
    double *ones = (double *)malloc(sizeof(double) * (size_t)(s->n_rows > 0 ? s->n_rows : 1));
    for (int64_t i = 0; i < nv; ++i) A2[i] = s->A[i] * s->A[i];
    for (int64_t i = 0; i < s->n_rows; ++i) ones[i] = 1.0;
    sq.A = A2;
    for (int64_t j = 0; j < nc; ++j) p[j] = 0.0;
    aprod2_impl(&sq, ones, p);
    for (int64_t j = 0; j < nc; ++j) p[j] = (p[j] > 0.0) ? 1.0 / sqrt(p[j]) : 1.0;
    free(A2);
    free(ones);
}

/* "Normalization of A by p" (Alg. 1): every coefficient times p of its column */
ORACLE_API void oracle_scale_columns(const oracle_sys *s, const double *p, double *A_out)
{
    const int na = s->n_astro, ni = s->n_ipr;
    const int64_t att0 = (int64_t)na * s->n_stars;
    const int64_t instr0 = att0 + (int64_t)N_AXES * s->n_dfa;
    const int64_t glob0 = instr0 + s->n_instr;
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
            for (; k < s->npar; ++k) o[k] = 0.0; /* the standard row's unused global slot */
        }
    }
}

/* the elementary vector steps of the LSQR driver, one plain loop each */
static void vec_scale(int64_t n, double a, const double *x, double *y)
{
    for (int64_t i = 0; i < n; ++i) y[i] = a * x[i];
}

static void vec_copy(int64_t n, const double *x, double *y)
{
    for (int64_t i = 0; i < n; ++i) y[i] = x[i];
}

static void vec_div(int64_t n, double *x, double d)
{
    for (int64_t i = 0; i < n; ++i) x[i] = x[i] / d;
}

/* dk = w / rho (var += dk^2), x += t1 w, w = v + t2 w; returns sum dk^2 */
static double vec_xw_update(int64_t n, double rho, double t1, double t2, const double *v, double *w, double *x,
                            double *var)
{
    double dknorm = 0.0;
    for (int64_t j = 0; j < n; ++j) {
        const double dk = w[j] / rho;
        dknorm = dknorm + dk * dk;
        if (var) var[j] = var[j] + dk * dk;
        x[j] = x[j] + t1 * w[j];
        w[j] = v[j] + t2 * w[j];
    }
    return dknorm;
}

static const oracle_ops plain_ops = {aprod1_impl, aprod2_impl, oracle_precond, oracle_scale_columns, oracle_norm2,
                                     vec_scale, vec_copy, vec_div, vec_xw_update};

/*
 * LSQR (Paige & Saunders 1982, the algorithm the paper's solver runs, Sec. 1
 * and Alg. 1) for min |A~ y - b|^2 + damp^2 |y|^2 with A~ = A diag(p) when
 * preconditioning is on (p from oracle_precond), and x = diag(p) y at the end
 * ("re-multiplication of the solution by p", Alg. 1). Steps in the published
 * order:
 *   beta_1 u_1 = b,  alpha_1 v_1 = A~^T u_1,  w_1 = v_1,  x_0 = 0,
 *   phibar_1 = beta_1,  rhobar_1 = alpha_1, then per iteration
 *   bidiagonalisation: beta u = A~ v - alpha u;  alpha v = A~^T u - beta v
 *   a plane rotation that eliminates damp, then the rotation that eliminates
 *   beta, the updates of x and w, and the norm, condition and residual
 *   estimates with the stopping tests 1..7.
 * The norms alpha and beta use Eq. 4. var (may be NULL) accumulates the sum of
 * (w_k / rho_k)^2, the diagonal estimate of (A~^T A~ + damp^2 I)^-1, in the
 * scaled variables.
 * Returns 0 on success, -1 on allocation failure.
 */
int oracle_lsqr_core(const oracle_sys *s, const double *b, const oracle_lsqr_params *prm, double *x, double *var,
                     oracle_lsqr_info *info, const oracle_ops *ops)
{
    const int64_t m = s->n_rows, n = oracle_ncols(s);
    double *p = (double *)malloc(sizeof(double) * (size_t)n);
    double *At = (double *)malloc(sizeof(double) * (size_t)(m * s->npar > 0 ? m * s->npar : 1));
    double *u = (double *)malloc(sizeof(double) * (size_t)(m > 0 ? m : 1));
    double *v = (double *)malloc(sizeof(double) * (size_t)n);
    double *w = (double *)malloc(sizeof(double) * (size_t)n);
    double *t = (double *)malloc(sizeof(double) * (size_t)(m > n ? m : n));
    if (!p || !At || !u || !v || !w || !t) {
        free(p); free(At); free(u); free(v); free(w); free(t);
        return -1;
    }

    /* preconditioning (Alg. 1: p, then normalisation of A by p) */
    if (prm->precond) ops->precond(s, p);
    else for (int64_t j = 0; j < n; ++j) p[j] = 1.0;
    ops->scale_columns(s, p, At);
    oracle_sys st = *s;
    st.A = At;

    const double damp = prm->damp, dampsq = damp * damp;
    const double ctol = prm->conlim > 0.0 ? 1.0 / prm->conlim : 0.0;

    for (int64_t j = 0; j < n; ++j) { x[j] = 0.0; if (var) var[j] = 0.0; }

    /* beta_1 u_1 = b */
    ops->copy(m, b, u);
    double beta = ops->norm2(m, u);
    if (beta > 0.0) ops->div(m, u, beta);
    /* alpha_1 v_1 = A~^T u_1 (the start through aprod 2, Alg. 1) */
    for (int64_t j = 0; j < n; ++j) v[j] = 0.0;
    if (beta > 0.0) ops->aprod2(&st, u, v);
    double alpha = ops->norm2(n, v);
    if (alpha > 0.0) ops->div(n, v, alpha);
    for (int64_t j = 0; j < n; ++j) w[j] = v[j];

    double rhobar = alpha, phibar = beta;
    double anorm = 0.0, acond = 0.0, ddnorm = 0.0, res2 = 0.0, xnorm = 0.0, xxnorm = 0.0, z = 0.0;
    double cs2 = -1.0, sn2 = 0.0;
    const double bnorm = beta;
    double rnorm = beta, r1norm = beta, r2norm = beta, arnorm = alpha * beta;
    int32_t istop = 0, itn = 0;

    if (arnorm != 0.0) {
        while (itn < prm->itnlim) {
            itn = itn + 1;
            /* beta u = A~ v - alpha u */
            ops->scale(m, -alpha, u, t);
            ops->aprod1(&st, v, t);
            ops->copy(m, t, u);
            beta = ops->norm2(m, u);
            if (beta > 0.0) {
                ops->div(m, u, beta);
                anorm = sqrt(anorm * anorm + alpha * alpha + beta * beta + dampsq);
                /* alpha v = A~^T u - beta v */
                ops->scale(n, -beta, v, t);
                ops->aprod2(&st, u, t);
                ops->copy(n, t, v);
                alpha = ops->norm2(n, v);
                if (alpha > 0.0) ops->div(n, v, alpha);
            }

            /* rotation eliminating the damping parameter */
            const double rhobar1 = sqrt(rhobar * rhobar + dampsq);
            const double cs1 = rhobar / rhobar1;
            const double sn1 = damp / rhobar1;
            const double psi = sn1 * phibar;
            phibar = cs1 * phibar;

            /* rotation eliminating beta: the next row of the bidiagonal */
            const double rho = sqrt(rhobar1 * rhobar1 + beta * beta);
            const double cs = rhobar1 / rho;
            const double sn = beta / rho;
            const double theta = sn * alpha;
            rhobar = -cs * alpha;
            const double phi = cs * phibar;
            phibar = sn * phibar;
            const double tau = sn * phi;

            /* x and w updates */
            const double t1 = phi / rho;
            const double t2 = -theta / rho;
            ddnorm = ddnorm + ops->xw_update(n, rho, t1, t2, v, w, x, var);

            /* estimate of |x| from the plane rotation on the right */
            const double delta = sn2 * rho;
            const double gambar = -cs2 * rho;
            const double rhs = phi - delta * z;
            const double zbar = rhs / gambar;
            xnorm = sqrt(xxnorm + zbar * zbar);
            const double gamma = sqrt(gambar * gambar + theta * theta);
            cs2 = gambar / gamma;
            sn2 = theta / gamma;
            z = rhs / gamma;
            xxnorm = xxnorm + z * z;

            /* norm, condition and residual estimates */
            acond = anorm * sqrt(ddnorm);
            const double res1 = phibar * phibar;
            res2 = res2 + psi * psi;
            rnorm = sqrt(res1 + res2);
            arnorm = alpha * fabs(tau);
            const double r1sq = rnorm * rnorm - dampsq * xxnorm;
            r1norm = sqrt(fabs(r1sq));
            if (r1sq < 0.0) r1norm = -r1norm;
            r2norm = rnorm;

            /* stopping tests */
            const double test1 = rnorm / bnorm;
            const double test2 = arnorm / (anorm * rnorm);
            const double test3 = 1.0 / acond;
            const double tt1 = test1 / (1.0 + anorm * xnorm / bnorm);
            const double rtol = prm->btol + prm->atol * anorm * xnorm / bnorm;
            if (itn >= prm->itnlim) istop = 7;
            if (1.0 + test3 <= 1.0) istop = 6;
            if (1.0 + test2 <= 1.0) istop = 5;
            if (1.0 + tt1 <= 1.0) istop = 4;
            if (test3 <= ctol) istop = 3;
            if (test2 <= prm->atol) istop = 2;
            if (test1 <= rtol) istop = 1;
            if (istop != 0) break;
        }
    }

    /* back to the unscaled unknowns: x = p * y, var = p^2 * var_y */
    for (int64_t j = 0; j < n; ++j) {
        x[j] = x[j] * p[j];
        if (var) var[j] = var[j] * p[j] * p[j];
    }
    if (info) {
        info->istop = istop;
        info->itn = itn;
        info->anorm = anorm;
        info->acond = acond;
        info->rnorm = rnorm;
        info->r1norm = r1norm;
        info->r2norm = r2norm;
        info->arnorm = arnorm;
        info->xnorm = xnorm;
        info->bnorm = bnorm;
    }
    free(p); free(At); free(u); free(v); free(w); free(t);
    return 0;
}

/* the plain single-threaded LSQR: the core with the plain loops above */
ORACLE_API int oracle_lsqr(const oracle_sys *s, const double *b, const oracle_lsqr_params *prm, double *x, double *var,
                           oracle_lsqr_info *info)
{
    return oracle_lsqr_core(s, b, prm, x, var, info, &plain_ops);
}
