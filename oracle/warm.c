/*
 * warm.c -- plain FP64 reference of the learned warm start (test infrastructure).
 *
 * TEST INFRASTRUCTURE (see oracle.h): loaded only by the tests, the smoke
 * check and the benchmark's CPU baseline; shares no code with the GPU library.
 *
 * The warm start is not part of the paper; it follows the benchmark spec:
 * attitude features from the Jacobi estimate, a six-layer 1D convolutional
 * network over the attitude knots, and per-star 5x5 (n_astro x n_astro) least-squares solves for
 * the astrometric block. Activations are stored position-major: a[b][p][c]
 * (sequence b, position p, channel c). A convolution layer with kernel 5 and
 * zero padding 2 computes
 *     out[b][p][co] = bias[co] + sum_{ci, t} W[co][ci][t] * in[b][p + t - 2][ci].
 * The "mirrored" switch rounds to bfloat16 (round to nearest even) at the
 * points where the GPU stores bfloat16: the weights, every layer input, and
 * every output gradient fed to a backward convolution.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#include "oracle.h"

#define ORACLE_API __attribute__((visibility("default")))

/* binary32 -> bfloat16 -> binary32, round to nearest even (finite inputs) */
ORACLE_API double oracle_bf16(double v)
{
    union { float f; uint32_t u; } c;
    c.f = (float)v;
    const uint32_t lsb = (c.u >> 16) & 1u;
    c.u = (c.u + 0x7fffu + lsb) & 0xffff0000u;
    return (double)c.f;
}

static double rnd(double v, int mirrored) { return mirrored ? oracle_bf16(v) : v; }

/* forward of one layer; relu != 0 applies max(0, .) to the output */
ORACLE_API void oracle_conv_fwd(const double *in, int64_t nb, int64_t L, int cin, const double *W, const double *bias,
                                int cout, int relu, int mirrored, double *out)
{
    for (int64_t b = 0; b < nb; ++b)
        for (int64_t p = 0; p < L; ++p)
            for (int co = 0; co < cout; ++co) {
                double s = 0.0;
                for (int t = 0; t < 5; ++t) {
                    const int64_t q = p + t - 2;
                    if (q < 0 || q >= L) continue;
                    for (int ci = 0; ci < cin; ++ci)
                        s = s + rnd(W[((int64_t)co * cin + ci) * 5 + t], mirrored) *
                                    rnd(in[(b * L + q) * cin + ci], mirrored);
                }
                s = s + bias[co];
                if (relu && s < 0.0) s = 0.0;
                out[(b * L + p) * cout + co] = s;
            }
}

/*
 * Backward of one layer given dout = dLoss/d(layer output before ReLU).
 * din (may be NULL) = dLoss/d(input); dW, dbias are accumulated (+=).
 */
ORACLE_API void oracle_conv_bwd(const double *in, const double *dout, int64_t nb, int64_t L, int cin, const double *W,
                                int cout, int mirrored, double *din, double *dW, double *dbias)
{
    if (din) memset(din, 0, sizeof(double) * (size_t)(nb * L * cin));
    for (int64_t b = 0; b < nb; ++b)
        for (int64_t p = 0; p < L; ++p)
            for (int co = 0; co < cout; ++co) {
                const double g = rnd(dout[(b * L + p) * cout + co], mirrored);
                dbias[co] = dbias[co] + dout[(b * L + p) * cout + co];
                for (int t = 0; t < 5; ++t) {
                    const int64_t q = p + t - 2;
                    if (q < 0 || q >= L) continue;
                    for (int ci = 0; ci < cin; ++ci) {
                        const int64_t wi = ((int64_t)co * cin + ci) * 5 + t;
                        dW[wi] = dW[wi] + g * rnd(in[(b * L + q) * cin + ci], mirrored);
                        if (din) din[(b * L + q) * cin + ci] = din[(b * L + q) * cin + ci] + g * rnd(W[wi], mirrored);
                    }
                }
            }
}

/* mean squared error over n values and its gradient 2 (y - t) / n */
ORACLE_API double oracle_mse(const double *y, const double *t, int64_t n, double *grad)
{
    double s = 0.0;
    for (int64_t i = 0; i < n; ++i) {
        const double d = y[i] - t[i];
        s = s + d * d;
        if (grad) grad[i] = 2.0 * d / (double)n;
    }
    return s / (double)n;
}

/*
 * Adam (Kingma & Ba 2015), step number `step` (1-based):
 *   m = b1 m + (1 - b1) g;  v = b2 v + (1 - b2) g^2
 *   w = w - lr * (m / (1 - b1^step)) / (sqrt(v / (1 - b2^step)) + eps)
 */
ORACLE_API void oracle_adam(double *w, double *m, double *v, const double *g, int64_t n, double lr, double b1, double b2,
                            double eps, int step)
{
    const double c1 = 1.0 - pow(b1, step), c2 = 1.0 - pow(b2, step);
    for (int64_t i = 0; i < n; ++i) {
        m[i] = b1 * m[i] + (1.0 - b1) * g[i];
        v[i] = b2 * v[i] + (1.0 - b2) * g[i] * g[i];
        w[i] = w[i] - lr * (m[i] / c1) / (sqrt(v[i] / c2) + eps);
    }
}

/*
 * Per-star astrometric solve: for each star s, with r_i = b_i minus the
 * attitude, instrumental and global parts of row i applied to x,
 *   G_s = sum_i a_i a_i^T + lambda_s I,   h_s = sum_i a_i r_i,   x_s = G_s^-1 h_s
 * over the star's rows (a_i = the n_astro astrometric coefficients, five for
 * the standard row), with lambda_s = 1e-12 * trace(sum a a^T) / n_astro so
 * that stars with fewer observations than unknowns still give a finite start.
 * Solved by Cholesky. Nothing to solve without an astrometric section.
 * x (n_cols): reads the attitude, instrumental and global parts, writes the
 * astrometric part.
 * Returns the number of stars whose G was not positive definite (x_s = 0).
 */
ORACLE_API int64_t oracle_astro_solve(const oracle_sys *s, const double *b, double *x)
{
    const int na = s->n_astro, ni = s->n_ipr;
    const int64_t att0 = (int64_t)na * s->n_stars;
    const int64_t instr0 = att0 + 3 * (int64_t)s->n_dfa, glob0 = instr0 + s->n_instr;
    int64_t bad = 0;
    if (na == 0) return 0;
    for (int64_t star = 0; star < s->n_stars; ++star) {
        double G[5][5] = {{0}}, h[5] = {0};
        for (int64_t i = s->star_ptr[star]; i < s->star_ptr[star + 1]; ++i) {
            const double *a = s->A + i * s->npar;
            double r = b[i];
            for (int ax = 0; ax < 3; ++ax)
                for (int j = 0; j < 4; ++j)
                    r = r - a[na + 4 * ax + j] * x[att0 + (int64_t)ax * s->n_dfa + s->knot[i] + j];
            for (int j = 0; j < ni; ++j) r = r - a[na + 12 + j] * x[instr0 + s->instr[i * ni + j]];
            for (int j = 0; j < s->n_glob; ++j) r = r - a[na + 12 + ni + j] * x[glob0 + j];
            for (int p = 0; p < na; ++p) {
                h[p] = h[p] + a[p] * r;
                for (int q = 0; q < na; ++q) G[p][q] = G[p][q] + a[p] * a[q];
            }
        }
        double tr = 0.0;
        for (int p = 0; p < na; ++p) tr = tr + G[p][p];
        const double lam = 1e-12 * tr / (double)na;
        for (int p = 0; p < na; ++p) G[p][p] = G[p][p] + lam;
        /* Cholesky G = L L^T */
        double Lm[5][5] = {{0}};
        int ok = 1;
        for (int j = 0; j < na && ok; ++j) {
            double d = G[j][j];
            for (int k = 0; k < j; ++k) d = d - Lm[j][k] * Lm[j][k];
            if (!(d > 0.0)) { ok = 0; break; }
            Lm[j][j] = sqrt(d);
            for (int i = j + 1; i < na; ++i) {
                double v = G[i][j];
                for (int k = 0; k < j; ++k) v = v - Lm[i][k] * Lm[j][k];
                Lm[i][j] = v / Lm[j][j];
            }
        }
        double y[5], xs[5];
        if (ok) {
            for (int i = 0; i < na; ++i) {
                double v = h[i];
                for (int k = 0; k < i; ++k) v = v - Lm[i][k] * y[k];
                y[i] = v / Lm[i][i];
            }
            for (int i = na - 1; i >= 0; --i) {
                double v = y[i];
                for (int k = i + 1; k < na; ++k) v = v - Lm[k][i] * xs[k];
                xs[i] = v / Lm[i][i];
            }
        } else {
            for (int i = 0; i < na; ++i) xs[i] = 0.0;
            ++bad;
        }
        for (int i = 0; i < na; ++i) x[(int64_t)na * star + i] = xs[i];
    }
    return bad;
}
