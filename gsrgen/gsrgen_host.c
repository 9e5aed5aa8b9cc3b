/*
 * gsrgen_host.c -- host side of the seeded synthetic-system generator.
 *
 * Fills caller-owned host arrays with the rows, planted solution and noise of
 * a synthetic Gaia-shaped system (see gsrgen_core.h for the model and the
 * random source). Build with -ffp-contract=off so values match the device
 * generator bit for bit. Independent rows are generated in parallel with
 * OpenMP when the library is built with -fopenmp; the output does not depend
 * on the thread count.
 */
#include "gsrgen_core.h"

#include <stddef.h>
#include <stdlib.h>
#include <string.h>

#define GSRGEN_API __attribute__((visibility("default")))

GSRGEN_API int64_t gsrgen_host_ncols(const gsrgen_cfg *c) { return gsrgen_ncols(c); }

/* star_ptr[0..n_stars]: first row of each star, star_ptr[n_stars] = n_rows */
GSRGEN_API int64_t gsrgen_host_star_ptr(const gsrgen_cfg *c, int64_t *star_ptr)
{
    int64_t acc = 0;
    for (int64_t s = 0; s < c->n_stars; ++s) {
        star_ptr[s] = acc;
        acc += gsrgen_obs_of_star(c, s);
    }
    star_ptr[c->n_stars] = acc;
    return acc;
}

static void sort_i32(int32_t *a, int32_t n)
{
    for (int32_t i = 1; i < n; ++i) {
        int32_t v = a[i];
        int32_t j = i - 1;
        while (j >= 0 && a[j] > v) {
            a[j + 1] = a[j];
            --j;
        }
        a[j + 1] = v;
    }
}

/*
 * Rows of stars [s0, s1). Output arrays are indexed from row star_ptr[s0]:
 *   vals64 : AoS, gsrgen_npar coefficients per row as doubles (24 for the
 *            standard sections); with round32 != 0 each
 *            value is first rounded to binary32 (what an FP32-stored system
 *            holds), widened back exactly. May be NULL.
 *   vals32 : AoS, the same coefficients rounded to binary32. May be NULL.
 *   knot   : first attitude knot of the row, nondecreasing within a star
 *   instr  : n_ipr instrumental columns per row
 */
GSRGEN_API void gsrgen_host_rows(const gsrgen_cfg *c, const int64_t *star_ptr, int64_t s0, int64_t s1,
                                 int32_t round32, double *vals64, float *vals32, int32_t *knot, int32_t *instr)
{
    const int64_t base = star_ptr[s0];
    const int32_t np = gsrgen_npar(c), ni = c->n_ipr;
#pragma omp parallel for schedule(dynamic, 64)
    for (int64_t s = s0; s < s1; ++s) {
        const int64_t r0 = star_ptr[s], r1 = star_ptr[s + 1];
        int32_t *kn = knot + (r0 - base);
        for (int64_t r = r0; r < r1; ++r) kn[r - r0] = gsrgen_knot_raw(c, r);
        sort_i32(kn, (int32_t)(r1 - r0));
        for (int64_t r = r0; r < r1; ++r) {
            const int64_t o = r - base;
            int32_t ic[6];
            gsrgen_instr_row(c, r, ic);
            for (int32_t j = 0; j < ni; ++j) instr[o * ni + j] = ic[j];
            for (int32_t j = 0; j < np; ++j) {
                double v = gsrgen_value(c, r, j);
                if (vals64) vals64[o * np + j] = round32 ? (double)(float)v : v;
                if (vals32) vals32[o * np + j] = (float)v;
            }
        }
    }
}

GSRGEN_API void gsrgen_host_xtrue(const gsrgen_cfg *c, int64_t col0, int64_t ncol, double *x)
{
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < ncol; ++i) x[i] = gsrgen_xtrue(c, col0 + i);
}

GSRGEN_API void gsrgen_host_noise(const gsrgen_cfg *c, int64_t row0, int64_t nrow, double *eps)
{
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < nrow; ++i) eps[i] = gsrgen_noise(c, row0 + i);
}

/* single draws, exposed so tests can check the distribution helpers */
GSRGEN_API double gsrgen_host_normal_at(uint64_t seed, uint32_t tag, uint64_t idx)
{
    return gsrgen_normal_at(seed, tag, idx);
}
GSRGEN_API double gsrgen_host_ln(double x) { return gsrgen_ln(x); }
GSRGEN_API double gsrgen_host_cos_turn(double u) { return gsrgen_cos_turn(u); }
GSRGEN_API uint64_t gsrgen_host_bits(uint64_t seed, uint32_t tag, uint64_t idx, uint32_t sub)
{
    return gsrgen_bits(seed, tag, idx, sub);
}
