/*
 * gsrgen_core.h -- seeded synthetic Gaia-shaped inputs, shared by host and device.
 *
 * This is the input generator that BOTH the CPU oracle (tests) and the GPU
 * path (benchmarks) draw their inputs from. It holds none of the solver's
 * arithmetic: it only produces the random values, indices, planted solution
 * and noise of a synthetic system. Assembling b = A*x_true + eps is left to
 * the caller (each side does it with its own aprod1).
 *
 * Row structure follows the paper's model of one observation equation
 * (Sec. 2): 24 coefficients per row, 5 astrometric (the observed star),
 * 3 axes x 4 consecutive attitude B-spline knots, 6 instrumental columns
 * with no fixed pattern, 1 global (PPN gamma). Rows are star-major
 * (the block-diagonal astrometric part, Sec. 2), with the observation times of
 * each star sorted, so the attitude knot of a row is nondecreasing within a
 * star.
 *
 * Section variants (Sec. 2 allows 0..5 astrometric and 0..6 instrumental
 * coefficients per row, and a global section of several unknowns or none):
 * n_astro, n_ipr (instrumental coefficients per row) and n_glob. The paper's
 * standard sections (5, 6, n_glob <= 1) keep the 24-slot row (slot 23 zero
 * without a global); any other choice gives the compact row of
 * n_astro + 12 + n_ipr + n_glob coefficients [astro | attitude | instr | glob].
 * A coefficient present in both draws the same number: compact position j
 * maps to the standard slot it stands for, and globals past the first draw
 * from a tag of their own.
 *
 * Random source: the SplitMix64 output function (Steele, Lea & Flood, "Fast
 * splittable pseudorandom number generators", OOPSLA 2014) applied to a
 * counter, keyed by (seed, tag). Each draw is a pure function of
 * (seed, tag, index, sub), so any row can be regenerated on its own.
 *
 * Gaussians: Box-Muller, z = sqrt(-2 ln u1) cos(2 pi u2), with ln and cos
 * written out here from their series (atanh series for ln, Taylor series for
 * sin/cos after an exact quarter-turn reduction). Every operation is a single
 * IEEE-754 binary64 add, multiply, divide or sqrt with round-to-nearest, and
 * the files that include this header are compiled without contraction
 * (gcc -ffp-contract=off, nvcc -fmad=false), so the host and the device
 * produce bit-identical values.
 */
#ifndef GSRGEN_CORE_H
#define GSRGEN_CORE_H

#include <stdint.h>
#include <math.h>

#if defined(__CUDACC__)
#define GSRGEN_FN static __host__ __device__ __forceinline__
#else
#define GSRGEN_FN static inline
#endif

#define GSRGEN_NPAR 24
#define GSRGEN_NASTRO 5
#define GSRGEN_NATT 12
#define GSRGEN_NINSTR 6
#define GSRGEN_MAX_OBS 4096
#define GSRGEN_MAX_GLOB 5

/* draw tags: one independent stream per kind of quantity */
enum {
    GSRGEN_TAG_OBS = 1,   /* observations per star          idx = star          */
    GSRGEN_TAG_TIME = 2,  /* attitude knot of an observation idx = row           */
    GSRGEN_TAG_INSTR = 3, /* instrumental columns            idx = row*64+try   */
    GSRGEN_TAG_VAL = 4,   /* coefficients                    idx = row*24+slot  */
    GSRGEN_TAG_XTRUE = 5, /* planted solution                idx = column       */
    GSRGEN_TAG_SIN = 6,   /* attitude sinusoid parameters    idx = axis*8+m     */
    GSRGEN_TAG_NOISE = 7, /* observation noise               idx = row          */
    GSRGEN_TAG_GLOB = 8   /* global coefficients 2..         idx = row*8+g-1    */
};

typedef struct {
    uint64_t seed;
    int64_t n_stars;
    int32_t obs_min, obs_max; /* observations per star, uniform in [min, max] */
    int32_t n_dfa;            /* attitude degrees of freedom per axis (>= 4)  */
    int32_t n_instr;          /* instrumental columns (>= 6)                   */
    int32_t n_glob;           /* global columns, 0 or 1                        */
    int32_t att_kind;         /* planted attitude: 0 = N(0,1), 1 = 8 sinusoids */
    double noise_sigma;       /* standard deviation of the observation noise   */
    int32_t n_astro;          /* astrometric coefficients per row, 0..5        */
    int32_t n_ipr;            /* instrumental coefficients per row, 0..6       */
} gsrgen_cfg;

GSRGEN_FN uint64_t gsrgen_mix64(uint64_t z)
{
    z ^= z >> 30;
    z *= 0xbf58476d1ce4e5b9ULL;
    z ^= z >> 27;
    z *= 0x94d049bb133111ebULL;
    z ^= z >> 31;
    return z;
}

GSRGEN_FN uint64_t gsrgen_bits(uint64_t seed, uint32_t tag, uint64_t idx, uint32_t sub)
{
    const uint64_t gamma = 0x9e3779b97f4a7c15ULL;
    uint64_t key = gsrgen_mix64(seed + gamma * ((((uint64_t)tag) << 1) | 1ULL));
    return gsrgen_mix64(key + gamma * (idx * 4ULL + (uint64_t)sub + 1ULL));
}

/* uniform on (0, 1]: 53 random bits, never zero */
GSRGEN_FN double gsrgen_u01(uint64_t bits)
{
    return (double)((bits >> 11) + 1ULL) * 0x1.0p-53;
}

/* uniform integer in [0, m) from the top 32 bits (m < 2^31) */
GSRGEN_FN int32_t gsrgen_below(uint64_t bits, int32_t m)
{
    return (int32_t)(((bits >> 32) * (uint64_t)(uint32_t)m) >> 32);
}

GSRGEN_FN double gsrgen_from_bits(uint64_t b)
{
#if defined(__CUDA_ARCH__)
    return __longlong_as_double((long long)b);
#else
    union { uint64_t u; double d; } c;
    c.u = b;
    return c.d;
#endif
}

GSRGEN_FN uint64_t gsrgen_to_bits(double d)
{
#if defined(__CUDA_ARCH__)
    return (uint64_t)__double_as_longlong(d);
#else
    union { uint64_t u; double d; } c;
    c.d = d;
    return c.u;
#endif
}

/* natural log of a normal positive double: x = m 2^e with m in [1/sqrt2, sqrt2),
 * ln m = 2 atanh(s), s = (m-1)/(m+1), |s| <= 0.1716, series to s^25. */
GSRGEN_FN double gsrgen_ln(double x)
{
    uint64_t b = gsrgen_to_bits(x);
    int32_t e = (int32_t)((b >> 52) & 0x7ffULL) - 1023;
    double m = gsrgen_from_bits((b & 0x000fffffffffffffULL) | 0x3ff0000000000000ULL);
    if (m > 1.4142135623730951) {
        m = m * 0.5;
        e = e + 1;
    }
    double s = (m - 1.0) / (m + 1.0);
    double s2 = s * s;
    double p = 1.0 / 25.0;
    p = p * s2 + 1.0 / 23.0;
    p = p * s2 + 1.0 / 21.0;
    p = p * s2 + 1.0 / 19.0;
    p = p * s2 + 1.0 / 17.0;
    p = p * s2 + 1.0 / 15.0;
    p = p * s2 + 1.0 / 13.0;
    p = p * s2 + 1.0 / 11.0;
    p = p * s2 + 1.0 / 9.0;
    p = p * s2 + 1.0 / 7.0;
    p = p * s2 + 1.0 / 5.0;
    p = p * s2 + 1.0 / 3.0;
    p = p * s2 + 1.0;
    const double ln2 = 0.6931471805599453;
    return (double)e * ln2 + 2.0 * s * p;
}

/* sin and cos of theta in [0, pi/4] by Taylor series (Horner) */
GSRGEN_FN double gsrgen_sin_small(double t)
{
    double t2 = t * t;
    double p = -1.0 / 1307674368000.0;      /* -1/15! */
    p = p * t2 + 1.0 / 6227020800.0;        /*  1/13! */
    p = p * t2 - 1.0 / 39916800.0;          /* -1/11! */
    p = p * t2 + 1.0 / 362880.0;            /*  1/9!  */
    p = p * t2 - 1.0 / 5040.0;              /* -1/7!  */
    p = p * t2 + 1.0 / 120.0;               /*  1/5!  */
    p = p * t2 - 1.0 / 6.0;                 /* -1/3!  */
    return t + t * (t2 * p);
}

GSRGEN_FN double gsrgen_cos_small(double t)
{
    double t2 = t * t;
    double p = 1.0 / 20922789888000.0;      /*  1/16! */
    p = p * t2 - 1.0 / 87178291200.0;       /* -1/14! */
    p = p * t2 + 1.0 / 479001600.0;         /*  1/12! */
    p = p * t2 - 1.0 / 3628800.0;           /* -1/10! */
    p = p * t2 + 1.0 / 40320.0;             /*  1/8!  */
    p = p * t2 - 1.0 / 720.0;               /* -1/6!  */
    p = p * t2 + 1.0 / 24.0;                /*  1/4!  */
    p = p * t2 - 0.5;                       /* -1/2!  */
    return 1.0 + t2 * p;
}

/* cos(2 pi u) for u in [0, 1): exact reduction to a quarter turn */
GSRGEN_FN double gsrgen_cos_turn(double u)
{
    const double half_pi = 1.5707963267948966;
    double t = 4.0 * u;               /* exact */
    int32_t q = (int32_t)t;           /* 0..3 */
    double f = t - (double)q;         /* exact, in [0, 1) */
    double c, s;                      /* cos, sin of f*pi/2 */
    if (f <= 0.5) {
        double th = f * half_pi;
        c = gsrgen_cos_small(th);
        s = gsrgen_sin_small(th);
    } else {
        double th = (1.0 - f) * half_pi;
        c = gsrgen_sin_small(th);
        s = gsrgen_cos_small(th);
    }
    switch (q & 3) {
    case 0: return c;
    case 1: return -s;
    case 2: return -c;
    default: return s;
    }
}

/* standard normal from two 64-bit draws (Box-Muller, cosine branch) */
GSRGEN_FN double gsrgen_normal(uint64_t b1, uint64_t b2)
{
    double u1 = gsrgen_u01(b1);
    double u2 = (double)(b2 >> 11) * 0x1.0p-53; /* [0, 1) */
    double r = (-2.0) * gsrgen_ln(u1);
    if (r < 0.0) r = 0.0; /* ln(1) may round to a tiny negative */
    return sqrt(r) * gsrgen_cos_turn(u2);
}

GSRGEN_FN double gsrgen_normal_at(uint64_t seed, uint32_t tag, uint64_t idx)
{
    return gsrgen_normal(gsrgen_bits(seed, tag, idx, 0), gsrgen_bits(seed, tag, idx, 1));
}

GSRGEN_FN int64_t gsrgen_ncols(const gsrgen_cfg *c)
{
    return (int64_t)c->n_astro * c->n_stars + 3LL * c->n_dfa + c->n_instr + c->n_glob;
}

/* the paper's standard sections: 24-slot rows */
GSRGEN_FN int32_t gsrgen_standard(const gsrgen_cfg *c)
{
    return c->n_astro == GSRGEN_NASTRO && c->n_ipr == GSRGEN_NINSTR && c->n_glob <= 1;
}

/* coefficients per generated row */
GSRGEN_FN int32_t gsrgen_npar(const gsrgen_cfg *c)
{
    return gsrgen_standard(c) ? GSRGEN_NPAR : c->n_astro + GSRGEN_NATT + c->n_ipr + c->n_glob;
}

GSRGEN_FN int32_t gsrgen_obs_of_star(const gsrgen_cfg *c, int64_t star)
{
    int32_t span = c->obs_max - c->obs_min + 1;
    if (span <= 1) return c->obs_min;
    return c->obs_min + gsrgen_below(gsrgen_bits(c->seed, GSRGEN_TAG_OBS, (uint64_t)star, 0), span);
}

/* raw (unsorted) knot draw of a row: floor(t * (n_dfa - 3)), t = u32 / 2^32 */
GSRGEN_FN int32_t gsrgen_knot_raw(const gsrgen_cfg *c, int64_t row)
{
    return gsrgen_below(gsrgen_bits(c->seed, GSRGEN_TAG_TIME, (uint64_t)row, 0), c->n_dfa - 3);
}

/* n_ipr distinct instrumental columns of a row in [0, n_instr), in draw order
 * (a prefix of the same draws for every n_ipr) */
GSRGEN_FN void gsrgen_instr_row(const gsrgen_cfg *c, int64_t row, int32_t out[6])
{
    const int32_t want = c->n_ipr;
    int32_t got = 0;
    for (int32_t a = 0; a < 64 && got < want; ++a) {
        int32_t v = gsrgen_below(gsrgen_bits(c->seed, GSRGEN_TAG_INSTR, (uint64_t)row * 64ULL + (uint64_t)a, 0),
                                 c->n_instr);
        int32_t dup = 0;
        for (int32_t k = 0; k < got; ++k) dup |= (out[k] == v);
        if (!dup) out[got++] = v;
    }
    /* deterministic completion in the (astronomically rare) case of 64 collisions */
    for (int32_t v = 0; got < want; ++v) {
        int32_t dup = 0;
        for (int32_t k = 0; k < got; ++k) dup |= (out[k] == v);
        if (!dup) out[got++] = v;
    }
}

/* coefficient j (0 <= j < gsrgen_npar) of a row */
GSRGEN_FN double gsrgen_value(const gsrgen_cfg *c, int64_t row, int32_t j)
{
    int32_t slot = j; /* the standard slot it stands for */
    if (!gsrgen_standard(c)) {
        const int32_t na = c->n_astro, ni = c->n_ipr;
        if (j < na) slot = j;
        else if (j < na + GSRGEN_NATT) slot = GSRGEN_NASTRO + (j - na);
        else if (j < na + GSRGEN_NATT + ni) slot = GSRGEN_NASTRO + GSRGEN_NATT + (j - na - GSRGEN_NATT);
        else {
            const int32_t g = j - (na + GSRGEN_NATT + ni);
            if (g > 0)
                return gsrgen_normal_at(c->seed, GSRGEN_TAG_GLOB, (uint64_t)row * 8ULL + (uint64_t)(g - 1));
            slot = GSRGEN_NPAR - 1;
        }
    }
    if (slot == GSRGEN_NPAR - 1 && c->n_glob == 0) return 0.0;
    return gsrgen_normal_at(c->seed, GSRGEN_TAG_VAL, (uint64_t)row * GSRGEN_NPAR + (uint64_t)slot);
}

GSRGEN_FN double gsrgen_noise(const gsrgen_cfg *c, int64_t row)
{
    return c->noise_sigma * gsrgen_normal_at(c->seed, GSRGEN_TAG_NOISE, (uint64_t)row);
}

/* planted solution, column layout [astro n_astro*n_stars | att axis0 | axis1 | axis2 | instr | glob] */
GSRGEN_FN double gsrgen_xtrue(const gsrgen_cfg *c, int64_t col)
{
    int64_t att0 = (int64_t)c->n_astro * c->n_stars;
    int64_t att1 = att0 + 3LL * c->n_dfa;
    if (c->att_kind == 1 && col >= att0 && col < att1) {
        int64_t a = col - att0;
        int32_t axis = (int32_t)(a / c->n_dfa);
        int64_t k = a - (int64_t)axis * c->n_dfa;
        double x = 0.0;
        for (int32_t m = 0; m < 8; ++m) {
            uint64_t id = (uint64_t)(axis * 8 + m);
            /* amplitude ~ N(0, 1/8) (variance 1/8) */
            double amp = gsrgen_normal_at(c->seed, GSRGEN_TAG_SIN, id * 4ULL + 0ULL) * 0.35355339059327373;
            /* frequency ~ U(0.5, 10) cycles per 1000 knots */
            double f = 0.5 + 9.5 * gsrgen_u01(gsrgen_bits(c->seed, GSRGEN_TAG_SIN, id * 4ULL + 1ULL, 0));
            /* phase ~ U(0, 1) turns */
            double ph = gsrgen_u01(gsrgen_bits(c->seed, GSRGEN_TAG_SIN, id * 4ULL + 2ULL, 0));
            double turn = f * ((double)k / 1000.0) + ph;
            turn = turn - floor(turn);
            /* sin(2 pi turn) = cos(2 pi (turn - 1/4)) */
            double tt = turn - 0.25;
            if (tt < 0.0) tt = tt + 1.0;
            x = x + amp * gsrgen_cos_turn(tt);
        }
        return x;
    }
    return gsrgen_normal_at(c->seed, GSRGEN_TAG_XTRUE, (uint64_t)col);
}

#endif /* GSRGEN_CORE_H */
