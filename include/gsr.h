/*
 * gsr.h -- C ABI of libgsr: the LSQR hot path of the Gaia AVU-GSR solver
 * (Cesare et al., arXiv 2308.00778) on one NVIDIA GB300 (sm_103a).
 *
 * The problem (Sec. 1, Eq. 1): an overdetermined sparse system A x = b solved
 * in the least-squares sense by LSQR. Each row (observation) of A has 24
 * nonzeros (Sec. 2): 5 astrometric coefficients of the observed star, 3 axes x
 * 4 consecutive attitude B-spline coefficients (axis stride n_dfa), 6
 * instrumental coefficients at arbitrary instrumental columns and 1 global
 * (PPN gamma) coefficient. Rows are grouped by star (the block-diagonal
 * astrometric part). The unknowns are laid out as
 *     [astro 5*n_stars | attitude axis0 | axis1 | axis2 (n_dfa each) | instr n_instr | glob n_glob].
 *
 * Conventions for every entry point:
 *   - Every call returns a gsr_status and never aborts; on failure
 *     gsr_last_error(ctx) holds a one-line message. Nothing is written on
 *     GSR_EINVAL.
 *   - The context owns all device memory it allocates; caller pointers are
 *     borrowed for the duration of the call only.
 *   - "where" arguments say whether a caller pointer is host (GSR_HOST) or
 *     device (GSR_DEVICE) memory; device pointers must be on the context's
 *     device.
 *   - stream is a cudaStream_t passed as void* (NULL = legacy default
 *     stream). Calls that take a stream are asynchronous with respect to the
 *     host unless stated otherwise.
 *   - A context is not thread-safe; use one context per host thread. Its
 *     calls must not overlap on the GPU either (they share the context's
 *     scratch: the workspace, the attitude window accumulators and window
 *     copies); calls on one stream are ordered.
 */
#ifndef GSR_H
#define GSR_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct gsr_ctx gsr_ctx;

typedef enum {
    GSR_OK = 0,
    GSR_EINVAL = 1,   /* bad argument: sizes, indices, ordering, null pointers   */
    GSR_ENOMEM = 2,   /* a device or pinned-host allocation failed               */
    GSR_ECUDA = 3,    /* a CUDA runtime call failed                              */
    GSR_ESTATE = 4,   /* call out of order (e.g. solve before the system is set) */
    GSR_ENUMERIC = 5, /* NaN/Inf in the inputs or in the LSQR scalars            */
    GSR_ETIMEOUT = 6  /* the solve exceeded gsr_solve_params.timeout_s           */
} gsr_status;

enum { GSR_FP64 = 0, GSR_FP32 = 1 };   /* storage precision of the coefficients  */
enum { GSR_HOST = 0, GSR_DEVICE = 1 }; /* where a caller pointer lives            */
enum { GSR_AOS = 0, GSR_SOA = 1 };     /* layout of caller coefficient arrays     */
enum { GSR_PLAIN = 0, GSR_MIXED = 1 }; /* solver mode                             */
enum { GSR_WARM_NONE = 0, GSR_WARM_JACOBI = 1, GSR_WARM_LEARNED = 2 };
#define GSR_MAX_GLOB 5 /* global unknowns of a section variant (gsr_create_sections) */

/*
 * gsr_create -- size a context for one system and allocate its device memory.
 *   n_stars       number of stars (>= 1); astrometric unknowns are 5*n_stars (Sec. 2).
 *   obs_per_star  observations per star when every star has the same count (>= 1),
 *                 or 0 when star_ptr gives the grouping.
 *   star_ptr      host array [n_stars+1] of first rows, star_ptr[0] = 0,
 *                 nondecreasing; NULL when obs_per_star > 0. Copied.
 *   n_dfa         attitude degrees of freedom per axis (>= 4): N_DFA of Sec. 2.
 *   n_instr       instrumental unknowns (>= 6).
 *   n_glob        global unknowns: 0 or 1 (PPN gamma).
 *   value_precision GSR_FP64 or GSR_FP32: how the coefficients are stored.
 *                 FP32 storage is required for GSR_MIXED solves.
 *   device        CUDA device ordinal.
 * Errors: GSR_EINVAL (sizes, star_ptr), GSR_ENOMEM, GSR_ECUDA. On failure
 * *out is NULL.
 */
gsr_status gsr_create(gsr_ctx **out, int64_t n_stars, int32_t obs_per_star, const int64_t *star_ptr, int32_t n_dfa,
                      int32_t n_instr, int32_t n_glob, int32_t value_precision, int32_t device);

/*
 * gsr_create_sections -- gsr_create for any choice of the sections of a row.
 * Sec. 2 allows 0 to 5 astrometric and 0 to 6 instrumental coefficients per
 * row beside the 12 attitude ones, and a global section or none; Sec. 4.2
 * runs systems with one and with five global unknowns.
 *   n_astro   astrometric unknowns per star = coefficients per row, 0..5.
 *   n_instr   instrumental unknowns (>= n_ipr; may be 0 when n_ipr = 0).
 *   n_ipr     instrumental coefficients per row, 0..6 (distinct columns per row
 *             are not required).
 *   n_glob    global unknowns = global coefficients per row, 0..GSR_MAX_GLOB.
 *   Other arguments as gsr_create.
 * Unknowns: [astro n_astro*n_stars | attitude 3*n_dfa | instr n_instr | glob n_glob].
 * Rows passed to gsr_set_rows / gsr_set_system then hold
 * n_astro + 12 + n_ipr + n_glob coefficients in that order (the compact row;
 * 23 or 24 for the standard sections 5, 6 and 0 or 1 global) and n_ipr
 * instrumental columns. The context stores only the planes present: a
 * variant streams (n_astro + 12 + n_ipr + n_glob) values per row, the
 * standard sections run the same kernels as gsr_create. Errors as gsr_create.
 */
gsr_status gsr_create_sections(gsr_ctx **out, int64_t n_stars, int32_t obs_per_star, const int64_t *star_ptr,
                               int32_t n_astro, int32_t n_dfa, int32_t n_instr, int32_t n_ipr, int32_t n_glob,
                               int32_t value_precision, int32_t device);

/*
 * gsr_sections -- the context's sections: astrometric, instrumental and global
 * coefficients per row, and coefficients per row of the caller's arrays
 * (any pointer may be NULL).
 */
gsr_status gsr_sections(const gsr_ctx *ctx, int32_t *n_astro, int32_t *n_ipr, int32_t *n_glob, int32_t *row_width);

/* gsr_destroy -- free everything the context owns. NULL is accepted. */
gsr_status gsr_destroy(gsr_ctx *ctx);

/* gsr_last_error -- message of the last failed call on ctx ("" if none; a
 * static message when ctx is NULL). Valid until the next call on ctx. */
const char *gsr_last_error(const gsr_ctx *ctx);

/* gsr_dims -- rows and unknowns of the system (either pointer may be NULL). */
gsr_status gsr_dims(const gsr_ctx *ctx, int64_t *n_rows, int64_t *n_cols);

/*
 * gsr_set_rows -- load rows [row0, row0+nrows) of the coefficient matrix in the
 * paper's storage (Sec. 2: A_d with 24 values per row, the attitude index map
 * M_i and the instrumental map I_c) and convert them to the context's layout.
 *   values      coefficients, binary64 (values_fp32 = 0) or binary32 (= 1).
 *               GSR_AOS: row-major nrows x 24 (A_d: element (i, j) at i*24 + j).
 *               GSR_SOA: 24 planes, plane j at values + j*plane_stride elements.
 *               Slots [0,5) astro, [5,17) attitude axis-major (4 knots each),
 *               [17,23) instrumental, 23 global (ignored when n_glob = 0).
 *               A gsr_create_sections context takes W = n_astro + 12 + n_ipr +
 *               n_glob coefficients per row (rows of W, or W planes), in the
 *               order astro, attitude, instrumental, global.
 *   att_knot    nrows first attitude knots, each in [0, n_dfa-4]; slot
 *               5+4a+k of a row multiplies unknown 5*n_stars + a*n_dfa + knot + k
 *               (n_astro+4a+k and n_astro*n_stars + a*n_dfa + knot + k for a
 *               gsr_create_sections context).
 *   instr_col   instrumental columns in [0, n_instr): GSR_AOS nrows x 6 row-major,
 *               GSR_SOA 6 planes at instr_col + j*plane_stride (n_ipr per row for
 *               a gsr_create_sections context; may be NULL when n_ipr = 0).
 *   where       GSR_HOST or GSR_DEVICE (all three arrays).
 * FP64 values into an FP32 context are rounded to nearest; FP32 values into an
 * FP64 context are widened exactly. GSR_EINVAL on an out-of-range index,
 * GSR_ENUMERIC on a NaN or Inf coefficient. Device arrays, and host arrays in
 * pageable memory, are validated before anything is committed (the rows are
 * left unchanged on an error). GSR_AOS host arrays in pinned (page-locked,
 * mapped) memory, values 16-byte and instr_col 8-byte aligned, are converted
 * straight from host memory in one pass that also validates them: on an error
 * the rows of the call are then not loaded (their previous content is lost and
 * the calls that need every row return GSR_ESTATE until they are set again).
 * Synchronous: returns after the rows are in place.
 */
gsr_status gsr_set_rows(gsr_ctx *ctx, int64_t row0, int64_t nrows, const void *values, int32_t values_fp32,
                        int32_t layout, int64_t plane_stride, const int32_t *att_knot, const int32_t *instr_col,
                        int32_t where, void *stream);

/*
 * gsr_set_rhs -- load the known terms b (n_rows binary64; Eq. 1). Copied, then
 * checked on the device: GSR_ENUMERIC if b holds a NaN or Inf, and b is then
 * not loaded (a solve returns GSR_ESTATE until b is set again). Synchronous.
 */
gsr_status gsr_set_rhs(gsr_ctx *ctx, const double *b, int32_t where, void *stream);

/*
 * gsr_set_system -- gsr_set_rows over all rows (AoS, like the paper's A_d),
 * then gsr_set_rhs(b) when b is not NULL.
 */
gsr_status gsr_set_system(gsr_ctx *ctx, const void *values, int32_t values_fp32, const int32_t *att_knot,
                          const int32_t *instr_col, const double *b, int32_t where, void *stream);

/*
 * gsr_aprod1 -- y += A x (aprod 1, Eq. 2; Alg. 2).
 *   x  device array of n_cols binary64 (read only).
 *   y  device array of n_rows binary64, updated in place.
 * Runs on stream; does not synchronise. Arithmetic is binary64 whatever the
 * storage precision. Errors: GSR_EINVAL (null vector), GSR_ESTATE (before
 * every row has been set), GSR_ECUDA.
 */
gsr_status gsr_aprod1(gsr_ctx *ctx, const double *x, double *y, void *stream);

/*
 * gsr_aprod2 -- x += A^T y (aprod 2, Eq. 3; Alg. 3).
 *   y  device array of n_rows binary64 (read only).
 *   x  device array of n_cols binary64, updated in place.
 * Runs on stream. Partial sums (per star segment, per attitude knot run,
 * per block for the instrumental and global unknowns) are added with atomic
 * adds, so the low bits of the results can differ from run to run (the sums
 * are reordered). With binary64 storage and the standard row, the
 * instrumental products are summed per block as 64-bit fixed point: each is
 * rounded once, exactly from the product of the two significands, to a grid
 * of about 2^-53 of (its column's max |coefficient| x the most terms one
 * block adds to that column x y_t), where y_t is a power of two above all
 * but about 1/1024 of the |y_i| (rows at or above it add theirs in binary64);
 * the block sums are exact, whatever their order. The first call after the
 * rows change builds the knot-ordered attitude copy (52 B a row for binary32
 * storage, 100 B for binary64, plus temporaries while it is sorted) and, for
 * binary64 storage, the statistics of the fixed-point sums, and synchronises
 * stream.
 * Errors: GSR_EINVAL (null vector), GSR_ESTATE (rows not loaded),
 * GSR_ENOMEM, GSR_ECUDA.
 */
gsr_status gsr_aprod2(gsr_ctx *ctx, const double *y, double *x, void *stream);

/*
 * gsr_aprod1_f32 -- y += A x in binary32 arithmetic (the kernel of the inner
 * solves of GSR_MIXED; Eq. 2). FP32-stored contexts only (GSR_EINVAL
 * otherwise).
 *   x  device array of n_cols binary32.   y  device array of n_rows binary32.
 * Errors: GSR_EINVAL (binary64-stored context, null vector), GSR_ESTATE (rows
 * not loaded), GSR_ECUDA.
 */
gsr_status gsr_aprod1_f32(gsr_ctx *ctx, const float *x, float *y, void *stream);

/*
 * gsr_aprod2_f32 -- x += A^T y with binary32 products (Eq. 3), added into
 * binary64 x. FP32-stored contexts only.
 *   y  device array of n_rows binary32.   x  device array of n_cols binary64.
 * Astrometric and global partial sums are binary32. The instrumental sums,
 * and the attitude sums when the row tiles are read in one pass, are 32-bit
 * fixed point per block (each contribution rounded to 2^-20 or finer of its
 * column's bound max|a_j| max|y|) and then exact in binary64, so those
 * entries do not depend on the order of the additions; gsr_aprod2_plan says
 * which form the loaded rows take. The first call after the rows change
 * takes the statistics of that choice (one pass, then a synchronisation of
 * stream), and builds the knot-ordered copy when the two-pass form applies.
 * Errors: as gsr_aprod1_f32, and GSR_ENOMEM.
 */
gsr_status gsr_aprod2_f32(gsr_ctx *ctx, const float *y, double *x, void *stream);

/*
 * gsr_aprod12_f32 -- one Golub-Kahan step's two products (Eq. 2 then Eq. 3,
 * the bidiagonalisation of Sec. 1): y <- A x + coef y, then z += A^T y with
 * the new y; binary32 values, products and y, binary64 z. On attitude blocks
 * too wide for the one-pass shared-memory aprod 2 (gsr_aprod2_plan passes 3)
 * both products come from one read of each row tile (the inner iterations'
 * fused pass, gsr_solve_params.inner_fused); otherwise y is scaled and the
 * two products run as gsr_aprod1_f32 and gsr_aprod2_f32.
 *   x  device, n_cols binary32.   y  device, n_rows binary32 (read, written).
 *   z  device, n_cols binary64 (accumulated).
 * FP32-stored contexts only. The first call after the rows change takes the
 * statistics of the aprod 2 form (as gsr_aprod2_f32). Errors: as
 * gsr_aprod2_f32.
 */
gsr_status gsr_aprod12_f32(gsr_ctx *ctx, const float *x, float *y, double *z, float coef, void *stream);

/*
 * gsr_aprod2_plan -- the form gsr_aprod2_f32 (and the inner iterations of
 * GSR_MIXED) takes on the loaded rows. FP32-stored contexts only.
 *   passes     1: one pass over the row tiles also sums the attitude columns
 *              (block-private fixed point, one scale for all of them);
 *              2: a second pass over a knot-ordered copy sums them (section
 *              variants whose attitude columns do not fit the one-pass form);
 *              3: one pass over the row tiles adds each row's attitude
 *              products per axis as one 4-wide binary32 reduction into window
 *              accumulators that stay in L2, then a pass over the attitude
 *              columns folds the windows into x (binary64): the standard row
 *              when the attitude columns do not fit the one-pass form.
 *   fx_bits    fewest fixed-point bits of an instrumental column's per-block
 *              sums (>= 20), or 0 when those sums are binary32.
 *   ins_group  1 when the instrumental columns share one scale (one-pass form
 *              only), else 0.
 * Any pointer may be NULL. The choice rests on per-column statistics of the
 * rows (the largest count a block adds to a column, the largest |a_j|); a
 * group shares one scale only if its smallest column still keeps >= 20 bits.
 * When the rows changed since the statistics were taken, computes them (one
 * pass over the tiles on stream, then a synchronisation of stream).
 * Errors: GSR_EINVAL (binary64-stored context), GSR_ESTATE (rows not
 * loaded), GSR_ECUDA.
 */
gsr_status gsr_aprod2_plan(gsr_ctx *ctx, void *stream, int32_t *passes, int32_t *fx_bits, int32_t *ins_group);

/*
 * gsr_residual -- r = b - A x (the residual of Eq. 1) for the loaded b, with
 * every product and sum carried in double-float (pairs of binary32 with
 * error-free transforms: about 2^-44 relative to the sum of |terms|), the
 * outer residual of the GSR_MIXED refinement. FP32-stored contexts only; b
 * must be loaded.
 *   x  device array of n_cols binary64.   r  device array of n_rows binary32.
 * Errors: GSR_EINVAL (binary64-stored context, null vector), GSR_ESTATE (rows
 * or b not loaded), GSR_ENOMEM (the workspace, allocated on first use),
 * GSR_ECUDA.
 */
gsr_status gsr_residual(gsr_ctx *ctx, const double *x, float *r, void *stream);

/*
 * gsr_residual_static -- the same r = b - A x as gsr_residual (same arithmetic),
 * for callers that must not allocate device memory at call time: a process
 * whose device memory is already reserved by another allocator's pool, or a
 * latency-critical loop that cannot afford cudaMalloc's implicit device
 * synchronisation. (The paper has no counterpart; this is a library
 * convenience.) gsr_residual takes its scratch from the context's workspace,
 * allocated on first use; this entry point calls no allocating routine.
 *   - Its scratch is a file-scope device array of 2^20 binary32 pairs
 *     (8 MiB): n_cols above 1048576 is rejected with GSR_EINVAL.
 *   - Set-up: creating a context (gsr_create / gsr_create_sections) places
 *     the array on that context's device and loads the two kernels this
 *     entry point launches, once per device, while allocating is expected;
 *     the array then stays there until the process exits. A call looks the
 *     array's device address up again (cudaGetSymbolAddress, a host-side
 *     lookup while it is loaded) and allocates nothing. A cudaDeviceReset
 *     removes the array with every context of the device: create a context
 *     again, which places it anew, before the next call.
 *   - Every call shares the one array, which keeps the last call's contents;
 *     each call writes every element it reads first, so nothing needs
 *     clearing. Calls that overlap on the GPU (different streams, or
 *     contexts on the same device) race on it: order them.
 *   x  device array of n_cols binary64.   r  device array of n_rows binary32.
 * FP32-stored contexts only; b must be loaded. Runs on stream.
 */
gsr_status gsr_residual_static(gsr_ctx *ctx, const double *x, float *r, void *stream);

/*
 * gsr_fp64_fma_rate -- the binary64 fused multiply-add rate of `device`, in
 * TFLOP/s (2 flops per FMA): the arithmetic ceiling of the binary64 aprods
 * (Eq. 2 / Eq. 3 with binary64 values and products: 24 multiply-adds per row).
 * Runs a probe kernel of independent FMA chains for a few tens of ms on the
 * default stream; synchronous. (The paper has no counterpart; it measures the
 * roofline the binary64 kernels are reported against.)
 * Errors: GSR_EINVAL (null tflops), GSR_ECUDA.
 */
gsr_status gsr_fp64_fma_rate(int32_t device, double *tflops);

/*
 * gsr_tc_wait_check -- exercises the tensor-core kernels' bounded wait on its
 * timeout path: one CTA of 128 threads allocates 32 TMEM columns, waits on an
 * mbarrier that nothing arrives on for limit_ms, records whether the wait
 * gave up, releases the TMEM and exits (what the network's convolution does
 * when its MMAs have not completed within 1 s: it sets its net's fault word,
 * which the next call on the net, or the solve that ran it, reports as
 * GSR_ECUDA). Synchronous, on the default stream of `device`; the context
 * stays usable afterwards.
 *   limit_ms   in (0, 2000].
 *   timed_out  1 if the wait gave up (the expected result), 0 if it completed.
 *   waited_ms  the kernel's duration (CUDA events).
 * Errors: GSR_EINVAL (bad limit or null output), GSR_ECUDA.
 */
gsr_status gsr_tc_wait_check(int32_t device, double limit_ms, int32_t *timed_out, double *waited_ms);

typedef struct {
    int32_t itnlim;     /* maximum LSQR iterations (>= 0)                               */
    double atol, btol;  /* Paige-Saunders tolerances (0 disables the test)              */
    double conlim;      /* condition limit (0 disables)                                 */
    double damp;        /* damping of the scaled problem (>= 0)                         */
    int32_t precond;    /* 1: column-norm preconditioning (Alg. 1), 0: none             */
    int32_t mode;       /* GSR_PLAIN or GSR_MIXED                                       */
    int32_t warm;       /* GSR_WARM_NONE / _JACOBI / _LEARNED                           */
    const char *weights_path; /* learned warm start: weights file (see gsr_warm.h)      */
    double timeout_s;   /* wall-clock limit of the solve (0 = none)                     */
    int32_t graph_k;    /* LSQR iterations per CUDA-graph launch (0 = automatic)        */
    int32_t where;      /* GSR_HOST / GSR_DEVICE: x0, x_out and se_out                  */
    int32_t inner_itn;  /* MIXED: iterations per inner FP32 solve (0 = automatic)       */
    double inner_tol;   /* MIXED: an inner solve stops when its |A~^T r| estimate is below
                           inner_tol times its value at the start of that solve (0 = 1e-6) */
    double refine_tol;  /* MIXED: stop when every block's |dx|/|x| < refine_tol (0 = 1e-10) */
    int32_t max_outer;  /* MIXED: maximum refinement steps (0 = 20)                     */
    int32_t inner_itn_next; /* MIXED: inner iteration limit of the refinement steps after
                               the first (0 = inner_itn); the first step solves for the whole
                               error of x0, the later ones only for its binary32 residue     */
    int32_t refine_grad;    /* MIXED: the start of each inner solve after the first,
                               alpha_1 v_1 = A~^T r / |r|: 0 = binary32 until the refinement
                               stalls (a step's largest block |dx|/|x| above half the previous
                               step's), binary64 from then on; 1 = binary64 from the second
                               step on; -1 = always binary32. The binary64 gradient of the
                               double-float residual r keeps the solution within the inner
                               solve's relative accuracy of the least-squares solution when
                               the column norms spread widely (the binary32 rounding of r
                               otherwise limits column j to about 2^-24 |r| / |A_:,j|)     */
    int32_t inner_fused;    /* MIXED, attitude blocks too wide for the one-pass shared-memory
                               aprod 2 (gsr_aprod2_plan passes 3): each inner iteration's
                               aprod 1 and aprod 2 in one pass over the row tiles, the new u's
                               contributions to A^T u added while its coefficients are in
                               registers (13% faster per iteration than the two passes on
                               5e8 rows). 1 (default) = on; 0 or -1 = the two separate
                               passes                                                        */
    int32_t inner_close;    /* MIXED: the last iteration of an inner solve that runs to its
                               iteration limit forms x_k from beta_{k+1} alone (LSQR's x update
                               uses beta_{k+1}, not v_{k+1}): aprod 1 and the x update, no
                               aprod 2 (on 5e8 rows 10.7 instead of 20.3 ms per refinement
                               step). x is the same iterate up to rounding; that solve's
                               |A~^T r| estimate (gsr_solve_info.arnorm) is the one of the
                               iteration before. 1 (default) = on; 0 or -1 = every iteration
                               in full. Applies when the limit is a multiple of the iterations
                               per graph launch: graph_k if set, else the largest divisor of
                               the limit up to 8 when that is at least half of min(8, limit)
                               (every limit up to 8, and 10, 12, 14, 15, 16, 18, 20, 21, ...) */
} gsr_solve_params;

typedef struct {
    int32_t istop;      /* Paige-Saunders stop reason 0..7 (7 = itnlim reached)          */
    int32_t itn;        /* LSQR iterations run (all inner iterations in MIXED)          */
    int32_t outer_itn;  /* MIXED: refinement steps                                      */
    double r1norm;      /* |b - A x|                                                    */
    double r2norm;      /* sqrt(|b - A x|^2 + damp^2 |y|^2)                             */
    double anorm;       /* Frobenius-norm estimate of the scaled [A; damp I]            */
    double acond;       /* condition estimate                                           */
    double arnorm;      /* |A~^T r - damp^2 y| estimate                                  */
    double xnorm;       /* |y| estimate (scaled unknowns)                               */
    double ms_total;    /* wall time of the call                                        */
    double ms_warm;     /* part of ms_total spent on the warm start                     */
} gsr_solve_info;

/* gsr_default_params -- fill p with the defaults (itnlim 2000, atol = btol =
 * 1e-12, conlim 1e12, damp 0, precond 1, PLAIN, no warm start, host buffers). */
void gsr_default_params(gsr_solve_params *p);

/*
 * gsr_lsqr_solve -- damped LSQR (Paige & Saunders 1982, the solver of Sec. 1-2)
 * on the column-preconditioned system (Alg. 1), with every step on the GPU:
 * aprod 1/2, the Eq. 4 norms, the vector updates and the scalar recurrences,
 * one iteration per CUDA-graph segment and no per-iteration host copies
 * (replacing the copies of Alg. 1 and Sec. 4.4).
 *   x0      NULL or n_cols starting guess; LSQR then solves for the correction
 *           of r0 = b - A x0 and returns x0 + correction.
 *   x_out   n_cols solution (required).
 *   se_out  NULL or n_cols standard errors of the unknowns.
 *   info    NULL or filled on return (also on GSR_ETIMEOUT / GSR_ENUMERIC).
 * Synchronous (returns after x_out is written). GSR_ESTATE if the rows or b
 * are missing; GSR_EINVAL for MIXED on an FP64-stored context.
 */
gsr_status gsr_lsqr_solve(gsr_ctx *ctx, const gsr_solve_params *params, const double *x0, double *x_out,
                          double *se_out, gsr_solve_info *info, void *stream);

#ifdef __cplusplus
}
#endif

#endif /* GSR_H */
