// gsr_internal.cuh -- context, device views and helpers shared by the libgsr translation units.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <algorithm>
#include <chrono>
#include <string>
#include <utility>
#include <vector>

#include "../../include/gsr.h"

struct gsr_net;  // the warm start's network (net.cu, include/gsr_warm.h)

namespace gsr {

constexpr int NPAR = 24;     // coefficients per observation row (Sec. 2)
constexpr int NASTRO = 5;    // astrometric unknowns per star
constexpr int NAXES = 3;     // attitude axes
constexpr int NPARAXIS = 4;  // attitude B-spline knots per axis touched by a row
constexpr int NINSTR = 6;    // instrumental coefficients per row
constexpr int NGLOB_MAX = GSR_MAX_GLOB;  // global unknowns of a section variant
// register slots of a row's coefficients in the kernels, by section (the standard row's slots)
constexpr int A_ATT = NASTRO, A_INS = NASTRO + NAXES * NPARAXIS, A_GLOB = NPAR - 1;
constexpr int MAX_PARTIALS = 4096;  // per-block partial sums kept for the norms
// fixed-point words after the per-column ones (fx_word[3 nc + 1 ...]): the attitude columns' largest
// |a| and smallest |a| (complemented), the instrumental columns' likewise, then the bits of the
// attitude group scale and of the instrumental group scale (0: per-column scales)
constexpr int FX_GROUP = 6;

// ---------------------------------------------------------------- device views
// The coefficient matrix lives in tiles of rows (tiles.cuh): `tiles` holds the
// star-ordered tile records, `atiles` the knot-ordered attitude tiles
// (layout.cu). Rows of star s are [star_ptr[s], star_ptr[s+1]); first_star[t]
// is the star of the first row of tile t (first_star[n_tiles] = last star).
// The section geometry (na, ni, n_glob, planes) is the standard row's
// (5, 6, 0|1; planes 5, 17, 23 of 24) unless the context holds a section
// variant (Sec. 2: 0..5 astrometric, 0..6 instrumental, 0..NGLOB_MAX globals).
template <typename VT>
struct SysView {
    const uint8_t *__restrict__ tiles;
    const uint8_t *__restrict__ atiles;
    const int64_t *__restrict__ star_ptr;
    const int32_t *__restrict__ first_star;
    const int64_t *__restrict__ knot_ptr;  // first knot-ordered position of each knot, [n_dfa-2]
    int64_t n_tiles;
    int64_t n_stars, n_rows;
    int32_t n_dfa, n_instr, n_glob;
    int64_t att0, instr0, glob0;  // first column of each section
    int64_t tile_bytes;           // bytes of one star-ordered tile record (tiles.cuh)
    int32_t iw16;                 // instrumental columns stored as 16-bit (1) or 32-bit (0) integers
    int32_t na, ni;               // astrometric / instrumental coefficients per row
    int32_t npl;                  // value planes per tile record
    int32_t p_att, p_ins, p_glob; // plane of the first attitude / instrumental / global coefficient
    // wide attitude blocks of binary32 storage (att_red / att_window below): the window accumulators
    // aw[(a n_dfa + k) 4 + q] (squares: aw2) of the column k + q of axis a from the rows starting at
    // knot k, and the window copy xw[a n_dfa + k] = x_att[a][k .. k+3] of the vector aprod 1 gathers
    float *aw, *aw2;
    const float4 *xw;
    const float4 *xw2;  // the double-float residual's window: x_att[a][k .. k+3] as (hi, lo) pairs, 2 float4
};

// LSQR scalars shared between the kernels of one solve (one instance in device
// memory). Written only by the single-thread scalar kernels; read by all.
struct LsqrState {
    double alpha, beta;          // current alpha_i, beta_i
    double rhobar, phibar;
    double anorm, acond, ddnorm, res2, xnorm, xxnorm, zeta, cs2, sn2;
    double bnorm, rnorm, r1norm, r2norm, arnorm;
    double damp, atol, btol, ctol;
    // relative gradient test of the mixed solver's inner solves: stop (istop 2) once the
    // |A~^T r| estimate is below artol times its value at the start, arnorm0 (0: off)
    double artol, arnorm0;
    double coef_u;     // aprod1: u_next = A pv + coef_u * u   (= -alpha/beta)
    double inv_alpha;  // colB: v = vhat * inv_alpha
    double t1, t2;     // colB: x += t1 w, w = v + t2 w
    double inv_rho;    // colB: var += (w * inv_rho)^2
    int32_t itn, itnlim, istop, done, colb_skip, numeric;
};

struct GraphCache {
    cudaGraphExec_t exec = nullptr;
    int k = 0;
    bool var = false, inner32 = false;
    int fused = 0;
    bool close = false;  // the last iteration is a closing one (no aprod 2)
};

struct Workspace {
    int64_t n_rows = 0, n_cols = 0;
    double *u = nullptr;        // n_rows: unnormalised bidiagonalisation vector beta*u
    double *z = nullptr;        // n_cols: aprod2 accumulator (kept zero between uses)
    double *v = nullptr;        // n_cols: v (holds vhat between colA and colB)
    double *w = nullptr;        // n_cols
    double *x = nullptr;        // n_cols: solution of the scaled problem
    double *pv = nullptr;       // n_cols: p * v, the vector aprod1 gathers
    double *p = nullptr;        // n_cols: preconditioner, 1/|A_:,j|
    double *var = nullptr;      // n_cols: sum of (w/rho)^2
    double *tmp = nullptr;      // n_cols scratch
    double *part_u = nullptr;   // MAX_PARTIALS: per-block sums of squares of u
    double *part_v = nullptr;   // MAX_PARTIALS: of vhat
    double *part_w = nullptr;   // MAX_PARTIALS: of w
    float *u32 = nullptr;       // n_rows: binary32 row vector of the inner solves (FP32-stored systems)
    float *pv32 = nullptr;      // n_cols: binary32 copy of p * v for the inner aprod1
    double *xo = nullptr;       // n_cols: refined solution (unscaled) of the mixed solver
    float2 *xhl = nullptr;      // n_cols: xo split into two binary32 parts
    double *blk = nullptr;      // 16: per-block sums of squares of the correction and of x
    float *feats = nullptr;     // n_dfa x 6: warm-start features
    float *netout = nullptr;    // n_dfa x 3: network output
    double *wacc = nullptr;     // 4: feature sums [0..1], scale [2]
    double *x0w = nullptr;      // n_cols: warm start vector
    void *astro_n = nullptr;    // n_stars x 20: per-star normal equations of the warm start (binary32 for
                                // binary32 storage, binary64 for binary64 storage)
    std::vector<GraphCache> graphs;
    LsqrState *st = nullptr;    // device
    int32_t *flag_h = nullptr;  // pinned mapped host word: 1 when the solve has stopped
    int32_t *flag_d = nullptr;  // device alias of flag_h
    LsqrState *fin_h = nullptr;   // pinned: the final state of the last run_lsqr
    double *blk_h = nullptr;      // pinned, 8: the mixed solver's correction and solution norms per block
    uint32_t *counter = nullptr;  // finished-block count of k_colA (zero between launches)
};

}  // namespace gsr

struct gsr_ctx {
    int device = 0;
    int prec = GSR_FP64;
    int sm_count = 0;
    int64_t n_stars = 0, n_rows = 0, n_cols = 0;
    int32_t n_dfa = 0, n_instr = 0, n_glob = 0;
    // sections of a row (Sec. 2): astrometric and instrumental coefficients per row; sv marks a
    // section variant (anything but 5 and 6 with at most one global), stored in compact tiles of
    // npl = n_astro + 12 + n_ipr + n_glob value planes and run by the kernels' variant instances;
    // the standard row keeps 24 planes (plane 23 zero without a global). in_w: coefficients per
    // row of the caller's arrays (24 for gsr_create, the compact count for gsr_create_sections).
    int32_t n_astro = gsr::NASTRO, n_ipr = gsr::NINSTR, npl = gsr::NPAR, in_w = gsr::NPAR;
    bool sv = false;
    int64_t n_tiles = 0;             // row tiles (tiles.cuh); rows per tile depend on the precision
    int64_t tile_bytes = 0;          // bytes of one tile record
    int32_t iw16 = 0;                // instrumental columns in 16-bit planes (n_instr <= 65536)
    void *tiles = nullptr;           // star-ordered tile records
    void *atiles = nullptr;          // knot-ordered attitude tile records
    int32_t *first_star = nullptr;   // [n_tiles + 1] star of the first row of each tile
    int64_t *knot_ptr = nullptr;     // [n_dfa-2] first position of each knot
    bool att_valid = false;          // atiles / knot_ptr match the loaded rows
    int32_t fx_sig = -1;             // kernel choice the cached graphs were captured with
    // fixed-point instrumental sums of the binary32 star pass (layout.cu): the fewest bits per
    // contribution over the columns (0: binary32 shared atomics instead), the pass's fixed
    // partition, and device words: [n_instr] max |coefficient| per column (binary32 bits),
    // [n_instr] bits per column, max |y| of the current aprod 2 (binary32 bits), scratch
    int32_t fx_bits = 0;
    int64_t fx_per = 0, fx_blocks = 0;
    uint32_t *fx_word = nullptr;
    // fixed-point columns: the instrumental ones, then (fx_att) the 3 n_dfa attitude columns, whose
    // products the star pass then adds into shared memory as well (no attitude pass; the knot-ordered
    // copy is built only for the binary64 aprod 2). fx_word holds [fx_nc] max |a| per column, [fx_nc]
    // bits per column, max |y|, [fx_nc] scratch, then FX_GROUP words of the group scales.
    int32_t fx_nc = 0;
    bool fx_att = false;
    bool fx_uni = false;             // the one-pass aprod 2 gives the instrumental columns one scale too
    bool fx_valid = false;           // the statistics match the loaded rows
    // fixed-point instrumental sums of the binary64 star pass (binary64 storage, standard row; built
    // with the knot-ordered copy, layout.cu): the pass's partition (fx64_per tiles a warp, fx64_blocks
    // blocks of fx64_nt threads) and fx64_word: [FX64_BINS] the sampled binary64 exponents of |y| of the
    // current aprod 2, its y_t (binary64, 2 words), [n_instr] the largest number of contributions one
    // block adds to each instrumental column, [n_instr] each column's largest |coefficient| (binary32
    // bits, rounded up)
    int64_t fx64_per = 0, fx64_blocks = 0;
    int32_t fx64_nt = 0;
    uint32_t *fx64_word = nullptr;
    bool fx64 = false;               // the statistics are built (valid while att_valid holds)
    int32_t fused_inner = 0;         // the current solve's inner iterations take the fused pass (> 0)
    // wide attitude blocks (binary32 storage, standard row): attw holds the window accumulators of the
    // binary32 aprod 2 (2 x 3 n_dfa x 4 binary32: products, then squares; zero between uses), xwin the
    // window copy aprod 1 gathers from (n_dfa x 4 float4, knot-major: axes 0-2, one unused)
    float *attw = nullptr;
    float *xwin = nullptr;
    float4 *xhlwin = nullptr;  // the double-float residual's window copy (3 n_dfa x 2 float4), wide blocks
    int64_t *star_ptr = nullptr;     // device copy
    std::vector<int64_t> star_ptr_h; // host copy
    int32_t max_obs = 0;             // longest star
    double *b = nullptr;             // n_rows
    bool rhs_set = false;
    std::vector<std::pair<int64_t, int64_t>> rows_set;  // merged [lo, hi) ranges of loaded rows
    int32_t *errw = nullptr;         // device error words for validation (4 int32)
    cudaStream_t own = nullptr;      // non-blocking stream the solve runs (and captures) on
    struct gsr_net *warm_net = nullptr;  // network of GSR_WARM_LEARNED solves, loaded from warm_path
    std::string warm_path;
    cudaEvent_t ev = nullptr;        // orders `own` after the caller's stream
    cudaEvent_t ev_w0 = nullptr, ev_w1 = nullptr;  // the warm start's span inside a solve (timing)
    cudaMemPool_t pool = nullptr;    // stream-ordered scratch of the layout build, kept between builds
    gsr::Workspace ws;
    std::string err;
};

namespace gsr {

// ---------------------------------------------------------------- host helpers
gsr_status fail(gsr_ctx *c, gsr_status s, const std::string &msg);
gsr_status cuda_fail(gsr_ctx *c, cudaError_t e, const char *what);
bool rows_complete(const gsr_ctx *c);

template <typename VT>
SysView<VT> view(const gsr_ctx *c)
{
    SysView<VT> s;
    s.tiles = static_cast<const uint8_t *>(c->tiles);
    s.atiles = static_cast<const uint8_t *>(c->atiles);
    s.star_ptr = c->star_ptr;
    s.first_star = c->first_star;
    s.knot_ptr = c->knot_ptr;
    s.n_tiles = c->n_tiles;
    s.n_stars = c->n_stars;
    s.n_rows = c->n_rows;
    s.n_dfa = c->n_dfa;
    s.n_instr = c->n_instr;
    s.n_glob = c->n_glob;
    s.att0 = (int64_t)c->n_astro * c->n_stars;
    s.instr0 = s.att0 + (int64_t)NAXES * c->n_dfa;
    s.glob0 = s.instr0 + c->n_instr;
    s.tile_bytes = c->tile_bytes;
    s.iw16 = c->iw16;
    s.na = c->n_astro;
    s.ni = c->n_ipr;
    s.npl = c->npl;
    s.p_att = c->sv ? c->n_astro : A_ATT;
    s.p_ins = s.p_att + NAXES * NPARAXIS;
    s.p_glob = c->sv ? s.p_ins + c->n_ipr : A_GLOB;
    s.aw = c->attw;
    s.aw2 = c->attw ? c->attw + (size_t)NAXES * c->n_dfa * 4 : nullptr;
    s.xw = reinterpret_cast<const float4 *>(c->xwin);
    s.xw2 = c->xhlwin;
    return s;
}

// kernels launchers (aprod.cu)
// inner32: the binary32 kernels of the mixed solver's inner LSQR (x / y are float*)
cudaError_t launch_aprod1(const gsr_ctx *c, const void *x, void *y, const LsqrState *st, double *part,
                          cudaStream_t s, bool inner32 = false);
cudaError_t launch_aprod2(const gsr_ctx *c, const void *y, double *x, bool square, const LsqrState *st,
                          cudaStream_t s, bool inner32 = false);
// one pass computing x += A^T y and sq += the column sums of squares (the warm start)
cudaError_t launch_aprod2_both(const gsr_ctx *c, const void *y, double *x, double *sq, cudaStream_t s, bool inner32);
int aprod1_grid(const gsr_ctx *c, bool inner32 = false);
// one LSQR iteration's aprod 1 and aprod 2 in one pass over the tiles (binary32 inner solve of a wide
// attitude block: att_red and att_window); with grid_out only the number of partials it writes
cudaError_t launch_iter_fused(const gsr_ctx *c, const float *pv, float *u, double *z, const LsqrState *st,
                              double *part, cudaStream_t s, int *grid_out = nullptr, float coef = 1.f);
// y <- A x + coef y, z += A^T y (binary32 storage, products and y): the fused pass or the two products
cudaError_t launch_aprod12_f32(const gsr_ctx *c, const float *x, float *y, double *z, float coef, cudaStream_t s);

// per-system layout work (layout.cu), once per loaded system: the fixed-point statistics of binary32
// storage, and the knot-ordered attitude copy when binary64 aprod 2 passes will run (binary64) or the
// binary32 star pass does not take the attitude columns (fx_att false)
gsr_status ensure_att_layout(gsr_ctx *c, cudaStream_t s, bool binary64);
// the binary32 aprod 2 adds the attitude products in its star pass (no attitude pass)
inline bool att_fused(const gsr_ctx *c) { return c->prec == GSR_FP32 && c->fx_bits > 0 && c->fx_att && !c->sv; }
// the binary32 aprod 2 adds each row's attitude products with vector reductions into the window
// accumulators (the attitude columns do not fit the one-pass form's shared memory)
inline bool att_red(const gsr_ctx *c)
{
    return c->prec == GSR_FP32 && !c->sv && c->fx_valid && !att_fused(c) && c->attw;
}
// the binary32 aprod 1 gathers the attitude unknowns through the window copy (one 16-byte load per axis;
// every binary32 standard-row context: c2 0.394 -> 0.366 ms, c5 14.5 -> 10.9 ms)
inline bool att_window(const gsr_ctx *c) { return c->prec == GSR_FP32 && !c->sv && c->xwin; }
// the double-float residual gathers the attitude pairs through their window copy (wide blocks only)
inline bool res_window(const gsr_ctx *c) { return c->prec == GSR_FP32 && !c->sv && c->xhlwin; }
// the inner solves take the fused iteration pass (set per solve from gsr_solve_params.inner_fused)
inline bool iter_fused(const gsr_ctx *c) { return c->fused_inner && att_red(c) && att_window(c); }
// attitude columns above which the double-float residual uses the window copy of the pairs: beyond ~16K
// the gathered pairs no longer stay in L1 beside the streamed tiles (below, the window made it slower:
// c2, 9,000 columns, 0.550 -> 0.608 ms)
constexpr int64_t ATT_WINDOW_MIN_COLS = 16384;
// max |y| word of the fixed-point sums (nullptr when they are off)
constexpr int FX64_BINS = 2048;  // binary64 exponent values
// the binary64 star pass takes the fixed-point instrumental sums
inline bool star_fx64(const gsr_ctx *c) { return c->prec == GSR_FP64 && !c->sv && c->fx64 && c->att_valid; }
// its partition for the loaded dimensions (aprod.cu): per tiles a warp, blocks, threads a block
void fx64_partition(const gsr_ctx *c, int64_t *per, int64_t *blocks, int32_t *nt);
// bytes of the pass's dynamic shared memory: int64 sums and int16 shifts of the instrumental columns
inline size_t fx64_smem(const gsr_ctx *c) { return (sizeof(long long) + sizeof(int16_t)) * (size_t)c->n_instr; }
inline uint32_t *fx_ymax(const gsr_ctx *c) { return c->fx_bits > 0 ? c->fx_word + 2 * (size_t)c->fx_nc : nullptr; }

// the allocation-free residual's scratch array (residual_static.cu): load its module and the kernels
// the entry point launches on the current device and look up the array's address (context creation
// calls it, so that no later call of the entry point loads anything)
cudaError_t static_scratch_load(bool sv);
// load the split and residual kernels (mixed.cu) of a context with (sv) or without run-time sections
cudaError_t residual_kernels_load(bool sv);

// LSQR driver (lsqr.cu)
// x0_dev: x0 is device memory whatever prm->where says (the warm start's vector)
// p_ready: ws.p already holds this solve's column scaling (computed by the warm
// start of the same call, with the same precision), so the pass is skipped
gsr_status lsqr_solve(gsr_ctx *c, const gsr_solve_params *prm, const double *x0, bool x0_dev, double *x_out,
                      double *se_out, gsr_solve_info *info, cudaStream_t s, bool p_ready = false);
gsr_status ensure_workspace(gsr_ctx *c);
void free_workspace(gsr_ctx *c);
void drop_graphs(gsr_ctx *c);  // forget the cached iteration graphs (recaptured on next use)
void default_params(gsr_solve_params *p);
int col_grid(const gsr_ctx *c, int64_t n);
// with y (and use): the same pass also adds A^T y to z (binary32 products when f32)
gsr_status precond_pass(gsr_ctx *c, bool use, cudaStream_t s, bool f32 = false, const void *y = nullptr,
                        double *z = nullptr);
LsqrState initial_state(const gsr_solve_params *prm);
// defer_fin: leave the final state's download (into ws.fin_h) pending on s, for a caller that
// synchronises s itself after more work; *fin is then not written. start64 (inner32 only): the
// start's aprod 2 reads the binary64 right-hand side in ws.u with binary64 products and sums. close:
// a solve that reaches its iteration limit ends with a closing iteration (aprod 1 and the x update;
// the limit's estimates that need alpha_{k+1} keep the previous iteration's values)
gsr_status run_lsqr(gsr_ctx *c, const LsqrState &init, bool inner32, bool want_var, int n_part_u, int graph_k,
                    double timeout_s, std::chrono::steady_clock::time_point t0, cudaStream_t s, LsqrState *fin,
                    bool defer_fin = false, bool start64 = false, bool close = false);
void fill_info(gsr_solve_info *info, const LsqrState &fin, std::chrono::steady_clock::time_point t0);
// warm start (warm.cu)
// r0_parts (may be null): for binary32 storage the residual of x0 is also left in ws.u32, in
// binary32, with its per-block sums of squares in ws.part_u (*r0_parts partials; 0 when not)
gsr_status warm_start_dev(gsr_ctx *c, gsr_net *net, double *x0, cudaStream_t s, int *r0_parts);
// a convolution of the net found its tensor-core wait run out since the last look (then cleared)
bool net_take_fault(gsr_net *n);
// mixed-precision solver (mixed.cu)
gsr_status residual_f32(gsr_ctx *c, const double *x, float *r, cudaStream_t s);
// window: the attitude gathers read the context's window copy (split_launch with window built it);
// without, only xhl is read (the allocation-free entry point's path)
// r64 (may be null): the double-float residual also in binary64 (before its rounding to binary32)
cudaError_t residual_launch(const gsr_ctx *c, const float2 *xhl, const double *b64, float *r,
                            double *part, cudaStream_t s, int *grid_out, bool window = false,
                            double *r64 = nullptr);
// x -> (hi, lo) pairs into out; window (wide attitude blocks, att_window): also the window copy
cudaError_t split_launch(const gsr_ctx *c, const double *x, float2 *out, int64_t n, cudaStream_t s,
                         bool window = false);
// r0_parts > 0: ws.u32 / ws.part_u already hold the residual of x0 (from the warm start) for the
// first refinement step
gsr_status mixed_solve(gsr_ctx *c, const gsr_solve_params *prm, const double *x0, bool x0_dev, double *x_out,
                       gsr_solve_info *info, cudaStream_t s, bool p_ready = false, int r0_parts = 0);

// ---------------------------------------------------------------- device helpers
__device__ __forceinline__ double warp_sum(double v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// Deterministic sum of n partials by one warp: each lane keeps eight independent
// lane-strided sums (eight loads in flight instead of one dependent chain), then a
// fixed tree. The order depends only on n. Loads bypass L1 (partials may come from
// other blocks of the running kernel).
__device__ __forceinline__ double warp_sum_partials(const double *__restrict__ part, int n)
{
    double acc[8] = {0.0, 0.0, 0.0, 0.0, 0.0, 0.0, 0.0, 0.0};
    int i = threadIdx.x & 31;
    for (; i + 7 * 32 < n; i += 8 * 32) {
#pragma unroll
        for (int q = 0; q < 8; ++q) acc[q] += __ldcg(part + i + q * 32);
    }
#pragma unroll
    for (int q = 0; q < 8; ++q)
        if (i + q * 32 < n) acc[q] += __ldcg(part + i + q * 32);
    const double s = ((acc[0] + acc[1]) + (acc[2] + acc[3])) + ((acc[4] + acc[5]) + (acc[6] + acc[7]));
    return warp_sum(s);
}

// Block-wide sum; every thread must call it; result valid in thread 0.
__device__ __forceinline__ double block_sum(double v, double *sm32)
{
    v = warp_sum(v);
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    __syncthreads();
    if (lane == 0) sm32[wid] = v;
    __syncthreads();
    double r = 0.0;
    if (wid == 0) {
        const int nw = (blockDim.x + 31) >> 5;
        r = lane < nw ? sm32[lane] : 0.0;
        r = warp_sum(r);
    }
    return r;
}

// Two block-wide sums at once (one pair of barriers and one shuffle tree); every thread must call it;
// results valid in thread 0. sm64: 64 doubles of shared memory.
__device__ __forceinline__ double2 block_sum2(double a, double b, double *sm64)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        a += __shfl_xor_sync(0xffffffffu, a, o);
        b += __shfl_xor_sync(0xffffffffu, b, o);
    }
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    __syncthreads();
    if (lane == 0) {
        sm64[wid] = a;
        sm64[32 + wid] = b;
    }
    __syncthreads();
    double2 r = make_double2(0.0, 0.0);
    if (wid == 0) {
        const int nw = (blockDim.x + 31) >> 5;
        r.x = lane < nw ? sm64[lane] : 0.0;
        r.y = lane < nw ? sm64[32 + lane] : 0.0;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            r.x += __shfl_xor_sync(0xffffffffu, r.x, o);
            r.y += __shfl_xor_sync(0xffffffffu, r.y, o);
        }
    }
    return r;
}

// Block-wide maximum of non-negative values; every thread must call it; result valid in thread 0.
__device__ __forceinline__ float block_max(float v, float *sm32)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = fmaxf(v, __shfl_xor_sync(0xffffffffu, v, o));
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    __syncthreads();
    if (lane == 0) sm32[wid] = v;
    __syncthreads();
    float r = 0.f;
    if (wid == 0) {
        const int nw = (blockDim.x + 31) >> 5;
        r = lane < nw ? sm32[lane] : 0.f;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) r = fmaxf(r, __shfl_xor_sync(0xffffffffu, r, o));
    }
    return r;
}

}  // namespace gsr
