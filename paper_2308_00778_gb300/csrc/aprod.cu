// aprod.cu -- aprod 1 (y += A x, Eq. 2) and aprod 2 (x += A^T y, Eq. 3) over row tiles.
//
// All kernels are persistent grids in which a warp handles one tile of
// T = 32*R rows at a time (tiles.cuh): lane l owns R consecutive rows and reads
// every plane of the tile with one 16-byte load. Warps take tiles in a
// grid-stride order, so the warps running at one time stream consecutive
// tiles of memory.
//
// aprod 1: per row, the 5 astrometric unknowns of the row's star (the star
// of each row comes from star_ptr, searched from the tile's first star), the
// 12 attitude and 6 instrumental unknowns gathered through the read-only
// cache, 1 global. In the LSQR form it computes u <- A (p v) + coef * u and
// emits per-block sums of squares of the new u (the norm beta).
//
// aprod 2 runs as two passes. The star pass reads the astrometric,
// instrumental and global coefficients. Each warp owns a contiguous range of
// tiles; astrometric products of the current star accumulate in registers
// and are added once per star (run) and warp; instrumental products go to
// block-private shared-memory accumulators flushed once per block (global
// atomic adds when n_instr is too large); the global column is reduced per
// block and added once per block (the two-stage reduction of the paper's
// global kernels, Sec. 4.2, folded into one pass). The attitude pass reads the
// knot-ordered copy of the 12 attitude coefficients (layout.cu): each warp
// owns a contiguous range of tiles, sums runs of equal knot in registers and
// adds each run once, instead of 12 atomic adds per row.
//
// Every kernel is templated on the stored value type VT, the type of the
// gathered / streamed vectors (XT for x in aprod 1, UT for the row vector) and
// the arithmetic type AT: binary64 for the plain solver (on FP64- or
// FP32-stored values) and binary32 throughout for the inner solve of the
// mixed-precision solver. Column accumulators (z) are always binary64.
#include "tiles.cuh"

namespace gsr {

// what an aprod 2 pass accumulates per column: sum a y, sum a^2, or both (into a second vector)
enum { A2_PROD = 0, A2_SQUARE = 1, A2_BOTH = 2 };

// four binary32 additions at a 16-byte aligned global address in one reduction (no value returned)
__device__ __forceinline__ void red_add_v4(float *p, float a, float b, float c, float d)
{
    asm volatile("red.global.add.v4.f32 [%0], {%1, %2, %3, %4};" ::"l"(p), "f"(a), "f"(b), "f"(c), "f"(d)
                 : "memory");
}

template <typename T>
__device__ __forceinline__ T warp_sum_t(T v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

template <typename VT, typename XT, typename UT, typename AT, bool LSQR, bool SV = false, bool ATTW = false,
          bool XS = false>
__global__ void __launch_bounds__(256) k_aprod1(SysView<VT> S, const XT *__restrict__ x, UT *__restrict__ y,
                                                const LsqrState *__restrict__ st, double *__restrict__ part,
                                                uint32_t *__restrict__ ymax)
{
    constexpr int R = Tile<VT>::R;
    constexpr int T = Tile<VT>::T;
    constexpr int MG = Sec<SV>::MAXG;
    const Sec<SV> G(S);
    __shared__ double sm32[32];
    AT coef = (AT)1;
    if (LSQR) {
        if (st->done) return;  // same value for every thread of the grid
        coef = (AT)st->coef_u;
    }
    const int lane = threadIdx.x & 31;
    const int64_t gw = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
    const XT *__restrict__ xt = x + S.att0;
    const XT *__restrict__ xi = x + S.instr0;
    // XS: x of the instrumental columns copied to shared memory, its 6 gathers a row shared-memory loads
    extern __shared__ __align__(16) unsigned char smem_raw[];
    XT *sm_xi = reinterpret_cast<XT *>(smem_raw);
    if constexpr (XS) {
        for (int32_t i = threadIdx.x; i < S.n_instr; i += blockDim.x) sm_xi[i] = __ldg(xi + i);
        __syncthreads();
    }
    AT xg[MG];
#pragma unroll
    for (int q = 0; q < MG; ++q) xg[q] = q < S.n_glob ? (AT)__ldg(x + S.glob0 + q) : (AT)0;
    AT ssq = (AT)0;
    float amx = 0.f;
    for (int64_t t = gw; t < S.n_tiles; t += nw) {
        const uint8_t *tb = S.tiles + t * S.tile_bytes;
        const uint8_t *ti = tb + (int64_t)G.npl * Tile<VT>::VBLK;
        int32_t kn[R];
        load_ints<R>(ti, 0, kn);
        int32_t ic[NINSTR][R];
        AT a[A_GLOB + MG][R];
        if constexpr (SV) {
            // run-time sections: every load is unconditional (absent slots read an attitude plane or
            // the knot plane, always present in the record) and what an absent slot gathers is
            // masked to zero, so the loads schedule together as in the standard instance
#pragma unroll
            for (int j = 0; j < NINSTR; ++j) load_instr_or_knot<VT>(tb, G.npl, G.ni, S.iw16, j, ic[j]);
#pragma unroll
            for (int j = 0; j < NASTRO; ++j) load_vals<VT, AT>(tb, j < G.na ? j : G.p_att, a[j]);
#pragma unroll
            for (int j = 0; j < NAXES * NPARAXIS; ++j) load_vals<VT, AT>(tb, G.p_att + j, a[A_ATT + j]);
#pragma unroll
            for (int j = 0; j < NINSTR; ++j) load_vals<VT, AT>(tb, j < G.ni ? G.p_ins + j : G.p_att, a[A_INS + j]);
#pragma unroll
            for (int q = 0; q < MG; ++q) load_vals<VT, AT>(tb, q < G.ng ? G.p_glob + q : G.p_att, a[A_GLOB + q]);
        } else {
#pragma unroll
            for (int j = 0; j < NINSTR; ++j) load_instr<VT>(tb, S.iw16, j, ic[j]);
#pragma unroll
            for (int j = 0; j < A_GLOB + MG; ++j) load_vals<VT, AT>(tb, j, a[j]);
        }
        const int64_t r0 = t * T + lane * R;
        int64_t sr[R];
        stars_of_rows<R>(S.star_ptr, S.first_star, t, r0, sr);
#pragma unroll
        for (int i = 0; i < R; ++i) {
            AT v;
            if constexpr (SV) {
                const XT *__restrict__ xa = x + (int64_t)G.na * sr[i];
                v = (AT)0;
#pragma unroll
                for (int j = 0; j < NASTRO; ++j) {
                    const AT xv = (AT)__ldg(j < G.na ? xa + j : x);
                    v = fma(a[j][i], j < G.na ? xv : (AT)0, v);
                }
            } else {
                const XT *__restrict__ xa = x + NASTRO * sr[i];
                v = a[0][i] * (AT)__ldg(xa);
#pragma unroll
                for (int j = 1; j < NASTRO; ++j) v = fma(a[j][i], (AT)__ldg(xa + j), v);
            }
            float4 wv[NAXES];
            if constexpr (ATTW) att_window_load(S.xw, kn[i], wv);
#pragma unroll
            for (int ax = 0; ax < NAXES; ++ax) {
                if constexpr (ATTW) {
                    // the axis's 4 consecutive unknowns from the window copy
                    const float4 w = wv[ax];
                    v = fma(a[A_ATT + NPARAXIS * ax + 0][i], (AT)w.x, v);
                    v = fma(a[A_ATT + NPARAXIS * ax + 1][i], (AT)w.y, v);
                    v = fma(a[A_ATT + NPARAXIS * ax + 2][i], (AT)w.z, v);
                    v = fma(a[A_ATT + NPARAXIS * ax + 3][i], (AT)w.w, v);
                } else {
                    const XT *__restrict__ xk = xt + (int64_t)ax * S.n_dfa + kn[i];
#pragma unroll
                    for (int j = 0; j < NPARAXIS; ++j) v = fma(a[A_ATT + NPARAXIS * ax + j][i], (AT)__ldg(xk + j), v);
                }
            }
#pragma unroll
            for (int j = 0; j < NINSTR; ++j) {
                if constexpr (SV) {
                    const AT xv = (AT)__ldg(j < G.ni ? xi + ic[j][i] : x);
                    v = fma(a[A_INS + j][i], j < G.ni ? xv : (AT)0, v);
                } else {
                    v = fma(a[A_INS + j][i], (AT)(XS ? sm_xi[ic[j][i]] : __ldg(xi + ic[j][i])), v);
                }
            }
#pragma unroll
            for (int q = 0; q < MG; ++q) v = fma(a[A_GLOB + q][i], xg[q], v);  // xg[q] = 0 past n_glob
            const int64_t r = r0 + i;
            if (r < S.n_rows) {
                AT yn;
                if (LSQR) {
                    yn = fma(coef, (AT)y[r], v);
                    ssq = fma(yn, yn, ssq);
                } else {
                    yn = (AT)y[r] + v;
                }
                y[r] = (UT)yn;
                if constexpr (LSQR && sizeof(AT) == 4) amx = fmaxf(amx, fabsf((float)yn));
            }
        }
    }
    if (LSQR) {
        const double t = block_sum((double)ssq, sm32);
        if (threadIdx.x == 0) part[blockIdx.x] = t;
    }
    if constexpr (LSQR && sizeof(AT) == 4) {
        if (ymax) {  // max |new y| of the warp (binary32 bits of non-negative values order as integers)
            const uint32_t m = __reduce_max_sync(0xffffffffu, __float_as_uint(amx));
            if ((threadIdx.x & 31) == 0 && m) atomicMax(ymax, m);
        }
    }
}

// Add a warp's per-lane partial sums of the na (5 in the standard row)
// astrometric columns of star k: the 32 x 5 partials go through a per-warp
// shared-memory buffer and lanes 0..na-1 each sum one column (31 adds per
// column instead of a 5-step shuffle tree per value on every lane). Column j
// sits at j * WSTRIDE with WSTRIDE = 33 words: the summing lanes then read
// different banks (with 32 they read one bank, a 5-way conflict on every load).
// Warp-collective.
constexpr int WSTRIDE = 33;

template <typename AT>
__device__ __forceinline__ void flush_astro_run(AT (&acc)[NASTRO], int64_t k, AT *__restrict__ wbuf,
                                                double *__restrict__ z, int na = NASTRO)
{
    const int lane = threadIdx.x & 31;
#pragma unroll
    for (int j = 0; j < NASTRO; ++j) {
        wbuf[j * WSTRIDE + lane] = acc[j];
        acc[j] = (AT)0;
    }
    __syncwarp();
    if (lane < na) {
        AT t = (AT)0;
#pragma unroll 8
        for (int l = 0; l < 32; ++l) t += wbuf[lane * WSTRIDE + l];
        atomicAdd(z + (int64_t)na * k + lane, (double)t);
    }
    __syncwarp();
}

// the instrumental products of a lane's rows that the fixed-point sums leave out (rare), by binary64
// atomics; kept out of line so that the pass's own registers and schedule do not change
__device__ __noinline__ void fx64_lane_outliers(double *__restrict__ zi, const double (&ai)[NINSTR][2],
                                                const int32_t (&ic)[NINSTR][2], const double (&yr)[2], unsigned mask)
{
#pragma unroll
    for (int i = 0; i < 2; ++i)
        if (mask & (1u << i))
#pragma unroll
            for (int j = 0; j < NINSTR; ++j) atomicAdd(zi + ic[j][i], ai[j][i] * yr[i]);
}

// round(a y 2^sh) as an int64 from the exact product of the significands (a 53 x 53-bit integer
// multiply), for |a y 2^sh| <= 2^62: a y 2^sh = ma my 2^-t with t = 2150 - ea - ey - sh >= 42 (ea, ey the
// biased exponents, 1 for subnormals), rounded half away from zero by a right shift of t places. No
// binary64 operation: the product never passes through a rounded binary64 value.
__device__ __forceinline__ long long fx64_mulround(double a, double y, int sh)
{
    const unsigned long long ba = (unsigned long long)__double_as_longlong(a);
    const unsigned long long by = (unsigned long long)__double_as_longlong(y);
    const int ea = (int)((ba >> 52) & 0x7ff), ey = (int)((by >> 52) & 0x7ff);
    const unsigned long long ma = (ba & 0xfffffffffffffull) | (ea ? 0x10000000000000ull : 0ull);
    const unsigned long long my = (by & 0xfffffffffffffull) | (ey ? 0x10000000000000ull : 0ull);
    const int t = 2150 - max(ea, 1) - max(ey, 1) - sh;
    const unsigned __int128 p = (unsigned __int128)ma * my;
    unsigned long long q = 0ull;
    if (t > 0 && t < 128) q = (unsigned long long)((p + ((unsigned __int128)1 << (t - 1))) >> t);
    return ((ba ^ by) >> 63) ? -(long long)q : (long long)q;
}

// aprod 2, star pass: astrometric, instrumental and global parts. Each warp
// owns a contiguous range of tiles; astrometric products of the current star
// accumulate per lane and are flushed once when the star changes (a tile that
// crosses a star boundary moves its rows of the next star into a second
// accumulator; rows of stars that begin and end inside one tile are added
// directly).
//
// FX (binary32 products only): the instrumental sums are kept in block-private
// 32-bit integers, fixed point with a power-of-two scale per column and
// launch, added with the integer shared-memory atomics (the binary32 ones cost
// several times more per add). Column j's contributions are bounded by
// max|a_j| max|y| (fx_word), and its bits b_j are chosen per system so that no
// block of this fixed partition can overflow it (the most contributions one
// block adds to column j, times 2^b_j, stays below 2^31); each contribution is
// rounded to 2^-b_j of its column's bound (b_j >= 20), at the level of
// binary32 accumulation. The per-block integer sums convert exactly to binary64
// and sum exactly there, so these columns of A^T y do not depend on the order
// of the additions.
//
// FX64 (binary64 storage, products): the same for binary64, in 64-bit integers
// with a power-of-two scale per column and call (below), each product formed
// and rounded by integer operations (fx64_mulround): the binary64 shared-memory
// atomic adds they replace, and the products themselves, occupied the binary64
// pipe (on 2e7 rows with 1,000 instrumental columns the whole aprod 2 went from
// 1.70 to 1.29 ms). NW: warps per block (16 when the 20,000 columns of the
// 5e8-row system leave room for one block per SM only).
template <typename VT, typename UT, typename AT, bool INSTR_SMEM, int MODE, bool LSQR, bool FX, bool SV,
          bool ATT = false, bool UNI = false, bool ATTRED = false, bool FX64 = false, int NW = 8>
__device__ __forceinline__ void aprod2_star_body(const SysView<VT> &S, const UT *__restrict__ y,
                                                 double *__restrict__ z, double *__restrict__ z2,
                                                 const LsqrState *__restrict__ st, int64_t tiles_per_warp,
                                                 const uint32_t *__restrict__ fx_word, int32_t fxs)
{
    constexpr bool SQUARE = MODE == A2_SQUARE;
    constexpr bool BOTH = MODE == A2_BOTH;
    constexpr int MG = Sec<SV>::MAXG;
    const Sec<SV> G(S);
    static_assert(!FX || (INSTR_SMEM && sizeof(AT) == 4), "fixed point: binary32 products and squares");
    static_assert(!ATT || (FX && !SV), "attitude columns: fixed point, standard row");
    static_assert(!ATTRED || (!ATT && !SV && sizeof(AT) == 4), "attitude reductions: binary32, standard row");
    static_assert(!FX64 || (INSTR_SMEM && !FX && !SV && !ATT && !ATTRED && sizeof(AT) == 8 && MODE == A2_PROD),
                  "binary64 fixed point: the products of the standard row's instrumental columns");
    __shared__ int s_bad;
    constexpr int R = Tile<VT>::R;
    constexpr int T = Tile<VT>::T;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    __shared__ double sm32[32];
    __shared__ AT wred[NW][NASTRO * WSTRIDE];
    if (LSQR && st->done) return;
    // block-private columns: the instrumental ones, then (ATT) the attitude ones at n_instr + a*n_dfa + k
    const int32_t ncol = ATT ? S.n_instr + NAXES * S.n_dfa : S.n_instr;
    AT *sm_ins = reinterpret_cast<AT *>(smem_raw);
    AT *sm_sq = sm_ins + ncol;  // BOTH: the squares' accumulators follow the products'
    const int32_t nsm = INSTR_SMEM ? (BOTH ? 2 * ncol : ncol) : 0;
    for (int32_t i = threadIdx.x; i < nsm; i += blockDim.x) sm_ins[i] = (AT)0;  // also integer zero
    // FX: per-column scales of the instrumental columns after the accumulators (BOTH: products', then
    // squares'); fx_word holds fxs columns of max |a| and of bits, then max |y|. In the one-pass form
    // the attitude columns share one scale, and the instrumental ones too when the statistics allow
    // (group bits > 0: no column loses more than the spread of |a| in its group): from the group's
    // largest |a| and bits (fx_word[3 fxs + 1 ...], FX_GROUP words), one shared-memory read less per
    // product.
    __shared__ float s_att_sc, s_att_qsc, s_ins_sc, s_ins_qsc;
    float *sm_scale = reinterpret_cast<float *>(smem_raw) + nsm;
    float *sm_qscale = sm_scale + S.n_instr;
    if (FX) {
        const float ymax = SQUARE ? 1.f : __uint_as_float(fx_word[2 * fxs]);
        if (threadIdx.x == 0) s_bad = !(ymax < INFINITY);  // non-finite y: the sums are made NaN below
        if (ATT && threadIdx.x < 2) {  // thread 0: the attitude group, thread 1: the instrumental group
            const uint32_t *gw = fx_word + 3 * fxs + 1;
            const float am = __uint_as_float(gw[2 * threadIdx.x]);
            const uint32_t bits = gw[4 + threadIdx.x];
            const float lim = (float)((1u << bits) - 1u);
            const float bound = SQUARE ? am * am : am * ymax;
            float sc = 1.f, qs = 1.f;
            if (bound > 0.f && bound < INFINITY) sc = ldexpf(1.f, min(ilogbf(lim / bound), 126));
            if (am * am > 0.f && am * am < INFINITY) qs = ldexpf(1.f, min(ilogbf(lim / (am * am)), 126));
            if (threadIdx.x == 0) {
                s_att_sc = sc;
                s_att_qsc = qs;
            } else {
                s_ins_sc = sc;
                s_ins_qsc = qs;
            }
        }
        for (int32_t i = threadIdx.x; i < S.n_instr; i += blockDim.x) {
            // the largest power of two with bound * scale <= 2^b_j - 1, bound = max|a_j| max|y|
            // for the products and max|a_j|^2 for the squares (and for the squares' pass)
            const float am = __uint_as_float(fx_word[i]);
            const float lim = (float)((1u << fx_word[fxs + i]) - 1u);
            const float bound = SQUARE ? am * am : am * ymax;
            float sc = 1.f;
            if (bound > 0.f && bound < INFINITY) sc = ldexpf(1.f, min(ilogbf(lim / bound), 126));
            sm_scale[i] = sc;
            if (BOTH) {
                const float qb = am * am;
                float qs = 1.f;
                if (qb > 0.f && qb < INFINITY) qs = ldexpf(1.f, min(ilogbf(lim / qb), 126));
                sm_qscale[i] = qs;
            }
        }
    }
    // FX64: the instrumental sums as int64 fixed point, column j in units of 2^-sh_j, with sh_j the
    // largest shift for which (the most contributions one block adds to j) x max|a_j| x y_t stays
    // within 2^62: no block sum can overflow, and each contribution is rounded to 2^-(sh_j + 1), about
    // 2^-53 of its column's bound times that count (from the exact product, fx64_mulround). y_t is a
    // power of two above all but about 1/1024 of the rows' |y| (k_fx64_yt); the rows at or above it
    // (and non-finite or subnormal ones) add their instrumental products with binary64 atomics instead
    // (fx64_lane_outliers), so that one large entry of y does not coarsen every column's grid. Any y_t
    // gives the right sums; it only decides how fine the grid is. fx_word: the 2048 exponent bins, y_t (binary64), the counts,
    // max|a_j| (binary32 bits, rounded up). The fixed-point sums are exact integers, whatever their order.
    int16_t *sm_sh = reinterpret_cast<int16_t *>(smem_raw + sizeof(long long) * (size_t)S.n_instr);
    __shared__ double s_yt;
    if constexpr (FX64) {
        if (threadIdx.x == 0) s_yt = __longlong_as_double(*reinterpret_cast<const long long *>(fx_word + FX64_BINS));
        __syncthreads();
        const double yt = s_yt;
        const uint32_t *kmx = fx_word + FX64_BINS + 2, *amx = fx_word + FX64_BINS + 2 + S.n_instr;
        int bad = 0;
        for (int32_t i = threadIdx.x; i < S.n_instr; i += blockDim.x) {
            const double bound = (double)kmx[i] * (double)__uint_as_float(amx[i]) * yt;
            int sh = 0;
            if (bound > 0.0 && bound < INFINITY)
                sh = 61 - ilogb(bound);  // bound < 2^(ilogb + 1), so bound 2^sh <= 2^62
            else if (bound != 0.0)
                bad = 1;  // beyond the binary64 range: the column cannot be held in fixed point
            sm_sh[i] = (int16_t)max(min(sh, 30000), -30000);
        }
        bad = __syncthreads_or(bad);
        if (threadIdx.x == 0) s_bad = bad;
    }
    __syncthreads();
    // UNI: the instrumental group scale applies (the host chose this instance from the statistics)
    const bool ins_uni = ATT && UNI;
    const float ins_sc = ins_uni ? s_ins_sc : 1.f, ins_qsc = ins_uni ? s_ins_qsc : 1.f;

    const int lane = threadIdx.x & 31;
    AT *wbuf = wred[threadIdx.x >> 5];
    const int64_t gw = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t t0 = gw * tiles_per_warp;
    const int64_t t1 = min(S.n_tiles, t0 + tiles_per_warp);
    double *__restrict__ zi = z + S.instr0;
    double *__restrict__ z2i = BOTH ? z2 + S.instr0 : nullptr;
    AT gsum[MG], gsq[MG];
#pragma unroll
    for (int q = 0; q < MG; ++q) gsum[q] = gsq[q] = (AT)0;
    AT acc[NASTRO], acc2[NASTRO], sacc[NASTRO], sacc2[NASTRO];
#pragma unroll
    for (int j = 0; j < NASTRO; ++j) acc[j] = acc2[j] = sacc[j] = sacc2[j] = (AT)0;
    int64_t k = t0 < S.n_tiles ? S.first_star[t0] : 0;  // the star of the current run
    // a lane's R = 4 binary32 values of y in one 16-byte load where y is 16-byte aligned (the caller's
    // vector may be a view at any offset; measured 12.75 -> 12.65 ms on 5e8 rows)
    const bool y4 = (reinterpret_cast<uintptr_t>(y) & 15) == 0;
    for (int64_t t = t0; t < t1; ++t) {
        const uint8_t *tb = S.tiles + t * S.tile_bytes;
        // the one-pass form: the next tile of the warp's range into L2 (measured: 0.430 -> 0.422 ms
        // on 2e7 rows; in the grid-stride kernels and the two-pass forms it made the pass slower)
        if (ATT && t + 1 < t1) prefetch_l2(tb + S.tile_bytes, S.tile_bytes);
        int32_t ic[NINSTR][R];
        AT a[NASTRO][R], ai[NINSTR][R], ag[MG][R];
        if constexpr (SV) {
            // run-time sections: unconditional loads (absent slots read an attitude plane or the knot
            // plane) so that they schedule together; absent astrometric and global slots are zeroed
            // after the load, absent instrumental slots add nothing (their atomics are skipped)
#pragma unroll
            for (int j = 0; j < NINSTR; ++j) load_instr_or_knot<VT>(tb, G.npl, G.ni, S.iw16, j, ic[j]);
#pragma unroll
            for (int j = 0; j < NASTRO; ++j) {
                load_vals<VT, AT>(tb, j < G.na ? j : G.p_att, a[j]);
#pragma unroll
                for (int i = 0; i < R; ++i) a[j][i] = j < G.na ? a[j][i] : (AT)0;
            }
#pragma unroll
            for (int j = 0; j < NINSTR; ++j) load_vals<VT, AT>(tb, j < G.ni ? G.p_ins + j : G.p_att, ai[j]);
#pragma unroll
            for (int q = 0; q < MG; ++q) {
                load_vals<VT, AT>(tb, q < G.ng ? G.p_glob + q : G.p_att, ag[q]);
#pragma unroll
                for (int i = 0; i < R; ++i) ag[q][i] = q < G.ng ? ag[q][i] : (AT)0;
            }
        } else {
#pragma unroll
            for (int j = 0; j < NINSTR; ++j) load_instr<VT>(tb, S.iw16, j, ic[j]);
#pragma unroll
            for (int j = 0; j < NASTRO; ++j) load_vals<VT, AT>(tb, j, a[j]);
#pragma unroll
            for (int j = 0; j < NINSTR; ++j) load_vals<VT, AT>(tb, A_INS + j, ai[j]);
            load_vals<VT, AT>(tb, A_GLOB, ag[0]);
        }
        const int64_t r0 = t * T + lane * R;
        bool in[R];
        AT yr[R];
#pragma unroll
        for (int i = 0; i < R; ++i) in[i] = r0 + i < S.n_rows;
        if constexpr (!SQUARE && R == 4 && sizeof(UT) == 4) {
            if (y4 && r0 + R <= S.n_rows) {
                const float4 v = __ldg(reinterpret_cast<const float4 *>(y + r0));
                yr[0] = (AT)v.x;
                yr[1] = (AT)v.y;
                yr[2] = (AT)v.z;
                yr[3] = (AT)v.w;
            } else {
#pragma unroll
                for (int i = 0; i < R; ++i) yr[i] = in[i] ? (AT)y[r0 + i] : (AT)0;
            }
        } else {
#pragma unroll
            for (int i = 0; i < R; ++i) yr[i] = SQUARE ? (in[i] ? (AT)1 : (AT)0) : (in[i] ? (AT)y[r0 + i] : (AT)0);
        }
        // FX64: y of the rows whose instrumental products go to the fixed-point sums, 0 for the others
        // (|y| >= y_t, non-finite or subnormal y), which fx64_lane_outliers adds at once
        // (the tests on the bits of |y|: non-negative binary64 values, NaN above infinity, order as
        // integers, so the binary64 pipe stays with the products)
        AT yfx[R];
        unsigned omask = 0u;
        if constexpr (FX64) {
            const unsigned long long yt_bits = (unsigned long long)__double_as_longlong(s_yt);
#pragma unroll
            for (int i = 0; i < R; ++i) {
                const unsigned long long ya = (unsigned long long)__double_as_longlong((double)yr[i]) & 0x7fffffffffffffffull;
                const bool fx_row = ya < yt_bits && ya >= 0x0010000000000000ull;  // 2^-1022 <= |y| < y_t
                yfx[i] = fx_row ? yr[i] : (AT)0;
                if (!fx_row && ya != 0ull && in[i]) omask |= 1u << i;
            }
        }
        if constexpr (FX64 && R == 2) {
            if (omask) fx64_lane_outliers(zi, ai, ic, yr, omask);
        }
#pragma unroll
        for (int i = 0; i < R; ++i) {
#pragma unroll
            for (int j = 0; j < NINSTR; ++j) {
                const AT av = SQUARE ? ai[j][i] * ai[j][i] : ai[j][i];
                if constexpr (SV) {
                    // every contribution is formed from a valid column (an absent slot's index, read
                    // from the knot plane, is replaced by 0) and only the atomic is predicated, so the
                    // scale loads and products of the row overlap as in the standard instance
                    const bool on = j < G.ni && in[i];
                    const int32_t cj = j < G.ni ? ic[j][i] : 0;
                    if (FX) {
                        const int qv = __float2int_rn(av * yr[i] * sm_scale[cj]);
                        if (on) atomicAdd(reinterpret_cast<int *>(sm_ins) + cj, qv);
                    } else if (INSTR_SMEM) {
                        if (on) atomicAdd(sm_ins + cj, av * yr[i]);
                    } else {
                        if (on) atomicAdd(zi + cj, (double)(av * yr[i]));
                    }
                    if constexpr (BOTH) {
                        if (FX) {
                            const int qq = __float2int_rn(av * av * sm_qscale[cj]);
                            if (on) atomicAdd(reinterpret_cast<int *>(sm_sq) + cj, qq);
                        } else if (INSTR_SMEM) {
                            if (on) atomicAdd(sm_sq + cj, av * av);
                        } else {
                            if (on) atomicAdd(z2i + cj, (double)(av * av));
                        }
                    }
                    continue;
                }
                if (in[i]) {
                    if (FX64)  // straight-line: a row left to fx64_lane_outliers adds 0 here
                        atomicAdd(reinterpret_cast<unsigned long long *>(sm_ins) + ic[j][i],
                                  (unsigned long long)fx64_mulround((double)av, (double)yfx[i], sm_sh[ic[j][i]]));
                    else if (FX)
                        atomicAdd(reinterpret_cast<int *>(sm_ins) + ic[j][i],
                                  __float2int_rn(av * yr[i] * (ATT && ins_uni ? ins_sc : sm_scale[ic[j][i]])));
                    else if (INSTR_SMEM)
                        atomicAdd(sm_ins + ic[j][i], av * yr[i]);
                    else
                        atomicAdd(zi + ic[j][i], (double)(av * yr[i]));
                    if constexpr (BOTH) {
                        if (FX)
                            atomicAdd(reinterpret_cast<int *>(sm_sq) + ic[j][i],
                                      __float2int_rn(av * av * (ATT && ins_uni ? ins_qsc : sm_qscale[ic[j][i]])));
                        else if (INSTR_SMEM)
                            atomicAdd(sm_sq + ic[j][i], av * av);
                        else
                            atomicAdd(z2i + ic[j][i], (double)(av * av));
                    }
                }
            }
#pragma unroll
            for (int q = 0; q < MG; ++q) {
                const AT gv = SQUARE ? ag[q][i] * ag[q][i] : ag[q][i];
                gsum[q] = fma(gv, yr[i], gsum[q]);
                if constexpr (BOTH) gsq[q] = fma(gv, in[i] ? gv : (AT)0, gsq[q]);
            }
        }
        // astrometric part: does the whole tile belong to star k?
        const int64_t tile_end = min((t + 1) * T, S.n_rows);  // one past the tile's last row
        if constexpr (BOTH) {  // squares of padding rows (past n_rows) are masked here
#pragma unroll
            for (int i = 0; i < R; ++i)
                if (!in[i])
#pragma unroll
                    for (int j = 0; j < NASTRO; ++j) a[j][i] = (AT)0;
        }
        if (__ldg(S.star_ptr + k + 1) >= tile_end) {
#pragma unroll
            for (int i = 0; i < R; ++i)
#pragma unroll
                for (int j = 0; j < NASTRO; ++j) {
                    const AT av = SQUARE ? a[j][i] * a[j][i] : a[j][i];
                    acc[j] = fma(av, yr[i], acc[j]);
                    if constexpr (BOTH) sacc[j] = fma(av, av, sacc[j]);
                }
        } else {
            // the star of the tile's last row ends the next run
            const int64_t kn = star_of_row(S.star_ptr, S.first_star, t, tile_end - 1);
            int64_t sr[R];
            stars_of_rows<R>(S.star_ptr, S.first_star, t, r0, sr);
#pragma unroll
            for (int i = 0; i < R; ++i) {
#pragma unroll
                for (int j = 0; j < NASTRO; ++j) {
                    const AT av = SQUARE ? a[j][i] * a[j][i] : a[j][i];
                    const AT pv = av * yr[i];
                    const AT qv = BOTH ? av * av : (AT)0;
                    if (sr[i] == k) {
                        acc[j] += pv;
                        if constexpr (BOTH) sacc[j] += qv;
                    } else if (sr[i] == kn) {
                        acc2[j] += pv;
                        if constexpr (BOTH) sacc2[j] += qv;
                    } else if (in[i] && j < G.na) {
                        atomicAdd(z + (int64_t)G.na * sr[i] + j, (double)pv);
                        if constexpr (BOTH) atomicAdd(z2 + (int64_t)G.na * sr[i] + j, (double)qv);
                    }
                }
            }
            flush_astro_run(acc, k, wbuf, z, G.na);
            if constexpr (BOTH) flush_astro_run(sacc, k, wbuf, z2, G.na);
#pragma unroll
            for (int j = 0; j < NASTRO; ++j) {
                acc[j] = acc2[j];
                acc2[j] = (AT)0;
                sacc[j] = sacc2[j];
                sacc2[j] = (AT)0;
            }
            k = kn;
        }
        if constexpr (ATT) {
            // the 12 attitude products of each row into the block-private fixed-point columns
            // (after the rest of the tile: fewer registers live than with all planes loaded at once)
            int32_t knot[R];
            load_ints<R>(tb + NPAR * Tile<VT>::VBLK, 0, knot);
            int *acc_a = reinterpret_cast<int *>(sm_ins) + S.n_instr;
            int *accq_a = reinterpret_cast<int *>(sm_ins) + ncol + S.n_instr;
            const float sc_a = s_att_sc, qsc_a = s_att_qsc;
#pragma unroll
            for (int ax = 0; ax < NAXES; ++ax) {
                AT at[NPARAXIS][R];
#pragma unroll
                for (int j = 0; j < NPARAXIS; ++j) load_vals<VT, AT>(tb, A_ATT + NPARAXIS * ax + j, at[j]);
#pragma unroll
                for (int i = 0; i < R; ++i)
#pragma unroll
                    for (int j = 0; j < NPARAXIS; ++j) {
                        const int32_t col = ax * S.n_dfa + knot[i] + j;
                        const AT av = SQUARE ? at[j][i] * at[j][i] : at[j][i];
                        const int qv = __float2int_rn(av * yr[i] * sc_a);
                        if (in[i]) atomicAdd(acc_a + col, qv);
                        if constexpr (BOTH) {
                            const int qq = __float2int_rn(av * av * qsc_a);
                            if (in[i]) atomicAdd(accq_a + col, qq);
                        }
                    }
            }
        }
        if constexpr (ATTRED) {
            // the 12 attitude products of each row as three 16-byte reductions (one per axis) into the
            // window accumulators, which stay in L2 (aw[a][k][q] collects column k + q of axis a from the
            // rows starting at knot k; k_att_fold adds the windows into z)
            int32_t knot[R];
            load_ints<R>(tb + NPAR * Tile<VT>::VBLK, 0, knot);
#pragma unroll
            for (int ax = 0; ax < NAXES; ++ax) {
                AT at[NPARAXIS][R];
#pragma unroll
                for (int j = 0; j < NPARAXIS; ++j) load_vals<VT, AT>(tb, A_ATT + NPARAXIS * ax + j, at[j]);
#pragma unroll
                for (int i = 0; i < R; ++i) {
                    if (!in[i]) continue;
                    const int64_t wi = ((int64_t)ax * S.n_dfa + knot[i]) * 4;
                    AT q[NPARAXIS];
#pragma unroll
                    for (int j = 0; j < NPARAXIS; ++j) q[j] = SQUARE ? at[j][i] * at[j][i] : at[j][i];
                    red_add_v4(S.aw + wi, q[0] * yr[i], q[1] * yr[i], q[2] * yr[i], q[3] * yr[i]);
                    if constexpr (BOTH) red_add_v4(S.aw2 + wi, q[0] * q[0], q[1] * q[1], q[2] * q[2], q[3] * q[3]);
                }
            }
        }
    }
    if (t0 < t1) {
        flush_astro_run(acc, k, wbuf, z, G.na);
        if constexpr (BOTH) flush_astro_run(sacc, k, wbuf, z2, G.na);
    }
    __syncthreads();
    if (FX) {
        for (int32_t i = threadIdx.x; i < nsm; i += blockDim.x) {
            const int q = reinterpret_cast<const int *>(sm_ins)[i];
            if (q == 0) continue;
            const bool sq = BOTH && i >= ncol;
            const int32_t col = sq ? i - ncol : i;
            // column col of the block-private space: instrumental, or (ATT) attitude
            const bool ins = col < S.n_instr;
            const int64_t dst = ins ? S.instr0 + col : S.att0 + (col - S.n_instr);
            const float sc = !ins ? (sq ? s_att_qsc : s_att_sc)
                             : ATT && ins_uni ? (sq ? s_ins_qsc : s_ins_sc) : (sq ? sm_qscale[col] : sm_scale[col]);
            atomicAdd((sq ? z2 : z) + dst, (double)q / (double)sc);  // the scale is a power of two: exact
        }
        if (s_bad && threadIdx.x == 0) atomicAdd(S.n_instr ? zi : z + S.att0, (double)NAN);
    } else if (FX64) {
        for (int32_t i = threadIdx.x; i < S.n_instr; i += blockDim.x) {
            const long long q = reinterpret_cast<const long long *>(sm_ins)[i];
            if (q != 0) atomicAdd(zi + i, ldexp((double)q, -(int)sm_sh[i]));  // a power of two: exact
        }
        if (s_bad && threadIdx.x == 0) atomicAdd(zi, (double)NAN);
    } else {
        for (int32_t i = threadIdx.x; i < nsm; i += blockDim.x) {
            const AT v = sm_ins[i];
            if (v != (AT)0) atomicAdd(BOTH && i >= S.n_instr ? z2i + (i - S.n_instr) : zi + i, (double)v);
        }
    }
#pragma unroll
    for (int q = 0; q < MG; ++q) {
        if (q < S.n_glob) {  // the same for every thread of the block
            const double tot = block_sum((double)gsum[q], sm32);
            if (threadIdx.x == 0 && tot != 0.0) atomicAdd(z + S.glob0 + q, tot);
            if constexpr (BOTH) {
                const double tq = block_sum((double)gsq[q], sm32);
                if (threadIdx.x == 0 && tq != 0.0) atomicAdd(z2 + S.glob0 + q, tq);
            }
        }
    }
}

// The standard row's instance, and a section variant's (run-time geometry) with
// its registers capped for two resident blocks per SM, as the standard one has.
template <typename VT, typename UT, typename AT, bool INSTR_SMEM, int MODE, bool LSQR, bool FX = false,
          bool ATTRED = false>
__global__ void __launch_bounds__(256) k_aprod2_star(SysView<VT> S, const UT *__restrict__ y, double *__restrict__ z,
                                                     double *__restrict__ z2, const LsqrState *__restrict__ st,
                                                     int64_t tiles_per_warp, const uint32_t *__restrict__ fx_word,
                                                     int32_t fxs)
{
    aprod2_star_body<VT, UT, AT, INSTR_SMEM, MODE, LSQR, FX, false, false, false, ATTRED>(S, y, z, z2, st,
                                                                                        tiles_per_warp, fx_word, fxs);
}

// The binary64 star pass with int64 fixed-point instrumental sums (binary64 storage, standard row,
// products): NT threads a block, 256 where two blocks' sums fit an SM, else 512 (one block of 16 warps:
// the 20,000 columns' 200 KB of sums and shifts leave room for one block only). fx_word: the context's
// fx64_word (max |y| of this call, the per-column counts and bounds).
template <bool LSQR, int NT>
__global__ void __launch_bounds__(NT) k_aprod2_star_fx64(SysView<double> S, const double *__restrict__ y,
                                                         double *__restrict__ z, const LsqrState *__restrict__ st,
                                                         int64_t tiles_per_warp, const uint32_t *__restrict__ fx_word)
{
    aprod2_star_body<double, double, double, true, A2_PROD, LSQR, false, false, false, false, false, true, NT / 32>(
        S, y, z, nullptr, st, tiles_per_warp, fx_word, 0);
}

// The binary64 exponents of |y| over a sample of the rows (every 64th) into FX64_BINS bins (zero on
// entry), from which the fixed-point star pass picks the magnitude that all but about 1/1024 of the
// rows stay below; nothing once the solve has stopped (st)
__global__ void k_ybins64(const double *__restrict__ y, int64_t n, uint32_t *__restrict__ bins,
                          const LsqrState *__restrict__ st)
{
    __shared__ uint32_t hb[FX64_BINS];
    if (st && st->done) return;
    for (int i = threadIdx.x; i < FX64_BINS; i += blockDim.x) hb[i] = 0u;
    __syncthreads();
    const int64_t ns = (n + 63) / 64;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < ns; i += (int64_t)gridDim.x * blockDim.x)
        atomicAdd(hb + (int)((__double_as_longlong(y[64 * i]) >> 52) & 0x7ff), 1u);
    __syncthreads();
    for (int i = threadIdx.x; i < FX64_BINS; i += blockDim.x)
        if (hb[i]) atomicAdd(bins + i, hb[i]);
}

// z[att] += the window accumulators of the attitude reductions: column k of axis a collects
// aw[a][k - q][q] for q = 0..3 (the rows starting q knots before it), summed in binary64 in that fixed
// order; each window entry is read once and cleared for the next aprod 2. After the star pass, which
// also no longer needs the max |y| word: cleared here for the next aprod 2 (ymax_reset).
template <int MODE, bool LSQR>
__global__ void k_att_fold(SysView<float> S, double *__restrict__ z, double *__restrict__ z2,
                           const LsqrState *__restrict__ st, uint32_t *__restrict__ ymax_reset)
{
    if (LSQR && st->done) return;
    if (ymax_reset && blockIdx.x == 0 && threadIdx.x == 0) *ymax_reset = 0u;
    const int64_t nat = (int64_t)NAXES * S.n_dfa;
    for (int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; c < nat; c += (int64_t)gridDim.x * blockDim.x) {
        const int32_t k = (int32_t)(c % S.n_dfa);
        double s = 0.0, s2 = 0.0;
#pragma unroll
        for (int q = 0; q < NPARAXIS; ++q) {
            const int32_t k0 = k - q;  // the window starting at knot k0 (rows start at knots 0..n_dfa-4)
            if (k0 < 0 || k0 > S.n_dfa - NPARAXIS) continue;
            const int64_t wi = (c - q) * 4 + q;
            s += (double)S.aw[wi];
            S.aw[wi] = 0.f;
            if (MODE == A2_BOTH) {
                s2 += (double)S.aw2[wi];
                S.aw2[wi] = 0.f;
            }
        }
        if (s != 0.0) z[S.att0 + c] += s;
        if (MODE == A2_BOTH && s2 != 0.0) z2[S.att0 + c] += s2;
    }
}

// the window copy of the binary32 attitude unknowns, knot-major in 64-byte records:
// xw[4 k + a] = x[att0 + a n_dfa + k .. +3] (zero past the axis's end), xw[4 k + 3] unused, so that a
// row's axes 0 and 1 are one 32-byte load and axis 2 a 16-byte one (att_window_load)
__global__ void k_att_window(const float *__restrict__ x, int64_t att0, int32_t n_dfa, float4 *__restrict__ xw)
{
    const int64_t nat = (int64_t)NAXES * n_dfa;
    for (int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; c < nat; c += (int64_t)gridDim.x * blockDim.x) {
        const int32_t a = (int32_t)(c / n_dfa), k = (int32_t)(c % n_dfa);
        const float *xa = x + att0 + c;
        xw[4 * (int64_t)k + a] = make_float4(xa[0], k + 1 < n_dfa ? xa[1] : 0.f, k + 2 < n_dfa ? xa[2] : 0.f,
                                             k + 3 < n_dfa ? xa[3] : 0.f);
    }
}

template <typename VT, typename UT, typename AT, bool INSTR_SMEM, int MODE, bool LSQR, bool FX = false>
__global__ void __launch_bounds__(256, 2) k_aprod2_star_sv(SysView<VT> S, const UT *__restrict__ y,
                                                           double *__restrict__ z, double *__restrict__ z2,
                                                           const LsqrState *__restrict__ st, int64_t tiles_per_warp,
                                                           const uint32_t *__restrict__ fx_word, int32_t fxs)
{
    aprod2_star_body<VT, UT, AT, INSTR_SMEM, MODE, LSQR, FX, true>(S, y, z, z2, st, tiles_per_warp, fx_word, fxs);
}

// The star pass that also takes the attitude columns (binary32 fixed point, standard row): the whole
// aprod 2 in one pass over the row tiles, two blocks per SM as the plain star pass.
template <typename VT, int MODE, bool LSQR, bool UNI>
__global__ void __launch_bounds__(256, 2) k_aprod2_star_att(SysView<VT> S, const float *__restrict__ y,
                                                            double *__restrict__ z, double *__restrict__ z2,
                                                            const LsqrState *__restrict__ st, int64_t tiles_per_warp,
                                                            const uint32_t *__restrict__ fx_word, int32_t fxs)
{
    aprod2_star_body<VT, float, float, true, MODE, LSQR, true, false, true, UNI>(S, y, z, z2, st, tiles_per_warp,
                                                                                 fx_word, fxs);
}

// Add a warp's run sums of the 12 attitude columns of knot k (warp-collective).
template <typename AT>
__device__ __forceinline__ void flush_att_run(AT (&acc)[NAXES * NPARAXIS], int32_t k, int32_t n_dfa,
                                              double *__restrict__ zt)
{
    const int lane = threadIdx.x & 31;
#pragma unroll
    for (int j = 0; j < NAXES * NPARAXIS; ++j) {
        const AT t = warp_sum_t(acc[j]);
        if (lane == 0 && t != (AT)0) atomicAdd(zt + (j / NPARAXIS) * n_dfa + k + (j % NPARAXIS), (double)t);
        acc[j] = (AT)0;
    }
}

// aprod 2, attitude pass over the knot-ordered tiles: each warp owns the tiles
// [w*tiles_per_warp, (w+1)*tiles_per_warp); runs of equal knot are summed in
// registers and added once per run (one atomic add per column per run).
template <typename VT, typename UT, typename AT, int MODE, bool LSQR>
__global__ void __launch_bounds__(256) k_aprod2_att(SysView<VT> S, const UT *__restrict__ y,
                                                    double *__restrict__ z, double *__restrict__ z2,
                                                    const LsqrState *__restrict__ st, int64_t tiles_per_warp,
                                                    uint32_t *__restrict__ ymax_reset)
{
    constexpr bool SQUARE = MODE == A2_SQUARE;
    constexpr bool BOTH = MODE == A2_BOTH;
    constexpr int R = Tile<VT>::R;
    constexpr int T = Tile<VT>::T;
    constexpr int NA = NAXES * NPARAXIS;
    if (LSQR && st->done) return;
    // the star pass of this aprod 2 has finished: the max |y| word is free for the next one
    if (ymax_reset && blockIdx.x == 0 && threadIdx.x == 0) *ymax_reset = 0u;
    const int lane = threadIdx.x & 31;
    const int64_t gw = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t n = S.n_rows;
    const int64_t t0 = gw * tiles_per_warp;
    if (t0 >= S.n_tiles) return;
    const int64_t t1 = min(S.n_tiles, t0 + tiles_per_warp);
    const int32_t nk = S.n_dfa - 3;
    const int64_t p0 = t0 * T;
    // knot of p0: the largest k with knot_ptr[k] <= p0
    int32_t lo = 0, hi = nk - 1;
    while (lo < hi) {
        const int32_t mid = (lo + hi + 1) >> 1;
        if (S.knot_ptr[mid] <= p0)
            lo = mid;
        else
            hi = mid - 1;
    }
    int32_t k = lo;
    int64_t next = S.knot_ptr[k + 1];
    double *__restrict__ zt = z + S.att0;
    double *__restrict__ z2t = BOTH ? z2 + S.att0 : nullptr;
    AT acc[NA], sacc[BOTH ? NA : 1];
#pragma unroll
    for (int j = 0; j < NA; ++j) acc[j] = (AT)0;
#pragma unroll
    for (int j = 0; j < (BOTH ? NA : 1); ++j) sacc[j] = (AT)0;
    // the row permutation is read one tile ahead, so that the gather of y through it is issued
    // together with the tile's coefficient loads instead of after a dependent load
    int32_t pr_next[R];
    if (!SQUARE) load_ints<R>(S.atiles + t0 * Tile<VT>::ABYTES + NA * Tile<VT>::VBLK, 0, pr_next);
    for (int64_t t = t0; t < t1; ++t) {
        const uint8_t *tb = S.atiles + t * Tile<VT>::ABYTES;
        const int64_t q = t * T;
        const int64_t lastp = min(q + T - 1, n - 1);
        const int64_t pl = q + lane * R;
        int32_t pr[R];
#pragma unroll
        for (int i = 0; i < R; ++i) pr[i] = pr_next[i];
        AT yr[R];
        if (!SQUARE) {
#pragma unroll
            for (int i = 0; i < R; ++i) yr[i] = (pl + i < n) ? (AT)y[pr[i]] : (AT)0;
            if (t + 1 < t1) load_ints<R>(tb + Tile<VT>::ABYTES + NA * Tile<VT>::VBLK, 0, pr_next);
        }
        AT a[NA][R];
#pragma unroll
        for (int j = 0; j < NA; ++j) load_vals<VT, AT>(tb, j, a[j]);
        if (SQUARE) {
#pragma unroll
            for (int i = 0; i < R; ++i) yr[i] = (pl + i < n) ? (AT)1 : (AT)0;
#pragma unroll
            for (int j = 0; j < NA; ++j)
#pragma unroll
                for (int i = 0; i < R; ++i) a[j][i] = a[j][i] * a[j][i];
        } else {
            if constexpr (BOTH) {
#pragma unroll
                for (int i = 0; i < R; ++i)
                    if (pl + i >= n)
#pragma unroll
                        for (int j = 0; j < NA; ++j) a[j][i] = (AT)0;
            }
        }
        if (lastp < next) {  // every position of this tile is on knot k
#pragma unroll
            for (int j = 0; j < NA; ++j)
#pragma unroll
                for (int i = 0; i < R; ++i) {
                    acc[j] = fma(a[j][i], yr[i], acc[j]);
                    if constexpr (BOTH) sacc[j] = fma(a[j][i], a[j][i], sacc[j]);
                }
        } else {  // the tile crosses knot boundaries: add its products position by position
            flush_att_run(acc, k, S.n_dfa, zt);
            if constexpr (BOTH) flush_att_run(sacc, k, S.n_dfa, z2t);
#pragma unroll
            for (int i = 0; i < R; ++i) {
                const int64_t p = pl + i;
                if (p < n) {
                    int32_t kl = k;
                    while (S.knot_ptr[kl + 1] <= p) ++kl;
#pragma unroll
                    for (int j = 0; j < NA; ++j) {
                        const int64_t col = (j / NPARAXIS) * S.n_dfa + kl + (j % NPARAXIS);
                        const AT pv = a[j][i] * yr[i];
                        if (pv != (AT)0) atomicAdd(zt + col, (double)pv);
                        if constexpr (BOTH) {
                            const AT qv = a[j][i] * a[j][i];
                            if (qv != (AT)0) atomicAdd(z2t + col, (double)qv);
                        }
                    }
                }
            }
            while (S.knot_ptr[k + 1] <= lastp) ++k;
            next = S.knot_ptr[k + 1];
        }
    }
    flush_att_run(acc, k, S.n_dfa, zt);
    if constexpr (BOTH) flush_att_run(sacc, k, S.n_dfa, z2t);
}

// One LSQR iteration's two products in one pass over the row tiles (the binary32 inner solve of a
// wide attitude block, att_red). The Golub-Kahan step u_{i+1} = A v_i - alpha_i u_i depends on each
// row alone, so once a tile's new u is formed its contributions to A^T u_{i+1} can be added from the
// coefficients still in registers: the tile is read once instead of twice. The 1/beta_{i+1} of the
// normalised u is applied afterwards (k_colA takes z = A^T u unnormalised, with beta from the
// per-block sums of squares written here). Per tile: the aprod 1 part as k_aprod1 (attitude
// unknowns through the window copy), then the aprod 2 part as the star pass with the attitude
// reductions (astrometric runs in registers, instrumental sums in shared memory, the global column
// per block, the attitude products as three 16-byte reductions per row into the L2 windows).
// Each warp owns a contiguous range of tiles (the astrometric runs need them in order).
// (A form in which a warp takes each tile in two halves, each lane two rows with 8-byte loads, half
// the registers and two resident blocks per SM, ran 40% slower on 5e8 rows: 31.6 vs 22.7 ms.)
// LSQR: coef = -alpha/beta from the solver state (and nothing to do once it has stopped), the per-block
// sums of squares of the new u into part; otherwise coef_arg, and part may be null.
// XS: the block also keeps x of the instrumental columns in shared memory (after its sums), so that
// the 6 gathers a row makes of it are shared-memory loads: a random 4-byte gather from global memory
// costs the L1 data pipe about one pass per lane, and that pipe, not DRAM, bounds this pass.
template <bool INSTR_SMEM, bool LSQR, bool XS = false>
__device__ __forceinline__ void iter_fused_body(const SysView<float> &S, const float *__restrict__ x,
                                                float *__restrict__ y, double *__restrict__ z,
                                                const LsqrState *__restrict__ st, double *__restrict__ part,
                                                int64_t tiles_per_warp, float coef_arg)
{
    constexpr int R = Tile<float>::R;
    constexpr int T = Tile<float>::T;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    __shared__ double sm64[64];
    __shared__ float wred[8][NASTRO * WSTRIDE];
    if (LSQR && st->done) return;
    const float coef = LSQR ? (float)st->coef_u : coef_arg;
    static_assert(!XS || INSTR_SMEM, "x in shared memory follows the block's sums");
    float *sm_ins = reinterpret_cast<float *>(smem_raw);
    float *sm_xi = sm_ins + S.n_instr;
    if (INSTR_SMEM)
        for (int32_t i = threadIdx.x; i < S.n_instr; i += blockDim.x) sm_ins[i] = 0.f;
    if (XS)
        for (int32_t i = threadIdx.x; i < S.n_instr; i += blockDim.x) sm_xi[i] = __ldg(x + S.instr0 + i);
    __syncthreads();
    const int lane = threadIdx.x & 31;
    float *wbuf = wred[threadIdx.x >> 5];
    const int64_t gw = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t t0 = gw * tiles_per_warp;
    const int64_t t1 = min(S.n_tiles, t0 + tiles_per_warp);
    const float *__restrict__ xi = x + S.instr0;
    double *__restrict__ zi = z + S.instr0;
    const float xg = S.n_glob ? __ldg(x + S.glob0) : 0.f;
    float gsum = 0.f, ssq = 0.f;
    float acc[NASTRO], acc2[NASTRO];
#pragma unroll
    for (int j = 0; j < NASTRO; ++j) acc[j] = acc2[j] = 0.f;
    int64_t k = t0 < S.n_tiles ? S.first_star[t0] : 0;  // the star of the current astrometric run
    for (int64_t t = t0; t < t1; ++t) {
        const uint8_t *tb = S.tiles + t * S.tile_bytes;
        if (t + 1 < t1) prefetch_l2(tb + S.tile_bytes, S.tile_bytes);  // the warp's next tile into L2
        {
            int32_t kn[R];
            int32_t ic[NINSTR][R];
            float a[NPAR][R];
            load_ints<R>(tb + NPAR * Tile<float>::VBLK, 0, kn);
#pragma unroll
            for (int j = 0; j < NINSTR; ++j) load_instr<float>(tb, S.iw16, j, ic[j]);
#pragma unroll
            for (int j = 0; j < NPAR; ++j) load_vals<float, float>(tb, j, a[j]);
            const int64_t r0 = t * T + lane * R;
            int64_t sr[R];
            stars_of_rows<R>(S.star_ptr, S.first_star, t, r0, sr);
            bool in[R];
            float yr[R];
            // aprod 1: the new u of this lane's rows
#pragma unroll
            for (int i = 0; i < R; ++i) {
                const float *__restrict__ xa = x + NASTRO * sr[i];
                float v = a[0][i] * __ldg(xa);
#pragma unroll
                for (int j = 1; j < NASTRO; ++j) v = fmaf(a[j][i], __ldg(xa + j), v);
                float4 wv[NAXES];
                att_window_load(S.xw, kn[i], wv);
#pragma unroll
                for (int ax = 0; ax < NAXES; ++ax) {
                    const float4 w = wv[ax];
                    v = fmaf(a[A_ATT + NPARAXIS * ax + 0][i], w.x, v);
                    v = fmaf(a[A_ATT + NPARAXIS * ax + 1][i], w.y, v);
                    v = fmaf(a[A_ATT + NPARAXIS * ax + 2][i], w.z, v);
                    v = fmaf(a[A_ATT + NPARAXIS * ax + 3][i], w.w, v);
                }
#pragma unroll
                for (int j = 0; j < NINSTR; ++j) v = fmaf(a[A_INS + j][i], XS ? sm_xi[ic[j][i]] : __ldg(xi + ic[j][i]), v);
                v = fmaf(a[A_GLOB][i], xg, v);
                const int64_t r = r0 + i;
                in[i] = r < S.n_rows;
                float yn = 0.f;
                if (in[i]) {
                    yn = fmaf(coef, y[r], v);
                    y[r] = yn;
                    ssq = fmaf(yn, yn, ssq);
                }
                yr[i] = yn;
            }
            // aprod 2 with the new u: instrumental and global columns
#pragma unroll
            for (int i = 0; i < R; ++i) {
#pragma unroll
                for (int j = 0; j < NINSTR; ++j) {
                    if (!in[i]) continue;
                    if (INSTR_SMEM)
                        atomicAdd(sm_ins + ic[j][i], a[A_INS + j][i] * yr[i]);
                    else
                        atomicAdd(zi + ic[j][i], (double)(a[A_INS + j][i] * yr[i]));
                }
                gsum = fmaf(a[A_GLOB][i], yr[i], gsum);
            }
            // attitude columns: one 16-byte reduction per axis and row into the windows
#pragma unroll
            for (int ax = 0; ax < NAXES; ++ax)
#pragma unroll
                for (int i = 0; i < R; ++i) {
                    if (!in[i]) continue;
                    const int64_t wi = ((int64_t)ax * S.n_dfa + kn[i]) * 4;
                    red_add_v4(S.aw + wi, a[A_ATT + NPARAXIS * ax + 0][i] * yr[i],
                               a[A_ATT + NPARAXIS * ax + 1][i] * yr[i], a[A_ATT + NPARAXIS * ax + 2][i] * yr[i],
                               a[A_ATT + NPARAXIS * ax + 3][i] * yr[i]);
                }
            // astrometric columns: runs of the current star in registers (as the star pass)
            const int64_t part_end = min((t + 1) * T, S.n_rows);
            if (__ldg(S.star_ptr + k + 1) >= part_end) {
#pragma unroll
                for (int i = 0; i < R; ++i)
#pragma unroll
                    for (int j = 0; j < NASTRO; ++j) acc[j] = fmaf(a[j][i], yr[i], acc[j]);
            } else {
                const int64_t kl = star_of_row(S.star_ptr, S.first_star, t, part_end - 1);
#pragma unroll
                for (int i = 0; i < R; ++i) {
#pragma unroll
                    for (int j = 0; j < NASTRO; ++j) {
                        const float pv = a[j][i] * yr[i];
                        if (sr[i] == k)
                            acc[j] += pv;
                        else if (sr[i] == kl)
                            acc2[j] += pv;
                        else if (in[i])
                            atomicAdd(z + (int64_t)NASTRO * sr[i] + j, (double)pv);
                    }
                }
                flush_astro_run(acc, k, wbuf, z);
#pragma unroll
                for (int j = 0; j < NASTRO; ++j) {
                    acc[j] = acc2[j];
                    acc2[j] = 0.f;
                }
                k = kl;
            }
        }
    }
    if (t0 < t1) flush_astro_run(acc, k, wbuf, z);
    __syncthreads();
    if (INSTR_SMEM) {
        for (int32_t i = threadIdx.x; i < S.n_instr; i += blockDim.x) {
            const float v = sm_ins[i];
            if (v != 0.f) atomicAdd(zi + i, (double)v);
        }
    }
    const double2 tot = block_sum2((double)ssq, (double)gsum, sm64);
    if (threadIdx.x == 0) {
        if (part) part[blockIdx.x] = tot.x;
        if (S.n_glob && tot.y != 0.0) atomicAdd(z + S.glob0, tot.y);
    }
}

template <bool INSTR_SMEM, bool LSQR, bool XS>
__global__ void __launch_bounds__(256) k_iter_fused(SysView<float> S, const float *__restrict__ x,
                                                    float *__restrict__ y, double *__restrict__ z,
                                                    const LsqrState *__restrict__ st, double *__restrict__ part,
                                                    int64_t tiles_per_warp, float coef_arg)
{
    iter_fused_body<INSTR_SMEM, LSQR, XS>(S, x, y, z, st, part, tiles_per_warp, coef_arg);
}

// ---------------------------------------------------------------- launchers
static constexpr int kThreads = 256;
static constexpr size_t kSmemBudget = 100 * 1024;  // bytes of block-private accumulators
// the pass that sums products and squares together (the warm start's, once per solve) keeps its
// block-private accumulators in shared memory up to one block per SM
static constexpr size_t kSmemBudgetBoth = 200 * 1024;

template <typename KernelT>
static int persistent_blocks(const gsr_ctx *c, KernelT kern, size_t dyn_smem)
{
    int per_sm = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, kThreads, dyn_smem) != cudaSuccess || per_sm < 1)
        per_sm = 1;
    int64_t blocks = (int64_t)per_sm * c->sm_count;
    // no more warps than tiles, at least one block
    const int64_t max_blocks = (c->n_tiles + (kThreads / 32) - 1) / (kThreads / 32);
    if (blocks > max_blocks) blocks = max_blocks;
    if (blocks < 1) blocks = 1;
    if (blocks > MAX_PARTIALS) blocks = MAX_PARTIALS;
    return (int)blocks;
}

// Contiguous tile ranges for the aprod 2 passes: one range per warp of the
// resident grid, at least 8 tiles per warp.
template <typename KernelT>
static void tile_ranges(const gsr_ctx *c, KernelT kern, size_t dyn_smem, int64_t *per_warp, int64_t *blocks)
{
    int per_sm = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, kThreads, dyn_smem) != cudaSuccess || per_sm < 1)
        per_sm = 1;
    const int64_t wpb = kThreads / 32;
    const int64_t max_warps = (int64_t)per_sm * c->sm_count * wpb;
    int64_t per = (c->n_tiles + max_warps - 1) / max_warps;
    if (per < 8) per = 8;
    const int64_t warps = (c->n_tiles + per - 1) / per;
    *per_warp = per;
    *blocks = std::max<int64_t>((warps + wpb - 1) / wpb, 1);
}

template <typename VT, typename XT, typename UT, typename AT>
static cudaError_t aprod1_t(const gsr_ctx *c, const void *x, void *y, const LsqrState *st, double *part,
                            cudaStream_t s, int *grid_out)
{
    const SysView<VT> S = view<VT>(c);
    auto pick = [&](auto kern, size_t dyn) -> cudaError_t {
        if (dyn > 48 * 1024) {
            const cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)dyn);
            if (e != cudaSuccess) return e;
        }
        const int g = persistent_blocks(c, kern, dyn);
        if (grid_out) {
            *grid_out = g;
            return cudaSuccess;
        }
        if (!x || !y) return cudaErrorInvalidValue;
        // the inner iteration's star pass reads max |u| (fixed-point instrumental sums)
        uint32_t *ymax = (sizeof(AT) == 4 && st) ? fx_ymax(c) : nullptr;
        kern<<<g, kThreads, dyn, s>>>(S, (const XT *)x, (UT *)y, st, part, ymax);
        return cudaGetLastError();
    };
    if (c->sv) {  // a section variant (run-time section geometry)
        if (st) return pick(k_aprod1<VT, XT, UT, AT, true, true>, 0);
        return pick(k_aprod1<VT, XT, UT, AT, false, true>, 0);
    }
    if constexpr (sizeof(XT) == 4 && sizeof(VT) == 4) {
        if (att_window(c)) {
            // wide attitude block: the window copy of x first (a few MB, stays in L2), then one 16-byte
            // gather per axis and row; x of the instrumental columns in shared memory where it fits
            if (!grid_out) {
                if (!x) return cudaErrorInvalidValue;
                k_att_window<<<col_grid(c, (int64_t)NAXES * c->n_dfa), kThreads, 0, s>>>(
                    (const float *)x, S.att0, c->n_dfa, reinterpret_cast<float4 *>(c->xwin));
                const cudaError_t e = cudaGetLastError();
                if (e != cudaSuccess) return e;
            }
            const size_t dxs = sizeof(XT) * (size_t)c->n_instr;
            if (dxs <= kSmemBudget) {
                if (st) return pick(k_aprod1<VT, XT, UT, AT, true, false, true, true>, dxs);
                return pick(k_aprod1<VT, XT, UT, AT, false, false, true, true>, dxs);
            }
            if (st) return pick(k_aprod1<VT, XT, UT, AT, true, false, true>, 0);
            return pick(k_aprod1<VT, XT, UT, AT, false, false, true>, 0);
        }
    }
    if constexpr (sizeof(VT) == 8) {
        // binary64 storage (one block per SM at its registers): x of the instrumental columns in shared
        // memory where it fits
        const size_t dxs = sizeof(XT) * (size_t)c->n_instr;
        if (dxs <= kSmemBudgetBoth) {
            if (st) return pick(k_aprod1<VT, XT, UT, AT, true, false, false, true>, dxs);
            return pick(k_aprod1<VT, XT, UT, AT, false, false, false, true>, dxs);
        }
    }
    if (st) return pick(k_aprod1<VT, XT, UT, AT, true>, 0);
    return pick(k_aprod1<VT, XT, UT, AT, false>, 0);
}

static cudaError_t aprod1_dispatch(const gsr_ctx *c, const void *x, void *y, const LsqrState *st, double *part,
                                   cudaStream_t s, bool inner32, int *grid_out)
{
    if (inner32) return aprod1_t<float, float, float, float>(c, x, y, st, part, s, grid_out);
    if (c->prec == GSR_FP32) return aprod1_t<float, double, double, double>(c, x, y, st, part, s, grid_out);
    return aprod1_t<double, double, double, double>(c, x, y, st, part, s, grid_out);
}

int aprod1_grid(const gsr_ctx *c, bool inner32)
{
    int g = 1;
    static LsqrState dummy;  // only selects the LSQR kernel variant; never dereferenced on the host
    aprod1_dispatch(c, nullptr, nullptr, &dummy, nullptr, nullptr, inner32, &g);
    return g;
}

cudaError_t launch_aprod1(const gsr_ctx *c, const void *x, void *y, const LsqrState *st, double *part,
                          cudaStream_t s, bool inner32)
{
    if (c->n_rows == 0) return cudaSuccess;
    return aprod1_dispatch(c, x, y, st, part, s, inner32, nullptr);
}

template <typename VT, typename UT, typename AT, bool INS, int MODE, bool LS, bool FX, bool SV, bool ATTRED = false>
static cudaError_t aprod2_star_launch_t(const gsr_ctx *c, const void *y, double *x, double *x2, const LsqrState *st,
                                        cudaStream_t s)
{
    auto kern = SV ? k_aprod2_star_sv<VT, UT, AT, INS, MODE, LS, FX>
                   : k_aprod2_star<VT, UT, AT, INS, MODE, LS, FX, ATTRED>;
    const size_t dyn = INS ? sizeof(AT) * (size_t)c->n_instr * ((MODE == A2_BOTH ? 2 : 1) * (FX ? 2 : 1)) : 0;
    if (dyn > 48 * 1024) {
        cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)dyn);
        if (e != cudaSuccess) return e;
    }
    int64_t per = 0, blocks = 0;
    if (FX) {  // the partition the overflow bound was computed for
        per = c->fx_per;
        blocks = c->fx_blocks;
    } else {
        tile_ranges(c, kern, dyn, &per, &blocks);
    }
    kern<<<(unsigned)blocks, kThreads, dyn, s>>>(view<VT>(c), (const UT *)y, x, x2, st, per, c->fx_word, c->fx_nc);
    return cudaGetLastError();
}

// the whole binary32 aprod 2 as one star pass with the attitude columns (att_fused)
template <int MODE, bool LS>
static cudaError_t aprod2_fused_launch(const gsr_ctx *c, const void *y, double *x, double *x2, const LsqrState *st,
                                       cudaStream_t s)
{
    // one scale for the instrumental columns too when the statistics allow it (fx_uni)
    auto kern = c->fx_uni ? k_aprod2_star_att<float, MODE, LS, true> : k_aprod2_star_att<float, MODE, LS, false>;
    const int32_t ncol = c->n_instr + NAXES * c->n_dfa;
    // accumulators of every column (twice for products and squares), scales of the instrumental ones
    const size_t dyn = sizeof(float) * ((size_t)ncol + (size_t)c->n_instr) * (MODE == A2_BOTH ? 2 : 1);
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)dyn);
    if (e != cudaSuccess) return e;
    kern<<<(unsigned)c->fx_blocks, kThreads, dyn, s>>>(view<float>(c), (const float *)y, x, x2, st, c->fx_per,
                                                      c->fx_word, c->fx_nc);
    return cudaGetLastError();
}

template <typename VT, typename UT, typename AT, bool INS, int MODE, bool LS, bool FX = false>
static cudaError_t aprod2_star_launch(const gsr_ctx *c, const void *y, double *x, double *x2, const LsqrState *st,
                                      cudaStream_t s)
{
    if (c->sv) return aprod2_star_launch_t<VT, UT, AT, INS, MODE, LS, FX, true>(c, y, x, x2, st, s);
    return aprod2_star_launch_t<VT, UT, AT, INS, MODE, LS, FX, false>(c, y, x, x2, st, s);
}

// max |y| of a binary32 row vector into *ymax (binary32 bits; the word is zero on entry)
__global__ void k_absmax(const float *__restrict__ y, int64_t n, uint32_t *__restrict__ ymax)
{
    __shared__ float sm32[32];
    float m = 0.f;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        m = fmaxf(m, fabsf(__ldcs(y + i)));
    m = block_max(m, sm32);
    if (threadIdx.x == 0) atomicMax(ymax, __float_as_uint(m));
}

// y_t of the binary64 fixed-point star pass from the sampled exponent bins (one warp): the power of two
// 2^(E - 1023) with E >= 1 the smallest exponent whose bin and those above hold at most 1/1024 of the
// sample; into fx_word[FX64_BINS ..] as binary64. Nothing once the solve has stopped (st).
__global__ void k_fx64_yt(uint32_t *__restrict__ fx_word, const LsqrState *__restrict__ st)
{
    if (st && st->done) return;
    const uint32_t *bins = fx_word;
    const int l = threadIdx.x;  // lane l holds bins [64 l, 64 l + 64)
    uint32_t mine = 0u;
    for (int b = 0; b < 64; ++b) mine += bins[64 * l + b];
    uint32_t incl = mine;  // sum over lanes l..31 (inclusive suffix scan)
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const uint32_t t = __shfl_down_sync(0xffffffffu, incl, o);
        if (l + o < 32) incl += t;
    }
    const uint32_t total = __shfl_sync(0xffffffffu, incl, 0);
    const uint32_t lim = total >> 10;
    int cand = 0;  // the largest bin b of this lane with (bins b and above) > lim, if any
    uint32_t run = incl - mine;
    for (int b = 63; b >= 0; --b) {
        run += bins[64 * l + b];
        if (run > lim) {
            cand = 64 * l + b;
            break;
        }
    }
    const int E = max(__reduce_max_sync(0xffffffffu, cand) + 1, 1);
    if (l == 0) *reinterpret_cast<long long *>(fx_word + FX64_BINS) = __double_as_longlong(ldexp(1.0, min(E, 2046) - 1023));
}


// The partition of the binary64 fixed-point star pass (the statistics of layout.cu are taken over it):
// two blocks of 256 threads per SM where their shared memory fits, else one block of 512; contiguous
// ranges of at least 8 tiles a warp.
void fx64_partition(const gsr_ctx *c, int64_t *per, int64_t *blocks, int32_t *nt)
{
    const size_t dyn = fx64_smem(c);
    int per_sm = 0;
    auto k256 = k_aprod2_star_fx64<false, 256>;
    if (dyn > 48 * 1024) cudaFuncSetAttribute(k256, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)dyn);
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k256, 256, dyn) != cudaSuccess) per_sm = 0;
    cudaGetLastError();
    *nt = per_sm >= 2 ? 256 : 512;
    const int64_t wpb = *nt / 32;
    const int64_t max_warps = (per_sm >= 2 ? (int64_t)per_sm : 1) * c->sm_count * wpb;
    *per = std::max<int64_t>((c->n_tiles + max_warps - 1) / max_warps, 8);
    const int64_t warps = (c->n_tiles + *per - 1) / *per;
    *blocks = std::max<int64_t>((warps + wpb - 1) / wpb, 1);
}

// the binary64 star pass with the fixed-point instrumental sums: the sampled exponents of |y| and y_t
// first, then the pass over the partition its statistics were taken for
template <bool LS>
static cudaError_t aprod2_star_fx64_launch(const gsr_ctx *c, const double *y, double *x, const LsqrState *st,
                                           cudaStream_t s)
{
    cudaError_t e = cudaMemsetAsync(c->fx64_word, 0, sizeof(uint32_t) * FX64_BINS, s);
    if (e != cudaSuccess) return e;
    const int64_t ns = (c->n_rows + 63) / 64;
    k_ybins64<<<(unsigned)std::min<int64_t>(std::max<int64_t>((ns + kThreads - 1) / kThreads, 1), c->sm_count),
                kThreads, 0, s>>>(y, c->n_rows, c->fx64_word, st);
    k_fx64_yt<<<1, 32, 0, s>>>(c->fx64_word, st);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    const size_t dyn = fx64_smem(c);
    auto kern = c->fx64_nt == 256 ? k_aprod2_star_fx64<LS, 256> : k_aprod2_star_fx64<LS, 512>;
    if (dyn > 48 * 1024 &&
        (e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)dyn)) != cudaSuccess)
        return e;
    kern<<<(unsigned)c->fx64_blocks, (unsigned)c->fx64_nt, dyn, s>>>(view<double>(c), y, x, st, c->fx64_per,
                                                                    c->fx64_word);
    return cudaGetLastError();
}

// the binary32 aprod 2 of a wide attitude block (att_red): one star pass whose attitude products go to the
// window accumulators by vector reductions, then the fold into z (which also clears max |y|)
template <int MODE, bool LS>
static cudaError_t aprod2_red_t(const gsr_ctx *c, const void *y, double *x, double *x2, const LsqrState *st,
                                cudaStream_t s)
{
    cudaError_t e = cudaSuccess;
    const bool fx = c->fx_bits > 0 && (MODE != A2_BOTH || 4 * sizeof(float) * (size_t)c->n_instr <= kSmemBudget);
    if (fx) {
        if (MODE != A2_SQUARE && !LS) {
            k_absmax<<<col_grid(c, c->n_rows), kThreads, 0, s>>>((const float *)y, c->n_rows, fx_ymax(c));
            if ((e = cudaGetLastError()) != cudaSuccess) return e;
        }
        e = aprod2_star_launch_t<float, float, float, true, MODE, LS, true, false, true>(c, y, x, x2, st, s);
    } else if (sizeof(float) * (size_t)c->n_instr * (MODE == A2_BOTH ? 2 : 1) <=
               (MODE == A2_BOTH ? kSmemBudgetBoth : kSmemBudget)) {
        e = aprod2_star_launch_t<float, float, float, true, MODE, LS, false, false, true>(c, y, x, x2, st, s);
    } else {
        e = aprod2_star_launch_t<float, float, float, false, MODE, LS, false, false, true>(c, y, x, x2, st, s);
    }
    if (e != cudaSuccess) return e;
    k_att_fold<MODE, LS><<<col_grid(c, (int64_t)NAXES * c->n_dfa), kThreads, 0, s>>>(
        view<float>(c), x, x2, st, fx && MODE != A2_SQUARE ? fx_ymax(c) : nullptr);
    return cudaGetLastError();
}

template <typename VT, typename UT, typename AT, int MODE, bool LS>
static cudaError_t aprod2_t(const gsr_ctx *c, const void *y, double *x, double *x2, const LsqrState *st,
                            cudaStream_t s)
{
    if (LS != (st != nullptr)) return cudaErrorInvalidValue;  // the LSQR variants read the solver state
    if (MODE != A2_SQUARE && !y) return cudaErrorInvalidValue;
    if (MODE == A2_BOTH && !x2) return cudaErrorInvalidValue;
    cudaError_t e = cudaSuccess;
    constexpr bool F32 = sizeof(AT) == 4;
    if constexpr (F32 && sizeof(VT) == 4) {
        if (att_red(c)) return aprod2_red_t<MODE, LS>(c, y, x, x2, st, s);
        if (att_fused(c)) {
            // one pass: the star pass takes the attitude columns too (no attitude pass); max |y| comes
            // from the LSQR aprod 1 of the same iteration (the LSQR colA clears it for the next one),
            // else from a pass over y here, cleared after the star pass
            if (MODE != A2_SQUARE && !LS) {
                k_absmax<<<col_grid(c, c->n_rows), kThreads, 0, s>>>((const float *)y, c->n_rows, fx_ymax(c));
                if ((e = cudaGetLastError()) != cudaSuccess) return e;
            }
            if ((e = aprod2_fused_launch<MODE, LS>(c, y, x, x2, st, s)) != cudaSuccess) return e;
            if (MODE != A2_SQUARE && !LS) e = cudaMemsetAsync(fx_ymax(c), 0, sizeof(uint32_t), s);
            return e;
        }
    }
    // the combined pass needs twice the shared words; it keeps binary32 atomics when they do not fit
    const bool fx = F32 && c->fx_bits > 0 &&
                    (MODE != A2_BOTH || 4 * sizeof(float) * (size_t)c->n_instr <= kSmemBudget);
    bool fx64 = false;
    if constexpr (sizeof(VT) == 8 && MODE == A2_PROD) fx64 = star_fx64(c);
    if (fx64) {
        // binary64 storage: int64 fixed-point instrumental sums (integer operations and atomics, off
        // the binary64 pipe that the products keep busy)
        if constexpr (sizeof(VT) == 8 && MODE == A2_PROD) e = aprod2_star_fx64_launch<LS>(c, (const double *)y, x, st, s);
    } else if (fx) {
        // fixed-point instrumental sums: max |y| comes from the LSQR aprod 1 of the same iteration,
        // else from a pass over y here
        if (MODE != A2_SQUARE && !LS) {
            k_absmax<<<col_grid(c, c->n_rows), kThreads, 0, s>>>((const float *)y, c->n_rows, fx_ymax(c));
            if ((e = cudaGetLastError()) != cudaSuccess) return e;
        }
        if constexpr (F32) e = aprod2_star_launch<VT, UT, AT, true, MODE, LS, true>(c, y, x, x2, st, s);
    } else if (sizeof(AT) * (size_t)c->n_instr * (MODE == A2_BOTH ? 2 : 1) <=
               (MODE == A2_BOTH || sizeof(VT) == 8 ? kSmemBudgetBoth : kSmemBudget)) {
        // binary64 storage: up to one block per SM's worth of shared sums (on 1e8 rows with 20,000
        // instrumental columns, 160 KB of shared binary64 sums at one block per SM ran 8.49 ms against
        // 10.20 ms for global binary64 atomics at two blocks per SM; with binary32 storage the same
        // change made the binary64 products slower, 53.4 -> 59.4 ms on 5e8 rows)
        e = aprod2_star_launch<VT, UT, AT, true, MODE, LS>(c, y, x, x2, st, s);
    } else {
        e = aprod2_star_launch<VT, UT, AT, false, MODE, LS>(c, y, x, x2, st, s);
    }
    if (e != cudaSuccess) return e;
    // attitude pass (resets the max |y| word after a fixed-point star pass) over the knot-ordered copy,
    // which the caller built (ensure_att_layout)
    if (!c->atiles || !c->att_valid) return cudaErrorNotReady;
    auto kern = k_aprod2_att<VT, UT, AT, MODE, LS>;
    int64_t per = 0, blocks = 0;
    tile_ranges(c, kern, 0, &per, &blocks);
    kern<<<(unsigned)blocks, kThreads, 0, s>>>(view<VT>(c), (const UT *)y, x, x2, st, per,
                                               fx && MODE != A2_SQUARE ? fx_ymax(c) : nullptr);
    return cudaGetLastError();
}

cudaError_t launch_aprod2(const gsr_ctx *c, const void *y, double *x, bool square, const LsqrState *st,
                          cudaStream_t s, bool inner32)
{
    if (c->n_rows == 0) return cudaSuccess;
    if (inner32) {
        if (square) return aprod2_t<float, float, float, A2_SQUARE, false>(c, y, x, nullptr, nullptr, s);
        if (st) return aprod2_t<float, float, float, A2_PROD, true>(c, y, x, nullptr, st, s);
        return aprod2_t<float, float, float, A2_PROD, false>(c, y, x, nullptr, nullptr, s);
    }
    if (c->prec == GSR_FP32) {
        if (square) return aprod2_t<float, double, double, A2_SQUARE, false>(c, y, x, nullptr, nullptr, s);
        if (st) return aprod2_t<float, double, double, A2_PROD, true>(c, y, x, nullptr, st, s);
        return aprod2_t<float, double, double, A2_PROD, false>(c, y, x, nullptr, nullptr, s);
    }
    if (square) return aprod2_t<double, double, double, A2_SQUARE, false>(c, y, x, nullptr, nullptr, s);
    if (st) return aprod2_t<double, double, double, A2_PROD, true>(c, y, x, nullptr, st, s);
    return aprod2_t<double, double, double, A2_PROD, false>(c, y, x, nullptr, nullptr, s);
}

// y <- coef y (binary32)
__global__ void k_scale_f32(float *__restrict__ y, float coef, int64_t n)
{
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        y[i] *= coef;
}

// y <- A x + coef y, then z += A^T y with the new y (binary32 storage and products): the fused pass when
// the context's form allows it, else the two products after scaling y
cudaError_t launch_aprod12_f32(const gsr_ctx *c, const float *x, float *y, double *z, float coef, cudaStream_t s)
{
    if (c->n_rows == 0) return cudaSuccess;
    if (att_red(c) && att_window(c)) return launch_iter_fused(c, x, y, z, nullptr, nullptr, s, nullptr, coef);
    cudaError_t e = cudaSuccess;
    if (coef != 1.f) {
        k_scale_f32<<<col_grid(c, c->n_rows), kThreads, 0, s>>>(y, coef, c->n_rows);
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
    }
    if ((e = launch_aprod1(c, x, y, nullptr, nullptr, s, true)) != cudaSuccess) return e;
    return launch_aprod2(c, y, z, false, nullptr, s, true);
}

// The fused iteration pass of a wide attitude block (k_iter_fused): the window copy of p v, the pass,
// the fold of the attitude windows into z. grid_out: only the pass's block count (its partials).
cudaError_t launch_iter_fused(const gsr_ctx *c, const float *pv, float *u, double *z, const LsqrState *st,
                              double *part, cudaStream_t s, int *grid_out, float coef)
{
    const bool ins = sizeof(float) * (size_t)c->n_instr <= kSmemBudget;
    // the instrumental x beside the sums where both fit (the pass runs one block per SM either way)
    const bool xs = ins && 2 * sizeof(float) * (size_t)c->n_instr <= kSmemBudgetBoth;
    auto kern = st ? (xs ? k_iter_fused<true, true, true> : ins ? k_iter_fused<true, true, false>
                                                                : k_iter_fused<false, true, false>)
                   : (xs ? k_iter_fused<true, false, true> : ins ? k_iter_fused<true, false, false>
                                                                 : k_iter_fused<false, false, false>);
    const size_t dyn = (xs ? 2 : ins ? 1 : 0) * sizeof(float) * (size_t)c->n_instr;
    if (dyn > 48 * 1024) {
        const cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)dyn);
        if (e != cudaSuccess) return e;
    }
    int64_t per = 0, blocks = 0;
    tile_ranges(c, kern, dyn, &per, &blocks);
    if (grid_out) {
        *grid_out = (int)blocks;
        return cudaSuccess;
    }
    if (!att_red(c) || !att_window(c)) return cudaErrorInvalidValue;
    const SysView<float> S = view<float>(c);
    k_att_window<<<col_grid(c, (int64_t)NAXES * c->n_dfa), kThreads, 0, s>>>(pv, S.att0, c->n_dfa,
                                                                           reinterpret_cast<float4 *>(c->xwin));
    kern<<<(unsigned)blocks, kThreads, dyn, s>>>(S, pv, u, z, st, part, per, coef);
    if (st)
        k_att_fold<A2_PROD, true><<<col_grid(c, (int64_t)NAXES * c->n_dfa), kThreads, 0, s>>>(S, z, nullptr, st,
                                                                                            nullptr);
    else
        k_att_fold<A2_PROD, false><<<col_grid(c, (int64_t)NAXES * c->n_dfa), kThreads, 0, s>>>(S, z, nullptr,
                                                                                             nullptr, nullptr);
    return cudaGetLastError();
}

cudaError_t launch_aprod2_both(const gsr_ctx *c, const void *y, double *x, double *sq, cudaStream_t s, bool inner32)
{
    if (c->n_rows == 0) return cudaSuccess;
    if (inner32) return aprod2_t<float, float, float, A2_BOTH, false>(c, y, x, sq, nullptr, s);
    if (c->prec == GSR_FP32) return aprod2_t<float, double, double, A2_BOTH, false>(c, y, x, sq, nullptr, s);
    return aprod2_t<double, double, double, A2_BOTH, false>(c, y, x, sq, nullptr, s);
}

}  // namespace gsr
