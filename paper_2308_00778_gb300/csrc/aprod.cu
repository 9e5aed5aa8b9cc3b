// aprod.cu -- aprod 1 (y += A x, Eq. 2) and aprod 2 (x += A^T y, Eq. 3) on SoA planes.
//
// Both kernels are persistent grids with one warp per star: the rows of a star
// are contiguous (the block-diagonal astrometric part, Sec. 2), so each warp
// streams 32 consecutive rows per step with coalesced loads of the 24 value
// planes, the knot plane and the 6 instrumental planes.
//
// aprod 1: the 5 astrometric unknowns of the star are loaded once per star
// (broadcast), the 12 attitude and 6 instrumental unknowns are gathered
// through the read-only cache, and each lane writes its row's result. In the
// LSQR form it computes u <- A (p v) + coef * u and emits per-block sums of
// squares of the new u (the norm beta).
//
// Every kernel is templated on the stored value type VT, the type of the
// gathered / streamed vectors (XT for x in aprod 1, UT for the row vector) and
// the arithmetic type AT: binary64 for the plain solver (on FP64- or
// FP32-stored values) and binary32 throughout for the inner solve of the
// mixed-precision solver. Column accumulators (z) are always binary64.
//
// aprod 2 runs as two passes. The star-ordered pass reads the astrometric,
// instrumental and global coefficients: the astrometric part is a per-star
// register accumulation and one warp reduction per star, written without
// atomics (one warp owns a star); instrumental products go to block-private
// shared-memory accumulators flushed once per block (global atomic adds when
// n_instr is too large); the global column is reduced per block and added
// once per block (the two-stage reduction of the paper's global kernels,
// Sec. 4.2, folded into one pass). The attitude pass reads the knot-ordered
// copy of the 12 attitude coefficients (layout.cu) and gathers y through the
// row permutation: runs of equal knot are summed in registers and added once
// per run, instead of 12 atomic adds per row.
#include "gsr_internal.cuh"

namespace gsr {

template <typename T>
__device__ __forceinline__ T ld_stream(const T *p)
{
    return __ldcs(p);
}

template <typename T>
__device__ __forceinline__ T warp_sum_t(T v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// STAGE: the attitude and instrumental parts of x (3 n_dfa + n_instr values)
// are copied into shared memory once per block; the per-row gathers then hit
// shared memory instead of issuing scattered L1 requests.
template <typename VT, typename XT, typename UT, typename AT, bool LSQR, bool STAGE>
__global__ void __launch_bounds__(256) k_aprod1(SysView<VT> S, const XT *__restrict__ x, UT *__restrict__ y,
                                                const LsqrState *__restrict__ st, double *__restrict__ part)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
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
    if (STAGE) {
        XT *sx = reinterpret_cast<XT *>(smem_raw);
        const int32_t n_att = NAXES * S.n_dfa, n_st = n_att + S.n_instr;
        for (int32_t i = threadIdx.x; i < n_st; i += blockDim.x) sx[i] = x[S.att0 + i];
        __syncthreads();
        xt = sx;
        xi = sx + n_att;
    }
    const AT xg = S.n_glob ? (AT)__ldg(x + S.glob0) : (AT)0;
    AT ssq = (AT)0;
    for (int64_t s = gw; s < S.n_stars; s += nw) {
        const int64_t r0 = S.star_ptr[s], r1 = S.star_ptr[s + 1];
        const XT *__restrict__ xa = x + NASTRO * s;
        const AT xa0 = (AT)__ldg(xa + 0), xa1 = (AT)__ldg(xa + 1), xa2 = (AT)__ldg(xa + 2),
                 xa3 = (AT)__ldg(xa + 3), xa4 = (AT)__ldg(xa + 4);
        for (int64_t r = r0 + lane; r < r1; r += 32) {
            AT a[NPAR];
#pragma unroll
            for (int j = 0; j < NPAR; ++j) a[j] = (AT)ld_stream(S.val + j * S.plane + r);
            const int32_t k = ld_stream(S.knot + r);
            int32_t ic[NINSTR];
#pragma unroll
            for (int j = 0; j < NINSTR; ++j) ic[j] = ld_stream(S.instr + j * S.plane + r);
            AT sum = a[0] * xa0;
            sum = fma(a[1], xa1, sum);
            sum = fma(a[2], xa2, sum);
            sum = fma(a[3], xa3, sum);
            sum = fma(a[4], xa4, sum);
#pragma unroll
            for (int ax = 0; ax < NAXES; ++ax) {
                const XT *xk = xt + (int64_t)ax * S.n_dfa + k;
#pragma unroll
                for (int j = 0; j < NPARAXIS; ++j) sum = fma(a[NASTRO + NPARAXIS * ax + j], (AT)xk[j], sum);
            }
#pragma unroll
            for (int j = 0; j < NINSTR; ++j) sum = fma(a[17 + j], (AT)xi[ic[j]], sum);
            sum = fma(a[23], xg, sum);
            AT yn;
            if (LSQR) {
                yn = fma(coef, (AT)y[r], sum);
                ssq = fma(yn, yn, ssq);
            } else {
                yn = (AT)y[r] + sum;
            }
            y[r] = (UT)yn;
        }
    }
    if (LSQR) {
        const double t = block_sum((double)ssq, sm32);
        if (threadIdx.x == 0) part[blockIdx.x] = t;
    }
}

// aprod 2, star-ordered pass: astrometric (per-star warp reduction, no atomics),
// instrumental (block-private shared-memory accumulators, or global atomics
// when n_instr is too large) and global (block reduction) parts.
template <typename VT, typename UT, typename AT, bool INSTR_SMEM, bool SQUARE, bool LSQR>
__global__ void __launch_bounds__(256) k_aprod2_star(SysView<VT> S, const UT *__restrict__ y,
                                                     double *__restrict__ z, const LsqrState *__restrict__ st)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    __shared__ double sm32[32];
    if (LSQR && st->done) return;
    AT *sm_ins = reinterpret_cast<AT *>(smem_raw);
    const int32_t nsm = INSTR_SMEM ? S.n_instr : 0;
    for (int32_t i = threadIdx.x; i < nsm; i += blockDim.x) sm_ins[i] = (AT)0;
    __syncthreads();

    const int lane = threadIdx.x & 31;
    const int64_t gw = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
    double *__restrict__ zi = z + S.instr0;
    AT gsum = (AT)0;
    for (int64_t s = gw; s < S.n_stars; s += nw) {
        const int64_t r0 = S.star_ptr[s], r1 = S.star_ptr[s + 1];
        AT acc[NASTRO] = {(AT)0, (AT)0, (AT)0, (AT)0, (AT)0};
        for (int64_t r = r0 + lane; r < r1; r += 32) {
            AT a[NASTRO], ai[NINSTR];
#pragma unroll
            for (int j = 0; j < NASTRO; ++j) a[j] = (AT)ld_stream(S.val + j * S.plane + r);
#pragma unroll
            for (int j = 0; j < NINSTR; ++j) ai[j] = (AT)ld_stream(S.val + (17 + j) * S.plane + r);
            AT ag = (AT)ld_stream(S.val + 23 * S.plane + r);
            int32_t ic[NINSTR];
#pragma unroll
            for (int j = 0; j < NINSTR; ++j) ic[j] = ld_stream(S.instr + j * S.plane + r);
            AT yr;
            if (SQUARE) {
                yr = (AT)1;
#pragma unroll
                for (int j = 0; j < NASTRO; ++j) a[j] = a[j] * a[j];
#pragma unroll
                for (int j = 0; j < NINSTR; ++j) ai[j] = ai[j] * ai[j];
                ag = ag * ag;
            } else {
                yr = (AT)y[r];
            }
#pragma unroll
            for (int j = 0; j < NASTRO; ++j) acc[j] = fma(a[j], yr, acc[j]);
#pragma unroll
            for (int j = 0; j < NINSTR; ++j) {
                const AT pr = ai[j] * yr;
                if (INSTR_SMEM)
                    atomicAdd(sm_ins + ic[j], pr);
                else
                    atomicAdd(zi + ic[j], (double)pr);
            }
            gsum = fma(ag, yr, gsum);
        }
#pragma unroll
        for (int j = 0; j < NASTRO; ++j) acc[j] = warp_sum_t(acc[j]);
        if (lane < NASTRO) {
            AT mine = acc[0];
#pragma unroll
            for (int j = 1; j < NASTRO; ++j) mine = (lane == j) ? acc[j] : mine;
            z[NASTRO * s + lane] += (double)mine;
        }
    }
    __syncthreads();
    for (int32_t i = threadIdx.x; i < nsm; i += blockDim.x) {
        const AT v = sm_ins[i];
        if (v != (AT)0) atomicAdd(zi + i, (double)v);
    }
    if (S.n_glob) {
        const double t = block_sum((double)gsum, sm32);
        if (threadIdx.x == 0 && t != 0.0) atomicAdd(z + S.glob0, t);
    }
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

// aprod 2, attitude pass over the knot-ordered copy: each warp owns a
// contiguous range of positions; runs of equal knot are summed in registers
// and added once per run (one atomic add per column per run).
template <typename VT, typename UT, typename AT, bool SQUARE, bool LSQR>
__global__ void __launch_bounds__(256) k_aprod2_att(SysView<VT> S, const UT *__restrict__ y,
                                                    double *__restrict__ z, const LsqrState *__restrict__ st,
                                                    int64_t per_warp)
{
    if (LSQR && st->done) return;
    const int lane = threadIdx.x & 31;
    const int64_t gw = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t n = S.n_rows;
    const int64_t p0 = gw * per_warp;
    if (p0 >= n) return;
    const int64_t p1 = min(n, p0 + per_warp);
    const int32_t nk = S.n_dfa - 3;
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
    AT acc[NAXES * NPARAXIS];
#pragma unroll
    for (int j = 0; j < NAXES * NPARAXIS; ++j) acc[j] = (AT)0;
    for (int64_t q = p0; q < p1; q += 32) {
        const int64_t i = q + lane;
        const bool active = i < p1;
        const int64_t last = min(q + 31, p1 - 1);
        AT a[NAXES * NPARAXIS];
        AT yr = (AT)0;
        if (active) {
#pragma unroll
            for (int j = 0; j < NAXES * NPARAXIS; ++j) a[j] = (AT)ld_stream(S.att_k + j * S.plane + i);
            if (SQUARE) {
                yr = (AT)1;
#pragma unroll
                for (int j = 0; j < NAXES * NPARAXIS; ++j) a[j] = a[j] * a[j];
            } else {
                yr = (AT)y[ld_stream(S.perm + i)];
            }
        }
        if (last < next) {  // every position of this step is on knot k
            if (active) {
#pragma unroll
                for (int j = 0; j < NAXES * NPARAXIS; ++j) acc[j] = fma(a[j], yr, acc[j]);
            }
        } else {  // the step crosses knot boundaries
            flush_att_run(acc, k, S.n_dfa, zt);
            int32_t kl = k;
            if (active) {
                while (S.knot_ptr[kl + 1] <= i) ++kl;
#pragma unroll
                for (int j = 0; j < NAXES * NPARAXIS; ++j)
                    atomicAdd(zt + (j / NPARAXIS) * S.n_dfa + kl + (j % NPARAXIS), (double)(a[j] * yr));
            }
            k = __shfl_sync(0xffffffffu, kl, (int)(last - q));
            next = S.knot_ptr[k + 1];
        }
    }
    flush_att_run(acc, k, S.n_dfa, zt);
}

// ---------------------------------------------------------------- launchers
static constexpr int kThreads = 256;
static constexpr size_t kSmemBudget = 100 * 1024;  // bytes of block-private accumulators

template <typename KernelT>
static int persistent_blocks(const gsr_ctx *c, KernelT kern, size_t dyn_smem)
{
    int per_sm = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, kThreads, dyn_smem) != cudaSuccess || per_sm < 1)
        per_sm = 1;
    int64_t blocks = (int64_t)per_sm * c->sm_count;
    // no more warps than stars, at least one block
    const int64_t max_blocks = (c->n_stars + (kThreads / 32) - 1) / (kThreads / 32);
    if (blocks > max_blocks) blocks = max_blocks;
    if (blocks < 1) blocks = 1;
    if (blocks > MAX_PARTIALS) blocks = MAX_PARTIALS;
    return (int)blocks;
}

// bytes of shared memory that staging the gathered part of x needs (0 = too large, gather from L1)
static constexpr size_t kStageBudget = 160 * 1024;

template <typename XT>
static size_t stage_bytes(const gsr_ctx *c)
{
    const size_t b = sizeof(XT) * ((size_t)NAXES * c->n_dfa + (size_t)c->n_instr);
    return b <= kStageBudget ? b : 0;
}

template <typename VT, typename XT, typename UT, typename AT>
static cudaError_t aprod1_t(const gsr_ctx *c, const void *x, void *y, const LsqrState *st, double *part,
                            cudaStream_t s, int *grid_out)
{
    const SysView<VT> S = view<VT>(c);
    const size_t dyn = stage_bytes<XT>(c);
    auto pick = [&](auto kern) -> cudaError_t {
        if (dyn > 48 * 1024) {
            cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)dyn);
            if (e != cudaSuccess) return e;
        }
        const int g = persistent_blocks(c, kern, dyn);
        if (grid_out) {
            *grid_out = g;
            return cudaSuccess;
        }
        if (!x || !y) return cudaErrorInvalidValue;
        kern<<<g, kThreads, dyn, s>>>(S, (const XT *)x, (UT *)y, st, part);
        return cudaGetLastError();
    };
    if (st) {
        if (dyn) return pick(k_aprod1<VT, XT, UT, AT, true, true>);
        return pick(k_aprod1<VT, XT, UT, AT, true, false>);
    }
    if (dyn) return pick(k_aprod1<VT, XT, UT, AT, false, true>);
    return pick(k_aprod1<VT, XT, UT, AT, false, false>);
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

template <typename VT, typename UT, typename AT, bool INS, bool SQ, bool LS>
static cudaError_t aprod2_star_launch(const gsr_ctx *c, const void *y, double *x, const LsqrState *st,
                                      cudaStream_t s)
{
    auto kern = k_aprod2_star<VT, UT, AT, INS, SQ, LS>;
    const size_t dyn = INS ? sizeof(AT) * (size_t)c->n_instr : 0;
    if (dyn > 48 * 1024) {
        cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)dyn);
        if (e != cudaSuccess) return e;
    }
    const int g = persistent_blocks(c, kern, dyn);
    kern<<<g, kThreads, dyn, s>>>(view<VT>(c), (const UT *)y, x, st);
    return cudaGetLastError();
}

template <typename VT, typename UT, typename AT, bool SQ, bool LS>
static cudaError_t aprod2_t(const gsr_ctx *c, const void *y, double *x, const LsqrState *st, cudaStream_t s)
{
    if (LS != (st != nullptr)) return cudaErrorInvalidValue;  // the LSQR variants read the solver state
    if (!SQ && !y) return cudaErrorInvalidValue;
    cudaError_t e;
    if (sizeof(AT) * (size_t)c->n_instr <= kSmemBudget)
        e = aprod2_star_launch<VT, UT, AT, true, SQ, LS>(c, y, x, st, s);
    else
        e = aprod2_star_launch<VT, UT, AT, false, SQ, LS>(c, y, x, st, s);
    if (e != cudaSuccess) return e;
    // attitude pass: at least 256 positions per warp
    auto kern = k_aprod2_att<VT, UT, AT, SQ, LS>;
    int per_sm = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, kThreads, 0) != cudaSuccess || per_sm < 1)
        per_sm = 1;
    const int64_t wpb = kThreads / 32;
    const int64_t max_warps = (int64_t)per_sm * c->sm_count * wpb;
    int64_t per = (c->n_rows + max_warps - 1) / max_warps;
    if (per < 256) per = 256;
    const int64_t warps = (c->n_rows + per - 1) / per;
    const int64_t blocks = (warps + wpb - 1) / wpb;
    kern<<<(unsigned)blocks, kThreads, 0, s>>>(view<VT>(c), (const UT *)y, x, st, per);
    return cudaGetLastError();
}

cudaError_t launch_aprod2(const gsr_ctx *c, const void *y, double *x, bool square, const LsqrState *st,
                          cudaStream_t s, bool inner32)
{
    if (c->n_rows == 0) return cudaSuccess;
    if (inner32) {
        if (st) return aprod2_t<float, float, float, false, true>(c, y, x, st, s);
        return aprod2_t<float, float, float, false, false>(c, y, x, nullptr, s);
    }
    if (c->prec == GSR_FP32) {
        if (square) return aprod2_t<float, double, double, true, false>(c, y, x, nullptr, s);
        if (st) return aprod2_t<float, double, double, false, true>(c, y, x, st, s);
        return aprod2_t<float, double, double, false, false>(c, y, x, nullptr, s);
    }
    if (square) return aprod2_t<double, double, double, true, false>(c, y, x, nullptr, s);
    if (st) return aprod2_t<double, double, double, false, true>(c, y, x, st, s);
    return aprod2_t<double, double, double, false, false>(c, y, x, nullptr, s);
}

}  // namespace gsr
