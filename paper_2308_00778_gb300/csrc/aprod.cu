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

template <typename VT, bool LSQR>
__global__ void __launch_bounds__(256) k_aprod1(SysView<VT> S, const double *__restrict__ x, double *__restrict__ y,
                                                const LsqrState *__restrict__ st, double *__restrict__ part)
{
    __shared__ double sm32[32];
    double coef = 1.0;
    if (LSQR) {
        if (st->done) return;  // same value for every thread of the grid
        coef = st->coef_u;
    }
    const int lane = threadIdx.x & 31;
    const int64_t gw = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
    const double *__restrict__ xt = x + S.att0;
    const double *__restrict__ xi = x + S.instr0;
    const double xg = S.n_glob ? __ldg(x + S.glob0) : 0.0;
    double ssq = 0.0;
    for (int64_t s = gw; s < S.n_stars; s += nw) {
        const int64_t r0 = S.star_ptr[s], r1 = S.star_ptr[s + 1];
        const double *__restrict__ xa = x + NASTRO * s;
        const double xa0 = __ldg(xa + 0), xa1 = __ldg(xa + 1), xa2 = __ldg(xa + 2), xa3 = __ldg(xa + 3),
                     xa4 = __ldg(xa + 4);
        for (int64_t r = r0 + lane; r < r1; r += 32) {
            double a[NPAR];
#pragma unroll
            for (int j = 0; j < NPAR; ++j) a[j] = (double)ld_stream(S.val + j * S.plane + r);
            const int32_t k = ld_stream(S.knot + r);
            int32_t ic[NINSTR];
#pragma unroll
            for (int j = 0; j < NINSTR; ++j) ic[j] = ld_stream(S.instr + j * S.plane + r);
            double sum = a[0] * xa0;
            sum = fma(a[1], xa1, sum);
            sum = fma(a[2], xa2, sum);
            sum = fma(a[3], xa3, sum);
            sum = fma(a[4], xa4, sum);
#pragma unroll
            for (int ax = 0; ax < NAXES; ++ax) {
                const double *__restrict__ xk = xt + (int64_t)ax * S.n_dfa + k;
#pragma unroll
                for (int j = 0; j < NPARAXIS; ++j) sum = fma(a[NASTRO + NPARAXIS * ax + j], __ldg(xk + j), sum);
            }
#pragma unroll
            for (int j = 0; j < NINSTR; ++j) sum = fma(a[17 + j], __ldg(xi + ic[j]), sum);
            sum = fma(a[23], xg, sum);
            double yn;
            if (LSQR) {
                yn = fma(coef, y[r], sum);
                ssq = fma(yn, yn, ssq);
            } else {
                yn = y[r] + sum;
            }
            y[r] = yn;
        }
    }
    if (LSQR) {
        const double t = block_sum(ssq, sm32);
        if (threadIdx.x == 0) part[blockIdx.x] = t;
    }
}

// aprod 2, star-ordered pass: astrometric (per-star warp reduction, no atomics),
// instrumental (block-private shared-memory accumulators, or global atomics
// when n_instr is too large) and global (block reduction) parts.
template <typename VT, bool INSTR_SMEM, bool SQUARE, bool LSQR>
__global__ void __launch_bounds__(256) k_aprod2_star(SysView<VT> S, const double *__restrict__ y,
                                                     double *__restrict__ z, const LsqrState *__restrict__ st)
{
    extern __shared__ double smem[];
    __shared__ double sm32[32];
    if (LSQR && st->done) return;
    double *sm_ins = smem;
    const int32_t nsm = INSTR_SMEM ? S.n_instr : 0;
    for (int32_t i = threadIdx.x; i < nsm; i += blockDim.x) smem[i] = 0.0;
    __syncthreads();

    const int lane = threadIdx.x & 31;
    const int64_t gw = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
    double *__restrict__ zi = z + S.instr0;
    double gsum = 0.0;
    for (int64_t s = gw; s < S.n_stars; s += nw) {
        const int64_t r0 = S.star_ptr[s], r1 = S.star_ptr[s + 1];
        double acc[NASTRO] = {0.0, 0.0, 0.0, 0.0, 0.0};
        for (int64_t r = r0 + lane; r < r1; r += 32) {
            double a[NASTRO], ai[NINSTR];
#pragma unroll
            for (int j = 0; j < NASTRO; ++j) a[j] = (double)ld_stream(S.val + j * S.plane + r);
#pragma unroll
            for (int j = 0; j < NINSTR; ++j) ai[j] = (double)ld_stream(S.val + (17 + j) * S.plane + r);
            double ag = (double)ld_stream(S.val + 23 * S.plane + r);
            int32_t ic[NINSTR];
#pragma unroll
            for (int j = 0; j < NINSTR; ++j) ic[j] = ld_stream(S.instr + j * S.plane + r);
            double yr;
            if (SQUARE) {
                yr = 1.0;
#pragma unroll
                for (int j = 0; j < NASTRO; ++j) a[j] = a[j] * a[j];
#pragma unroll
                for (int j = 0; j < NINSTR; ++j) ai[j] = ai[j] * ai[j];
                ag = ag * ag;
            } else {
                yr = y[r];
            }
#pragma unroll
            for (int j = 0; j < NASTRO; ++j) acc[j] = fma(a[j], yr, acc[j]);
#pragma unroll
            for (int j = 0; j < NINSTR; ++j) {
                const double pr = ai[j] * yr;
                if (INSTR_SMEM)
                    atomicAdd(sm_ins + ic[j], pr);
                else
                    atomicAdd(zi + ic[j], pr);
            }
            gsum = fma(ag, yr, gsum);
        }
#pragma unroll
        for (int j = 0; j < NASTRO; ++j) acc[j] = warp_sum(acc[j]);
        if (lane < NASTRO) {
            double mine = acc[0];
#pragma unroll
            for (int j = 1; j < NASTRO; ++j) mine = (lane == j) ? acc[j] : mine;
            z[NASTRO * s + lane] += mine;
        }
    }
    __syncthreads();
    for (int32_t i = threadIdx.x; i < nsm; i += blockDim.x) {
        const double v = smem[i];
        if (v != 0.0) atomicAdd(zi + i, v);
    }
    if (S.n_glob) {
        const double t = block_sum(gsum, sm32);
        if (threadIdx.x == 0 && t != 0.0) atomicAdd(z + S.glob0, t);
    }
}

// Add a warp's run sums of the 12 attitude columns of knot k (warp-collective).
__device__ __forceinline__ void flush_att_run(double (&acc)[NAXES * NPARAXIS], int32_t k, int32_t n_dfa,
                                              double *__restrict__ zt)
{
    const int lane = threadIdx.x & 31;
#pragma unroll
    for (int j = 0; j < NAXES * NPARAXIS; ++j) {
        const double t = warp_sum(acc[j]);
        if (lane == 0 && t != 0.0) atomicAdd(zt + (j / NPARAXIS) * n_dfa + k + (j % NPARAXIS), t);
        acc[j] = 0.0;
    }
}

// aprod 2, attitude pass over the knot-ordered copy: each warp owns a
// contiguous range of positions; runs of equal knot are summed in registers
// and added once per run (one atomic add per column per run).
template <typename VT, bool SQUARE, bool LSQR>
__global__ void __launch_bounds__(256) k_aprod2_att(SysView<VT> S, const double *__restrict__ y,
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
    double acc[NAXES * NPARAXIS];
#pragma unroll
    for (int j = 0; j < NAXES * NPARAXIS; ++j) acc[j] = 0.0;
    for (int64_t q = p0; q < p1; q += 32) {
        const int64_t i = q + lane;
        const bool active = i < p1;
        const int64_t last = min(q + 31, p1 - 1);
        double a[NAXES * NPARAXIS];
        double yr = 0.0;
        if (active) {
#pragma unroll
            for (int j = 0; j < NAXES * NPARAXIS; ++j) a[j] = (double)ld_stream(S.att_k + j * S.plane + i);
            if (SQUARE) {
                yr = 1.0;
#pragma unroll
                for (int j = 0; j < NAXES * NPARAXIS; ++j) a[j] = a[j] * a[j];
            } else {
                yr = y[ld_stream(S.perm + i)];
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
                    atomicAdd(zt + (j / NPARAXIS) * S.n_dfa + kl + (j % NPARAXIS), a[j] * yr);
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

int aprod1_grid(const gsr_ctx *c)
{
    if (c->prec == GSR_FP32) return persistent_blocks(c, k_aprod1<float, true>, 0);
    return persistent_blocks(c, k_aprod1<double, true>, 0);
}

template <typename VT>
static cudaError_t aprod1_t(const gsr_ctx *c, const double *x, double *y, const LsqrState *st, double *part,
                            cudaStream_t s)
{
    const SysView<VT> S = view<VT>(c);
    if (st) {
        const int g = persistent_blocks(c, k_aprod1<VT, true>, 0);
        k_aprod1<VT, true><<<g, kThreads, 0, s>>>(S, x, y, st, part);
    } else {
        const int g = persistent_blocks(c, k_aprod1<VT, false>, 0);
        k_aprod1<VT, false><<<g, kThreads, 0, s>>>(S, x, y, nullptr, nullptr);
    }
    return cudaGetLastError();
}

cudaError_t launch_aprod1(const gsr_ctx *c, const double *x, double *y, const LsqrState *st, double *part,
                          cudaStream_t s)
{
    if (c->n_rows == 0) return cudaSuccess;
    return c->prec == GSR_FP32 ? aprod1_t<float>(c, x, y, st, part, s) : aprod1_t<double>(c, x, y, st, part, s);
}

template <typename VT, bool INS, bool SQ, bool LS>
static cudaError_t aprod2_star_launch(const gsr_ctx *c, const double *y, double *x, const LsqrState *st,
                                      cudaStream_t s)
{
    auto kern = k_aprod2_star<VT, INS, SQ, LS>;
    const size_t dyn = INS ? sizeof(double) * (size_t)c->n_instr : 0;
    if (dyn > 48 * 1024) {
        cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)dyn);
        if (e != cudaSuccess) return e;
    }
    const int g = persistent_blocks(c, kern, dyn);
    kern<<<g, kThreads, dyn, s>>>(view<VT>(c), y, x, st);
    return cudaGetLastError();
}

template <typename VT, bool SQ, bool LS>
static cudaError_t aprod2_t(const gsr_ctx *c, const double *y, double *x, const LsqrState *st, cudaStream_t s)
{
    cudaError_t e;
    if (sizeof(double) * (size_t)c->n_instr <= kSmemBudget)
        e = aprod2_star_launch<VT, true, SQ, LS>(c, y, x, st, s);
    else
        e = aprod2_star_launch<VT, false, SQ, LS>(c, y, x, st, s);
    if (e != cudaSuccess) return e;
    // attitude pass: at least 256 positions per warp
    auto kern = k_aprod2_att<VT, SQ, LS>;
    int per_sm = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, kThreads, 0) != cudaSuccess || per_sm < 1)
        per_sm = 1;
    const int64_t wpb = kThreads / 32;
    const int64_t max_warps = (int64_t)per_sm * c->sm_count * wpb;
    int64_t per = (c->n_rows + max_warps - 1) / max_warps;
    if (per < 256) per = 256;
    const int64_t warps = (c->n_rows + per - 1) / per;
    const int64_t blocks = (warps + wpb - 1) / wpb;
    kern<<<(unsigned)blocks, kThreads, 0, s>>>(view<VT>(c), y, x, st, per);
    return cudaGetLastError();
}

cudaError_t launch_aprod2(const gsr_ctx *c, const double *y, double *x, bool square, const LsqrState *st,
                          cudaStream_t s)
{
    if (c->n_rows == 0) return cudaSuccess;
    if (c->prec == GSR_FP32) {
        if (square) return aprod2_t<float, true, false>(c, y, x, nullptr, s);
        if (st) return aprod2_t<float, false, true>(c, y, x, st, s);
        return aprod2_t<float, false, false>(c, y, x, nullptr, s);
    }
    if (square) return aprod2_t<double, true, false>(c, y, x, nullptr, s);
    if (st) return aprod2_t<double, false, true>(c, y, x, st, s);
    return aprod2_t<double, false, false>(c, y, x, nullptr, s);
}

}  // namespace gsr
