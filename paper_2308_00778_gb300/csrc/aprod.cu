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
// aprod 2: the astrometric part is a per-star register accumulation and one
// warp reduction per star, written without atomics (one warp owns a star).
// Attitude and instrumental products go to block-private shared-memory
// accumulators when they fit (flushed once per block with atomic adds),
// otherwise straight to global memory with atomic adds resolved in L2. The
// global column is reduced per block in registers and added once per block
// (the two-stage reduction of the paper's global kernels, Sec. 4.2, folded
// into one pass).
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

template <typename VT, bool ATT_SMEM, bool INSTR_SMEM, bool SQUARE, bool LSQR>
__global__ void __launch_bounds__(256) k_aprod2(SysView<VT> S, const double *__restrict__ y, double *__restrict__ z,
                                                const LsqrState *__restrict__ st)
{
    extern __shared__ double smem[];
    __shared__ double sm32[32];
    if (LSQR && st->done) return;
    const int32_t n_att = NAXES * S.n_dfa;
    double *sm_att = smem;
    double *sm_ins = smem + (ATT_SMEM ? n_att : 0);
    const int32_t nsm = (ATT_SMEM ? n_att : 0) + (INSTR_SMEM ? S.n_instr : 0);
    for (int32_t i = threadIdx.x; i < nsm; i += blockDim.x) smem[i] = 0.0;
    __syncthreads();

    const int lane = threadIdx.x & 31;
    const int64_t gw = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
    double *__restrict__ zt = z + S.att0;
    double *__restrict__ zi = z + S.instr0;
    double gsum = 0.0;
    for (int64_t s = gw; s < S.n_stars; s += nw) {
        const int64_t r0 = S.star_ptr[s], r1 = S.star_ptr[s + 1];
        double acc[NASTRO] = {0.0, 0.0, 0.0, 0.0, 0.0};
        for (int64_t r = r0 + lane; r < r1; r += 32) {
            double a[NPAR];
#pragma unroll
            for (int j = 0; j < NPAR; ++j) a[j] = (double)ld_stream(S.val + j * S.plane + r);
            const int32_t k = ld_stream(S.knot + r);
            int32_t ic[NINSTR];
#pragma unroll
            for (int j = 0; j < NINSTR; ++j) ic[j] = ld_stream(S.instr + j * S.plane + r);
            double yr;
            if (SQUARE) {
                yr = 1.0;
#pragma unroll
                for (int j = 0; j < NPAR; ++j) a[j] = a[j] * a[j];
            } else {
                yr = y[r];
            }
#pragma unroll
            for (int j = 0; j < NASTRO; ++j) acc[j] = fma(a[j], yr, acc[j]);
#pragma unroll
            for (int ax = 0; ax < NAXES; ++ax) {
                const int32_t base = ax * S.n_dfa + k;
#pragma unroll
                for (int j = 0; j < NPARAXIS; ++j) {
                    const double pr = a[NASTRO + NPARAXIS * ax + j] * yr;
                    if (ATT_SMEM)
                        atomicAdd(sm_att + base + j, pr);
                    else
                        atomicAdd(zt + base + j, pr);
                }
            }
#pragma unroll
            for (int j = 0; j < NINSTR; ++j) {
                const double pr = a[17 + j] * yr;
                if (INSTR_SMEM)
                    atomicAdd(sm_ins + ic[j], pr);
                else
                    atomicAdd(zi + ic[j], pr);
            }
            gsum = fma(a[23], yr, gsum);
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
        if (v != 0.0) {
            if (ATT_SMEM && i < n_att)
                atomicAdd(zt + i, v);
            else
                atomicAdd(zi + (i - (ATT_SMEM ? n_att : 0)), v);
        }
    }
    if (S.n_glob) {
        const double t = block_sum(gsum, sm32);
        if (threadIdx.x == 0 && t != 0.0) atomicAdd(z + S.glob0, t);
    }
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

template <typename VT, bool ATT, bool INS, bool SQ, bool LS>
static cudaError_t aprod2_launch(const gsr_ctx *c, const double *y, double *x, const LsqrState *st, cudaStream_t s)
{
    auto kern = k_aprod2<VT, ATT, INS, SQ, LS>;
    const size_t dyn = sizeof(double) * ((ATT ? (size_t)NAXES * c->n_dfa : 0) + (INS ? (size_t)c->n_instr : 0));
    if (dyn > 48 * 1024) {
        cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)dyn);
        if (e != cudaSuccess) return e;
    }
    const int g = persistent_blocks(c, kern, dyn);
    kern<<<g, kThreads, dyn, s>>>(view<VT>(c), y, x, st);
    return cudaGetLastError();
}

template <typename VT, bool SQ, bool LS>
static cudaError_t aprod2_modes(const gsr_ctx *c, const double *y, double *x, const LsqrState *st, cudaStream_t s)
{
    const size_t att_b = sizeof(double) * (size_t)NAXES * c->n_dfa;
    const size_t ins_b = sizeof(double) * (size_t)c->n_instr;
    if (att_b + ins_b <= kSmemBudget) return aprod2_launch<VT, true, true, SQ, LS>(c, y, x, st, s);
    if (ins_b <= kSmemBudget) return aprod2_launch<VT, false, true, SQ, LS>(c, y, x, st, s);
    return aprod2_launch<VT, false, false, SQ, LS>(c, y, x, st, s);
}

cudaError_t launch_aprod2(const gsr_ctx *c, const double *y, double *x, bool square, const LsqrState *st,
                          cudaStream_t s)
{
    if (c->n_rows == 0) return cudaSuccess;
    if (c->prec == GSR_FP32) {
        if (square) return aprod2_modes<float, true, false>(c, y, x, nullptr, s);
        if (st) return aprod2_modes<float, false, true>(c, y, x, st, s);
        return aprod2_modes<float, false, false>(c, y, x, nullptr, s);
    }
    if (square) return aprod2_modes<double, true, false>(c, y, x, nullptr, s);
    if (st) return aprod2_modes<double, false, true>(c, y, x, st, s);
    return aprod2_modes<double, false, false>(c, y, x, nullptr, s);
}

}  // namespace gsr
