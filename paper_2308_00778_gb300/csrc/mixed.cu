// mixed.cu -- mixed-precision LSQR: binary32 inner solves, iterative refinement in binary64.
//
// The coefficients are stored and streamed in binary32. Each refinement step
//   1. computes the residual r = b - A x of the current solution x with the
//      products and sums carried in double-float (pairs of binary32: Dekker /
//      Knuth error-free transforms), so no binary64 arithmetic runs per row;
//      r is stored in binary32 as the inner right-hand side,
//   2. runs LSQR (the same start / graph-captured iteration as the plain
//      solver, with the binary32 aprod kernels) on A d ~ r to a loose
//      tolerance,
//   3. adds the correction x += d in binary64 and measures |d| and |x| per
//      block (astro / attitude / instrumental / global);
// until every block's |d|/|x| is below refine_tol. The norms, the alpha / beta
// / rho / phi recurrences, the column vectors and x stay binary64.
//
// The refined solution is the least-squares solution of the system; with a
// damped inner solve the damping acts on the correction only, so the fixed
// point is the undamped minimiser (it differs from the damped one by
// O(damp^2), far below the binary32 noise for the damping used here).
#include "gsr_internal.cuh"
#include "dfloat.cuh"

namespace gsr {

static constexpr int kThreads = 256;

__global__ void k_split(const double *__restrict__ a, float2 *__restrict__ out, int64_t n)
{
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        out[i] = split_double(a[i]);
    }
}

// r = b - A x for every row (one warp per star), stored in binary32, with
// per-block sums of squares of r.
// STAGE: the attitude and instrumental parts of x are copied to shared memory
// once per block (as in aprod 1), so the per-row gathers stay on chip.
template <bool STAGE>
__global__ void __launch_bounds__(256) k_residual(SysView<float> S, const float2 *__restrict__ xhl,
                                                  const float2 *__restrict__ bhl, float *__restrict__ r_out,
                                                  double *__restrict__ part)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    __shared__ double sm32[32];
    const int lane = threadIdx.x & 31;
    const int64_t gw = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
    const float2 *xt = xhl + S.att0;
    const float2 *xi = xhl + S.instr0;
    if (STAGE) {
        float2 *sx = reinterpret_cast<float2 *>(smem_raw);
        const int32_t n_att = NAXES * S.n_dfa, n_st = n_att + S.n_instr;
        for (int32_t i = threadIdx.x; i < n_st; i += blockDim.x) sx[i] = xhl[S.att0 + i];
        __syncthreads();
        xt = sx;
        xi = sx + n_att;
    }
    const float2 xg = S.n_glob ? xhl[S.glob0] : make_float2(0.f, 0.f);
    float ssq = 0.f;
    for (int64_t s = gw; s < S.n_stars; s += nw) {
        const int64_t r0 = S.star_ptr[s], r1 = S.star_ptr[s + 1];
        float2 xa[NASTRO];
#pragma unroll
        for (int j = 0; j < NASTRO; ++j) xa[j] = xhl[NASTRO * s + j];
        for (int64_t r = r0 + lane; r < r1; r += 32) {
            float a[NPAR];
#pragma unroll
            for (int j = 0; j < NPAR; ++j) a[j] = __ldcs(S.val + j * S.plane + r);
            const int32_t k = __ldcs(S.knot + r);
            int32_t ic[NINSTR];
#pragma unroll
            for (int j = 0; j < NINSTR; ++j) ic[j] = __ldcs(S.instr + j * S.plane + r);
            float sh = 0.f, c = 0.f;
#pragma unroll
            for (int j = 0; j < NASTRO; ++j) acc_term(a[j], xa[j], sh, c);
#pragma unroll
            for (int ax = 0; ax < NAXES; ++ax) {
                const float2 *xk = xt + (int64_t)ax * S.n_dfa + k;
#pragma unroll
                for (int j = 0; j < NPARAXIS; ++j) acc_term(a[NASTRO + NPARAXIS * ax + j], xk[j], sh, c);
            }
#pragma unroll
            for (int j = 0; j < NINSTR; ++j) acc_term(a[17 + j], xi[ic[j]], sh, c);
            acc_term(a[23], xg, sh, c);
            const float2 b = __ldcs(bhl + r);
            float t, e;
            two_sum(b.x, -sh, t, e);  // b_hi - s exactly
            const float lo = __fadd_rn(__fadd_rn(e, b.y), -c);
            const float rv = __fadd_rn(t, lo);
            r_out[r] = rv;
            ssq = fmaf(rv, rv, ssq);
        }
    }
    const double tot = block_sum((double)ssq, sm32);
    if (threadIdx.x == 0) part[blockIdx.x] = tot;
}

// x += p * y (the inner solution, scaled back); per-block sums of squares of
// the correction (blk[0..3]) and of the new x (blk[4..7]).
__global__ void k_correct(double *__restrict__ x, const double *__restrict__ p, const double *__restrict__ y,
                          int64_t n, int64_t att0, int64_t instr0, int64_t glob0, double *__restrict__ blk)
{
    __shared__ double sm32[32];
    double sd[4] = {0.0, 0.0, 0.0, 0.0}, sx[4] = {0.0, 0.0, 0.0, 0.0};
    for (int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; j < n; j += (int64_t)gridDim.x * blockDim.x) {
        const double d = p[j] * y[j];
        const double xn = x[j] + d;
        x[j] = xn;
        const int b = j < att0 ? 0 : (j < instr0 ? 1 : (j < glob0 ? 2 : 3));
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            sd[q] += (q == b) ? d * d : 0.0;
            sx[q] += (q == b) ? xn * xn : 0.0;
        }
    }
#pragma unroll
    for (int q = 0; q < 4; ++q) {
        const double a = block_sum(sd[q], sm32);
        if (threadIdx.x == 0 && a != 0.0) atomicAdd(blk + q, a);
        const double bx = block_sum(sx[q], sm32);
        if (threadIdx.x == 0 && bx != 0.0) atomicAdd(blk + 4 + q, bx);
    }
}

static constexpr size_t kStageBudget = 160 * 1024;

static size_t residual_stage_bytes(const gsr_ctx *c)
{
    const size_t b = sizeof(float2) * ((size_t)NAXES * c->n_dfa + (size_t)c->n_instr);
    return b <= kStageBudget ? b : 0;
}

// launch (or, with grid_out, only size) the residual kernel
static cudaError_t residual_launch(const gsr_ctx *c, const float2 *xhl, const float2 *bhl, float *r, double *part,
                                   cudaStream_t s, int *grid_out)
{
    const size_t dyn = residual_stage_bytes(c);
    auto kern = dyn ? k_residual<true> : k_residual<false>;
    if (dyn > 48 * 1024) {
        cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)dyn);
        if (e != cudaSuccess) return e;
    }
    int per_sm = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, kThreads, dyn) != cudaSuccess || per_sm < 1)
        per_sm = 1;
    int64_t blocks = (int64_t)per_sm * c->sm_count;
    const int64_t max_blocks = (c->n_stars + (kThreads / 32) - 1) / (kThreads / 32);
    blocks = std::min(blocks, max_blocks);
    blocks = std::max<int64_t>(blocks, 1);
    blocks = std::min<int64_t>(blocks, MAX_PARTIALS);
    if (grid_out) {
        *grid_out = (int)blocks;
        return cudaSuccess;
    }
    kern<<<(unsigned)blocks, kThreads, dyn, s>>>(view<float>(c), xhl, bhl, r, part);
    return cudaGetLastError();
}

gsr_status residual_f32(gsr_ctx *c, const double *x, float *r, cudaStream_t s)
{
    gsr_status rc = ensure_workspace(c);
    if (rc != GSR_OK) return rc;
    if (c->n_rows == 0) return GSR_OK;
    Workspace &ws = c->ws;
    k_split<<<col_grid(c, c->n_rows), kThreads, 0, s>>>(c->b, ws.bhl, c->n_rows);
    k_split<<<col_grid(c, c->n_cols), kThreads, 0, s>>>(x, ws.xhl, c->n_cols);
    const cudaError_t e = residual_launch(c, ws.xhl, ws.bhl, r, ws.part_u, s, nullptr);
    if (e != cudaSuccess) return cuda_fail(c, e, "residual");
    return GSR_OK;
}

gsr_status mixed_solve(gsr_ctx *c, const gsr_solve_params *prm, const double *x0, double *x_out,
                       gsr_solve_info *info, cudaStream_t s)
{
    const auto t0 = std::chrono::steady_clock::now();
    gsr_status rc = ensure_workspace(c);
    if (rc != GSR_OK) return rc;
    Workspace &ws = c->ws;
    const int64_t nc = c->n_cols, nr = c->n_rows;
    const int gcol = col_grid(c, nc);
    const int grow = col_grid(c, nr);
    const bool dev_io = prm->where == GSR_DEVICE;
    cudaError_t e;

    if ((rc = precond_pass(c, prm->precond != 0, s)) != GSR_OK) return rc;
    k_split<<<grow, kThreads, 0, s>>>(c->b, ws.bhl, nr);
    if (x0)
        e = cudaMemcpyAsync(ws.xo, x0, nc * sizeof(double), dev_io ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice,
                            s);
    else
        e = cudaMemsetAsync(ws.xo, 0, nc * sizeof(double), s);
    if (e != cudaSuccess) return cuda_fail(c, e, "mixed start");

    LsqrState init = initial_state(prm);
    init.itnlim = prm->inner_itn > 0 ? prm->inner_itn : prm->itnlim;
    init.atol = init.btol = prm->inner_tol > 0.0 ? prm->inner_tol : 1e-6;
    const int max_outer = prm->max_outer > 0 ? prm->max_outer : 20;
    const double refine_tol = prm->refine_tol != 0.0 ? prm->refine_tol : 1e-10;
    int gres = 1;
    residual_launch(c, nullptr, nullptr, nullptr, nullptr, s, &gres);
    const int64_t att0 = (int64_t)NASTRO * c->n_stars, instr0 = att0 + (int64_t)NAXES * c->n_dfa,
                  glob0 = instr0 + c->n_instr;

    LsqrState fin = LsqrState();
    int total_itn = 0, outer = 0;
    gsr_status status = GSR_OK;
    for (; outer < max_outer; ++outer) {
        k_split<<<gcol, kThreads, 0, s>>>(ws.xo, ws.xhl, nc);
        if (nr > 0 && (e = residual_launch(c, ws.xhl, ws.bhl, ws.u32, ws.part_u, s, nullptr)) != cudaSuccess)
            return cuda_fail(c, e, "residual");
        if ((e = cudaGetLastError()) != cudaSuccess) return cuda_fail(c, e, "residual");
        status = run_lsqr(c, init, true, false, nr > 0 ? gres : 0, prm->graph_k, prm->timeout_s, t0, s, &fin);
        total_itn += fin.itn;
        if (status != GSR_OK && status != GSR_ETIMEOUT) return status;
        double hb[8];
        if ((e = cudaMemsetAsync(ws.blk, 0, 8 * sizeof(double), s)) != cudaSuccess) return cuda_fail(c, e, "memset");
        k_correct<<<gcol, kThreads, 0, s>>>(ws.xo, ws.p, ws.x, nc, att0, instr0, glob0, ws.blk);
        if ((e = cudaMemcpyAsync(hb, ws.blk, sizeof(hb), cudaMemcpyDeviceToHost, s)) != cudaSuccess ||
            (e = cudaStreamSynchronize(s)) != cudaSuccess)
            return cuda_fail(c, e, "refinement");
        if (status == GSR_ETIMEOUT) {
            ++outer;
            break;
        }
        if (fin.numeric) {
            ++outer;
            status = fail(c, GSR_ENUMERIC, "non-finite value in the inner LSQR scalars");
            break;
        }
        bool converged = refine_tol > 0.0;
        for (int q = 0; q < 4; ++q) {
            const double dn = std::sqrt(hb[q]), xn = std::sqrt(hb[4 + q]);
            if (dn > refine_tol * xn) converged = false;
        }
        if (converged) {
            ++outer;
            break;
        }
    }
    e = cudaMemcpyAsync(x_out, ws.xo, nc * sizeof(double), dev_io ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost,
                        s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return cuda_fail(c, e, "result");
    fill_info(info, fin, t0);
    if (info) {
        info->itn = total_itn;
        info->outer_itn = outer;
    }
    return status;
}

}  // namespace gsr
