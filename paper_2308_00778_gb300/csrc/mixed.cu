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
#include "dfloat.cuh"
#include "tiles.cuh"

namespace gsr {

static constexpr int kThreads = 256;

__global__ void k_split(const double *__restrict__ a, float2 *__restrict__ out, int64_t n)
{
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        out[i] = split_double(a[i]);
    }
}

// r = b - A x for every row, stored in binary32, over the binary32 row tiles
// (one warp per tile, 4 rows per lane: four independent double-float chains).
// b is read in binary64 and split here (the same 8 bytes per row as a pre-split
// copy, without the pass that would make it); `part` (may be null) receives
// per-block sums of squares of r.
// the window copy of the attitude unknowns as (hi, lo) pairs: xw2[2 c], xw2[2 c + 1] = the pairs of
// x[att0 + c .. c + 3] (zero past the axis's end), c = a n_dfa + k
__global__ void k_split_window(const double *__restrict__ x, int64_t att0, int32_t n_dfa, float4 *__restrict__ xw2)
{
    const int64_t nat = (int64_t)NAXES * n_dfa;
    for (int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; c < nat; c += (int64_t)gridDim.x * blockDim.x) {
        const int32_t k = (int32_t)(c % n_dfa);
        float2 v[NPARAXIS];
#pragma unroll
        for (int q = 0; q < NPARAXIS; ++q) v[q] = k + q < n_dfa ? split_double(x[att0 + c + q]) : make_float2(0.f, 0.f);
        xw2[2 * c] = make_float4(v[0].x, v[0].y, v[1].x, v[1].y);
        xw2[2 * c + 1] = make_float4(v[2].x, v[2].y, v[3].x, v[3].y);
    }
}

// ATTW: the attitude pairs come from the window copy (one 32-byte load per axis and row instead of
// four 8-byte gathers); the terms and their order are the same, so the result is bitwise the same.
// XS: the block copies the instrumental pairs to shared memory first and gathers them there (a random
// 8-byte gather from global memory costs the L1 data pipe about a pass per lane); again the same terms.
template <bool SV = false, bool ATTW = false, bool R64 = false, bool XS = false>
__global__ void __launch_bounds__(256) k_residual(SysView<float> S, const float2 *__restrict__ xhl,
                                                  const double *__restrict__ b64, float *__restrict__ r_out,
                                                  double *__restrict__ part, double *__restrict__ r64)
{
    constexpr int R = Tile<float>::R;
    constexpr int T = Tile<float>::T;
    constexpr int MG = Sec<SV>::MAXG;
    const Sec<SV> G(S);
    __shared__ double sm32[32];
    const int lane = threadIdx.x & 31;
    const int64_t gw = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
    const float2 *__restrict__ xt = xhl + S.att0;
    const float2 *__restrict__ xi = xhl + S.instr0;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    float2 *sm_xi = reinterpret_cast<float2 *>(smem_raw);
    if constexpr (XS) {
        for (int32_t i = threadIdx.x; i < S.n_instr; i += blockDim.x) sm_xi[i] = xi[i];
        __syncthreads();
    }
    float2 xg[MG];
#pragma unroll
    for (int q = 0; q < MG; ++q) xg[q] = q < S.n_glob ? xhl[S.glob0 + q] : make_float2(0.f, 0.f);
    float ssq = 0.f;
    for (int64_t t = gw; t < S.n_tiles; t += nw) {
        const uint8_t *tb = S.tiles + t * S.tile_bytes;
        const uint8_t *ti = tb + (int64_t)G.npl * Tile<float>::VBLK;
        int32_t kn[R];
        load_ints<R>(ti, 0, kn);
        int32_t ic[NINSTR][R];
        float a[A_GLOB + MG][R];
        if constexpr (SV) {
            // run-time sections: unconditional loads (absent slots read an attitude plane or the
            // knot plane) and masked gathers, as in aprod 1
#pragma unroll
            for (int j = 0; j < NINSTR; ++j) load_instr_or_knot<float>(tb, G.npl, G.ni, S.iw16, j, ic[j]);
#pragma unroll
            for (int j = 0; j < NASTRO; ++j) load_vals<float, float>(tb, j < G.na ? j : G.p_att, a[j]);
#pragma unroll
            for (int j = 0; j < NAXES * NPARAXIS; ++j) load_vals<float, float>(tb, G.p_att + j, a[A_ATT + j]);
#pragma unroll
            for (int j = 0; j < NINSTR; ++j)
                load_vals<float, float>(tb, j < G.ni ? G.p_ins + j : G.p_att, a[A_INS + j]);
#pragma unroll
            for (int q = 0; q < MG; ++q)
                load_vals<float, float>(tb, q < G.ng ? G.p_glob + q : G.p_att, a[A_GLOB + q]);
        } else {
#pragma unroll
            for (int j = 0; j < NINSTR; ++j) load_instr<float>(tb, S.iw16, j, ic[j]);
#pragma unroll
            for (int j = 0; j < A_GLOB + MG; ++j) load_vals<float, float>(tb, j, a[j]);
        }
        const int64_t r0 = t * T + lane * R;
        int64_t sr[R];
        stars_of_rows<R>(S.star_ptr, S.first_star, t, r0, sr);
        float sh[R], c[R];
#pragma unroll
        for (int i = 0; i < R; ++i) {
            sh[i] = 0.f;
            c[i] = 0.f;
        }
        const float2 zero2 = make_float2(0.f, 0.f);
#pragma unroll
        for (int j = 0; j < NASTRO; ++j)
#pragma unroll
            for (int i = 0; i < R; ++i) {
                if constexpr (SV) {
                    const float2 xv = xhl[j < G.na ? (int64_t)G.na * sr[i] + j : 0];
                    acc_term(a[j][i], j < G.na ? xv : zero2, sh[i], c[i]);
                } else {
                    acc_term(a[j][i], xhl[NASTRO * sr[i] + j], sh[i], c[i]);
                }
            }
#pragma unroll
        for (int ax = 0; ax < NAXES; ++ax) {
            if constexpr (ATTW) {
#pragma unroll
                for (int i = 0; i < R; ++i) {
                    float4 p, q;  // the pairs of columns k, k+1 and k+2, k+3: one 32-byte load
                    ldg_v8(S.xw2 + 2 * ((int64_t)ax * S.n_dfa + kn[i]), p, q);
                    acc_term(a[A_ATT + NPARAXIS * ax + 0][i], make_float2(p.x, p.y), sh[i], c[i]);
                    acc_term(a[A_ATT + NPARAXIS * ax + 1][i], make_float2(p.z, p.w), sh[i], c[i]);
                    acc_term(a[A_ATT + NPARAXIS * ax + 2][i], make_float2(q.x, q.y), sh[i], c[i]);
                    acc_term(a[A_ATT + NPARAXIS * ax + 3][i], make_float2(q.z, q.w), sh[i], c[i]);
                }
            } else {
#pragma unroll
                for (int j = 0; j < NPARAXIS; ++j)
#pragma unroll
                    for (int i = 0; i < R; ++i)
                        acc_term(a[A_ATT + NPARAXIS * ax + j][i], xt[(int64_t)ax * S.n_dfa + kn[i] + j], sh[i], c[i]);
            }
        }
#pragma unroll
        for (int j = 0; j < NINSTR; ++j)
#pragma unroll
            for (int i = 0; i < R; ++i) {
                if constexpr (SV) {
                    const float2 xv = xhl[j < G.ni ? S.instr0 + ic[j][i] : 0];
                    acc_term(a[A_INS + j][i], j < G.ni ? xv : zero2, sh[i], c[i]);
                } else {
                    acc_term(a[A_INS + j][i], XS ? sm_xi[ic[j][i]] : xi[ic[j][i]], sh[i], c[i]);
                }
            }
#pragma unroll
        for (int i = 0; i < R; ++i) {
#pragma unroll
            for (int q = 0; q < MG; ++q) acc_term(a[A_GLOB + q][i], xg[q], sh[i], c[i]);  // xg[q] = 0 past n_glob
            const int64_t r = r0 + i;
            if (r < S.n_rows) {
                const float2 bb = split_double(__ldcs(b64 + r));
                float tt, e;
                two_sum(bb.x, -sh[i], tt, e);  // b_hi - s exactly
                const float lo = __fadd_rn(__fadd_rn(e, bb.y), -c[i]);
                const float rv = __fadd_rn(tt, lo);
                r_out[r] = rv;
                if constexpr (R64) r64[r] = (double)tt + (double)lo;  // exact in binary64
                ssq = fmaf(rv, rv, ssq);
            }
        }
    }
    if (part) {
        const double tot = block_sum((double)ssq, sm32);
        if (threadIdx.x == 0) part[blockIdx.x] = tot;
    }
}

// The residual of x = 0: r = b rounded to binary32 (what k_residual computes
// for x = 0, without reading A); per-block sums of squares into part.
__global__ void k_rhs32(const double *__restrict__ b, float *__restrict__ r, double *__restrict__ part, int64_t n)
{
    __shared__ double sm32[32];
    float ssq = 0.f;
    // four rows per thread and round: two 16-byte loads of b and one 16-byte store of r (the grid is the
    // residual kernel's, a few blocks per SM, so each thread keeps several loads in flight)
    const int64_t n4 = n / 4;
    const double2 *__restrict__ b2 = reinterpret_cast<const double2 *>(b);
    float4 *__restrict__ r4 = reinterpret_cast<float4 *>(r);
    for (int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; q < n4; q += (int64_t)gridDim.x * blockDim.x) {
        const double2 lo = __ldcs(b2 + 2 * q), hi = __ldcs(b2 + 2 * q + 1);
        const float4 v = make_float4((float)lo.x, (float)lo.y, (float)hi.x, (float)hi.y);
        r4[q] = v;
        ssq = fmaf(v.x, v.x, ssq);
        ssq = fmaf(v.y, v.y, ssq);
        ssq = fmaf(v.z, v.z, ssq);
        ssq = fmaf(v.w, v.w, ssq);
    }
    for (int64_t i = 4 * n4 + (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x) {
        const float v = (float)__ldcs(b + i);
        r[i] = v;
        ssq = fmaf(v, v, ssq);
    }
    const double tot = block_sum((double)ssq, sm32);
    if (threadIdx.x == 0) part[blockIdx.x] = tot;
}

// x += p * y (the inner solution, scaled back); per-block sums of squares of the
// correction (blk[0..3]) and of the new x (blk[4..7]). Four columns per thread and
// round with their loads issued together (the pass is latency-bound), one block
// reduction for the eight sums.
__global__ void k_correct(double *__restrict__ x, const double *__restrict__ p, const double *__restrict__ y,
                          int64_t n, int64_t att0, int64_t instr0, int64_t glob0, double *__restrict__ blk)
{
    constexpr int E = 4;
    __shared__ double sm[kThreads / 32][8];
    double acc[8] = {0.0, 0.0, 0.0, 0.0, 0.0, 0.0, 0.0, 0.0};
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t j0 = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; j0 < n; j0 += E * stride) {
        double pr[E], yr[E], xr[E];
#pragma unroll
        for (int q = 0; q < E; ++q) {
            const int64_t j = j0 + q * stride;
            pr[q] = yr[q] = xr[q] = 0.0;
            if (j < n) {
                pr[q] = p[j];
                yr[q] = y[j];
                xr[q] = x[j];
            }
        }
#pragma unroll
        for (int q = 0; q < E; ++q) {
            const int64_t j = j0 + q * stride;
            if (j >= n) continue;
            const double d = pr[q] * yr[q];
            const double xn = xr[q] + d;
            x[j] = xn;
            const int b = j < att0 ? 0 : (j < instr0 ? 1 : (j < glob0 ? 2 : 3));
#pragma unroll
            for (int k = 0; k < 4; ++k) {
                acc[k] += (k == b) ? d * d : 0.0;
                acc[4 + k] += (k == b) ? xn * xn : 0.0;
            }
        }
    }
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
    for (int k = 0; k < 8; ++k) {
        const double v = warp_sum(acc[k]);
        if (lane == 0) sm[wid][k] = v;
    }
    __syncthreads();
    if (threadIdx.x < 8) {
        double tot = 0.0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) tot += sm[w][threadIdx.x];
        if (tot != 0.0) atomicAdd(blk + threadIdx.x, tot);
    }
}

// Launch (or, with grid_out, only size) the residual kernel. Allocates nothing.
static constexpr size_t kResidualXsBudget = 200 * 1024;  // bytes of instrumental pairs in shared memory

cudaError_t residual_launch(const gsr_ctx *c, const float2 *xhl, const double *b64, float *r,
                            double *part, cudaStream_t s, int *grid_out, bool window, double *r64)
{
    // a section variant runs the run-time-geometry instance; a wide attitude block the window instance;
    // r64: the instance that also keeps the residual in binary64
    const bool w = window && res_window(c);
    // the window instance keeps the instrumental pairs in shared memory where they fit (it runs one
    // block per SM either way)
    const size_t dxs = sizeof(float2) * (size_t)c->n_instr;
    const bool xs = w && dxs <= kResidualXsBudget;
    auto kern = c->sv ? (r64 ? k_residual<true, false, true> : k_residual<true>)
                : xs  ? (r64 ? k_residual<false, true, true, true> : k_residual<false, true, false, true>)
                : w   ? (r64 ? k_residual<false, true, true> : k_residual<false, true>)
                      : (r64 ? k_residual<false, false, true> : k_residual<false>);
    // the grid (and so the number of partial sums) is the instance without r64's, whichever runs
    auto sized = c->sv ? k_residual<true>
                 : xs  ? k_residual<false, true, false, true>
                 : w   ? k_residual<false, true>
                       : k_residual<false>;
    const size_t dyn = xs ? dxs : 0;
    if (dyn > 48 * 1024) {
        cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)dyn);
        if (e == cudaSuccess) e = cudaFuncSetAttribute(sized, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)dyn);
        if (e != cudaSuccess) return e;
    }
    int per_sm = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, sized, kThreads, dyn) != cudaSuccess || per_sm < 1)
        per_sm = 1;
    int64_t blocks = (int64_t)per_sm * c->sm_count;
    blocks = std::min<int64_t>(blocks, (c->n_tiles + (kThreads / 32) - 1) / (kThreads / 32));
    blocks = std::max<int64_t>(blocks, 1);
    blocks = std::min<int64_t>(blocks, MAX_PARTIALS);
    if (grid_out) {
        *grid_out = (int)blocks;
        return cudaSuccess;
    }
    kern<<<(unsigned)blocks, kThreads, dyn, s>>>(view<float>(c), xhl, b64, r, part, r64);
    return cudaGetLastError();
}

// x (binary64) -> (hi, lo) binary32 pairs. Allocates nothing.
cudaError_t residual_kernels_load(bool sv)
{
    // cudaFuncGetAttributes loads a kernel that lazy module loading has not loaded yet
    cudaFuncAttributes a;
    cudaError_t e = cudaFuncGetAttributes(&a, k_split);
    if (e == cudaSuccess) e = cudaFuncGetAttributes(&a, sv ? k_residual<true> : k_residual<false>);
    return e;
}

cudaError_t split_launch(const gsr_ctx *c, const double *x, float2 *out, int64_t n, cudaStream_t s, bool window)
{
    if (n <= 0) return cudaSuccess;
    k_split<<<col_grid(c, n), kThreads, 0, s>>>(x, out, n);
    if (window && res_window(c))
        k_split_window<<<col_grid(c, (int64_t)NAXES * c->n_dfa), kThreads, 0, s>>>(
            x, (int64_t)c->n_astro * c->n_stars, c->n_dfa, c->xhlwin);
    return cudaGetLastError();
}

gsr_status residual_f32(gsr_ctx *c, const double *x, float *r, cudaStream_t s)
{
    gsr_status rc = ensure_workspace(c);
    if (rc != GSR_OK) return rc;
    if (c->n_rows == 0) return GSR_OK;
    Workspace &ws = c->ws;
    cudaError_t e = split_launch(c, x, ws.xhl, c->n_cols, s, true);
    if (e == cudaSuccess) e = residual_launch(c, ws.xhl, c->b, r, ws.part_u, s, nullptr, true);
    if (e != cudaSuccess) return cuda_fail(c, e, "residual");
    return GSR_OK;
}

gsr_status mixed_solve(gsr_ctx *c, const gsr_solve_params *prm, const double *x0, bool x0_dev, double *x_out,
                       gsr_solve_info *info, cudaStream_t s, bool p_ready, int r0_parts)
{
    const auto t0 = std::chrono::steady_clock::now();
    gsr_status rc = ensure_workspace(c);
    if (rc != GSR_OK) return rc;
    Workspace &ws = c->ws;
    const int64_t nc = c->n_cols, nr = c->n_rows;
    // k_correct: four columns per thread and round, two blocks per SM
    const int gcor = (int)std::min<int64_t>(std::max<int64_t>((nc + 4 * kThreads - 1) / (4 * kThreads), 1),
                                            2 * (int64_t)c->sm_count);
    const bool dev_io = prm->where == GSR_DEVICE;
    cudaError_t e;

    if (!p_ready && (rc = precond_pass(c, prm->precond != 0, s, true)) != GSR_OK) return rc;
    c->fused_inner = prm->inner_fused > 0 ? 1 : 0;  // the inner iterations' pass (iteration_graph reads it)
    if (x0)
        e = cudaMemcpyAsync(ws.xo, x0, nc * sizeof(double),
                            (dev_io || x0_dev) ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, s);
    else
        e = cudaMemsetAsync(ws.xo, 0, nc * sizeof(double), s);
    if (e != cudaSuccess) return cuda_fail(c, e, "mixed start");

    LsqrState init = initial_state(prm);
    const int32_t itn_first = prm->inner_itn > 0 ? prm->inner_itn : prm->itnlim;
    const int32_t itn_next = prm->inner_itn_next > 0 ? prm->inner_itn_next : itn_first;
    // inner stop: the correction problem's gradient |A~^T r| reduced by inner_tol from its start. The
    // Paige-Saunders tests 1 and 2 compare with |r|, which is mostly the part of b no correction can
    // fit; on noisy systems they stop the inner solves after one to three iterations and the
    // refinement crawls
    init.atol = init.btol = 0.0;
    init.artol = prm->inner_tol > 0.0 ? prm->inner_tol : 1e-6;
    const int max_outer = prm->max_outer > 0 ? prm->max_outer : 20;
    const double refine_tol = prm->refine_tol != 0.0 ? prm->refine_tol : 1e-10;
    int gres = 1;
    residual_launch(c, nullptr, nullptr, nullptr, nullptr, s, &gres, true);  // the grid of the launches below
    const int64_t att0 = (int64_t)c->n_astro * c->n_stars, instr0 = att0 + (int64_t)NAXES * c->n_dfa,
                  glob0 = instr0 + c->n_instr;

    LsqrState fin = LsqrState();
    int total_itn = 0, outer = 0;
    gsr_status status = GSR_OK;
    // the binary64 gradient of the inner solves' start (refine_grad): once on, every later step's
    // residual is also kept in binary64 (ws.u) and A~^T r is summed in binary64 from it
    bool grad64 = false;
    double prev_ratio = -1.0;
    for (; outer < max_outer; ++outer) {
        init.itnlim = outer == 0 ? itn_first : itn_next;
        int n_part = gres;
        const bool start64 = outer > 0 && (grad64 || prm->refine_grad > 0);
        if (start64 && !c->att_valid) {  // the binary64 aprod 2 of binary32 storage: knot-ordered copy
            if ((rc = ensure_att_layout(c, s, true)) != GSR_OK) return rc;
        }
        if (outer == 0 && r0_parts > 0) {
            n_part = r0_parts;  // the warm start left the residual of x0 (binary32) in ws.u32
        } else if (outer == 0 && !x0) {
            if (nr > 0) k_rhs32<<<gres, kThreads, 0, s>>>(c->b, ws.u32, ws.part_u, nr);
        } else {
            if ((e = split_launch(c, ws.xo, ws.xhl, nc, s, true)) != cudaSuccess) return cuda_fail(c, e, "split");
            if (nr > 0 && (e = residual_launch(c, ws.xhl, c->b, ws.u32, ws.part_u, s, nullptr, true,
                                               start64 ? ws.u : nullptr)) != cudaSuccess)
                return cuda_fail(c, e, "residual");
        }
        if ((e = cudaGetLastError()) != cudaSuccess) return cuda_fail(c, e, "residual");
        // one host synchronisation per refinement step: the inner solve's final state and the
        // correction's norms come back together
        status = run_lsqr(c, init, true, false, nr > 0 ? n_part : 0, prm->graph_k, prm->timeout_s, t0, s, &fin,
                          true, start64, prm->inner_close > 0);
        if (status != GSR_OK && status != GSR_ETIMEOUT) return status;
        if ((e = cudaMemsetAsync(ws.blk, 0, 8 * sizeof(double), s)) != cudaSuccess) return cuda_fail(c, e, "memset");
        k_correct<<<gcor, kThreads, 0, s>>>(ws.xo, ws.p, ws.x, nc, att0, instr0, glob0, ws.blk);
        if ((e = cudaMemcpyAsync(ws.blk_h, ws.blk, 8 * sizeof(double), cudaMemcpyDeviceToHost, s)) != cudaSuccess ||
            (e = cudaStreamSynchronize(s)) != cudaSuccess)
            return cuda_fail(c, e, "refinement");
        fin = *ws.fin_h;
        total_itn += fin.itn;
        const double *hb = ws.blk_h;
        if (status == GSR_OK && prm->timeout_s > 0.0 &&
            std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count() > prm->timeout_s)
            status = fail(c, GSR_ETIMEOUT, "solve exceeded timeout_s");
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
        double ratio = 0.0;  // the largest block |dx| / |x| of this step
        for (int q = 0; q < 4; ++q) {
            const double dn = std::sqrt(hb[q]), xn = std::sqrt(hb[4 + q]);
            if (dn > refine_tol * xn) converged = false;
            if (xn > 0.0) ratio = std::max(ratio, dn / xn);
        }
        // refine_grad 0: a step that did not halve the largest block correction of the one before has
        // met the binary32 rounding of the residual; the binary64 gradient takes over
        if (prm->refine_grad == 0 && !grad64 && outer >= 1 && prev_ratio > 0.0 && ratio > 0.5 * prev_ratio)
            grad64 = true;
        prev_ratio = ratio;
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
