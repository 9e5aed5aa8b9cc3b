// lsqr.cu -- the LSQR iteration (Paige & Saunders 1982; the solver of Sec. 1-2) on the GPU.
//
// One iteration is five kernels, captured once into a CUDA graph and replayed
// (replacing the per-iteration host synchronisations and copies of Alg. 1 and
// Sec. 4.4):
//   aprod1  u <- A (p v) - (alpha/beta) u, per-block sums of squares of u
//   aprod2  z <- A^T u (z is zero on entry)
//   colA    beta = |u| (from the partials), vhat = p z / beta - beta v,
//           z <- 0, per-block sums of squares of vhat and of w
//   scalar  alpha = |vhat|, the two plane rotations, the norm / condition /
//           residual estimates and the stopping tests (one thread)
//   colB    v = vhat / alpha, pv = p v, x += t1 w, w = v + t2 w, var += (w/rho)^2
// The LSQR vectors u and v are kept unnormalised where that saves a pass: u is
// stored as beta*u (its scale folded into the aprod1 coefficient), and the
// preconditioner p (column norms, Alg. 1) is applied to column vectors rather
// than to A. Norms (alpha, beta) are exact 2-norms from per-block FP64 sums of
// squares reduced in a fixed order (Eq. 4's scaling only guards against
// overflow; a non-finite sum stops the solve with GSR_ENUMERIC).
//
// Stopping: the scalar kernel sets st->done when a test fires (after setting
// the coefficients of that iteration's x update). Later kernels read done and
// return at once; colB of the stopping iteration still runs (it reads
// st->colb_skip, which the scalar kernel clears when it ran). The host reads
// a pinned mapped flag after each graph launch.
#include <chrono>
#include <cmath>

#include "gsr_internal.cuh"

namespace gsr {

static constexpr int kColThreads = 256;
static constexpr int kColElems = 4;  // columns per thread and round in k_colA and k_colB

// ---------------------------------------------------------------- column kernels
// u <- b - (A x0 is added by a separate aprod1 on -x0); here: u <- src, partial sums of squares
__global__ void k_copy_ssq(const double *__restrict__ src, double *__restrict__ dst, int64_t n,
                           double *__restrict__ part)
{
    __shared__ double sm32[32];
    double ssq = 0.0;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const double v = src[i];
        dst[i] = v;
        ssq = fma(v, v, ssq);
    }
    const double t = block_sum(ssq, sm32);
    if (threadIdx.x == 0) part[blockIdx.x] = t;
}

// sums of squares of a row vector (used after u <- b - A x0)
__global__ void k_ssq(const double *__restrict__ a, int64_t n, double *__restrict__ part)
{
    __shared__ double sm32[32];
    double ssq = 0.0;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const double v = a[i];
        ssq = fma(v, v, ssq);
    }
    const double t = block_sum(ssq, sm32);
    if (threadIdx.x == 0) part[blockIdx.x] = t;
}

// p_j = 1/sqrt(colsq_j) (1 for an empty column), colsq reset to zero
__global__ void k_precond_finish(double *__restrict__ colsq, double *__restrict__ p, int64_t n, int32_t use)
{
    for (int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; j < n; j += (int64_t)gridDim.x * blockDim.x) {
        const double q = colsq[j];
        p[j] = (use && q > 0.0) ? 1.0 / sqrt(q) : 1.0;
        colsq[j] = 0.0;
    }
}

// One step of the recurrence (beta of this iteration and 1/beta given), by the
// first warp of the block that finishes k_colA last; thread 0 writes. Binary64
// divides and square roots are slow on this GPU (about 0.34 us each when
// dependent), so each rotation takes one reciprocal and multiplies by it.
// CLOSE: the last iteration of a solve that has reached its iteration limit, run
// without the aprod 2 (k_colA_close): the x update needs only beta_{k+1}, through
// rho_k and phi_k, so alpha_{k+1} is not formed. It enters theta and rhobar of the
// next step and the |A^T r| estimate; the first two are not used again, the last
// keeps the previous iteration's value, and the tests that read it are not made.
template <bool CLOSE = false>
__device__ void scalar_step(LsqrState *__restrict__ st, double beta, double inv_beta, const double *__restrict__ part_v,
                            const double *__restrict__ part_w, int n_part, int32_t *__restrict__ flag)
{
    const double ssq_v = CLOSE ? 0.0 : warp_sum_partials(part_v, n_part);
    const double ssq_w = warp_sum_partials(part_w, n_part);
    if (threadIdx.x != 0) return;
    st->colb_skip = 0;
    const double damp = st->damp, dampsq = damp * damp;
    st->beta = beta;
    double alpha = st->alpha;
    double anorm = st->anorm;
    if (beta > 0.0) {
        anorm = sqrt(anorm * anorm + alpha * alpha + beta * beta + dampsq);
        alpha = CLOSE ? 0.0 : sqrt(ssq_v);
    }
    const double inv_bnorm = 1.0 / st->bnorm;  // off the critical path
    // rotation eliminating damp
    const double rhobar = st->rhobar;
    double phibar = st->phibar;
    const double rhobar1 = sqrt(rhobar * rhobar + dampsq);
    const double i_rhobar1 = 1.0 / rhobar1;
    const double cs1 = rhobar * i_rhobar1;
    const double sn1 = damp * i_rhobar1;
    const double psi = sn1 * phibar;
    phibar = cs1 * phibar;
    // rotation eliminating beta
    const double rho = sqrt(rhobar1 * rhobar1 + beta * beta);
    const double i_rho = 1.0 / rho;
    const double cs = rhobar1 * i_rho;
    const double sn = beta * i_rho;
    const double theta = sn * alpha;
    const double rhobar_n = -cs * alpha;
    const double phi = cs * phibar;
    phibar = sn * phibar;
    const double tau = sn * phi;
    // coefficients of the x and w updates
    st->t1 = phi * i_rho;
    st->t2 = -theta * i_rho;
    st->inv_rho = i_rho;
    const double ddnorm = st->ddnorm + ssq_w * (i_rho * i_rho);
    // |x| estimate
    const double delta = st->sn2 * rho;
    const double gambar = -st->cs2 * rho;
    const double rhs = phi - delta * st->zeta;
    const double zbar = rhs / gambar;
    const double xnorm = sqrt(st->xxnorm + zbar * zbar);
    const double gamma = sqrt(gambar * gambar + theta * theta);
    const double i_gamma = 1.0 / gamma;
    st->cs2 = gambar * i_gamma;
    st->sn2 = theta * i_gamma;
    st->zeta = rhs * i_gamma;
    st->xxnorm = st->xxnorm + st->zeta * st->zeta;
    // estimates
    const double acond = anorm * sqrt(ddnorm);
    const double res1 = phibar * phibar;
    const double res2 = st->res2 + psi * psi;
    const double rnorm = sqrt(res1 + res2);
    const double arnorm = CLOSE ? st->arnorm : alpha * fabs(tau);
    const double r1sq = rnorm * rnorm - dampsq * st->xxnorm;
    double r1norm = sqrt(fabs(r1sq));
    if (r1sq < 0.0) r1norm = -r1norm;
    const int itn = st->itn + 1;
    // stopping tests
    const double test1 = rnorm * inv_bnorm;
    const double test2 = arnorm / (anorm * rnorm);
    const double test3 = 1.0 / acond;
    const double anx = anorm * xnorm * inv_bnorm;
    const double tt1 = test1 / (1.0 + anx);
    const double rtol = st->btol + st->atol * anx;
    int istop = 0;
    if (itn >= st->itnlim || CLOSE) istop = 7;
    if (1.0 + test3 <= 1.0) istop = 6;
    if (!CLOSE && 1.0 + test2 <= 1.0) istop = 5;
    if (1.0 + tt1 <= 1.0) istop = 4;
    if (test3 <= st->ctol) istop = 3;
    if (!CLOSE && test2 <= st->atol) istop = 2;
    if (!CLOSE && arnorm <= st->artol * st->arnorm0) istop = 2;
    if (test1 <= rtol) istop = 1;
    const bool bad = !(isfinite(alpha) && isfinite(rho) && isfinite(phi) && isfinite(theta) && isfinite(rnorm));
    // store
    if (!CLOSE) st->alpha = alpha;
    st->anorm = anorm;
    st->rhobar = rhobar_n;
    st->phibar = phibar;
    st->ddnorm = ddnorm;
    st->xnorm = xnorm;
    st->acond = acond;
    st->res2 = res2;
    st->rnorm = rnorm;
    st->r1norm = r1norm;
    st->r2norm = rnorm;
    st->arnorm = arnorm;
    st->itn = itn;
    st->inv_alpha = alpha > 0.0 ? 1.0 / alpha : 0.0;
    st->coef_u = beta > 0.0 ? -alpha * inv_beta : 0.0;
    if (bad) {
        st->numeric = 1;
        st->colb_skip = 1;
        istop = istop ? istop : 7;
    }
    st->istop = istop;
    if (istop) {
        st->done = 1;
        *flag = 1;
    }
}

// colA: beta from the aprod1 partials; vhat = p z / beta - beta v (first=1: no v term); z <- 0;
// per-block sums of squares of vhat (alpha) and of w (for the condition estimate). In the
// iterations (first=0) the block that finishes last also runs the scalar step (the grid's
// partials are complete then): `counter` counts finished blocks and is reset by that block.
//
// ymax_reset (may be null): the max |y| word of the fixed-point aprod 2 sums; the aprod 2 of this
// iteration has read it, the next iteration's aprod 1 rebuilds it from zero.
__global__ void k_colA(const double *__restrict__ part_u, int n_part_u, double *__restrict__ z,
                       const double *__restrict__ p, double *__restrict__ v, const double *__restrict__ w, int64_t n,
                       LsqrState *__restrict__ st, double *__restrict__ part_v, double *__restrict__ part_w,
                       int32_t first, uint32_t *__restrict__ counter, int32_t *__restrict__ flag,
                       uint32_t *__restrict__ ymax_reset)
{
    __shared__ double sm64[64];
    __shared__ double s_beta, s_ib;
    __shared__ int s_last;
    if (ymax_reset && blockIdx.x == 0 && threadIdx.x == 0) *ymax_reset = 0u;
    if (!first && st->done) {  // stopped: the x / w update of this iteration is skipped as well
        if (blockIdx.x == 0 && threadIdx.x == 0) st->colb_skip = 1;
        return;
    }
    if (threadIdx.x < 32) {
        const double ssq = warp_sum_partials(part_u, n_part_u);
        if (threadIdx.x == 0) {
            s_beta = sqrt(ssq);
            s_ib = 1.0 / s_beta;
        }
    }
    __syncthreads();
    const double beta = s_beta;
    double sv = 0.0, sw = 0.0;
    if (beta > 0.0 && isfinite(beta)) {
        const double ib = s_ib;
        // kColElems columns per thread and round, all loaded before any is used: the loop is
        // latency-bound (a few MB per call), so the loads of a round are issued together
        const int64_t stride = (int64_t)gridDim.x * blockDim.x;
        for (int64_t j0 = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; j0 < n; j0 += kColElems * stride) {
            double zr[kColElems], pr[kColElems], vr[kColElems], wr[kColElems];
#pragma unroll
            for (int q = 0; q < kColElems; ++q) {
                const int64_t j = j0 + q * stride;
                zr[q] = pr[q] = vr[q] = wr[q] = 0.0;
                if (j < n) {
                    zr[q] = z[j];
                    pr[q] = p[j];
                    if (!first) {
                        vr[q] = v[j];
                        wr[q] = w[j];
                    }
                }
            }
#pragma unroll
            for (int q = 0; q < kColElems; ++q) {
                const int64_t j = j0 + q * stride;
                if (j < n) {
                    z[j] = 0.0;
                    double vh = pr[q] * zr[q] * ib;
                    if (!first) vh = fma(-beta, vr[q], vh);
                    v[j] = vh;
                    sv = fma(vh, vh, sv);
                    sw = fma(wr[q], wr[q], sw);
                }
            }
        }
    } else {
        // beta = 0 (b in the range of A already reached) or non-finite: leave v as alpha*v,
        // so that colB restores it; the scalar kernel keeps alpha.
        const double a = first ? 0.0 : st->alpha;
        for (int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; j < n;
             j += (int64_t)gridDim.x * blockDim.x) {
            z[j] = 0.0;
            const double vh = a * v[j];
            v[j] = vh;
            sv = fma(vh, vh, sv);
            if (!first) {
                const double wj = w[j];
                sw = fma(wj, wj, sw);
            }
        }
    }
    const double2 t = block_sum2(sv, sw, sm64);
    if (threadIdx.x == 0) {
        part_v[blockIdx.x] = t.x;
        part_w[blockIdx.x] = t.y;
        if (first && blockIdx.x == 0) st->beta = beta;
        if (!first) {
            __threadfence();  // the partials are visible before the count
            s_last = atomicAdd(counter, 1u) == gridDim.x - 1;
        }
    }
    if (first) return;
    __syncthreads();
    if (!s_last) return;
    __threadfence();
    if (threadIdx.x < 32) scalar_step(st, beta, s_ib, part_v, part_w, gridDim.x, flag);
    if (threadIdx.x == 0) *counter = 0;
}

// colA of a closing iteration (the last of a solve that runs to its iteration limit; no aprod 2
// before it): beta from the aprod 1 partials, the per-block sums of squares of w (the condition
// estimate), and the closing scalar step by the block that finishes last. v, w and z are not
// touched (z stays zero). ymax_reset as in k_colA: the aprod 1 has built max |y|, which nothing
// reads in this iteration.
__global__ void k_colA_close(const double *__restrict__ part_u, int n_part_u, const double *__restrict__ w,
                             int64_t n, LsqrState *__restrict__ st, double *__restrict__ part_w,
                             uint32_t *__restrict__ counter, int32_t *__restrict__ flag,
                             uint32_t *__restrict__ ymax_reset)
{
    __shared__ double sm64[64];
    __shared__ double s_beta, s_ib;
    __shared__ int s_last;
    if (ymax_reset && blockIdx.x == 0 && threadIdx.x == 0) *ymax_reset = 0u;
    if (st->done) {
        if (blockIdx.x == 0 && threadIdx.x == 0) st->colb_skip = 1;
        return;
    }
    if (threadIdx.x < 32) {
        const double ssq = warp_sum_partials(part_u, n_part_u);
        if (threadIdx.x == 0) {
            s_beta = sqrt(ssq);
            s_ib = 1.0 / s_beta;
        }
    }
    double sw = 0.0;
    for (int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; j < n; j += (int64_t)gridDim.x * blockDim.x) {
        const double wj = w[j];
        sw = fma(wj, wj, sw);
    }
    const double2 t = block_sum2(0.0, sw, sm64);  // synchronises the block (s_beta is then visible)
    if (threadIdx.x == 0) {
        part_w[blockIdx.x] = t.y;
        __threadfence();
        s_last = atomicAdd(counter, 1u) == gridDim.x - 1;
    }
    __syncthreads();
    if (!s_last) return;
    __threadfence();
    const double beta = s_beta;
    if (threadIdx.x < 32) scalar_step<true>(st, beta, s_ib, nullptr, part_w, gridDim.x, flag);
    if (threadIdx.x == 0) *counter = 0;
}

// colB of a closing iteration: x += t1 w, var += (w / rho)^2 (v and w are not needed again)
__global__ void k_colB_close(const double *__restrict__ w, double *__restrict__ x, double *__restrict__ var, int64_t n,
                             const LsqrState *__restrict__ st)
{
    if (st->colb_skip) return;
    const double t1 = st->t1, ir = st->inv_rho;
    for (int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; j < n; j += (int64_t)gridDim.x * blockDim.x) {
        const double wj = w[j];
        x[j] = fma(t1, wj, x[j]);
        if (var) {
            const double d = wj * ir;
            var[j] = fma(d, d, var[j]);
        }
    }
}

// The start of LSQR: beta_1 u_1 = b, alpha_1 v_1 = A~^T u_1, w_1 = v_1, x_0 = 0,
// phibar_1 = beta_1, rhobar_1 = alpha_1 (one warp; thread 0 writes).
__global__ void k_scalar_init(LsqrState *__restrict__ st, const double *__restrict__ part_v, int n_part,
                              int32_t *__restrict__ flag)
{
    const double ssq = warp_sum_partials(part_v, n_part);
    if (threadIdx.x != 0) return;
    const double beta = st->beta;
    const double alpha = sqrt(ssq);
    st->alpha = alpha;
    st->rhobar = alpha;
    st->phibar = beta;
    st->anorm = 0.0;
    st->acond = 0.0;
    st->ddnorm = 0.0;
    st->res2 = 0.0;
    st->xnorm = 0.0;
    st->xxnorm = 0.0;
    st->zeta = 0.0;
    st->cs2 = -1.0;
    st->sn2 = 0.0;
    st->bnorm = beta;
    st->rnorm = beta;
    st->r1norm = beta;
    st->r2norm = beta;
    st->arnorm = alpha * beta;
    st->arnorm0 = alpha * beta;
    st->itn = 0;
    st->istop = 0;
    st->numeric = !(isfinite(alpha) && isfinite(beta));
    st->done = (st->arnorm == 0.0 || st->numeric || st->itnlim <= 0) ? 1 : 0;
    st->colb_skip = 0;
    st->inv_alpha = alpha > 0.0 ? 1.0 / alpha : 0.0;
    st->t1 = 0.0;
    st->t2 = 0.0;
    st->inv_rho = 0.0;
    st->coef_u = beta > 0.0 ? -alpha / beta : 0.0;
    *flag = st->done;
}

// colB (first=1: the start, w = v and x = 0)
__global__ void k_colB(double *__restrict__ v, double *__restrict__ pv, float *__restrict__ pv32,
                       const double *__restrict__ p, double *__restrict__ w, double *__restrict__ x,
                       double *__restrict__ var, int64_t n, const LsqrState *__restrict__ st, int32_t first)
{
    if (!first && st->colb_skip) return;
    const double ia = st->inv_alpha;
    const double t1 = st->t1, t2 = st->t2, ir = st->inv_rho;
    const bool has_alpha = st->alpha > 0.0;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t j0 = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; j0 < n; j0 += kColElems * stride) {
        double vr[kColElems], pr[kColElems], wr[kColElems], xr[kColElems];
#pragma unroll
        for (int q = 0; q < kColElems; ++q) {
            const int64_t j = j0 + q * stride;
            vr[q] = pr[q] = wr[q] = xr[q] = 0.0;
            if (j < n) {
                vr[q] = v[j];
                pr[q] = p[j];
                if (!first) {
                    wr[q] = w[j];
                    xr[q] = x[j];
                }
            }
        }
#pragma unroll
        for (int q = 0; q < kColElems; ++q) {
            const int64_t j = j0 + q * stride;
            if (j >= n) continue;
            const double vj = has_alpha ? vr[q] * ia : vr[q];
            v[j] = vj;
            const double pvj = pr[q] * vj;
            pv[j] = pvj;
            if (pv32) pv32[j] = (float)pvj;
            if (first) {
                w[j] = vj;
                x[j] = 0.0;
                if (var) var[j] = 0.0;
            } else {
                const double wj = wr[q];
                if (var) {
                    const double d = wj * ir;
                    var[j] = fma(d, d, var[j]);
                }
                x[j] = fma(t1, wj, xr[q]);
                w[j] = fma(t2, wj, vj);
            }
        }
    }
}

// x_out = p * x (+ x0); se = sqrt(var) * p * s (s = |r| / sqrt(max(m - n, 1)))
__global__ void k_finish(const double *__restrict__ x, const double *__restrict__ p, const double *__restrict__ x0,
                         double *__restrict__ out, const double *__restrict__ var, double *__restrict__ se,
                         const LsqrState *__restrict__ st, int64_t n, double dof)
{
    const double s = fabs(st->r1norm) / sqrt(dof);
    for (int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; j < n; j += (int64_t)gridDim.x * blockDim.x) {
        double xv = x[j] * p[j];
        if (x0) xv += x0[j];
        out[j] = xv;
        if (se) se[j] = sqrt(var[j]) * p[j] * s;
    }
}

__global__ void k_negate(const double *__restrict__ a, double *__restrict__ out, int64_t n)
{
    for (int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; j < n; j += (int64_t)gridDim.x * blockDim.x)
        out[j] = -a[j];
}

// ---------------------------------------------------------------- host side
// k_colA / k_colB: two blocks per SM (each thread takes kColElems columns a round)
static int colab_grid(const gsr_ctx *c, int64_t n)
{
    int64_t g = (n + (int64_t)kColThreads * kColElems - 1) / ((int64_t)kColThreads * kColElems);
    const int64_t cap = (int64_t)c->sm_count * 2;
    if (g > cap) g = cap;
    if (g < 1) g = 1;
    return (int)g;
}

int col_grid(const gsr_ctx *c, int64_t n)
{
    int64_t g = (n + kColThreads - 1) / kColThreads;
    const int64_t cap = (int64_t)c->sm_count * 4;
    if (g > cap) g = cap;
    if (g < 1) g = 1;
    return (int)g;
}

gsr_status ensure_workspace(gsr_ctx *c)
{
    Workspace &ws = c->ws;
    if (ws.u) return GSR_OK;
    const size_t nr = (size_t)(c->n_rows > 0 ? c->n_rows : 1), nc = (size_t)c->n_cols;
    cudaError_t e = cudaSuccess;
    double **cols[] = {&ws.z, &ws.v, &ws.w, &ws.x, &ws.pv, &ws.p, &ws.var, &ws.tmp};
    if ((e = cudaMalloc(&ws.u, nr * sizeof(double))) != cudaSuccess) goto oom;
    for (double **pp : cols)
        if ((e = cudaMalloc(pp, nc * sizeof(double))) != cudaSuccess) goto oom;
    if ((e = cudaMalloc(&ws.part_u, 3 * MAX_PARTIALS * sizeof(double))) != cudaSuccess) goto oom;
    ws.part_v = ws.part_u + MAX_PARTIALS;
    ws.part_w = ws.part_v + MAX_PARTIALS;
    if ((e = cudaMalloc(&ws.st, sizeof(LsqrState))) != cudaSuccess) goto oom;
    if ((e = cudaHostAlloc(&ws.flag_h, sizeof(int32_t), cudaHostAllocMapped)) != cudaSuccess) goto oom;
    if ((e = cudaHostAlloc(&ws.fin_h, sizeof(LsqrState), cudaHostAllocDefault)) != cudaSuccess) goto oom;
    if ((e = cudaHostAlloc(&ws.blk_h, 8 * sizeof(double), cudaHostAllocDefault)) != cudaSuccess) goto oom;
    if ((e = cudaHostGetDevicePointer(&ws.flag_d, ws.flag_h, 0)) != cudaSuccess) goto oom;
    if ((e = cudaMalloc(&ws.counter, sizeof(uint32_t))) != cudaSuccess) goto oom;
    if ((e = cudaMemset(ws.counter, 0, sizeof(uint32_t))) != cudaSuccess) goto oom;
    if ((e = cudaMemset(ws.z, 0, nc * sizeof(double))) != cudaSuccess) goto oom;
    if ((e = cudaMemset(ws.part_u, 0, 3 * MAX_PARTIALS * sizeof(double))) != cudaSuccess) goto oom;
    if (c->prec == GSR_FP32) {
        // mixed-precision solver: binary32 row vector, gathered column vector, split x
        if ((e = cudaMalloc(&ws.u32, nr * sizeof(float))) != cudaSuccess) goto oom;
        if ((e = cudaMalloc(&ws.pv32, nc * sizeof(float))) != cudaSuccess) goto oom;
        if ((e = cudaMalloc(&ws.xo, nc * sizeof(double))) != cudaSuccess) goto oom;
        if ((e = cudaMalloc(&ws.xhl, nc * sizeof(float2))) != cudaSuccess) goto oom;
        if ((e = cudaMalloc(&ws.blk, 16 * sizeof(double))) != cudaSuccess) goto oom;
    }
    ws.n_rows = c->n_rows;
    ws.n_cols = c->n_cols;
    return GSR_OK;
oom:
    free_workspace(c);
    cudaGetLastError();
    return fail(c, GSR_ENOMEM, std::string("workspace allocation failed: ") + cudaGetErrorString(e));
}

void free_workspace(gsr_ctx *c)
{
    Workspace &ws = c->ws;
    double *ptrs[] = {ws.u, ws.z, ws.v, ws.w, ws.x, ws.pv, ws.p, ws.var, ws.tmp, ws.part_u, ws.xo, ws.blk, ws.wacc,
                      ws.x0w};
    if (ws.feats) cudaFree(ws.feats);
    if (ws.netout) cudaFree(ws.netout);
    if (ws.astro_n) cudaFree(ws.astro_n);
    for (double *p : ptrs)
        if (p) cudaFree(p);
    if (ws.u32) cudaFree(ws.u32);
    if (ws.pv32) cudaFree(ws.pv32);
    if (ws.xhl) cudaFree(ws.xhl);
    if (ws.st) cudaFree(ws.st);
    if (ws.counter) cudaFree(ws.counter);
    if (ws.flag_h) cudaFreeHost(ws.flag_h);
    if (ws.fin_h) cudaFreeHost(ws.fin_h);
    if (ws.blk_h) cudaFreeHost(ws.blk_h);
    for (auto &gc : ws.graphs)
        if (gc.exec) cudaGraphExecDestroy(gc.exec);
    ws = Workspace();
}

void drop_graphs(gsr_ctx *c)
{
    for (auto &gc : c->ws.graphs)
        if (gc.exec) cudaGraphExecDestroy(gc.exec);
    c->ws.graphs.clear();
}

// The executable graph of `k` LSQR iterations (aprod 1, aprod 2 in one pass or two, colA
// with the scalar step, colB: 4 or 5 kernels each), captured on first use and cached on
// the context (kernel arguments are the context's fixed buffers; the iteration state lives
// in device memory); dropped when a reload changes the fixed-point kernel choice.
// close: the graph's last iteration is a closing one (aprod 1, k_colA_close, k_colB_close), for the
// last launch of a solve whose iteration limit is a multiple of k.
static cudaError_t iteration_graph(gsr_ctx *c, int k, bool want_var, bool inner32, cudaStream_t s,
                                   cudaGraphExec_t *out, bool close = false)
{
    Workspace &ws = c->ws;
    const int fused = inner32 && iter_fused(c) ? c->fused_inner : 0;
    for (auto &gc : ws.graphs) {
        if (gc.exec && gc.k == k && gc.var == want_var && gc.inner32 == inner32 && gc.fused == fused &&
            gc.close == close) {
            *out = gc.exec;
            return cudaSuccess;
        }
    }
    const int gu1 = aprod1_grid(c, inner32);  // the partials of a standalone aprod 1 (closing iteration)
    int gu = gu1;
    if (fused) launch_iter_fused(c, nullptr, nullptr, nullptr, nullptr, nullptr, s, &gu);
    const int gc = colab_grid(c, c->n_cols);
    // the fused binary32 aprod 2 leaves the max |y| word to colA (the attitude pass clears it otherwise)
    uint32_t *ymax_reset = inner32 && att_fused(c) ? fx_ymax(c) : nullptr;
    void *u = inner32 ? (void *)ws.u32 : (void *)ws.u;
    const void *pv = inner32 ? (const void *)ws.pv32 : (const void *)ws.pv;
    float *pv32 = c->prec == GSR_FP32 ? ws.pv32 : nullptr;
    cudaGraph_t g = nullptr;
    cudaGraphExec_t exec = nullptr;
    cudaError_t e = cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal);
    if (e != cudaSuccess) return e;
    for (int i = 0; i < k && e == cudaSuccess; ++i) {
        if (close && i == k - 1) {  // the x update from beta_{k+1}: aprod 1 only
            if ((e = launch_aprod1(c, pv, u, ws.st, ws.part_u, s, inner32)) != cudaSuccess) break;
            k_colA_close<<<gc, kColThreads, 0, s>>>(ws.part_u, gu1, ws.w, c->n_cols, ws.st, ws.part_w, ws.counter,
                                                    ws.flag_d, inner32 ? fx_ymax(c) : nullptr);
            k_colB_close<<<gc, kColThreads, 0, s>>>(ws.w, ws.x, want_var ? ws.var : nullptr, c->n_cols, ws.st);
            e = cudaGetLastError();
            break;
        }
        if (fused) {  // both products in one pass over the tiles
            if ((e = launch_iter_fused(c, (const float *)pv, (float *)u, ws.z, ws.st, ws.part_u, s)) != cudaSuccess)
                break;
        } else {
            if ((e = launch_aprod1(c, pv, u, ws.st, ws.part_u, s, inner32)) != cudaSuccess) break;
            if ((e = launch_aprod2(c, u, ws.z, false, ws.st, s, inner32)) != cudaSuccess) break;
        }
        k_colA<<<gc, kColThreads, 0, s>>>(ws.part_u, gu, ws.z, ws.p, ws.v, ws.w, c->n_cols, ws.st, ws.part_v,
                                          ws.part_w, 0, ws.counter, ws.flag_d, ymax_reset);
        k_colB<<<gc, kColThreads, 0, s>>>(ws.v, ws.pv, pv32, ws.p, ws.w, ws.x, want_var ? ws.var : nullptr,
                                          c->n_cols, ws.st, 0);
        e = cudaGetLastError();
    }
    cudaError_t e2 = cudaStreamEndCapture(s, &g);
    if (e == cudaSuccess) e = e2;
    if (e == cudaSuccess) e = cudaGraphInstantiate(&exec, g, 0);
    if (g) cudaGraphDestroy(g);
    if (e != cudaSuccess) return e;
    GraphCache gcache;
    gcache.exec = exec;
    gcache.k = k;
    gcache.var = want_var;
    gcache.inner32 = inner32;
    gcache.fused = fused;
    gcache.close = close;
    ws.graphs.push_back(gcache);
    *out = exec;
    return cudaSuccess;
}

void default_params(gsr_solve_params *p)
{
    *p = gsr_solve_params();
    p->itnlim = 2000;
    p->atol = 1e-12;
    p->btol = 1e-12;
    p->conlim = 1e12;
    p->damp = 0.0;
    p->precond = 1;
    p->mode = GSR_PLAIN;
    p->warm = GSR_WARM_NONE;
    p->weights_path = nullptr;
    p->timeout_s = 0.0;
    p->graph_k = 0;
    p->where = GSR_HOST;
    p->inner_itn = 0;
    p->inner_tol = 0.0;
    p->refine_tol = 0.0;
    p->max_outer = 0;
    p->inner_itn_next = 0;
    p->refine_grad = 0;
    p->inner_fused = 1;
    p->inner_close = 1;
}

// p = 1/|A_:,j| into ws.p. f32: squares and per-block partial sums in
// binary32 (binary32-stored systems; used by the mixed solver, whose
// refinement does not depend on the exact scaling), otherwise binary64.
gsr_status precond_pass(gsr_ctx *c, bool use, cudaStream_t s, bool f32, const void *y, double *z)
{
    Workspace &ws = c->ws;
    const int64_t nc = c->n_cols;
    cudaError_t e = cudaMemsetAsync(ws.tmp, 0, nc * sizeof(double), s);
    if (e != cudaSuccess) return cuda_fail(c, e, "memset");
    if (use && y) {
        if ((e = launch_aprod2_both(c, y, z, ws.tmp, s, f32)) != cudaSuccess) return cuda_fail(c, e, "A^T y + norms");
    } else if (use && (e = launch_aprod2(c, nullptr, ws.tmp, true, nullptr, s, f32)) != cudaSuccess) {
        return cuda_fail(c, e, "column norms");
    }
    k_precond_finish<<<col_grid(c, nc), kColThreads, 0, s>>>(ws.tmp, ws.p, nc, use ? 1 : 0);
    if ((e = cudaGetLastError()) != cudaSuccess) return cuda_fail(c, e, "preconditioner");
    return GSR_OK;
}

// LSQR from a prepared start: the row vector (ws.u, or ws.u32 when inner32)
// holds the right-hand side and part_u[0..n_part_u) its per-block sums of
// squares. Runs the start (alpha_1 v_1 = A~^T u_1) and the iterations; leaves
// the scaled solution in ws.x and the final scalars in *fin.
gsr_status run_lsqr(gsr_ctx *c, const LsqrState &init, bool inner32, bool want_var, int n_part_u, int graph_k,
                    double timeout_s, std::chrono::steady_clock::time_point t0, cudaStream_t s, LsqrState *fin,
                    bool defer_fin, bool start64, bool close)
{
    using clk = std::chrono::steady_clock;
    Workspace &ws = c->ws;
    const int64_t nc = c->n_cols;
    const int gc = colab_grid(c, nc);
    float *pv32 = c->prec == GSR_FP32 ? ws.pv32 : nullptr;
    cudaError_t e;
    if ((e = cudaMemcpyAsync(ws.st, &init, sizeof(init), cudaMemcpyHostToDevice, s)) != cudaSuccess)
        return cuda_fail(c, e, "state upload");
    // start64: the start's A^T u reads the binary64 copy of the right-hand side (ws.u) with binary64
    // products and sums, the iterations the binary32 one (inner32)
    void *u = inner32 && !start64 ? (void *)ws.u32 : (void *)ws.u;
    if ((e = launch_aprod2(c, u, ws.z, false, nullptr, s, inner32 && !start64)) != cudaSuccess)
        return cuda_fail(c, e, "start");
    k_colA<<<gc, kColThreads, 0, s>>>(ws.part_u, n_part_u, ws.z, ws.p, ws.v, ws.w, nc, ws.st, ws.part_v, ws.part_w, 1,
                                      ws.counter, ws.flag_d, nullptr);
    k_scalar_init<<<1, 32, 0, s>>>(ws.st, ws.part_v, gc, ws.flag_d);
    k_colB<<<gc, kColThreads, 0, s>>>(ws.v, ws.pv, pv32, ws.p, ws.w, ws.x, want_var ? ws.var : nullptr, nc, ws.st, 1);
    if ((e = cudaGetLastError()) != cudaSuccess) return cuda_fail(c, e, "LSQR start");

    int k = graph_k > 0 ? graph_k : 8;
    if (k > init.itnlim && init.itnlim > 0) k = init.itnlim;
    if (k < 1) k = 1;
    if (close && graph_k <= 0 && init.itnlim > 0) {
        // the largest divisor of the limit up to k, so that the last launch ends on the limit
        int d = k;
        while (init.itnlim % d) --d;
        if (2 * d >= k) k = d;
    }
    close = close && init.itnlim > 0 && init.itnlim % k == 0;
    cudaGraphExec_t exec = nullptr, exec_close = nullptr;
    if ((e = iteration_graph(c, k, want_var, inner32, s, &exec)) != cudaSuccess) return cuda_fail(c, e, "graph capture");
    if (close && (e = iteration_graph(c, k, want_var, inner32, s, &exec_close, true)) != cudaSuccess)
        return cuda_fail(c, e, "graph capture");
    // No host round trip between the start and the first launch, nor after the last one: errors of the
    // start surface at the next synchronisation, and the graph's kernels skip their work once the
    // device-side state says the solve has stopped. The host waits between launches only to read the
    // stop flag.
    gsr_status status = GSR_OK;
    int launched = 0;
    const int max_launch = init.itnlim > 0 ? (init.itnlim + k - 1) / k : 0;
    while (launched < max_launch) {
        if ((e = cudaGraphLaunch(close && launched == max_launch - 1 ? exec_close : exec, s)) != cudaSuccess) {
            status = cuda_fail(c, e, "graph launch");
            break;
        }
        if (++launched == max_launch) break;
        if ((e = cudaStreamSynchronize(s)) != cudaSuccess) {
            status = cuda_fail(c, e, "LSQR iteration");
            break;
        }
        if (*(volatile int32_t *)ws.flag_h) break;
        if (timeout_s > 0.0 && std::chrono::duration<double>(clk::now() - t0).count() > timeout_s) {
            status = fail(c, GSR_ETIMEOUT, "solve exceeded timeout_s");
            break;
        }
    }
    if ((e = cudaMemcpyAsync(ws.fin_h, ws.st, sizeof(LsqrState), cudaMemcpyDeviceToHost, s)) != cudaSuccess)
        return cuda_fail(c, e, "state download");
    if (defer_fin) return status;  // the caller synchronises s and reads ws.fin_h
    if ((e = cudaStreamSynchronize(s)) != cudaSuccess) return cuda_fail(c, e, "state download");
    *fin = *ws.fin_h;
    if (status == GSR_OK && timeout_s > 0.0 && std::chrono::duration<double>(clk::now() - t0).count() > timeout_s)
        status = fail(c, GSR_ETIMEOUT, "solve exceeded timeout_s");
    return status;
}

LsqrState initial_state(const gsr_solve_params *prm)
{
    LsqrState init = LsqrState();
    init.damp = prm->damp;
    init.atol = prm->atol;
    init.btol = prm->btol;
    init.ctol = prm->conlim > 0.0 ? 1.0 / prm->conlim : 0.0;
    init.itnlim = prm->itnlim;
    return init;
}

void fill_info(gsr_solve_info *info, const LsqrState &fin, std::chrono::steady_clock::time_point t0)
{
    if (!info) return;
    info->istop = fin.istop;
    info->itn = fin.itn;
    info->outer_itn = 0;
    info->r1norm = fin.r1norm;
    info->r2norm = fin.r2norm;
    info->anorm = fin.anorm;
    info->acond = fin.acond;
    info->arnorm = fin.arnorm;
    info->xnorm = fin.xnorm;
    info->ms_total = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
    info->ms_warm = 0.0;
}

gsr_status lsqr_solve(gsr_ctx *c, const gsr_solve_params *prm, const double *x0, bool x0_dev, double *x_out,
                      double *se_out, gsr_solve_info *info, cudaStream_t s, bool p_ready)
{
    const auto t0 = std::chrono::steady_clock::now();
    gsr_status rc = ensure_workspace(c);
    if (rc != GSR_OK) return rc;
    Workspace &ws = c->ws;
    const int64_t nc = c->n_cols, nr = c->n_rows;
    const bool dev_io = prm->where == GSR_DEVICE;
    const bool want_var = se_out != nullptr;
    const int gc = col_grid(c, nc);
    const int gr = col_grid(c, nr);
    cudaError_t e;

    // preconditioner p = 1/|A_:,j| (Alg. 1): one pass over A per solve
    if (!p_ready && (rc = precond_pass(c, prm->precond != 0, s)) != GSR_OK) return rc;

    // x0: u = b - A x0 ; otherwise u = b
    const double *x0d = nullptr;
    double *x0_buf = nullptr;
    if (x0) {
        if (dev_io || x0_dev) {
            x0d = x0;
        } else {
            if ((e = cudaMalloc(&x0_buf, nc * sizeof(double))) != cudaSuccess)
                return fail(c, GSR_ENOMEM, "x0 buffer allocation failed");
            if ((e = cudaMemcpyAsync(x0_buf, x0, nc * sizeof(double), cudaMemcpyHostToDevice, s)) != cudaSuccess) {
                cudaFree(x0_buf);
                return cuda_fail(c, e, "x0 copy");
            }
            x0d = x0_buf;
        }
        k_negate<<<gc, kColThreads, 0, s>>>(x0d, ws.x, nc);
        k_copy_ssq<<<gr, kColThreads, 0, s>>>(c->b, ws.u, nr, ws.part_u);
        launch_aprod1(c, ws.x, ws.u, nullptr, nullptr, s);  // u = b - A x0
        k_ssq<<<gr, kColThreads, 0, s>>>(ws.u, nr, ws.part_u);
    } else {
        k_copy_ssq<<<gr, kColThreads, 0, s>>>(c->b, ws.u, nr, ws.part_u);
    }
    LsqrState fin;
    gsr_status status = run_lsqr(c, initial_state(prm), false, want_var, gr, prm->graph_k, prm->timeout_s, t0, s, &fin);
    if (status != GSR_OK && status != GSR_ETIMEOUT) {
        if (x0_buf) cudaFree(x0_buf);
        return status;
    }
    // result
    double *out_d = dev_io ? x_out : ws.tmp;
    double *se_d = nullptr;
    if (se_out) se_d = dev_io ? se_out : ws.z;  // z is free after the loop (cleared again below)
    const double dof = (double)(nr - nc > 1 ? nr - nc : 1);
    k_finish<<<gc, kColThreads, 0, s>>>(ws.x, ws.p, x0d, out_d, ws.var, se_d, ws.st, nc, dof);
    if ((e = cudaGetLastError()) == cudaSuccess && !dev_io) {
        e = cudaMemcpyAsync(x_out, out_d, nc * sizeof(double), cudaMemcpyDeviceToHost, s);
        if (e == cudaSuccess && se_out) e = cudaMemcpyAsync(se_out, se_d, nc * sizeof(double), cudaMemcpyDeviceToHost, s);
    }
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e == cudaSuccess && se_d == ws.z) e = cudaMemsetAsync(ws.z, 0, nc * sizeof(double), s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (x0_buf) cudaFree(x0_buf);
    if (e != cudaSuccess) return cuda_fail(c, e, "result");
    fill_info(info, fin, t0);
    if (status != GSR_OK) return status;
    if (fin.numeric) return fail(c, GSR_ENUMERIC, "non-finite value in the LSQR scalars");
    return GSR_OK;
}

}  // namespace gsr
