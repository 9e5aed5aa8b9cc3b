// warm.cu -- the warm start of LSQR: attitude features, the network's attitude
// guess, and per-star 5x5 solves for the astrometric block (include/gsr_warm.h).
#include <cmath>

#include "../../include/gsr_warm.h"
#include "tiles.cuh"

#define GSR_API extern "C" __attribute__((visibility("default")))

namespace gsr {

static constexpr int kThreads = 256;

__global__ void k_to_f32(const double *__restrict__ a, float *__restrict__ out, int64_t n)
{
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        out[i] = (float)a[i];
}

// Jacobi estimate and log column norm of the attitude columns; sums for the
// normalisation (sum of squares of the estimate, sum of the logs) in acc[0..1].
__global__ void k_att_features(const double *__restrict__ z, const double *__restrict__ p, int64_t att0, int32_t n_dfa,
                               float *__restrict__ feats, double *__restrict__ acc)
{
    __shared__ double sm32[32];
    double s2 = 0.0, sl = 0.0;
    for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < n_dfa; k += (int64_t)gridDim.x * blockDim.x) {
#pragma unroll
        for (int a = 0; a < NAXES; ++a) {
            const int64_t j = att0 + (int64_t)a * n_dfa + k;
            const double pj = p[j];
            const double jac = z[j] * pj * pj;  // (A^T b)_j / |A_:,j|^2 with |A_:,j| = 1 / p_j
            const double lg = -2.0 * log(pj);   // log |A_:,j|^2 (0 for an empty column, p_j = 1)
            feats[k * 6 + a] = (float)jac;
            feats[k * 6 + 3 + a] = (float)lg;
            s2 += jac * jac;
            sl += lg;
        }
    }
    const double t2 = block_sum(s2, sm32);
    const double tl = block_sum(sl, sm32);
    if (threadIdx.x == 0) {
        atomicAdd(acc, t2);
        atomicAdd(acc + 1, tl);
    }
}

__global__ void k_normalise_features(float *__restrict__ feats, int32_t n_dfa, const double *__restrict__ acc,
                                     double *__restrict__ scale_out)
{
    const double n = 3.0 * (double)n_dfa;
    double scale = sqrt(acc[0] / n);
    if (!(scale > 0.0)) scale = 1.0;
    const float inv = (float)(1.0 / scale), mean = (float)(acc[1] / n);
    for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < n_dfa; k += (int64_t)gridDim.x * blockDim.x) {
#pragma unroll
        for (int a = 0; a < NAXES; ++a) {
            feats[k * 6 + a] *= inv;
            feats[k * 6 + 3 + a] -= mean;
        }
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) *scale_out = scale;
}

// x0: attitude part = scale * (feats[:, 0:3] + net_out), everything else 0
// (the instrumental and global parts are then set by k_rest_guess)
__global__ void k_att_guess(const float *__restrict__ feats, const float *__restrict__ net_out,
                            const double *__restrict__ scale, int64_t att0, int32_t n_dfa, int64_t n_cols,
                            double *__restrict__ x0)
{
    const double sc = *scale;
    for (int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; j < n_cols; j += (int64_t)gridDim.x * blockDim.x) {
        double v = 0.0;
        if (j >= att0 && j < att0 + (int64_t)NAXES * n_dfa) {
            const int64_t a = (j - att0) / n_dfa, k = (j - att0) % n_dfa;
            double f = feats[k * 6 + a];
            if (net_out) f += net_out[k * 3 + a];
            v = sc * f;
        }
        x0[j] = v;
    }
}

// x0 of the instrumental and global unknowns: their Jacobi estimates z_j p_j^2
__global__ void k_rest_guess(const double *__restrict__ z, const double *__restrict__ p, int64_t instr0,
                             int64_t n_cols, double *__restrict__ x0)
{
    for (int64_t j = instr0 + (int64_t)blockIdx.x * blockDim.x + threadIdx.x; j < n_cols;
         j += (int64_t)gridDim.x * blockDim.x)
        x0[j] = z[j] * p[j] * p[j];
}

// Per-star 5x5 solve (one warp per star): with r_i = b_i minus the attitude,
// instrumental and global parts of row i applied to x0, accumulate G = sum a a^T
// and h = sum a r over the star's rows
// (a = the 5 astrometric coefficients; binary32), add lambda = 1e-12 trace(G)/5
// to the diagonal and solve G x = h by Cholesky in binary64 (x = 0 when G is
// not positive definite).
template <typename VT>
__global__ void __launch_bounds__(256) k_astro_solve(SysView<VT> S, const double *__restrict__ b,
                                                     double *__restrict__ x0)
{
    using TL = Tile<VT>;
    const int lane = threadIdx.x & 31;
    const int64_t gw = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
    const double *xt = x0 + S.att0;
    for (int64_t s = gw; s < S.n_stars; s += nw) {
        float G[15], h[5];
#pragma unroll
        for (int q = 0; q < 15; ++q) G[q] = 0.f;
#pragma unroll
        for (int q = 0; q < 5; ++q) h[q] = 0.f;
        for (int64_t r = S.star_ptr[s] + lane; r < S.star_ptr[s + 1]; r += 32) {
            const uint8_t *tb = S.tiles + (r / TL::T) * TL::BYTES;
            const int64_t i = r % TL::T;
            const int32_t k = reinterpret_cast<const int32_t *>(tb + NPAR * TL::VBLK)[i];
            float rr = (float)b[r];
#pragma unroll
            for (int ax = 0; ax < NAXES; ++ax)
#pragma unroll
                for (int j = 0; j < NPARAXIS; ++j)
                    rr -= (float)reinterpret_cast<const VT *>(tb + (NASTRO + NPARAXIS * ax + j) * TL::VBLK)[i] *
                          (float)xt[(int64_t)ax * S.n_dfa + k + j];
#pragma unroll
            for (int j = 0; j < NINSTR; ++j) {
                const int32_t ic = reinterpret_cast<const int32_t *>(tb + NPAR * TL::VBLK + (1 + j) * TL::IBLK)[i];
                rr -= (float)reinterpret_cast<const VT *>(tb + (17 + j) * TL::VBLK)[i] * (float)x0[S.instr0 + ic];
            }
            if (S.n_glob) rr -= (float)reinterpret_cast<const VT *>(tb + 23 * TL::VBLK)[i] * (float)x0[S.glob0];
            float a[5];
#pragma unroll
            for (int p = 0; p < 5; ++p) a[p] = (float)reinterpret_cast<const VT *>(tb + p * TL::VBLK)[i];
            int q = 0;
#pragma unroll
            for (int p = 0; p < 5; ++p) {
                h[p] = fmaf(a[p], rr, h[p]);
#pragma unroll
                for (int c = p; c < 5; ++c) {
                    G[q] = fmaf(a[p], a[c], G[q]);
                    ++q;
                }
            }
        }
#pragma unroll
        for (int q = 0; q < 15; ++q)
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) G[q] += __shfl_xor_sync(0xffffffffu, G[q], o);
#pragma unroll
        for (int q = 0; q < 5; ++q)
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) h[q] += __shfl_xor_sync(0xffffffffu, h[q], o);
        if (lane == 0) {
            double M[5][5], L[5][5] = {{0}}, y[5], xs[5];
            int q = 0;
            for (int p = 0; p < 5; ++p)
                for (int c = p; c < 5; ++c) M[p][c] = M[c][p] = (double)G[q++];
            const double lam = 1e-12 * (M[0][0] + M[1][1] + M[2][2] + M[3][3] + M[4][4]) / 5.0;
            bool ok = true;
            for (int p = 0; p < 5; ++p) M[p][p] += lam;
            for (int j = 0; j < 5 && ok; ++j) {
                double d = M[j][j];
                for (int k2 = 0; k2 < j; ++k2) d -= L[j][k2] * L[j][k2];
                if (!(d > 0.0)) {
                    ok = false;
                    break;
                }
                L[j][j] = sqrt(d);
                for (int i2 = j + 1; i2 < 5; ++i2) {
                    double v = M[i2][j];
                    for (int k2 = 0; k2 < j; ++k2) v -= L[i2][k2] * L[j][k2];
                    L[i2][j] = v / L[j][j];
                }
            }
            if (ok) {
                for (int i2 = 0; i2 < 5; ++i2) {
                    double v = (double)h[i2];
                    for (int k2 = 0; k2 < i2; ++k2) v -= L[i2][k2] * y[k2];
                    y[i2] = v / L[i2][i2];
                }
                for (int i2 = 4; i2 >= 0; --i2) {
                    double v = y[i2];
                    for (int k2 = i2 + 1; k2 < 5; ++k2) v -= L[k2][i2] * xs[k2];
                    xs[i2] = v / L[i2][i2];
                }
            } else {
                for (int i2 = 0; i2 < 5; ++i2) xs[i2] = 0.0;
            }
            for (int i2 = 0; i2 < 5; ++i2) x0[NASTRO * s + i2] = xs[i2];
        }
    }
}

static int grid_for(const gsr_ctx *c, int64_t n)
{
    return (int)std::max<int64_t>(1, std::min<int64_t>((n + kThreads - 1) / kThreads, (int64_t)c->sm_count * 4));
}

// features of the loaded system into ws.feats, the device scale into ws.wacc[2];
// keep_z leaves z = A^T b in ws.z (the caller clears it)
gsr_status warm_features_dev(gsr_ctx *c, cudaStream_t s, bool keep_z)
{
    gsr_status rc = ensure_workspace(c);
    if (rc != GSR_OK) return rc;
    if ((rc = ensure_att_layout(c, s)) != GSR_OK) return rc;
    Workspace &ws = c->ws;
    cudaError_t e = cudaSuccess;
    if (!ws.feats) {
        if ((e = cudaMalloc(&ws.feats, sizeof(float) * 6 * (size_t)c->n_dfa)) != cudaSuccess ||
            (e = cudaMalloc(&ws.netout, sizeof(float) * 3 * (size_t)c->n_dfa)) != cudaSuccess ||
            (e = cudaMalloc(&ws.wacc, sizeof(double) * 4)) != cudaSuccess)
            return cuda_fail(c, e, "warm-start buffers");
    }
    const bool f32 = c->prec == GSR_FP32;
    if ((rc = precond_pass(c, true, s, f32)) != GSR_OK) return rc;
    // z = A^T b (z is zero between uses); binary32 products for binary32 storage
    if (f32) {
        k_to_f32<<<grid_for(c, c->n_rows), kThreads, 0, s>>>(c->b, ws.u32, c->n_rows);
        e = launch_aprod2(c, ws.u32, ws.z, false, nullptr, s, true);
    } else {
        e = launch_aprod2(c, c->b, ws.z, false, nullptr, s, false);
    }
    if (e != cudaSuccess) return cuda_fail(c, e, "features: A^T b");
    const int64_t att0 = (int64_t)NASTRO * c->n_stars;
    if ((e = cudaMemsetAsync(ws.wacc, 0, sizeof(double) * 4, s)) != cudaSuccess) return cuda_fail(c, e, "memset");
    k_att_features<<<grid_for(c, c->n_dfa), kThreads, 0, s>>>(ws.z, ws.p, att0, c->n_dfa, ws.feats, ws.wacc);
    k_normalise_features<<<grid_for(c, c->n_dfa), kThreads, 0, s>>>(ws.feats, c->n_dfa, ws.wacc, ws.wacc + 2);
    if (!keep_z && (e = cudaMemsetAsync(ws.z, 0, sizeof(double) * (size_t)c->n_cols, s)) != cudaSuccess)
        return cuda_fail(c, e, "memset");
    if ((e = cudaGetLastError()) != cudaSuccess) return cuda_fail(c, e, "features");
    return GSR_OK;
}

// x0 (device) from the features and (optionally) the network
gsr_status warm_start_dev(gsr_ctx *c, gsr_net *net, double *x0, cudaStream_t s)
{
    gsr_status rc = warm_features_dev(c, s, true);
    if (rc != GSR_OK) return rc;
    Workspace &ws = c->ws;
    if (net && (rc = gsr_net_forward(net, ws.feats, 1, c->n_dfa, ws.netout, s)) != GSR_OK)
        return fail(c, rc, std::string("warm start: ") + gsr_net_last_error(net));
    const int64_t att0 = (int64_t)NASTRO * c->n_stars, instr0 = att0 + (int64_t)NAXES * c->n_dfa;
    k_att_guess<<<grid_for(c, c->n_cols), kThreads, 0, s>>>(ws.feats, net ? ws.netout : nullptr, ws.wacc + 2, att0,
                                                            c->n_dfa, c->n_cols, x0);
    k_rest_guess<<<grid_for(c, c->n_cols - instr0), kThreads, 0, s>>>(ws.z, ws.p, instr0, c->n_cols, x0);
    cudaError_t ez = cudaMemsetAsync(ws.z, 0, sizeof(double) * (size_t)c->n_cols, s);
    if (ez != cudaSuccess) return cuda_fail(c, ez, "memset");
    const int g = (int)std::max<int64_t>(1, std::min<int64_t>((c->n_stars + 7) / 8, (int64_t)c->sm_count * 8));
    if (c->prec == GSR_FP32)
        k_astro_solve<float><<<g, kThreads, 0, s>>>(view<float>(c), c->b, x0);
    else
        k_astro_solve<double><<<g, kThreads, 0, s>>>(view<double>(c), c->b, x0);
    const cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(c, e, "warm start");
    return GSR_OK;
}

}  // namespace gsr

using namespace gsr;

GSR_API gsr_status gsr_warm_features(gsr_ctx *c, float *feats, double *scale, void *stream)
{
    if (!c || !feats) return GSR_EINVAL;
    if (!rows_complete(c)) return fail(c, GSR_ESTATE, "rows not loaded");
    if (!c->rhs_set) return fail(c, GSR_ESTATE, "b not loaded");
    cudaError_t e = cudaSetDevice(c->device);
    if (e != cudaSuccess) return cuda_fail(c, e, "cudaSetDevice");
    const cudaStream_t s = (cudaStream_t)stream;
    gsr_status rc = warm_features_dev(c, s, false);
    if (rc != GSR_OK) return rc;
    if ((e = cudaMemcpyAsync(feats, c->ws.feats, sizeof(float) * 6 * (size_t)c->n_dfa, cudaMemcpyDeviceToDevice, s)) !=
        cudaSuccess)
        return cuda_fail(c, e, "features copy");
    double sc = 1.0;
    if ((e = cudaMemcpyAsync(&sc, c->ws.wacc + 2, sizeof(double), cudaMemcpyDeviceToHost, s)) != cudaSuccess ||
        (e = cudaStreamSynchronize(s)) != cudaSuccess)
        return cuda_fail(c, e, "features");
    if (scale) *scale = sc;
    return GSR_OK;
}

GSR_API gsr_status gsr_warm_start(gsr_ctx *c, gsr_net *net, double *x0, void *stream)
{
    if (!c || !x0) return GSR_EINVAL;
    if (!rows_complete(c)) return fail(c, GSR_ESTATE, "rows not loaded");
    if (!c->rhs_set) return fail(c, GSR_ESTATE, "b not loaded");
    cudaError_t e = cudaSetDevice(c->device);
    if (e != cudaSuccess) return cuda_fail(c, e, "cudaSetDevice");
    const cudaStream_t s = (cudaStream_t)stream;
    gsr_status rc = warm_start_dev(c, net, x0, s);
    if (rc != GSR_OK) return rc;
    if ((e = cudaStreamSynchronize(s)) != cudaSuccess) return cuda_fail(c, e, "warm start");
    return GSR_OK;
}
