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

__global__ void k_neg_f32(const double *__restrict__ a, float *__restrict__ out, int64_t n)
{
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        out[i] = -(float)a[i];
}

__global__ void k_neg_f64(const double *__restrict__ a, double *__restrict__ out, int64_t n)
{
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        out[i] = -a[i];
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

// Per-star 5x5 solve of the astrometric block. With r_i = b_i minus the
// attitude, instrumental and global parts of row i applied to x0 (one aprod 1
// pass with the astrometric part of x0 still zero), k_astro_normal
// accumulates for every star G = sum a a^T (upper triangle, 15 values) and
// h = sum a r (5 values) over the star's rows (a = the row's 5 astrometric
// coefficients) into N[star][20], in binary32 for binary32 storage (the mixed
// solver's start, refined afterwards) and in binary64 for binary64 storage
// (the plain solver's start, whose products are exact and whose sums are then
// good to ~n_obs 2^-53 relative); k_astro_chol
// adds lambda = 1e-12 trace(G)/5 to the diagonal and solves G x = h by
// Cholesky in binary64, one thread per star (x = 0 when G is not positive
// definite).
static constexpr int NNORM = 20;

// Add a warp's per-lane partial sums of the 20 normal-equation values of star
// k to N (through a per-warp shared buffer: lanes 0..19 each sum one value;
// value j at j * NSTRIDE, 33 elements apart, so that the summing lanes do not
// all read one bank). Warp-collective.
constexpr int NSTRIDE = 33;

template <typename NT>
__device__ __forceinline__ void flush_normal_run(NT (&acc)[NNORM], int64_t k, NT *__restrict__ wbuf,
                                                 NT *__restrict__ N)
{
    const int lane = threadIdx.x & 31;
#pragma unroll
    for (int j = 0; j < NNORM; ++j) {
        wbuf[j * NSTRIDE + lane] = acc[j];
        acc[j] = (NT)0;
    }
    __syncwarp();
    if (lane < NNORM) {
        NT t = (NT)0;
#pragma unroll 8
        for (int l = 0; l < 32; ++l) t += wbuf[lane * NSTRIDE + l];
        atomicAdd(N + NNORM * k + lane, t);
    }
    __syncwarp();
}

// the 20 products of one row: a_p a_q (p <= q), then a_p r
template <typename NT>
__device__ __forceinline__ void normal_terms(const NT (&a)[NASTRO], NT r, NT (&out)[NNORM])
{
    int q = 0;
#pragma unroll
    for (int p = 0; p < NASTRO; ++p)
#pragma unroll
        for (int c = p; c < NASTRO; ++c) out[q++] = a[p] * a[c];
#pragma unroll
    for (int p = 0; p < NASTRO; ++p) out[15 + p] = a[p] * r;
}

// this lane's R consecutive entries of a row vector as NT (0 past n_rows)
template <typename RT, typename NT, int R>
__device__ __forceinline__ void load_rows(const RT *__restrict__ r, int64_t r0, int64_t n, NT (&out)[R])
{
#pragma unroll
    for (int i = 0; i < R; ++i) out[i] = r0 + i < n ? (NT)__ldcs(r + r0 + i) : (NT)0;
}

// Each warp owns a contiguous range of row tiles (as the star pass of aprod 2):
// products of the current star accumulate per lane and are flushed once per
// star; at a tile that crosses a star boundary the run of star k is flushed
// first, then the tile's rows of the next star start the new run, and stars
// that begin and end inside one tile are added directly. N must be zero on
// entry; r holds the residual of the non-astrometric parts (n_rows entries).
//
// A section variant with n_astro < 5 keeps the 20-value layout: its missing
// astrometric coefficients are zero, so their rows and columns of G and
// entries of h stay zero (k_astro_chol solves only the leading n_astro).
template <typename VT, typename RT, typename NT, bool SV = false>
__global__ void __launch_bounds__(256) k_astro_normal(SysView<VT> S, const RT *__restrict__ r,
                                                      NT *__restrict__ N, int64_t tiles_per_warp)
{
    const int na = SV ? S.na : NASTRO;
    constexpr int R = Tile<VT>::R;
    constexpr int T = Tile<VT>::T;
    __shared__ NT wred[8][NNORM * NSTRIDE];
    const int lane = threadIdx.x & 31;
    NT *wbuf = wred[threadIdx.x >> 5];
    const int64_t gw = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t t0 = gw * tiles_per_warp;
    const int64_t t1 = min(S.n_tiles, t0 + tiles_per_warp);
    NT acc[NNORM];
#pragma unroll
    for (int j = 0; j < NNORM; ++j) acc[j] = (NT)0;
    int64_t k = t0 < S.n_tiles ? S.first_star[t0] : 0;
    for (int64_t t = t0; t < t1; ++t) {
        const uint8_t *tb = S.tiles + t * S.tile_bytes;
        const int64_t r0 = t * T + lane * R;
        NT rv[R];
        load_rows<RT, NT, R>(r, r0, S.n_rows, rv);
        NT a[NASTRO][R];
#pragma unroll
        for (int j = 0; j < NASTRO; ++j) {
            // a variant's absent slots read an attitude plane (always present), zeroed after the load
            load_vals<VT, NT>(tb, j < na ? j : (SV ? S.p_att : A_ATT), a[j]);
#pragma unroll
            for (int i = 0; i < R; ++i) a[j][i] = j < na ? a[j][i] : (NT)0;
        }
#pragma unroll
        for (int i = 0; i < R; ++i)
            if (r0 + i >= S.n_rows)
#pragma unroll
                for (int j = 0; j < NASTRO; ++j) a[j][i] = (NT)0;
        const int64_t tile_end = min((t + 1) * T, S.n_rows);
        if (__ldg(S.star_ptr + k + 1) >= tile_end) {  // the whole tile belongs to star k
#pragma unroll
            for (int i = 0; i < R; ++i) {
                NT ar[NASTRO], tr[NNORM];
#pragma unroll
                for (int j = 0; j < NASTRO; ++j) ar[j] = a[j][i];
                normal_terms(ar, rv[i], tr);
#pragma unroll
                for (int j = 0; j < NNORM; ++j) acc[j] += tr[j];
            }
        } else {
            const int64_t kn2 = star_of_row(S.star_ptr, S.first_star, t, tile_end - 1);
            int64_t sr[R];
            stars_of_rows<R>(S.star_ptr, S.first_star, t, r0, sr);
#pragma unroll
            for (int i = 0; i < R; ++i)
                if (sr[i] == k) {
                    NT ar[NASTRO], tr[NNORM];
#pragma unroll
                    for (int j = 0; j < NASTRO; ++j) ar[j] = a[j][i];
                    normal_terms(ar, rv[i], tr);
#pragma unroll
                    for (int j = 0; j < NNORM; ++j) acc[j] += tr[j];
                }
            flush_normal_run(acc, k, wbuf, N);
#pragma unroll
            for (int i = 0; i < R; ++i) {
                if (sr[i] == k) continue;
                NT ar[NASTRO], tr[NNORM];
#pragma unroll
                for (int j = 0; j < NASTRO; ++j) ar[j] = a[j][i];
                normal_terms(ar, rv[i], tr);
                if (sr[i] == kn2) {
#pragma unroll
                    for (int j = 0; j < NNORM; ++j) acc[j] += tr[j];
                } else if (r0 + i < S.n_rows) {
#pragma unroll
                    for (int j = 0; j < NNORM; ++j) atomicAdd(N + NNORM * sr[i] + j, tr[j]);
                }
            }
            k = kn2;
        }
    }
    if (t0 < t1) flush_normal_run(acc, k, wbuf, N);
}

// r -= (astrometric part of the rows) x0, in binary32, over the row tiles in
// grid-stride order; per-block sums of squares of the new r into part. With r
// the residual of the other parts of x0 this gives the residual of the whole
// warm start, for the first refinement step of the mixed solver.
template <bool SV = false>
__global__ void __launch_bounds__(256) k_astro_residual(SysView<float> S, const double *__restrict__ x0,
                                                        float *__restrict__ r, double *__restrict__ part)
{
    const int na = SV ? S.na : NASTRO;
    constexpr int R = Tile<float>::R;
    constexpr int T = Tile<float>::T;
    __shared__ double sm32[32];
    const int lane = threadIdx.x & 31;
    const int64_t gw = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
    float ssq = 0.f;
    for (int64_t t = gw; t < S.n_tiles; t += nw) {
        const uint8_t *tb = S.tiles + t * S.tile_bytes;
        float a[NASTRO][R];
#pragma unroll
        for (int j = 0; j < NASTRO; ++j) load_vals<float, float>(tb, j < na ? j : (SV ? S.p_att : A_ATT), a[j]);
        const int64_t r0 = t * T + lane * R;
        int64_t sr[R];
        stars_of_rows<R>(S.star_ptr, S.first_star, t, r0, sr);
        const bool full = r0 + R <= S.n_rows;  // all of this lane's rows exist: one 16-byte access
        float v[R];
        if (full) {
            const float4 q = *reinterpret_cast<const float4 *>(r + r0);
            v[0] = q.x, v[1] = q.y, v[2] = q.z, v[3] = q.w;
        } else {
#pragma unroll
            for (int i = 0; i < R; ++i) v[i] = r0 + i < S.n_rows ? r[r0 + i] : 0.f;
        }
#pragma unroll
        for (int i = 0; i < R; ++i) {
            const double *xa = x0 + (int64_t)na * sr[i];
#pragma unroll
            for (int j = 0; j < NASTRO; ++j) {  // a variant's absent slots gather x0[0], masked to zero
                const float xv = (float)__ldg(j < na ? xa + j : x0);
                v[i] = fmaf(-a[j][i], j < na ? xv : 0.f, v[i]);
            }
            if (r0 + i < S.n_rows) ssq = fmaf(v[i], v[i], ssq);
        }
        if (full) {
            *reinterpret_cast<float4 *>(r + r0) = make_float4(v[0], v[1], v[2], v[3]);
        } else {
#pragma unroll
            for (int i = 0; i < R; ++i)
                if (r0 + i < S.n_rows) r[r0 + i] = v[i];
        }
    }
    const double tot = block_sum((double)ssq, sm32);
    if (threadIdx.x == 0) part[blockIdx.x] = tot;
}

// na: astrometric unknowns per star (5 in the standard row); a section variant's
// trailing rows and columns (zero in N) get a unit diagonal and give x = 0
template <typename NT>
__global__ void k_astro_chol(const NT *__restrict__ N, int64_t n_stars, double *__restrict__ x0, int na)
{
    for (int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; s < n_stars;
         s += (int64_t)gridDim.x * blockDim.x) {
        const NT *n = N + NNORM * s;
        double M[NASTRO][NASTRO], L[NASTRO][NASTRO], y[NASTRO], xs[NASTRO];
        int q = 0;
#pragma unroll
        for (int p = 0; p < NASTRO; ++p)
#pragma unroll
            for (int c = p; c < NASTRO; ++c) {
                M[p][c] = M[c][p] = (double)n[q];
                ++q;
            }
        double tr = 0.0;
#pragma unroll
        for (int p = 0; p < NASTRO; ++p) tr += p < na ? M[p][p] : 0.0;
        const double lam = 1e-12 * tr / (double)na;
#pragma unroll
        for (int p = 0; p < NASTRO; ++p) M[p][p] = p < na ? M[p][p] + lam : 1.0;
        bool ok = true;
#pragma unroll
        for (int j = 0; j < NASTRO; ++j) {
            double d = M[j][j];
#pragma unroll
            for (int k2 = 0; k2 < j; ++k2) d -= L[j][k2] * L[j][k2];
            ok = ok && d > 0.0;
            L[j][j] = sqrt(ok ? d : 1.0);
#pragma unroll
            for (int i2 = j + 1; i2 < NASTRO; ++i2) {
                double v = M[i2][j];
#pragma unroll
                for (int k2 = 0; k2 < j; ++k2) v -= L[i2][k2] * L[j][k2];
                L[i2][j] = v / L[j][j];
            }
        }
#pragma unroll
        for (int i2 = 0; i2 < NASTRO; ++i2) {
            double v = (double)n[15 + i2];
#pragma unroll
            for (int k2 = 0; k2 < i2; ++k2) v -= L[i2][k2] * y[k2];
            y[i2] = v / L[i2][i2];
        }
#pragma unroll
        for (int i2 = NASTRO - 1; i2 >= 0; --i2) {
            double v = y[i2];
#pragma unroll
            for (int k2 = i2 + 1; k2 < NASTRO; ++k2) v -= L[k2][i2] * xs[k2];
            xs[i2] = v / L[i2][i2];
        }
#pragma unroll
        for (int i2 = 0; i2 < NASTRO; ++i2)
            if (i2 < na) x0[(int64_t)na * s + i2] = ok ? xs[i2] : 0.0;
    }
}

static int grid_for(const gsr_ctx *c, int64_t n)
{
    return (int)std::max<int64_t>(1, std::min<int64_t>((n + kThreads - 1) / kThreads, (int64_t)c->sm_count * 4));
}

// k_astro_normal over contiguous tile ranges, one range per resident warp (at least 8 tiles each)
template <typename VT, typename RT, typename NT>
static cudaError_t astro_normal_launch(const gsr_ctx *c, const RT *r, cudaStream_t s)
{
    auto kern = c->sv ? k_astro_normal<VT, RT, NT, true> : k_astro_normal<VT, RT, NT, false>;
    int per_sm = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, kThreads, 0) != cudaSuccess || per_sm < 1)
        per_sm = 1;
    const int64_t wpb = kThreads / 32;
    const int64_t max_warps = (int64_t)per_sm * c->sm_count * wpb;
    const int64_t per = std::max<int64_t>((c->n_tiles + max_warps - 1) / max_warps, 8);
    const int64_t warps = (c->n_tiles + per - 1) / per;
    const int64_t blocks = std::max<int64_t>((warps + wpb - 1) / wpb, 1);
    kern<<<(unsigned)blocks, kThreads, 0, s>>>(view<VT>(c), r, static_cast<NT *>(c->ws.astro_n), per);
    return cudaGetLastError();
}

// features of the loaded system into ws.feats, the device scale into ws.wacc[2];
// keep_z leaves z = A^T b in ws.z (the caller clears it)
gsr_status warm_features_dev(gsr_ctx *c, cudaStream_t s, bool keep_z)
{
    gsr_status rc = ensure_workspace(c);
    if (rc != GSR_OK) return rc;
    // binary64 storage: the combined pass below runs in binary64 (attitude pass, knot-ordered copy)
    if ((rc = ensure_att_layout(c, s, c->prec == GSR_FP64)) != GSR_OK) return rc;
    Workspace &ws = c->ws;
    cudaError_t e = cudaSuccess;
    if (!ws.feats) {
        if ((e = cudaMalloc(&ws.feats, sizeof(float) * 6 * (size_t)c->n_dfa)) != cudaSuccess ||
            (e = cudaMalloc(&ws.netout, sizeof(float) * 3 * (size_t)c->n_dfa)) != cudaSuccess ||
            (e = cudaMalloc(&ws.wacc, sizeof(double) * 4)) != cudaSuccess)
            return cuda_fail(c, e, "warm-start buffers");
    }
    // p = 1/|A_:,j| and z = A^T b (z is zero between uses) in one pass over the rows; binary32
    // products and sums for binary32 storage (b rounded to binary32 in ws.u32)
    const bool f32 = c->prec == GSR_FP32;
    if (f32) k_to_f32<<<grid_for(c, c->n_rows), kThreads, 0, s>>>(c->b, ws.u32, c->n_rows);
    if ((rc = precond_pass(c, true, s, f32, f32 ? (const void *)ws.u32 : (const void *)c->b, ws.z)) != GSR_OK)
        return rc;
    const int64_t att0 = (int64_t)c->n_astro * c->n_stars;
    if ((e = cudaMemsetAsync(ws.wacc, 0, sizeof(double) * 4, s)) != cudaSuccess) return cuda_fail(c, e, "memset");
    k_att_features<<<grid_for(c, c->n_dfa), kThreads, 0, s>>>(ws.z, ws.p, att0, c->n_dfa, ws.feats, ws.wacc);
    k_normalise_features<<<grid_for(c, c->n_dfa), kThreads, 0, s>>>(ws.feats, c->n_dfa, ws.wacc, ws.wacc + 2);
    if (!keep_z && (e = cudaMemsetAsync(ws.z, 0, sizeof(double) * (size_t)c->n_cols, s)) != cudaSuccess)
        return cuda_fail(c, e, "memset");
    if ((e = cudaGetLastError()) != cudaSuccess) return cuda_fail(c, e, "features");
    return GSR_OK;
}

// x0 (device) from the features and (optionally) the network
gsr_status warm_start_dev(gsr_ctx *c, gsr_net *net, double *x0, cudaStream_t s, int *r0_parts)
{
    if (r0_parts) *r0_parts = 0;
    gsr_status rc = warm_features_dev(c, s, true);
    if (rc != GSR_OK) return rc;
    Workspace &ws = c->ws;
    if (net && (rc = gsr_net_forward(net, ws.feats, 1, c->n_dfa, ws.netout, s)) != GSR_OK)
        return fail(c, rc, std::string("warm start: ") + gsr_net_last_error(net));
    const int64_t att0 = (int64_t)c->n_astro * c->n_stars, instr0 = att0 + (int64_t)NAXES * c->n_dfa;
    k_att_guess<<<grid_for(c, c->n_cols), kThreads, 0, s>>>(ws.feats, net ? ws.netout : nullptr, ws.wacc + 2, att0,
                                                            c->n_dfa, c->n_cols, x0);
    k_rest_guess<<<grid_for(c, c->n_cols - instr0), kThreads, 0, s>>>(ws.z, ws.p, instr0, c->n_cols, x0);
    cudaError_t ez = cudaMemsetAsync(ws.z, 0, sizeof(double) * (size_t)c->n_cols, s);
    if (ez != cudaSuccess) return cuda_fail(c, ez, "memset");
    // per-star normal equations: binary32 for binary32 storage, binary64 for binary64 storage
    const size_t nt_size = c->prec == GSR_FP32 ? sizeof(float) : sizeof(double);
    if (!ws.astro_n && (ez = cudaMalloc(&ws.astro_n, nt_size * NNORM * (size_t)c->n_stars)) != cudaSuccess)
        return cuda_fail(c, ez, "normal-equation buffer");
    if ((ez = cudaMemsetAsync(ws.astro_n, 0, nt_size * NNORM * (size_t)c->n_stars, s)) != cudaSuccess)
        return cuda_fail(c, ez, "memset");
    if (c->n_rows > 0 && c->n_astro > 0) {
        // r = b - A x0 with the astrometric part of x0 still zero: the residual of the other parts
        const int64_t nc = c->n_cols;
        if (c->prec == GSR_FP32) {
            // ws.u32 still holds b rounded to binary32 (the features' pass only read it)
            k_neg_f32<<<grid_for(c, nc), kThreads, 0, s>>>(x0, ws.pv32, nc);
            if ((ez = launch_aprod1(c, ws.pv32, ws.u32, nullptr, nullptr, s, true)) == cudaSuccess)
                ez = astro_normal_launch<float, float, float>(c, ws.u32, s);
        } else {
            k_neg_f64<<<grid_for(c, nc), kThreads, 0, s>>>(x0, ws.tmp, nc);
            if ((ez = cudaMemcpyAsync(ws.u, c->b, sizeof(double) * (size_t)c->n_rows, cudaMemcpyDeviceToDevice,
                                      s)) == cudaSuccess &&
                (ez = launch_aprod1(c, ws.tmp, ws.u, nullptr, nullptr, s, false)) == cudaSuccess)
                ez = astro_normal_launch<double, double, double>(c, ws.u, s);
        }
        if (ez != cudaSuccess) return cuda_fail(c, ez, "warm start: normal equations");
    }
    if (c->n_astro > 0) {
        if (c->prec == GSR_FP32)
            k_astro_chol<float><<<grid_for(c, c->n_stars), kThreads, 0, s>>>(static_cast<const float *>(ws.astro_n),
                                                                             c->n_stars, x0, c->n_astro);
        else
            k_astro_chol<double><<<grid_for(c, c->n_stars), kThreads, 0, s>>>(
                static_cast<const double *>(ws.astro_n), c->n_stars, x0, c->n_astro);
    }
    if (r0_parts && c->prec == GSR_FP32 && c->n_rows > 0 && c->n_astro > 0) {
        // ws.u32 holds the residual of the non-astrometric parts: complete it (binary32) into the
        // residual of x0, with its per-block sums of squares in ws.part_u
        const int g = (int)std::min<int64_t>(std::max<int64_t>((c->n_tiles + 7) / 8, 1), (int64_t)c->sm_count * 4);
        if (c->sv)
            k_astro_residual<true><<<g, kThreads, 0, s>>>(view<float>(c), x0, ws.u32, ws.part_u);
        else
            k_astro_residual<false><<<g, kThreads, 0, s>>>(view<float>(c), x0, ws.u32, ws.part_u);
        *r0_parts = g;
    }
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
    gsr_status rc = warm_start_dev(c, net, x0, s, nullptr);
    if (rc != GSR_OK) return rc;
    if ((e = cudaStreamSynchronize(s)) != cudaSuccess) return cuda_fail(c, e, "warm start");
    return GSR_OK;
}
