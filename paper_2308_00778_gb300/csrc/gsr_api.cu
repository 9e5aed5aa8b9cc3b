// gsr_api.cu -- the C ABI of libgsr (include/gsr.h): contexts, loading the
// system into SoA device planes, aprod 1/2 on caller buffers, and the solve.
#include <algorithm>
#include <cmath>
#include <chrono>
#include <cstring>

#include "../../include/gsr_warm.h"
#include "tiles.cuh"

#define GSR_API extern "C" __attribute__((visibility("default")))

namespace gsr {

gsr_status fail(gsr_ctx *c, gsr_status s, const std::string &msg)
{
    if (c) c->err = msg;
    return s;
}

gsr_status cuda_fail(gsr_ctx *c, cudaError_t e, const char *what)
{
    const std::string m = std::string(what) + ": " + cudaGetErrorString(e);
    cudaGetLastError();
    if (e == cudaErrorMemoryAllocation) return fail(c, GSR_ENOMEM, m);
    return fail(c, GSR_ECUDA, m);
}

bool rows_complete(const gsr_ctx *c)
{
    if (c->n_rows == 0) return true;
    return c->rows_set.size() == 1 && c->rows_set[0].first == 0 && c->rows_set[0].second == c->n_rows;
}

static void mark_rows(gsr_ctx *c, int64_t lo, int64_t hi)
{
    if (hi <= lo) return;
    auto &v = c->rows_set;
    v.emplace_back(lo, hi);
    std::sort(v.begin(), v.end());
    std::vector<std::pair<int64_t, int64_t>> m;
    for (auto &r : v) {
        if (!m.empty() && r.first <= m.back().second)
            m.back().second = std::max(m.back().second, r.second);
        else
            m.push_back(r);
    }
    v.swap(m);
}

// remove [lo, hi) from the loaded ranges (rows whose content is no longer valid)
static void unmark_rows(gsr_ctx *c, int64_t lo, int64_t hi)
{
    std::vector<std::pair<int64_t, int64_t>> m;
    for (auto &r : c->rows_set) {
        if (r.second <= lo || r.first >= hi) {
            m.push_back(r);
            continue;
        }
        if (r.first < lo) m.emplace_back(r.first, lo);
        if (r.second > hi) m.emplace_back(hi, r.second);
    }
    c->rows_set.swap(m);
}

// ---------------------------------------------------------------- conversion kernels
// Caller rows: in_w coefficients and ni instrumental columns per row (24 and 6
// for the paper's standard row; the compact row of a section variant).
// error words: [0] knot out of range, [1] instr out of range, [2] non-finite value
template <typename ST>
__global__ void k_validate(const ST *__restrict__ vals, int32_t layout, int64_t vstride, const int32_t *__restrict__ knot,
                           const int32_t *__restrict__ instr, int64_t n, int32_t n_dfa, int32_t n_instr,
                           int32_t in_w, int32_t ni, int32_t *__restrict__ errw)
{
    int32_t bk = 0, bi = 0, bv = 0;
    for (int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; r < n; r += (int64_t)gridDim.x * blockDim.x) {
        const int32_t k = knot[r];
        bk |= (k < 0 || k > n_dfa - 4);
        for (int j = 0; j < ni; ++j) {
            const int32_t ic = layout == GSR_AOS ? instr[r * ni + j] : instr[j * vstride + r];
            bi |= (ic < 0 || ic >= n_instr);
        }
        for (int j = 0; j < in_w; ++j) {
            const double v = (double)(layout == GSR_AOS ? vals[r * in_w + j] : vals[j * vstride + r]);
            bv |= !isfinite(v);
        }
    }
    if (bk) atomicOr(errw + 0, 1);
    if (bi) atomicOr(errw + 1, 1);
    if (bv) atomicOr(errw + 2, 1);
}

// rows [0, n) of the caller's arrays -> rows [row0, row0 + n) of the tiled layout (tiles.cuh):
// value plane j < npl takes coefficient j of the row when j < in_used, else zero (the
// standard row's global slot without a global)
template <typename ST, typename DT>
__global__ void k_convert(const ST *__restrict__ vals, int32_t layout, int64_t vstride, const int32_t *__restrict__ knot,
                          const int32_t *__restrict__ instr, int64_t n, int32_t in_w, int32_t in_used, int32_t npl,
                          int32_t ni, uint8_t *__restrict__ tiles, int64_t tile_bytes, int32_t iw16, int64_t row0)
{
    using TL = Tile<DT>;
    for (int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; r < n; r += (int64_t)gridDim.x * blockDim.x) {
        const int64_t o = row0 + r;
        uint8_t *tb = tiles + (o / TL::T) * tile_bytes;
        const int64_t i = o % TL::T;
        for (int j = 0; j < npl; ++j) {
            ST v = (ST)0;
            if (j < in_used) v = layout == GSR_AOS ? vals[r * in_w + j] : vals[j * vstride + r];
            reinterpret_cast<DT *>(tb + j * TL::VBLK)[i] = (DT)v;
        }
        reinterpret_cast<int32_t *>(tb + npl * TL::VBLK)[i] = knot[r];
        for (int j = 0; j < ni; ++j)
            store_instr<DT>(tb, npl, iw16, j, (int)i, layout == GSR_AOS ? instr[r * ni + j] : instr[j * vstride + r]);
    }
}

// AoS rows [0, n) of the caller (any device-visible address: device memory or mapped
// pinned host memory) -> rows [row0, row0 + n) of the tiles, validated in the same
// pass (error words as k_validate). The paper's standard 24-coefficient rows only. One block per output tile: the tile's rows are
// read with 16-byte loads (8-byte for the instrumental columns) into shared memory,
// then written plane by plane. vals must be 16-byte aligned, instr 8-byte aligned.
template <typename ST, typename DT>
__global__ void __launch_bounds__(256) k_convert_aos(const ST *__restrict__ vals, const int32_t *__restrict__ knot,
                                                     const int32_t *__restrict__ instr, int64_t n, int64_t row0,
                                                     int32_t n_glob, int32_t n_dfa, int32_t n_instr,
                                                     uint8_t *__restrict__ tiles, int64_t tile_bytes, int32_t iw16,
                                                     int32_t *__restrict__ errw)
{
    using TL = Tile<DT>;
    constexpr int T = TL::T;
    __shared__ __align__(16) ST sv[T * NPAR];
    __shared__ __align__(16) int32_t si[T * NINSTR];
    __shared__ int32_t sk[T];
    int32_t bk = 0, bi = 0, bv = 0;
    const int64_t t_first = row0 / T, t_last = (row0 + n - 1) / T;
    for (int64_t t = t_first + blockIdx.x; t <= t_last; t += gridDim.x) {
        const int64_t o_lo = max(row0, t * T), o_hi = min(row0 + n, (t + 1) * T);
        const int64_t r_lo = o_lo - row0;  // first input row
        const int m = (int)(o_hi - o_lo), off = (int)(o_lo - t * T);
        {
            const int nv = m * NPAR * (int)sizeof(ST) / 16;
            const int4 *src = reinterpret_cast<const int4 *>(vals + r_lo * NPAR);
            int4 *dst = reinterpret_cast<int4 *>(sv + off * NPAR);
            for (int q = threadIdx.x; q < nv; q += blockDim.x) dst[q] = src[q];
            const int ni = m * NINSTR / 2;
            const int2 *srci = reinterpret_cast<const int2 *>(instr + r_lo * NINSTR);
            int2 *dsti = reinterpret_cast<int2 *>(si + off * NINSTR);
            for (int q = threadIdx.x; q < ni; q += blockDim.x) dsti[q] = srci[q];
            for (int q = threadIdx.x; q < m; q += blockDim.x) sk[off + q] = knot[r_lo + q];
        }
        __syncthreads();
        uint8_t *tb = tiles + t * tile_bytes;
        for (int i = off + (int)threadIdx.x; i < off + m; i += blockDim.x) {
#pragma unroll 4
            for (int j = 0; j < NPAR; ++j) {
                ST v = sv[i * NPAR + j];
                bv |= !isfinite((double)v);
                if (j == NPAR - 1 && n_glob == 0) v = (ST)0;
                reinterpret_cast<DT *>(tb + j * TL::VBLK)[i] = (DT)v;
            }
            const int32_t k = sk[i];
            bk |= (k < 0 || k > n_dfa - 4);
            reinterpret_cast<int32_t *>(tb + NPAR * TL::VBLK)[i] = k;
#pragma unroll
            for (int j = 0; j < NINSTR; ++j) {
                const int32_t ic = si[i * NINSTR + j];
                bi |= (ic < 0 || ic >= n_instr);
                store_instr<DT>(tb, NPAR, iw16, j, i, ic);
            }
        }
        __syncthreads();
    }
    if (__syncthreads_or(bk) && threadIdx.x == 0) atomicOr(errw + 0, 1);
    if (__syncthreads_or(bi) && threadIdx.x == 0) atomicOr(errw + 1, 1);
    if (__syncthreads_or(bv) && threadIdx.x == 0) atomicOr(errw + 2, 1);
}

__global__ void k_check_finite(const double *__restrict__ a, int64_t n, int32_t *__restrict__ errw)
{
    int32_t bad = 0;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        bad |= !isfinite(a[i]);
    if (bad) atomicOr(errw + 2, 1);
}

static int grid_for(const gsr_ctx *c, int64_t n, int threads = 256)
{
    int64_t g = (n + threads - 1) / threads;
    const int64_t cap = (int64_t)c->sm_count * 8;
    if (g > cap) g = cap;
    if (g < 1) g = 1;
    return (int)g;
}

template <typename ST>
static gsr_status set_rows_device(gsr_ctx *c, int64_t row0, int64_t nrows, const ST *vals, int32_t layout,
                                  int64_t vstride, const int32_t *knot, const int32_t *instr, cudaStream_t s)
{
    cudaError_t e;
    if ((e = cudaMemsetAsync(c->errw, 0, 4 * sizeof(int32_t), s)) != cudaSuccess) return cuda_fail(c, e, "memset");
    const int g = grid_for(c, nrows);
    k_validate<ST><<<g, 256, 0, s>>>(vals, layout, vstride, knot, instr, nrows, c->n_dfa, c->n_instr, c->in_w,
                                     c->n_ipr, c->errw);
    int32_t hw[4];
    if ((e = cudaMemcpyAsync(hw, c->errw, sizeof(hw), cudaMemcpyDeviceToHost, s)) != cudaSuccess ||
        (e = cudaStreamSynchronize(s)) != cudaSuccess)
        return cuda_fail(c, e, "validation");
    if (hw[0]) return fail(c, GSR_EINVAL, "att_knot out of range [0, n_dfa-4]");
    if (hw[1]) return fail(c, GSR_EINVAL, "instr_col out of range [0, n_instr)");
    if (hw[2]) return fail(c, GSR_ENUMERIC, "non-finite coefficient");
    // coefficients copied from the row: all of a compact row; the standard row's global slot only
    // with a global
    const int32_t in_used = c->sv ? c->in_w : std::min(c->in_w, A_GLOB + c->n_glob);
    if (c->prec == GSR_FP32)
        k_convert<ST, float><<<g, 256, 0, s>>>(vals, layout, vstride, knot, instr, nrows, c->in_w, in_used, c->npl,
                                                c->n_ipr, (uint8_t *)c->tiles, c->tile_bytes, c->iw16, row0);
    else
        k_convert<ST, double><<<g, 256, 0, s>>>(vals, layout, vstride, knot, instr, nrows, c->in_w, in_used, c->npl,
                                                 c->n_ipr, (uint8_t *)c->tiles, c->tile_bytes, c->iw16, row0);
    if ((e = cudaGetLastError()) != cudaSuccess || (e = cudaStreamSynchronize(s)) != cudaSuccess)
        return cuda_fail(c, e, "conversion");
    return GSR_OK;
}

// host input. When the rows fit in a quarter of the free device memory they
// are staged whole, validated on the device and converted (nothing is written
// on error). Otherwise they are validated on the host first, then staged and
// converted chunk by chunk.
// the device address of mapped pinned host memory (nullptr for pageable memory)
static const void *mapped(const void *p)
{
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return nullptr;
    }
    return a.type == cudaMemoryTypeHost ? a.devicePointer : nullptr;
}

// AoS rows in mapped pinned host memory: converted straight from host memory in one pass (the
// transfer is the bound), validated in the same pass; on an error the rows are marked not loaded.
template <typename ST>
static gsr_status set_rows_mapped(gsr_ctx *c, int64_t row0, int64_t nrows, const ST *vals, const int32_t *knot,
                                  const int32_t *instr, cudaStream_t s)
{
    cudaError_t e;
    if ((e = cudaMemsetAsync(c->errw, 0, 4 * sizeof(int32_t), s)) != cudaSuccess) return cuda_fail(c, e, "memset");
    const int g = (int)std::max<int64_t>(1, std::min<int64_t>(c->n_tiles, (int64_t)c->sm_count * 4));
    if (c->prec == GSR_FP32)
        k_convert_aos<ST, float><<<g, 256, 0, s>>>(vals, knot, instr, nrows, row0, c->n_glob, c->n_dfa, c->n_instr,
                                                    (uint8_t *)c->tiles, c->tile_bytes, c->iw16, c->errw);
    else
        k_convert_aos<ST, double><<<g, 256, 0, s>>>(vals, knot, instr, nrows, row0, c->n_glob, c->n_dfa, c->n_instr,
                                                     (uint8_t *)c->tiles, c->tile_bytes, c->iw16, c->errw);
    int32_t hw[4];
    if ((e = cudaGetLastError()) != cudaSuccess ||
        (e = cudaMemcpyAsync(hw, c->errw, sizeof(hw), cudaMemcpyDeviceToHost, s)) != cudaSuccess ||
        (e = cudaStreamSynchronize(s)) != cudaSuccess)
        return cuda_fail(c, e, "conversion");
    if (hw[0] || hw[1] || hw[2]) {
        unmark_rows(c, row0, row0 + nrows);
        c->att_valid = false;
        c->fx_valid = false;
        if (hw[0]) return fail(c, GSR_EINVAL, "att_knot out of range [0, n_dfa-4] (the rows are not loaded)");
        if (hw[1]) return fail(c, GSR_EINVAL, "instr_col out of range [0, n_instr) (the rows are not loaded)");
        return fail(c, GSR_ENUMERIC, "non-finite coefficient (the rows are not loaded)");
    }
    return GSR_OK;
}

template <typename ST>
static gsr_status set_rows_host(gsr_ctx *c, int64_t row0, int64_t nrows, const ST *vals, int32_t layout,
                                int64_t vstride, const int32_t *knot, const int32_t *instr, cudaStream_t s)
{
    if (layout == GSR_AOS && !c->sv && c->in_w == NPAR) {  // the standard row: the single-pass path
        const void *dv = mapped(vals), *dk = mapped(knot), *di = mapped(instr);
        if (dv && dk && di && (uintptr_t)dv % 16 == 0 && (uintptr_t)di % 8 == 0)
            return set_rows_mapped<ST>(c, row0, nrows, (const ST *)dv, (const int32_t *)dk, (const int32_t *)di, s);
    }
    const int32_t W = c->in_w, NI = c->n_ipr;  // coefficients and instrumental columns per caller row
    const size_t row_bytes = sizeof(ST) * W + sizeof(int32_t) * (1 + NI);
    size_t free_b = 0, total_b = 0;
    cudaMemGetInfo(&free_b, &total_b);
    const bool whole = (size_t)nrows * row_bytes <= free_b / 4;
    if (!whole) {
        for (int64_t r = 0; r < nrows; ++r) {
            if (knot[r] < 0 || knot[r] > c->n_dfa - 4)
                return fail(c, GSR_EINVAL, "att_knot out of range [0, n_dfa-4]");
            for (int j = 0; j < NI; ++j) {
                const int32_t ic = layout == GSR_AOS ? instr[r * NI + j] : instr[j * vstride + r];
                if (ic < 0 || ic >= c->n_instr) return fail(c, GSR_EINVAL, "instr_col out of range [0, n_instr)");
            }
            for (int j = 0; j < W; ++j) {
                const double v = (double)(layout == GSR_AOS ? vals[r * W + j] : vals[j * vstride + r]);
                if (!std::isfinite(v)) return fail(c, GSR_ENUMERIC, "non-finite coefficient");
            }
        }
    }
    const int64_t chunk = whole ? nrows : std::min<int64_t>(nrows, 1 << 21);
    ST *dv = nullptr;
    int32_t *dk = nullptr, *di = nullptr;
    cudaError_t e;
    if ((e = cudaMalloc(&dv, sizeof(ST) * W * (size_t)std::max<int64_t>(chunk, 1))) != cudaSuccess ||
        (e = cudaMalloc(&dk, sizeof(int32_t) * (size_t)std::max<int64_t>(chunk, 1))) != cudaSuccess ||
        (e = cudaMalloc(&di, sizeof(int32_t) * std::max(NI, 1) * (size_t)std::max<int64_t>(chunk, 1))) !=
            cudaSuccess) {
        cudaFree(dv);
        cudaFree(dk);
        cudaFree(di);
        return cuda_fail(c, e, "staging allocation");
    }
    gsr_status rc = GSR_OK;
    for (int64_t r = 0; r < nrows && rc == GSR_OK; r += chunk) {
        const int64_t m = std::min(chunk, nrows - r);
        if (layout == GSR_AOS) {
            e = cudaMemcpyAsync(dv, vals + r * W, sizeof(ST) * W * m, cudaMemcpyHostToDevice, s);
            if (e == cudaSuccess && NI > 0)
                e = cudaMemcpyAsync(di, instr + r * NI, sizeof(int32_t) * NI * m, cudaMemcpyHostToDevice, s);
        } else {
            e = cudaMemcpy2DAsync(dv, sizeof(ST) * m, vals + r, sizeof(ST) * vstride, sizeof(ST) * m, W,
                                  cudaMemcpyHostToDevice, s);
            if (e == cudaSuccess && NI > 0)
                e = cudaMemcpy2DAsync(di, sizeof(int32_t) * m, instr + r, sizeof(int32_t) * vstride,
                                      sizeof(int32_t) * m, NI, cudaMemcpyHostToDevice, s);
        }
        if (e == cudaSuccess) e = cudaMemcpyAsync(dk, knot + r, sizeof(int32_t) * m, cudaMemcpyHostToDevice, s);
        if (e != cudaSuccess) {
            rc = cuda_fail(c, e, "row upload");
            break;
        }
        // device-resident staged rows: validate then convert, exactly as for device input
        rc = set_rows_device<ST>(c, row0 + r, m, dv, layout, m, dk, di, s);
    }
    cudaFree(dv);
    cudaFree(dk);
    cudaFree(di);
    return rc;
}

}  // namespace gsr

using namespace gsr;

// ---------------------------------------------------------------- entry points
GSR_API const char *gsr_last_error(const gsr_ctx *ctx)
{
    if (!ctx) return "null context";
    return ctx->err.c_str();
}

GSR_API void gsr_default_params(gsr_solve_params *p)
{
    if (p) default_params(p);
}

// one context: sections (n_astro, n_ipr, n_glob), the caller's row width in_w and whether the
// tiles use the compact layout of a section variant (sv)
static gsr_status create_ctx(gsr_ctx **out, int64_t n_stars, int32_t obs_per_star, const int64_t *star_ptr,
                             int32_t n_astro, int32_t n_dfa, int32_t n_instr, int32_t n_ipr, int32_t n_glob,
                             int32_t in_w, bool sv, int32_t value_precision, int32_t device)
{
    if (!out) return GSR_EINVAL;
    *out = nullptr;
    if (n_stars < 1 || n_dfa < 4 || n_instr < n_ipr || n_ipr < 0 || n_ipr > NINSTR || n_astro < 0 ||
        n_astro > NASTRO || n_glob < 0 || n_glob > NGLOB_MAX ||
        (value_precision != GSR_FP64 && value_precision != GSR_FP32) || obs_per_star < 0 ||
        (obs_per_star == 0) != (star_ptr != nullptr))
        return GSR_EINVAL;
    gsr_ctx *c = new gsr_ctx();
    c->device = device;
    c->prec = value_precision;
    c->n_stars = n_stars;
    c->n_dfa = n_dfa;
    c->n_instr = n_instr;
    c->n_glob = n_glob;
    c->n_astro = n_astro;
    c->n_ipr = n_ipr;
    c->sv = sv;
    c->npl = sv ? n_astro + NAXES * NPARAXIS + n_ipr + n_glob : NPAR;
    c->in_w = in_w;
    c->star_ptr_h.resize((size_t)n_stars + 1);
    if (star_ptr) {
        if (star_ptr[0] != 0) {
            delete c;
            return GSR_EINVAL;
        }
        for (int64_t s = 0; s < n_stars; ++s) {
            if (star_ptr[s + 1] < star_ptr[s]) {
                delete c;
                return GSR_EINVAL;
            }
        }
        std::memcpy(c->star_ptr_h.data(), star_ptr, sizeof(int64_t) * (size_t)(n_stars + 1));
    } else {
        for (int64_t s = 0; s <= n_stars; ++s) c->star_ptr_h[s] = s * (int64_t)obs_per_star;
    }
    c->n_rows = c->star_ptr_h[n_stars];
    for (int64_t s = 0; s < n_stars; ++s)
        c->max_obs = std::max<int64_t>(c->max_obs, c->star_ptr_h[s + 1] - c->star_ptr_h[s]);
    c->n_cols = (int64_t)n_astro * n_stars + (int64_t)NAXES * n_dfa + n_instr + n_glob;
    const int64_t rows_per_tile = value_precision == GSR_FP32 ? Tile<float>::T : Tile<double>::T;
    // instrumental columns in 16-bit planes whenever they fit (12 bytes less per row to stream)
    c->iw16 = n_instr <= 65536 ? 1 : 0;
    const int64_t tile_bytes = value_precision == GSR_FP32 ? Tile<float>::bytes(c->npl, n_ipr, c->iw16 != 0)
                                                           : Tile<double>::bytes(c->npl, n_ipr, c->iw16 != 0);
    c->tile_bytes = tile_bytes;
    const int64_t atile_bytes = value_precision == GSR_FP32 ? Tile<float>::ABYTES : Tile<double>::ABYTES;
    c->n_tiles = (c->n_rows + rows_per_tile - 1) / rows_per_tile;
    // first star of each tile (host), star of the last row at index n_tiles
    std::vector<int32_t> first_star((size_t)c->n_tiles + 1, 0);
    {
        int64_t st = 0;
        for (int64_t t = 0; t <= c->n_tiles; ++t) {
            const int64_t row = std::min(t * rows_per_tile, std::max<int64_t>(c->n_rows - 1, 0));
            while (st + 1 < n_stars && c->star_ptr_h[st + 1] <= row) ++st;
            first_star[(size_t)t] = (int32_t)st;
        }
    }

    cudaError_t e = cudaSetDevice(device);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&c->sm_count, cudaDevAttrMultiProcessorCount, device);
    // the scratch array of gsr_residual_static is placed on the device here, while allocating is expected
    if (e == cudaSuccess) e = static_scratch_load(sv);
    if (e != cudaSuccess) {
        cudaGetLastError();
        delete c;
        return GSR_ECUDA;
    }
    const size_t tbytes = (size_t)std::max<int64_t>(c->n_tiles, 1) * (size_t)tile_bytes;
    const size_t abytes = (size_t)std::max<int64_t>(c->n_tiles, 1) * (size_t)atile_bytes;
    // the knot-ordered attitude copy (atiles) is allocated when a binary64 aprod 2 first needs it (layout.cu)
    (void)abytes;
    if ((e = cudaMalloc(&c->tiles, tbytes)) != cudaSuccess ||
        (e = cudaMalloc(&c->first_star, sizeof(int32_t) * first_star.size())) != cudaSuccess ||
        (e = cudaMalloc(&c->star_ptr, sizeof(int64_t) * (size_t)(n_stars + 1))) != cudaSuccess ||
        (e = cudaMalloc(&c->b, sizeof(double) * (size_t)std::max<int64_t>(c->n_rows, 1))) != cudaSuccess ||
        (e = cudaMalloc(&c->errw, 4 * sizeof(int32_t))) != cudaSuccess ||
        (e = cudaMalloc(&c->knot_ptr, sizeof(int64_t) * (size_t)(n_dfa - 2))) != cudaSuccess ||
        (e = cudaStreamCreateWithFlags(&c->own, cudaStreamNonBlocking)) != cudaSuccess ||
        (e = cudaEventCreateWithFlags(&c->ev, cudaEventDisableTiming)) != cudaSuccess ||
        (e = cudaEventCreate(&c->ev_w0)) != cudaSuccess || (e = cudaEventCreate(&c->ev_w1)) != cudaSuccess) {
        cudaGetLastError();
        gsr_destroy(c);
        return e == cudaErrorMemoryAllocation ? GSR_ENOMEM : GSR_ECUDA;
    }
    // the window copies of the binary32 attitude unknowns: binary32 for aprod 1 and the fused pass (one
    // 16-byte window per axis and row, knot-major in 64-byte records), double-float pairs for the
    // residual of a wide attitude block
    if (value_precision == GSR_FP32 && !sv &&
        ((e = cudaMalloc(&c->xwin, sizeof(float4) * 4 * (size_t)n_dfa)) != cudaSuccess ||
         ((int64_t)NAXES * n_dfa > ATT_WINDOW_MIN_COLS &&
          (e = cudaMalloc(&c->xhlwin, sizeof(float4) * 2 * (size_t)NAXES * (size_t)n_dfa)) != cudaSuccess))) {
        cudaGetLastError();
        gsr_destroy(c);
        return e == cudaErrorMemoryAllocation ? GSR_ENOMEM : GSR_ECUDA;
    }
    // padding rows of the last tile hold zeros (zero coefficients contribute nothing)
    e = cudaMemset(c->tiles, 0, tbytes);
    if (e == cudaSuccess)
        e = cudaMemcpy(c->first_star, first_star.data(), sizeof(int32_t) * first_star.size(), cudaMemcpyHostToDevice);
    if (e == cudaSuccess)
        e = cudaMemcpy(c->star_ptr, c->star_ptr_h.data(), sizeof(int64_t) * (size_t)(n_stars + 1),
                       cudaMemcpyHostToDevice);
    if (e != cudaSuccess) {
        cudaGetLastError();
        gsr_destroy(c);
        return GSR_ECUDA;
    }
    *out = c;
    return GSR_OK;
}

GSR_API gsr_status gsr_create(gsr_ctx **out, int64_t n_stars, int32_t obs_per_star, const int64_t *star_ptr,
                              int32_t n_dfa, int32_t n_instr, int32_t n_glob, int32_t value_precision, int32_t device)
{
    if (out) *out = nullptr;
    if (n_glob != 0 && n_glob != 1) return GSR_EINVAL;
    return create_ctx(out, n_stars, obs_per_star, star_ptr, NASTRO, n_dfa, n_instr, NINSTR, n_glob, NPAR, false,
                      value_precision, device);
}

GSR_API gsr_status gsr_create_sections(gsr_ctx **out, int64_t n_stars, int32_t obs_per_star, const int64_t *star_ptr,
                                       int32_t n_astro, int32_t n_dfa, int32_t n_instr, int32_t n_ipr, int32_t n_glob,
                                       int32_t value_precision, int32_t device)
{
    if (out) *out = nullptr;
    if (n_astro < 0 || n_astro > NASTRO || n_ipr < 0 || n_ipr > NINSTR || n_glob < 0 || n_glob > NGLOB_MAX)
        return GSR_EINVAL;
    // the standard sections keep the standard tiles and kernels; the caller's rows are compact
    const bool sv = !(n_astro == NASTRO && n_ipr == NINSTR && n_glob <= 1);
    return create_ctx(out, n_stars, obs_per_star, star_ptr, n_astro, n_dfa, n_instr, n_ipr, n_glob,
                      n_astro + NAXES * NPARAXIS + n_ipr + n_glob, sv, value_precision, device);
}

GSR_API gsr_status gsr_sections(const gsr_ctx *c, int32_t *n_astro, int32_t *n_ipr, int32_t *n_glob,
                                int32_t *row_width)
{
    if (!c) return GSR_EINVAL;
    if (n_astro) *n_astro = c->n_astro;
    if (n_ipr) *n_ipr = c->n_ipr;
    if (n_glob) *n_glob = c->n_glob;
    if (row_width) *row_width = c->in_w;
    return GSR_OK;
}

GSR_API gsr_status gsr_destroy(gsr_ctx *c)
{
    if (!c) return GSR_OK;
    cudaSetDevice(c->device);
    free_workspace(c);
    if (c->warm_net) gsr_net_destroy(c->warm_net);
    cudaFree(c->tiles);
    cudaFree(c->atiles);
    cudaFree(c->first_star);
    cudaFree(c->star_ptr);
    cudaFree(c->b);
    cudaFree(c->errw);
    cudaFree(c->knot_ptr);
    cudaFree(c->fx_word);
    cudaFree(c->fx64_word);
    cudaFree(c->attw);
    cudaFree(c->xwin);
    cudaFree(c->xhlwin);
    if (c->own) cudaStreamDestroy(c->own);
    if (c->pool) {
        cudaDeviceSynchronize();
        cudaMemPoolDestroy(c->pool);
    }
    if (c->ev) cudaEventDestroy(c->ev);
    if (c->ev_w0) cudaEventDestroy(c->ev_w0);
    if (c->ev_w1) cudaEventDestroy(c->ev_w1);
    cudaGetLastError();
    delete c;
    return GSR_OK;
}

GSR_API gsr_status gsr_dims(const gsr_ctx *c, int64_t *n_rows, int64_t *n_cols)
{
    if (!c) return GSR_EINVAL;
    if (n_rows) *n_rows = c->n_rows;
    if (n_cols) *n_cols = c->n_cols;
    return GSR_OK;
}

GSR_API gsr_status gsr_set_rows(gsr_ctx *c, int64_t row0, int64_t nrows, const void *values, int32_t values_fp32,
                                int32_t layout, int64_t plane_stride, const int32_t *att_knot,
                                const int32_t *instr_col, int32_t where, void *stream)
{
    if (!c) return GSR_EINVAL;
    if (row0 < 0 || nrows < 0 || row0 + nrows > c->n_rows) return fail(c, GSR_EINVAL, "row range outside the system");
    if (layout != GSR_AOS && layout != GSR_SOA) return fail(c, GSR_EINVAL, "layout must be GSR_AOS or GSR_SOA");
    if (where != GSR_HOST && where != GSR_DEVICE) return fail(c, GSR_EINVAL, "where must be GSR_HOST or GSR_DEVICE");
    if (values_fp32 != 0 && values_fp32 != 1) return fail(c, GSR_EINVAL, "values_fp32 must be 0 or 1");
    if (nrows == 0) return GSR_OK;
    if (!values || !att_knot || (!instr_col && c->n_ipr > 0)) return fail(c, GSR_EINVAL, "null array");
    if (layout == GSR_SOA && plane_stride < nrows) return fail(c, GSR_EINVAL, "plane_stride < nrows");
    cudaError_t e = cudaSetDevice(c->device);
    if (e != cudaSuccess) return cuda_fail(c, e, "cudaSetDevice");
    cudaStream_t s = (cudaStream_t)stream;
    gsr_status rc;
    if (where == GSR_DEVICE)
        rc = values_fp32 ? set_rows_device<float>(c, row0, nrows, (const float *)values, layout, plane_stride,
                                                  att_knot, instr_col, s)
                         : set_rows_device<double>(c, row0, nrows, (const double *)values, layout, plane_stride,
                                                   att_knot, instr_col, s);
    else
        rc = values_fp32 ? set_rows_host<float>(c, row0, nrows, (const float *)values, layout, plane_stride, att_knot,
                                                instr_col, s)
                         : set_rows_host<double>(c, row0, nrows, (const double *)values, layout, plane_stride,
                                                 att_knot, instr_col, s);
    if (rc == GSR_OK) {
        mark_rows(c, row0, row0 + nrows);
        c->att_valid = false;
        c->fx_valid = false;
    }
    return rc;
}

GSR_API gsr_status gsr_set_rhs(gsr_ctx *c, const double *b, int32_t where, void *stream)
{
    if (!c) return GSR_EINVAL;
    if (!b && c->n_rows > 0) return fail(c, GSR_EINVAL, "null b");
    if (where != GSR_HOST && where != GSR_DEVICE) return fail(c, GSR_EINVAL, "where must be GSR_HOST or GSR_DEVICE");
    cudaError_t e = cudaSetDevice(c->device);
    if (e != cudaSuccess) return cuda_fail(c, e, "cudaSetDevice");
    cudaStream_t s = (cudaStream_t)stream;
    if (c->n_rows == 0) {
        c->rhs_set = true;
        return GSR_OK;
    }
    // copy, then check on the device (a NaN or Inf leaves b unloaded)
    c->rhs_set = false;
    int32_t hw[4];
    e = cudaMemcpyAsync(c->b, b, sizeof(double) * (size_t)c->n_rows,
                        where == GSR_HOST ? cudaMemcpyHostToDevice : cudaMemcpyDeviceToDevice, s);
    if (e == cudaSuccess) e = cudaMemsetAsync(c->errw, 0, sizeof(hw), s);
    if (e == cudaSuccess) {
        k_check_finite<<<grid_for(c, c->n_rows), 256, 0, s>>>(c->b, c->n_rows, c->errw);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaMemcpyAsync(hw, c->errw, sizeof(hw), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return cuda_fail(c, e, "b upload");
    if (hw[2]) return fail(c, GSR_ENUMERIC, "non-finite b (b is not loaded)");
    c->rhs_set = true;
    return GSR_OK;
}

GSR_API gsr_status gsr_set_system(gsr_ctx *c, const void *values, int32_t values_fp32, const int32_t *att_knot,
                                  const int32_t *instr_col, const double *b, int32_t where, void *stream)
{
    if (!c) return GSR_EINVAL;
    gsr_status rc = gsr_set_rows(c, 0, c->n_rows, values, values_fp32, GSR_AOS, 0, att_knot, instr_col, where, stream);
    if (rc != GSR_OK || !b) return rc;
    return gsr_set_rhs(c, b, where, stream);
}

GSR_API gsr_status gsr_aprod1(gsr_ctx *c, const double *x, double *y, void *stream)
{
    if (!c) return GSR_EINVAL;
    if (!rows_complete(c)) return fail(c, GSR_ESTATE, "rows not loaded");
    if ((!x || !y) && c->n_rows > 0) return fail(c, GSR_EINVAL, "null vector");
    cudaError_t e = cudaSetDevice(c->device);
    if (e == cudaSuccess) e = launch_aprod1(c, x, y, nullptr, nullptr, (cudaStream_t)stream);
    if (e != cudaSuccess) return cuda_fail(c, e, "aprod1");
    return GSR_OK;
}

GSR_API gsr_status gsr_aprod2(gsr_ctx *c, const double *y, double *x, void *stream)
{
    if (!c) return GSR_EINVAL;
    if (!rows_complete(c)) return fail(c, GSR_ESTATE, "rows not loaded");
    if ((!x || !y) && c->n_rows > 0) return fail(c, GSR_EINVAL, "null vector");
    cudaError_t e = cudaSetDevice(c->device);
    if (e != cudaSuccess) return cuda_fail(c, e, "cudaSetDevice");
    const gsr_status rc = ensure_att_layout(c, (cudaStream_t)stream, true);
    if (rc != GSR_OK) return rc;
    if ((e = launch_aprod2(c, y, x, false, nullptr, (cudaStream_t)stream)) != cudaSuccess)
        return cuda_fail(c, e, "aprod2");
    return GSR_OK;
}

GSR_API gsr_status gsr_aprod1_f32(gsr_ctx *c, const float *x, float *y, void *stream)
{
    if (!c) return GSR_EINVAL;
    if (c->prec != GSR_FP32) return fail(c, GSR_EINVAL, "binary32 kernels need an FP32-stored context");
    if (!rows_complete(c)) return fail(c, GSR_ESTATE, "rows not loaded");
    if ((!x || !y) && c->n_rows > 0) return fail(c, GSR_EINVAL, "null vector");
    cudaError_t e = cudaSetDevice(c->device);
    if (e == cudaSuccess) e = launch_aprod1(c, x, y, nullptr, nullptr, (cudaStream_t)stream, true);
    if (e != cudaSuccess) return cuda_fail(c, e, "aprod1_f32");
    return GSR_OK;
}

GSR_API gsr_status gsr_aprod2_f32(gsr_ctx *c, const float *y, double *x, void *stream)
{
    if (!c) return GSR_EINVAL;
    if (c->prec != GSR_FP32) return fail(c, GSR_EINVAL, "binary32 kernels need an FP32-stored context");
    if (!rows_complete(c)) return fail(c, GSR_ESTATE, "rows not loaded");
    if ((!x || !y) && c->n_rows > 0) return fail(c, GSR_EINVAL, "null vector");
    cudaError_t e = cudaSetDevice(c->device);
    if (e != cudaSuccess) return cuda_fail(c, e, "cudaSetDevice");
    const gsr_status rc = ensure_att_layout(c, (cudaStream_t)stream, false);
    if (rc != GSR_OK) return rc;
    if ((e = launch_aprod2(c, y, x, false, nullptr, (cudaStream_t)stream, true)) != cudaSuccess)
        return cuda_fail(c, e, "aprod2_f32");
    return GSR_OK;
}

GSR_API gsr_status gsr_aprod12_f32(gsr_ctx *c, const float *x, float *y, double *z, float coef, void *stream)
{
    if (!c) return GSR_EINVAL;
    if (c->prec != GSR_FP32) return fail(c, GSR_EINVAL, "binary32 kernels need an FP32-stored context");
    if (!rows_complete(c)) return fail(c, GSR_ESTATE, "rows not loaded");
    if ((!x || !y || !z) && c->n_rows > 0) return fail(c, GSR_EINVAL, "null vector");
    cudaError_t e = cudaSetDevice(c->device);
    if (e != cudaSuccess) return cuda_fail(c, e, "cudaSetDevice");
    const gsr_status rc = ensure_att_layout(c, (cudaStream_t)stream, false);
    if (rc != GSR_OK) return rc;
    if ((e = launch_aprod12_f32(c, x, y, z, coef, (cudaStream_t)stream)) != cudaSuccess)
        return cuda_fail(c, e, "aprod12_f32");
    return GSR_OK;
}

GSR_API gsr_status gsr_aprod2_plan(gsr_ctx *c, void *stream, int32_t *passes, int32_t *fx_bits,
                                   int32_t *ins_group)
{
    if (!c) return GSR_EINVAL;
    if (c->prec != GSR_FP32) return fail(c, GSR_EINVAL, "binary32 kernels need an FP32-stored context");
    if (!rows_complete(c)) return fail(c, GSR_ESTATE, "rows not loaded");
    const cudaError_t e = cudaSetDevice(c->device);
    if (e != cudaSuccess) return cuda_fail(c, e, "cudaSetDevice");
    const gsr_status rc = ensure_att_layout(c, (cudaStream_t)stream, false);
    if (rc != GSR_OK) return rc;
    if (passes) *passes = att_fused(c) ? 1 : att_red(c) ? 3 : 2;
    if (fx_bits) *fx_bits = c->fx_bits;
    if (ins_group) *ins_group = att_fused(c) && c->fx_uni ? 1 : 0;
    return GSR_OK;
}

GSR_API gsr_status gsr_residual(gsr_ctx *c, const double *x, float *r, void *stream)
{
    if (!c) return GSR_EINVAL;
    if (c->prec != GSR_FP32) return fail(c, GSR_EINVAL, "gsr_residual needs an FP32-stored context");
    if (!rows_complete(c)) return fail(c, GSR_ESTATE, "rows not loaded");
    if (!c->rhs_set) return fail(c, GSR_ESTATE, "b not loaded");
    if ((!x || !r) && c->n_rows > 0) return fail(c, GSR_EINVAL, "null vector");
    const cudaError_t e = cudaSetDevice(c->device);
    if (e != cudaSuccess) return cuda_fail(c, e, "cudaSetDevice");
    return residual_f32(c, x, r, (cudaStream_t)stream);
}

GSR_API gsr_status gsr_lsqr_solve(gsr_ctx *c, const gsr_solve_params *params, const double *x0, double *x_out,
                                  double *se_out, gsr_solve_info *info, void *stream)
{
    const auto t_call = std::chrono::steady_clock::now();
    if (!c) return GSR_EINVAL;
    if (!x_out) return fail(c, GSR_EINVAL, "null x_out");
    gsr_solve_params prm;
    if (params)
        prm = *params;
    else
        default_params(&prm);
    if (prm.itnlim < 0 || prm.damp < 0.0 || prm.atol < 0.0 || prm.btol < 0.0 || prm.conlim < 0.0 ||
        (prm.where != GSR_HOST && prm.where != GSR_DEVICE) || (prm.mode != GSR_PLAIN && prm.mode != GSR_MIXED) ||
        prm.warm < GSR_WARM_NONE || prm.warm > GSR_WARM_LEARNED || prm.inner_itn < 0 || prm.inner_itn_next < 0 ||
        prm.max_outer < 0)
        return fail(c, GSR_EINVAL, "invalid solve parameters");
    if (!rows_complete(c)) return fail(c, GSR_ESTATE, "rows not loaded");
    if (!c->rhs_set) return fail(c, GSR_ESTATE, "b not loaded");
    if (prm.mode == GSR_MIXED && c->prec != GSR_FP32)
        return fail(c, GSR_EINVAL, "GSR_MIXED needs an FP32-stored context");
    if (prm.mode == GSR_MIXED && se_out) return fail(c, GSR_EINVAL, "se_out is computed by GSR_PLAIN solves only");
    if (prm.warm != GSR_WARM_NONE && x0) return fail(c, GSR_EINVAL, "x0 and a warm start are exclusive");
    if (prm.warm == GSR_WARM_LEARNED && !prm.weights_path)
        return fail(c, GSR_EINVAL, "GSR_WARM_LEARNED needs weights_path");
    cudaError_t e = cudaSetDevice(c->device);
    if (e != cudaSuccess) return cuda_fail(c, e, "cudaSetDevice");
    // run on the context's own stream (graph capture needs a non-legacy stream), after the caller's work
    if ((e = cudaEventRecord(c->ev, (cudaStream_t)stream)) != cudaSuccess ||
        (e = cudaStreamWaitEvent(c->own, c->ev, 0)) != cudaSuccess)
        return cuda_fail(c, e, "stream ordering");
    {
        // binary64 aprod 2 passes (the plain solver) read the knot-ordered attitude copy
        const gsr_status rl = ensure_att_layout(c, c->own, prm.mode == GSR_PLAIN);
        if (rl != GSR_OK) return rl;
    }
    // warm start: x0 on the device from the features (and the network)
    const double *x0_use = x0;
    bool x0_dev = false;
    int r0_parts = 0;  // mixed solve from a warm start on binary32 storage: the start's residual is ready
    double ms_warm = 0.0;
    gsr_net *net = nullptr;
    if (prm.warm != GSR_WARM_NONE) {
        if ((e = cudaEventRecord(c->ev_w0, c->own)) != cudaSuccess) return cuda_fail(c, e, "warm start");
        gsr_status rw = ensure_workspace(c);
        if (rw != GSR_OK) return rw;
        if (!c->ws.x0w && (e = cudaMalloc(&c->ws.x0w, sizeof(double) * (size_t)c->n_cols)) != cudaSuccess)
            return cuda_fail(c, e, "warm-start vector");
        if (prm.warm == GSR_WARM_LEARNED) {
            if (!c->warm_net || c->warm_path != prm.weights_path) {
                if (c->warm_net) gsr_net_destroy(c->warm_net);
                c->warm_net = nullptr;
                c->warm_path.clear();
                if ((rw = gsr_net_create(&c->warm_net, c->device)) != GSR_OK) return fail(c, rw, "network allocation");
                if ((rw = gsr_net_load(c->warm_net, prm.weights_path)) != GSR_OK) {
                    const std::string m = gsr_net_last_error(c->warm_net);
                    gsr_net_destroy(c->warm_net);
                    c->warm_net = nullptr;
                    return fail(c, rw, m);
                }
                c->warm_path = prm.weights_path;
            }
            net = c->warm_net;
        }
        if ((rw = warm_start_dev(c, net, c->ws.x0w, c->own, prm.mode == GSR_MIXED ? &r0_parts : nullptr)) != GSR_OK)
            return rw;
        // no host wait here: the warm start's time comes from events once the solve has synchronised
        if ((e = cudaEventRecord(c->ev_w1, c->own)) != cudaSuccess) return cuda_fail(c, e, "warm start");
        x0_use = c->ws.x0w;
        x0_dev = true;
    }
    // the warm start computed p with binary32 sums on binary32 storage and binary64 sums otherwise: the
    // mixed solver (binary32 storage) and the plain solver on binary64 storage reuse it
    const bool p_ready = prm.warm != GSR_WARM_NONE && prm.precond != 0 &&
                         (prm.mode == GSR_MIXED || c->prec == GSR_FP64);
    const gsr_status rc = prm.mode == GSR_MIXED
                              ? mixed_solve(c, &prm, x0_use, x0_dev, x_out, info, c->own, p_ready, r0_parts)
                              : lsqr_solve(c, &prm, x0_use, x0_dev, x_out, se_out, info, c->own, p_ready);
    if (prm.warm != GSR_WARM_NONE) {
        float ms = 0.f;
        if (cudaEventElapsedTime(&ms, c->ev_w0, c->ev_w1) == cudaSuccess) ms_warm = ms;
        cudaGetLastError();
    }
    if (info) {  // the solve ended with a synchronisation: the call's wall time so far is the whole of it
        info->ms_warm = ms_warm;
        info->ms_total = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t_call).count();
    }
    // the caller's stream continues after the solve's last kernel
    if (cudaEventRecord(c->ev, c->own) == cudaSuccess) cudaStreamWaitEvent((cudaStream_t)stream, c->ev, 0);
    cudaGetLastError();
    // the solve has synchronised: a network convolution whose tensor-core wait ran out has reported it
    if (net && net_take_fault(net) && (rc == GSR_OK || rc == GSR_ETIMEOUT))
        return fail(c, GSR_ECUDA, "warm start: a tensor-core wait of the network timed out");
    return rc;
}
