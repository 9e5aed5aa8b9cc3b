// layout.cu -- the knot-ordered ("time-local") copy of the attitude coefficients.
//
// aprod 2 scatters each row's 12 attitude products into the columns of its
// attitude knot. Rows are stored star by star (the astrometric blocks), so
// consecutive rows hit unrelated knots and every product would need an atomic
// add. This file builds, once per loaded system, a second copy of the 12
// attitude coefficients with the rows ordered by knot, in tiles of T positions
// (tiles.cuh; 13 planes per tile):
//   plane j < 12 : attitude coefficient j of row perm[p] at position p
//   plane 12     : perm[p], the row of position p (int32)
//   knot_ptr[k]  : first position of knot k (k = 0..n_dfa-3), knot_ptr[n_dfa-3] = n
// With it the attitude part of aprod 2 reduces runs of equal knot in registers
// and adds each run once (aprod.cu). The sort is CUB's stable radix sort on
// (knot, row) pairs; ties keep row order, so the layout is deterministic.
// For binary32-stored systems the same step measures what the fixed-point
// instrumental sums of the inner star pass need (k_instr_stats).
#include <cub/device/device_radix_sort.cuh>

#include "tiles.cuh"

namespace gsr {

__global__ void k_iota(int32_t *__restrict__ a, int64_t n)
{
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        a[i] = (int32_t)i;
}

// knot of every row, read from the tiles (npl value planes precede the knot plane)
template <typename VT>
__global__ void k_extract_knots(const uint8_t *__restrict__ tiles, int64_t tile_bytes, int32_t npl, int64_t n,
                                int32_t *__restrict__ keys)
{
    using TL = Tile<VT>;
    for (int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; r < n; r += (int64_t)gridDim.x * blockDim.x)
        keys[r] = reinterpret_cast<const int32_t *>(tiles + (r / TL::T) * tile_bytes + npl * TL::VBLK)[r % TL::T];
}

// knot_ptr[k] = first i with sorted_knot[i] >= k (lower bound), k = 0..nk
__global__ void k_knot_ptr(const int32_t *__restrict__ sorted_knot, int64_t n, int32_t nk, int64_t *__restrict__ ptr)
{
    for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k <= nk; k += (int64_t)gridDim.x * blockDim.x) {
        int64_t lo = 0, hi = n;
        while (lo < hi) {
            const int64_t mid = (lo + hi) >> 1;
            if (sorted_knot[mid] < (int32_t)k)
                lo = mid + 1;
            else
                hi = mid;
        }
        ptr[k] = lo;
    }
}

// the 12 attitude coefficients of every row (planes p_att..p_att+11) as one
// contiguous record per row (rows in star order, read plane by plane from the
// tiles: coalesced)
template <typename VT>
__global__ void k_att_rows(const uint8_t *__restrict__ tiles, int64_t tile_bytes, int32_t p_att, int64_t n,
                           VT *__restrict__ rec)
{
    using TL = Tile<VT>;
    constexpr int NA = NAXES * NPARAXIS;
    for (int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; r < n; r += (int64_t)gridDim.x * blockDim.x) {
        const uint8_t *src = tiles + (r / TL::T) * tile_bytes;
        const int64_t ri = r % TL::T;
        VT v[NA];
#pragma unroll
        for (int j = 0; j < NA; ++j) v[j] = reinterpret_cast<const VT *>(src + (p_att + j) * TL::VBLK)[ri];
        using V = typename Vec16<VT>::type;
        constexpr int PER = 16 / (int)sizeof(VT);
#pragma unroll
        for (int q = 0; q < NA / PER; ++q) {
            V w;
            VT *wp = reinterpret_cast<VT *>(&w);
#pragma unroll
            for (int e = 0; e < PER; ++e) wp[e] = v[q * PER + e];
            reinterpret_cast<V *>(rec + r * NA)[q] = w;
        }
    }
}

// position p of the knot-ordered tiles <- the attitude record of row perm[p]
// (one contiguous 48- or 96-byte record per gathered row instead of 12 scattered words)
template <typename VT>
__global__ void k_gather_att(const VT *__restrict__ rec, const int32_t *__restrict__ perm, int64_t n,
                             uint8_t *__restrict__ atiles)
{
    using TL = Tile<VT>;
    constexpr int NA = NAXES * NPARAXIS;
    using V = typename Vec16<VT>::type;
    constexpr int PER = 16 / (int)sizeof(VT);
    for (int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; p < n; p += (int64_t)gridDim.x * blockDim.x) {
        const int64_t r = perm[p];
        uint8_t *dst = atiles + (p / TL::T) * TL::ABYTES;
        const int64_t pi = p % TL::T;
#pragma unroll
        for (int q = 0; q < NA / PER; ++q) {
            const V w = __ldg(reinterpret_cast<const V *>(rec + r * NA) + q);
            const VT *wp = reinterpret_cast<const VT *>(&w);
#pragma unroll
            for (int e = 0; e < PER; ++e) reinterpret_cast<VT *>(dst + (q * PER + e) * TL::VBLK)[pi] = wp[e];
        }
        reinterpret_cast<int32_t *>(dst + NA * TL::VBLK)[pi] = (int32_t)r;
    }
}

// For the fixed-point instrumental sums of the binary32 star pass (aprod.cu),
// per instrumental column j over the pass's partition (each warp a contiguous
// range of `per` tiles, 8 warps a block): the largest number of contributions
// one block adds to column j (kmax[j]) and the largest |coefficient| of column
// j (amax[j], binary32 bits). Both arrays are zero on entry.
template <bool SV>
__global__ void __launch_bounds__(256) k_instr_stats(SysView<float> S, int64_t per, uint32_t *__restrict__ kmax,
                                                     uint32_t *__restrict__ amax)
{
    const Sec<SV> G(S);
    constexpr int R = Tile<float>::R;
    constexpr int T = Tile<float>::T;
    extern __shared__ uint32_t cnt[];  // [n_instr] counts, then [n_instr] max |a| bits
    uint32_t *am = cnt + S.n_instr;
    for (int32_t i = threadIdx.x; i < 2 * S.n_instr; i += blockDim.x) cnt[i] = 0u;
    __syncthreads();
    const int lane = threadIdx.x & 31;
    const int64_t gw = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t t0 = gw * per, t1 = min(S.n_tiles, t0 + per);
    for (int64_t t = t0; t < t1; ++t) {
        const uint8_t *tb = S.tiles + t * S.tile_bytes;
        const int64_t r0 = t * T + lane * R;
#pragma unroll
        for (int j = 0; j < NINSTR; ++j) {
            if (j >= G.ni) break;
            int32_t ic[R];
            load_instr<float>(tb, G.npl, S.iw16, j, ic);
            float a[R];
            load_vals<float, float>(tb, G.p_ins + j, a);
#pragma unroll
            for (int i = 0; i < R; ++i)
                if (r0 + i < S.n_rows) {
                    atomicAdd(cnt + ic[i], 1u);
                    atomicMax(am + ic[i], __float_as_uint(fabsf(a[i])));
                }
        }
    }
    __syncthreads();
    for (int32_t i = threadIdx.x; i < S.n_instr; i += blockDim.x) {
        if (cnt[i]) atomicMax(kmax + i, cnt[i]);
        if (am[i]) atomicMax(amax + i, am[i]);
    }
}

// Per-column bits of the fixed-point sums (all 0: keep binary32 atomics):
// bits_j = 31 - ceil(log2(kmax_j + 1)), so that no block can overflow column j;
// the sums are used only when every column gets at least 20 bits. Launches the
// statistics and the copy of kmax into *kmax_h (asynchronous); the caller
// synchronises s and calls fixed_point_finish.
static gsr_status fixed_point_launch(gsr_ctx *c, cudaStream_t s, std::vector<uint32_t> *kmax_h)
{
    c->fx_bits = 0;
    kmax_h->clear();
    if (c->prec != GSR_FP32 || c->n_rows == 0 || c->n_ipr == 0 || c->n_instr == 0) return GSR_OK;
    const int32_t ni = c->n_instr;
    const size_t smem = 2 * sizeof(uint32_t) * (size_t)ni;  // the stats kernel's and the star pass's
    if (smem > 100 * 1024) return GSR_OK;
    cudaError_t e = cudaSuccess;
    // device words: [0, ni) max |a| per column, [ni, 2ni) bits per column, [2ni] max |y| of the
    // current aprod 2, then [ni] scratch counts
    if (!c->fx_word && (e = cudaMalloc(&c->fx_word, sizeof(uint32_t) * (3 * (size_t)ni + 1))) != cudaSuccess)
        return cuda_fail(c, e, "fixed-point words");
    uint32_t *kcnt = c->fx_word + 2 * ni + 1;
    // the partition: two blocks of 8 warps per SM, contiguous ranges of at least 8 tiles per warp
    const int64_t warps = (int64_t)c->sm_count * 2 * 8;
    c->fx_per = std::max<int64_t>((c->n_tiles + warps - 1) / warps, 8);
    c->fx_blocks = std::max<int64_t>(((c->n_tiles + c->fx_per - 1) / c->fx_per + 7) / 8, 1);
    if ((e = cudaMemsetAsync(c->fx_word, 0, sizeof(uint32_t) * (3 * (size_t)ni + 1), s)) != cudaSuccess)
        return cuda_fail(c, e, "memset");
    auto stats = c->sv ? k_instr_stats<true> : k_instr_stats<false>;
    if (smem > 48 * 1024 &&
        (e = cudaFuncSetAttribute(stats, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem)) != cudaSuccess)
        return cuda_fail(c, e, "fixed-point statistics");
    stats<<<(unsigned)c->fx_blocks, 256, smem, s>>>(view<float>(c), c->fx_per, kcnt, c->fx_word);
    kmax_h->resize((size_t)ni);
    if ((e = cudaGetLastError()) != cudaSuccess ||
        (e = cudaMemcpyAsync(kmax_h->data(), kcnt, sizeof(uint32_t) * (size_t)ni, cudaMemcpyDeviceToHost, s)) !=
            cudaSuccess)
        return cuda_fail(c, e, "fixed-point statistics");
    return GSR_OK;
}

static gsr_status fixed_point_finish(gsr_ctx *c, cudaStream_t s, const std::vector<uint32_t> &kmax)
{
    if (kmax.empty()) return GSR_OK;
    std::vector<uint32_t> bits(kmax.size());
    int min_bits = 30;
    for (size_t j = 0; j < kmax.size(); ++j) {
        int lg = 0;  // ceil(log2(kmax + 1))
        while (lg < 32 && ((uint64_t)1 << lg) < (uint64_t)kmax[j] + 1) ++lg;
        bits[j] = (uint32_t)std::min(31 - lg, 30);
        min_bits = std::min(min_bits, (int)bits[j]);
    }
    if (min_bits < 20) return GSR_OK;
    // pageable source: the call returns once the bytes are staged, the kernels that read them follow on s
    const cudaError_t e = cudaMemcpyAsync(c->fx_word + kmax.size(), bits.data(), sizeof(uint32_t) * bits.size(),
                                          cudaMemcpyHostToDevice, s);
    if (e != cudaSuccess) return cuda_fail(c, e, "fixed-point setup");
    c->fx_bits = min_bits;
    return GSR_OK;
}

gsr_status ensure_att_layout(gsr_ctx *c, cudaStream_t s)
{
    if (c->att_valid) return GSR_OK;
    const int64_t n = c->n_rows;
    const int32_t nk = c->n_dfa - 3;  // knots a row may start at: 0..n_dfa-4
    cudaError_t e = cudaSuccess;
    if (n == 0) {
        e = cudaMemsetAsync(c->knot_ptr, 0, sizeof(int64_t) * (size_t)(nk + 1), s);
        if (e == cudaSuccess) e = cudaStreamSynchronize(s);
        if (e != cudaSuccess) return cuda_fail(c, e, "attitude layout");
        c->att_valid = true;
        return GSR_OK;
    }
    int32_t *keys_in = nullptr, *keys_out = nullptr, *vals_in = nullptr, *perm = nullptr;
    void *tmp = nullptr, *rec = nullptr;
    size_t tmp_bytes = 0;
    const int bits = 32 - __builtin_clz((unsigned)(nk > 1 ? nk : 1));
    const bool f32 = c->prec == GSR_FP32;
    const uint8_t *tiles = (const uint8_t *)c->tiles;
    int g = (int)std::min<int64_t>((n + 255) / 256, (int64_t)c->sm_count * 8);
    std::vector<uint32_t> kmax_h;
    gsr_status rf = GSR_OK;
    // scratch from the context's stream-ordered pool, which keeps its memory between builds (a
    // reloaded system rebuilds the layout without new device allocations or a device-wide sync)
    if (!c->pool) {
        cudaMemPoolProps props = {};
        props.allocType = cudaMemAllocationTypePinned;
        props.location.type = cudaMemLocationTypeDevice;
        props.location.id = c->device;
        if ((e = cudaMemPoolCreate(&c->pool, &props)) != cudaSuccess) return cuda_fail(c, e, "memory pool");
        uint64_t keep = UINT64_MAX;
        if ((e = cudaMemPoolSetAttribute(c->pool, cudaMemPoolAttrReleaseThreshold, &keep)) != cudaSuccess)
            return cuda_fail(c, e, "memory pool");
    }
    if ((e = cudaMallocFromPoolAsync(&keys_in, sizeof(int32_t) * (size_t)n, c->pool, s)) != cudaSuccess) goto done;
    if ((e = cudaMallocFromPoolAsync(&keys_out, sizeof(int32_t) * (size_t)n, c->pool, s)) != cudaSuccess) goto done;
    if ((e = cudaMallocFromPoolAsync(&vals_in, sizeof(int32_t) * (size_t)n, c->pool, s)) != cudaSuccess) goto done;
    if ((e = cudaMallocFromPoolAsync(&perm, sizeof(int32_t) * (size_t)n, c->pool, s)) != cudaSuccess) goto done;
    if (f32)
        k_extract_knots<float><<<g, 256, 0, s>>>(tiles, c->tile_bytes, c->npl, n, keys_in);
    else
        k_extract_knots<double><<<g, 256, 0, s>>>(tiles, c->tile_bytes, c->npl, n, keys_in);
    k_iota<<<g, 256, 0, s>>>(vals_in, n);
    if ((e = cub::DeviceRadixSort::SortPairs(nullptr, tmp_bytes, keys_in, keys_out, vals_in, perm, n, 0, bits, s)) !=
        cudaSuccess)
        goto done;
    if ((e = cudaMallocFromPoolAsync(&tmp, tmp_bytes, c->pool, s)) != cudaSuccess) goto done;
    if ((e = cub::DeviceRadixSort::SortPairs(tmp, tmp_bytes, keys_in, keys_out, vals_in, perm, n, 0, bits, s)) !=
        cudaSuccess)
        goto done;
    k_knot_ptr<<<(nk + 256) / 256, 256, 0, s>>>(keys_out, n, nk, c->knot_ptr);
    // the attitude records in star order, then gathered by the permutation
    if ((e = cudaMallocFromPoolAsync(&rec, (f32 ? sizeof(float) : sizeof(double)) * NAXES * NPARAXIS * (size_t)n,
                                     c->pool, s)) != cudaSuccess)
        goto done;
    if (f32) {
        k_att_rows<float><<<g, 256, 0, s>>>(tiles, c->tile_bytes, view<float>(c).p_att, n, (float *)rec);
        k_gather_att<float><<<g, 256, 0, s>>>((const float *)rec, perm, n, (uint8_t *)c->atiles);
    } else {
        k_att_rows<double><<<g, 256, 0, s>>>(tiles, c->tile_bytes, view<double>(c).p_att, n, (double *)rec);
        k_gather_att<double><<<g, 256, 0, s>>>((const double *)rec, perm, n, (uint8_t *)c->atiles);
    }
    if ((e = cudaGetLastError()) != cudaSuccess) goto done;
    rf = fixed_point_launch(c, s, &kmax_h);
done:
    if (keys_in) cudaFreeAsync(keys_in, s);
    if (keys_out) cudaFreeAsync(keys_out, s);
    if (vals_in) cudaFreeAsync(vals_in, s);
    if (perm) cudaFreeAsync(perm, s);
    if (tmp) cudaFreeAsync(tmp, s);
    if (rec) cudaFreeAsync(rec, s);
    {
        const cudaError_t es = cudaStreamSynchronize(s);
        if (e == cudaSuccess) e = es;
    }
    if (e != cudaSuccess) return cuda_fail(c, e, "attitude layout");
    if (rf != GSR_OK) return rf;
    if ((rf = fixed_point_finish(c, s, kmax_h)) != GSR_OK) return rf;
    c->att_valid = true;
    return GSR_OK;
}

}  // namespace gsr
