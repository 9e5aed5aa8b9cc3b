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

// For the fixed-point sums of the binary32 star pass (aprod.cu), per column j
// over the pass's partition (each warp a contiguous range of `per` tiles, 8
// warps a block): the largest number of contributions one block adds to
// column j (kmax[j]) and the largest |coefficient| of column j (amax[j],
// binary32 bits). Columns [0, n_instr) are the instrumental unknowns; with
// att, columns n_instr + a*n_dfa + k the attitude unknowns. Both arrays are
// zero on entry.
template <bool SV>
__global__ void __launch_bounds__(256) k_instr_stats(SysView<float> S, int64_t per, uint32_t *__restrict__ kmax,
                                                     uint32_t *__restrict__ amax, int32_t nc, int32_t att)
{
    const Sec<SV> G(S);
    constexpr int R = Tile<float>::R;
    constexpr int T = Tile<float>::T;
    extern __shared__ uint32_t cnt[];  // [nc] counts, then [nc] max |a| bits
    uint32_t *am = cnt + nc;
    for (int32_t i = threadIdx.x; i < 2 * nc; i += blockDim.x) cnt[i] = 0u;
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
        if (att) {
            int32_t kn[R];
            load_ints<R>(tb + (int64_t)G.npl * Tile<float>::VBLK, 0, kn);
#pragma unroll
            for (int q = 0; q < NAXES * NPARAXIS; ++q) {
                float a[R];
                load_vals<float, float>(tb, G.p_att + q, a);
#pragma unroll
                for (int i = 0; i < R; ++i)
                    if (r0 + i < S.n_rows) {
                        const int32_t col = S.n_instr + (q / NPARAXIS) * S.n_dfa + kn[i] + (q % NPARAXIS);
                        atomicAdd(cnt + col, 1u);
                        atomicMax(am + col, __float_as_uint(fabsf(a[i])));
                    }
            }
        }
    }
    __syncthreads();
    for (int32_t i = threadIdx.x; i < nc; i += blockDim.x) {
        if (cnt[i]) atomicMax(kmax + i, cnt[i]);
        if (am[i]) atomicMax(amax + i, am[i]);
    }
}

// The largest and the smallest nonzero column max |coefficient| (amax, after every block of
// k_instr_stats) of the attitude and of the instrumental columns, for the one scale the one-pass
// aprod 2 gives each group: binary32 bits order as integers, the smallest kept as its complement so
// that all four are maxima; into ext[0..4) = hi_att, ~lo_att, hi_ins, ~lo_ins (zero on entry). One
// block.
__global__ void __launch_bounds__(1024) k_group_extremes(const uint32_t *__restrict__ amax, int32_t nc,
                                                         int32_t n_instr, uint32_t *__restrict__ ext)
{
    uint32_t hi_a = 0u, lo_a = 0u, hi_i = 0u, lo_i = 0u;
    for (int32_t i = threadIdx.x; i < nc; i += blockDim.x) {
        const uint32_t a = amax[i];
        if (!a) continue;
        if (i >= n_instr) {
            hi_a = max(hi_a, a);
            lo_a = max(lo_a, ~a);
        } else {
            hi_i = max(hi_i, a);
            lo_i = max(lo_i, ~a);
        }
    }
    hi_a = __reduce_max_sync(0xffffffffu, hi_a);
    lo_a = __reduce_max_sync(0xffffffffu, lo_a);
    hi_i = __reduce_max_sync(0xffffffffu, hi_i);
    lo_i = __reduce_max_sync(0xffffffffu, lo_i);
    if ((threadIdx.x & 31) == 0) {
        if (hi_a) atomicMax(ext + 0, hi_a);
        if (lo_a) atomicMax(ext + 1, lo_a);
        if (hi_i) atomicMax(ext + 2, hi_i);
        if (lo_i) atomicMax(ext + 3, lo_i);
    }
}

// Shared memory of the fixed-point star pass (aprod.cu) per block: accumulators and scales of
// every column, twice for the pass that sums products and squares together.
static constexpr size_t kFxSmemOne = 100 * 1024;   // two blocks per SM
static constexpr size_t kFxSmemBoth = 200 * 1024;  // one block per SM
// the binary64 fixed-point star pass: its sums and shifts beside the 21 KB of static shared memory of a
// 512-thread block, within the 227 KB a block may hold
static constexpr size_t kFx64SmemMax = 204 * 1024;

// Per-column bits of the fixed-point sums (all 0: keep binary32 atomics):
// bits_j = 31 - ceil(log2(kmax_j + 1)), so that no block can overflow column j;
// the instrumental sums are used only when every instrumental column gets at
// least 20 bits, the attitude columns join them (fx_att) when every attitude
// column does too. Launches the statistics and the copy of kmax into *kmax_h
// (asynchronous); the caller synchronises s and calls fixed_point_finish.
static gsr_status fixed_point_launch(gsr_ctx *c, cudaStream_t s, std::vector<uint32_t> *kmax_h)
{
    c->fx_bits = 0;
    c->fx_att = false;
    c->fx_uni = false;
    kmax_h->clear();
    if (c->prec != GSR_FP32 || c->n_rows == 0 || c->n_ipr == 0 || c->n_instr == 0) return GSR_OK;
    const int32_t ni = c->n_instr;
    if (2 * sizeof(uint32_t) * (size_t)ni > kFxSmemOne) return GSR_OK;
    // the attitude columns join when their accumulators fit beside the instrumental ones
    const int64_t nc_att = (int64_t)ni + (int64_t)NAXES * c->n_dfa;
    const bool att = !c->sv && 2 * sizeof(uint32_t) * (size_t)nc_att <= kFxSmemOne &&
                     4 * sizeof(uint32_t) * (size_t)nc_att <= kFxSmemBoth;
    const int32_t nc = att ? (int32_t)nc_att : ni;
    cudaError_t e = cudaSuccess;
    // device words: [0, nc) max |a| per column, [nc, 2nc) bits per column, [2nc] max |y| of the
    // current aprod 2, then [nc] scratch counts, then (FX_GROUP words) the attitude and the
    // instrumental columns' largest and smallest |a| and the bits of their group scales
    if (c->fx_word && c->fx_nc != nc) {
        cudaFree(c->fx_word);
        c->fx_word = nullptr;
    }
    if (!c->fx_word &&
        (e = cudaMalloc(&c->fx_word, sizeof(uint32_t) * (3 * (size_t)nc + 1 + FX_GROUP))) != cudaSuccess)
        return cuda_fail(c, e, "fixed-point words");
    c->fx_nc = nc;
    uint32_t *kcnt = c->fx_word + 2 * nc + 1;
    // the partition: two blocks of 8 warps per SM, contiguous ranges of at least 8 tiles per warp
    const int64_t warps = (int64_t)c->sm_count * 2 * 8;
    c->fx_per = std::max<int64_t>((c->n_tiles + warps - 1) / warps, 8);
    c->fx_blocks = std::max<int64_t>(((c->n_tiles + c->fx_per - 1) / c->fx_per + 7) / 8, 1);
    if ((e = cudaMemsetAsync(c->fx_word, 0, sizeof(uint32_t) * (3 * (size_t)nc + 1 + FX_GROUP), s)) != cudaSuccess)
        return cuda_fail(c, e, "memset");
    const size_t smem = 2 * sizeof(uint32_t) * (size_t)nc;
    auto stats = c->sv ? k_instr_stats<true> : k_instr_stats<false>;
    if ((e = cudaFuncSetAttribute(stats, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem)) != cudaSuccess)
        return cuda_fail(c, e, "fixed-point statistics");
    stats<<<(unsigned)c->fx_blocks, 256, smem, s>>>(view<float>(c), c->fx_per, kcnt, c->fx_word, nc, att ? 1 : 0);
    if ((e = cudaGetLastError()) != cudaSuccess) return cuda_fail(c, e, "fixed-point statistics");
    k_group_extremes<<<1, 1024, 0, s>>>(c->fx_word, nc, c->n_instr, kcnt + nc);
    kmax_h->resize((size_t)nc + 4);  // the counts, then the four group extremes
    if ((e = cudaGetLastError()) != cudaSuccess ||
        (e = cudaMemcpyAsync(kmax_h->data(), kcnt, sizeof(uint32_t) * ((size_t)nc + 4), cudaMemcpyDeviceToHost,
                             s)) != cudaSuccess)
        return cuda_fail(c, e, "fixed-point statistics");
    return GSR_OK;
}

// bits lost by one scale for a group of columns: ceil(log2(largest / smallest |a|)) (binary32 bits,
// the smallest stored as its complement; 99 when the group has no coefficient)
static int group_loss(uint32_t hi_bits, uint32_t lo_compl)
{
    if (!hi_bits || !lo_compl) return 99;
    const double hi = (double)__builtin_bit_cast(float, hi_bits), lo = (double)__builtin_bit_cast(float, ~lo_compl);
    if (!(lo > 0.0) || !(hi >= lo)) return 99;
    return (int)std::ceil(std::log2(hi / lo));
}

static gsr_status fixed_point_finish(gsr_ctx *c, cudaStream_t s, const std::vector<uint32_t> &kmax_ext)
{
    if (kmax_ext.empty()) return GSR_OK;
    const size_t nc = kmax_ext.size() - 4;
    std::vector<uint32_t> bits(nc);
    int min_ins = 30, min_att = 30;
    for (size_t j = 0; j < nc; ++j) {
        int lg = 0;  // ceil(log2(kmax + 1))
        while (lg < 32 && ((uint64_t)1 << lg) < (uint64_t)kmax_ext[j] + 1) ++lg;
        bits[j] = (uint32_t)std::min(31 - lg, 30);
        if ((int64_t)j < c->n_instr)
            min_ins = std::min(min_ins, (int)bits[j]);
        else
            min_att = std::min(min_att, (int)bits[j]);
    }
    if (min_ins < 20) return GSR_OK;
    // One scale per group (the attitude columns; the instrumental ones in the one-pass pass) from the
    // group's largest |a| and fewest bits: no column can overflow, and a column's contributions keep
    // at least 20 bits of its own bound when the group's fewest bits minus the bits lost to the
    // spread of |a| stay >= 20. Otherwise the attitude columns take the two-pass aprod 2 and the
    // instrumental ones their per-column scales.
    const bool att_cols = (int64_t)nc > c->n_instr;
    const int loss_att = group_loss(kmax_ext[nc], kmax_ext[nc + 1]);
    const int loss_ins = group_loss(kmax_ext[nc + 2], kmax_ext[nc + 3]);
    const uint32_t group_bits[2] = {att_cols && min_att - loss_att >= 20 ? (uint32_t)min_att : 0u,
                                    min_ins - loss_ins >= 20 ? (uint32_t)min_ins : 0u};
    // pageable sources: each call returns once the bytes are staged, the kernels that read them follow on s
    cudaError_t e = cudaMemcpyAsync(c->fx_word + nc, bits.data(), sizeof(uint32_t) * nc, cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(c->fx_word + 3 * nc + 5, group_bits, sizeof(group_bits), cudaMemcpyHostToDevice, s);
    if (e != cudaSuccess) return cuda_fail(c, e, "fixed-point setup");
    c->fx_bits = min_ins;
    c->fx_att = group_bits[0] > 0;
    c->fx_uni = group_bits[1] > 0;
    return GSR_OK;
}

// For the int64 fixed-point instrumental sums of the binary64 star pass (aprod.cu), over its partition
// (warp w of that pass takes tiles [w per, (w + 1) per), wpb warps a block; this kernel runs one block
// per block of the pass, its own warps striding over the block's tiles): the largest number of
// contributions one block adds to each instrumental column (kmax) and each column's largest
// |coefficient| (amax, binary32 bits rounded up, so never below the binary64 value). Both zero on entry.
__global__ void __launch_bounds__(256) k_instr_stats64(SysView<double> S, int64_t per, int32_t wpb,
                                                       uint32_t *__restrict__ kmax, uint32_t *__restrict__ amax)
{
    constexpr int R = Tile<double>::R;
    constexpr int T = Tile<double>::T;
    extern __shared__ uint32_t cnt[];  // [n_instr] counts, then [n_instr] max |a| bits
    uint32_t *am = cnt + S.n_instr;
    for (int32_t i = threadIdx.x; i < 2 * S.n_instr; i += blockDim.x) cnt[i] = 0u;
    __syncthreads();
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    const int64_t b0 = (int64_t)blockIdx.x * wpb * per;
    const int64_t b1 = min(S.n_tiles, b0 + (int64_t)wpb * per);
    for (int64_t t = b0 + warp; t < b1; t += nw) {
        const uint8_t *tb = S.tiles + t * S.tile_bytes;
        const int64_t r0 = t * T + lane * R;
#pragma unroll
        for (int j = 0; j < NINSTR; ++j) {
            int32_t ic[R];
            double a[R];
            load_instr<double>(tb, S.iw16, j, ic);
            load_vals<double, double>(tb, A_INS + j, a);
#pragma unroll
            for (int i = 0; i < R; ++i)
                if (r0 + i < S.n_rows) {
                    atomicAdd(cnt + ic[i], 1u);
                    atomicMax(am + ic[i], __float_as_uint(__double2float_ru(fabs(a[i]))));
                }
        }
    }
    __syncthreads();
    for (int32_t i = threadIdx.x; i < S.n_instr; i += blockDim.x) {
        if (cnt[i]) atomicMax(kmax + i, cnt[i]);
        if (am[i]) atomicMax(amax + i, am[i]);
    }
}

// The statistics of the binary64 fixed-point star pass (asynchronous on s), where it applies: binary64
// storage, the standard row, and its sums and shifts within one block's shared memory.
static gsr_status fx64_stats(gsr_ctx *c, cudaStream_t s)
{
    const bool was = c->fx64;
    c->fx64 = false;
    const size_t dyn = fx64_smem(c);
    const bool fits = dyn <= kFx64SmemMax && 2 * sizeof(uint32_t) * (size_t)c->n_instr <= kFx64SmemMax;
    if (c->prec != GSR_FP64 || c->sv || c->n_rows == 0 || c->n_instr == 0 || !fits) {
        if (was) drop_graphs(c);
        return GSR_OK;
    }
    cudaError_t e = cudaSuccess;
    const size_t words = FX64_BINS + 2 + 2 * (size_t)c->n_instr;
    if (!c->fx64_word && (e = cudaMalloc(&c->fx64_word, sizeof(uint32_t) * words)) != cudaSuccess)
        return cuda_fail(c, e, "fixed-point words");
    fx64_partition(c, &c->fx64_per, &c->fx64_blocks, &c->fx64_nt);
    if ((e = cudaMemsetAsync(c->fx64_word, 0, sizeof(uint32_t) * words, s)) != cudaSuccess)
        return cuda_fail(c, e, "memset");
    const size_t smem = 2 * sizeof(uint32_t) * (size_t)c->n_instr;
    if (smem > 48 * 1024 &&
        (e = cudaFuncSetAttribute(k_instr_stats64, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem)) !=
            cudaSuccess)
        return cuda_fail(c, e, "fixed-point statistics");
    k_instr_stats64<<<(unsigned)c->fx64_blocks, 256, smem, s>>>(view<double>(c), c->fx64_per, c->fx64_nt / 32,
                                                                c->fx64_word + FX64_BINS + 2,
                                                                c->fx64_word + FX64_BINS + 2 + c->n_instr);
    if ((e = cudaGetLastError()) != cudaSuccess) return cuda_fail(c, e, "fixed-point statistics");
    c->fx64 = true;
    if (!was) drop_graphs(c);  // graphs captured before hold the binary64 atomics' pass
    return GSR_OK;
}

// the knot-ordered attitude copy of the loaded rows
static gsr_status build_att_copy(gsr_ctx *c, cudaStream_t s)
{
    const int64_t n = c->n_rows;
    const int32_t nk = c->n_dfa - 3;  // knots a row may start at: 0..n_dfa-4
    cudaError_t e = cudaSuccess;
    if (n == 0) {
        e = cudaMemsetAsync(c->knot_ptr, 0, sizeof(int64_t) * (size_t)(nk + 1), s);
        if (e == cudaSuccess) e = cudaStreamSynchronize(s);
        if (e != cudaSuccess) return cuda_fail(c, e, "attitude layout");
        return GSR_OK;
    }
    int32_t *keys_in = nullptr, *keys_out = nullptr, *vals_in = nullptr, *perm = nullptr;
    void *tmp = nullptr, *rec = nullptr;
    size_t tmp_bytes = 0;
    if (!c->atiles) {  // first use: the copy's tiles, zero in the padding positions of the last tile
        const size_t abytes = (size_t)std::max<int64_t>(c->n_tiles, 1) *
                              (size_t)(c->prec == GSR_FP32 ? Tile<float>::ABYTES : Tile<double>::ABYTES);
        if ((e = cudaMalloc(&c->atiles, abytes)) != cudaSuccess ||
            (e = cudaMemsetAsync(c->atiles, 0, abytes, s)) != cudaSuccess) {
            if (c->atiles) cudaFree(c->atiles);
            c->atiles = nullptr;
            return cuda_fail(c, e, "attitude layout");
        }
    }
    const int bits = 32 - __builtin_clz((unsigned)(nk > 1 ? nk : 1));
    const bool f32 = c->prec == GSR_FP32;
    const uint8_t *tiles = (const uint8_t *)c->tiles;
    int g = (int)std::min<int64_t>((n + 255) / 256, (int64_t)c->sm_count * 8);
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
    e = cudaGetLastError();
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
    return GSR_OK;
}

gsr_status ensure_att_layout(gsr_ctx *c, cudaStream_t s, bool binary64)
{
    if (!c->fx_valid) {
        std::vector<uint32_t> kmax_h;
        gsr_status rf = fixed_point_launch(c, s, &kmax_h);
        const cudaError_t e = cudaStreamSynchronize(s);
        if (rf != GSR_OK) return rf;
        if (e != cudaSuccess) return cuda_fail(c, e, "fixed-point statistics");
        if ((rf = fixed_point_finish(c, s, kmax_h)) != GSR_OK) return rf;
        c->fx_valid = true;
        // the cached iteration graphs hold the kernel choice they were captured with
        const int32_t sig = (c->fx_bits > 0 ? 1 : 0) | (c->fx_att ? 2 : 0) | (c->fx_uni ? 4 : 0);
        if (sig != c->fx_sig) {
            drop_graphs(c);
            c->fx_sig = sig;
        }
    }
    // a wide attitude block of binary32 storage: the window accumulators of the vector reductions
    if (c->prec == GSR_FP32 && !c->sv && !att_fused(c) && !c->attw) {
        const size_t bytes = sizeof(float) * 2 * 4 * (size_t)NAXES * (size_t)c->n_dfa;
        cudaError_t e = cudaMalloc(&c->attw, bytes);
        if (e == cudaSuccess) e = cudaMemsetAsync(c->attw, 0, bytes, s);
        if (e != cudaSuccess) {
            if (c->attw) cudaFree(c->attw);
            c->attw = nullptr;
            return cuda_fail(c, e, "attitude window accumulators");
        }
    }
    // the knot-ordered copy: for binary64 aprod 2 passes, and binary32 section variants whose
    // attitude columns do not fit the one-pass form
    if ((binary64 || (!att_fused(c) && !att_red(c))) && !c->att_valid) {
        gsr_status rc = build_att_copy(c, s);
        if (rc == GSR_OK) rc = fx64_stats(c, s);
        if (rc != GSR_OK) return rc;
        c->att_valid = true;
    }
    return GSR_OK;
}

}  // namespace gsr
