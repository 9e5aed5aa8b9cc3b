// layout.cu -- the knot-ordered ("time-local") copy of the attitude coefficients.
//
// aprod 2 scatters each row's 12 attitude products into the columns of its
// attitude knot. Rows are stored star by star (the astrometric blocks), so
// consecutive rows hit unrelated knots and every product would need an atomic
// add. This file builds, once per loaded system, a second copy of the 12
// attitude coefficients with the rows ordered by knot, in tiles of T positions
// (tiles.cuh; 13 planes per tile):
//   plane j < 12 : coefficient 5+j of row perm[p] at position p
//   plane 12     : perm[p], the row of position p (int32)
//   knot_ptr[k]  : first position of knot k (k = 0..n_dfa-3), knot_ptr[n_dfa-3] = n
// With it the attitude part of aprod 2 reduces runs of equal knot in registers
// and adds each run once (aprod.cu). The sort is CUB's stable radix sort on
// (knot, row) pairs; ties keep row order, so the layout is deterministic.
#include <cub/device/device_radix_sort.cuh>

#include "tiles.cuh"

namespace gsr {

__global__ void k_iota(int32_t *__restrict__ a, int64_t n)
{
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        a[i] = (int32_t)i;
}

// knot of every row, read from the tiles
template <typename VT>
__global__ void k_extract_knots(const uint8_t *__restrict__ tiles, int64_t n, int32_t *__restrict__ keys)
{
    using TL = Tile<VT>;
    for (int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; r < n; r += (int64_t)gridDim.x * blockDim.x)
        keys[r] = reinterpret_cast<const int32_t *>(tiles + (r / TL::T) * TL::BYTES + NPAR * TL::VBLK)[r % TL::T];
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

// position p of the knot-ordered tiles <- the attitude coefficients of row perm[p]
template <typename VT>
__global__ void k_gather_att(const uint8_t *__restrict__ tiles, const int32_t *__restrict__ perm, int64_t n,
                             uint8_t *__restrict__ atiles)
{
    using TL = Tile<VT>;
    for (int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; p < n; p += (int64_t)gridDim.x * blockDim.x) {
        const int64_t r = perm[p];
        const uint8_t *src = tiles + (r / TL::T) * TL::BYTES;
        const int64_t ri = r % TL::T;
        uint8_t *dst = atiles + (p / TL::T) * TL::ABYTES;
        const int64_t pi = p % TL::T;
#pragma unroll
        for (int j = 0; j < NAXES * NPARAXIS; ++j)
            reinterpret_cast<VT *>(dst + j * TL::VBLK)[pi] =
                reinterpret_cast<const VT *>(src + (NASTRO + j) * TL::VBLK)[ri];
        reinterpret_cast<int32_t *>(dst + NAXES * NPARAXIS * TL::VBLK)[pi] = (int32_t)r;
    }
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
    void *tmp = nullptr;
    size_t tmp_bytes = 0;
    const int bits = 32 - __builtin_clz((unsigned)(nk > 1 ? nk : 1));
    const bool f32 = c->prec == GSR_FP32;
    const uint8_t *tiles = (const uint8_t *)c->tiles;
    int g = (int)std::min<int64_t>((n + 255) / 256, (int64_t)c->sm_count * 8);
    if ((e = cudaMalloc(&keys_in, sizeof(int32_t) * (size_t)n)) != cudaSuccess) goto done;
    if ((e = cudaMalloc(&keys_out, sizeof(int32_t) * (size_t)n)) != cudaSuccess) goto done;
    if ((e = cudaMalloc(&vals_in, sizeof(int32_t) * (size_t)n)) != cudaSuccess) goto done;
    if ((e = cudaMalloc(&perm, sizeof(int32_t) * (size_t)n)) != cudaSuccess) goto done;
    if (f32)
        k_extract_knots<float><<<g, 256, 0, s>>>(tiles, n, keys_in);
    else
        k_extract_knots<double><<<g, 256, 0, s>>>(tiles, n, keys_in);
    k_iota<<<g, 256, 0, s>>>(vals_in, n);
    if ((e = cub::DeviceRadixSort::SortPairs(nullptr, tmp_bytes, keys_in, keys_out, vals_in, perm, n, 0, bits, s)) !=
        cudaSuccess)
        goto done;
    if ((e = cudaMalloc(&tmp, tmp_bytes)) != cudaSuccess) goto done;
    if ((e = cub::DeviceRadixSort::SortPairs(tmp, tmp_bytes, keys_in, keys_out, vals_in, perm, n, 0, bits, s)) !=
        cudaSuccess)
        goto done;
    k_knot_ptr<<<(nk + 256) / 256, 256, 0, s>>>(keys_out, n, nk, c->knot_ptr);
    if (f32)
        k_gather_att<float><<<g, 256, 0, s>>>(tiles, perm, n, (uint8_t *)c->atiles);
    else
        k_gather_att<double><<<g, 256, 0, s>>>(tiles, perm, n, (uint8_t *)c->atiles);
    if ((e = cudaGetLastError()) != cudaSuccess) goto done;
    e = cudaStreamSynchronize(s);
done:
    cudaFree(keys_in);
    cudaFree(keys_out);
    cudaFree(vals_in);
    cudaFree(perm);
    cudaFree(tmp);
    if (e != cudaSuccess) return cuda_fail(c, e, "attitude layout");
    c->att_valid = true;
    return GSR_OK;
}

}  // namespace gsr
