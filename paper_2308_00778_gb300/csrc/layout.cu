// layout.cu -- the knot-ordered ("time-local") copy of the attitude coefficients.
//
// aprod 2 scatters each row's 12 attitude products into the columns of its
// attitude knot. Rows are stored star by star (the astrometric blocks), so
// consecutive rows hit unrelated knots and every product would need an atomic
// add. This file builds, once per loaded system, a second copy of the 12
// attitude coefficients with the rows ordered by knot:
//   att_k[j][i] = coefficient 5+j of row perm[i], i = 0..n-1, knots nondecreasing in i
//   knot_ptr[k] = first position of knot k (k = 0..n_dfa-3), knot_ptr[n_dfa-3] = n
// With it the attitude part of aprod 2 reduces runs of equal knots in registers
// and adds each run once (see aprod.cu). The sort is CUB's stable radix sort on
// (knot, row) pairs; ties keep row order, so the layout is deterministic.
#include <cub/device/device_radix_sort.cuh>

#include "gsr_internal.cuh"

namespace gsr {

__global__ void k_iota(int32_t *__restrict__ a, int64_t n)
{
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        a[i] = (int32_t)i;
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

template <typename VT>
__global__ void k_gather_att(const VT *__restrict__ val, int64_t plane, const int32_t *__restrict__ perm, int64_t n,
                             VT *__restrict__ att_k)
{
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const int64_t r = perm[i];
#pragma unroll
        for (int j = 0; j < NAXES * NPARAXIS; ++j) att_k[j * plane + i] = val[(NASTRO + j) * plane + r];
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
    int32_t *keys_out = nullptr, *vals_in = nullptr;
    void *tmp = nullptr;
    size_t tmp_bytes = 0;
    const int bits = 32 - __builtin_clz((unsigned)(nk > 1 ? nk : 1));
    int g = (int)std::min<int64_t>((n + 255) / 256, (int64_t)c->sm_count * 8);
    if ((e = cudaMalloc(&keys_out, sizeof(int32_t) * (size_t)n)) != cudaSuccess) goto done;
    if ((e = cudaMalloc(&vals_in, sizeof(int32_t) * (size_t)n)) != cudaSuccess) goto done;
    k_iota<<<g, 256, 0, s>>>(vals_in, n);
    if ((e = cub::DeviceRadixSort::SortPairs(nullptr, tmp_bytes, c->knot, keys_out, vals_in, c->perm, n, 0, bits,
                                             s)) != cudaSuccess)
        goto done;
    if ((e = cudaMalloc(&tmp, tmp_bytes)) != cudaSuccess) goto done;
    if ((e = cub::DeviceRadixSort::SortPairs(tmp, tmp_bytes, c->knot, keys_out, vals_in, c->perm, n, 0, bits, s)) !=
        cudaSuccess)
        goto done;
    k_knot_ptr<<<(nk + 256) / 256, 256, 0, s>>>(keys_out, n, nk, c->knot_ptr);
    if (c->prec == GSR_FP32)
        k_gather_att<float><<<g, 256, 0, s>>>((const float *)c->vals, c->plane, c->perm, n, (float *)c->att_k);
    else
        k_gather_att<double><<<g, 256, 0, s>>>((const double *)c->vals, c->plane, c->perm, n, (double *)c->att_k);
    if ((e = cudaGetLastError()) != cudaSuccess) goto done;
    e = cudaStreamSynchronize(s);
done:
    cudaFree(keys_out);
    cudaFree(vals_in);
    cudaFree(tmp);
    if (e != cudaSuccess) return cuda_fail(c, e, "attitude layout");
    c->att_valid = true;
    return GSR_OK;
}

}  // namespace gsr
