// residual_static.cu -- gsr_residual_static: the double-float residual r = b - A x
// of an FP32-stored context, computed without allocating any memory.
//
// gsr_residual needs scratch for the split copy of x and for its partial
// sums, and takes it from the context's workspace, which is allocated with
// cudaMalloc on first use. This entry point runs the same kernels but keeps
// its only scratch, the split copy of x, in a file-scope __device__ array of
// fixed size and writes no partial sums, so a call allocates nothing. The
// array's module and the two kernels are loaded when a context is created on
// the device (gsr_create / gsr_create_sections call static_scratch_load), so
// the first call of this entry point does not load them either.
#include "gsr_internal.cuh"

#define GSR_API extern "C" __attribute__((visibility("default")))

namespace gsr {

// Capacity: 2^20 columns. The array (8 MiB) is part of this file's module: with
// CUDA's lazy module loading it is placed on a device when the module is loaded
// there, which static_scratch_load below does at context creation, and it stays
// until the process exits (or a cudaDeviceReset unloads the module).
static constexpr int64_t kStaticMaxCols = int64_t(1) << 20;
static __device__ __align__(256) float2 g_static_xhl[kStaticMaxCols];

// In host code the symbol name is only a host-side stand-in; the address a
// kernel can use comes from cudaGetSymbolAddress, with the device current.
static cudaError_t static_scratch(float2 **out)
{
    void *p = nullptr;
    const cudaError_t e = cudaGetSymbolAddress(&p, g_static_xhl);
    if (e != cudaSuccess) return e;
    *out = static_cast<float2 *>(p);
    return cudaSuccess;
}

// Set-up, once per created context, with its device current: loads this module
// (the allocation of the array happens here, where the caller expects
// allocations), checks that the address lookup works, and loads the two
// kernels the entry point launches (loading a kernel allocates device memory
// for its code).
cudaError_t static_scratch_load(bool sv)
{
    float2 *p = nullptr;
    const cudaError_t e = static_scratch(&p);
    return e == cudaSuccess ? residual_kernels_load(sv) : e;
}

}  // namespace gsr

using namespace gsr;

GSR_API gsr_status gsr_residual_static(gsr_ctx *c, const double *x, float *r, void *stream)
{
    if (!c) return GSR_EINVAL;
    if (c->prec != GSR_FP32) return fail(c, GSR_EINVAL, "gsr_residual_static needs an FP32-stored context");
    if (c->n_cols > kStaticMaxCols)
        return fail(c, GSR_EINVAL, "gsr_residual_static: n_cols exceeds the capacity of its static scratch (1048576 "
                                   "columns)");
    if (!rows_complete(c)) return fail(c, GSR_ESTATE, "rows not loaded");
    if (!c->rhs_set) return fail(c, GSR_ESTATE, "b not loaded");
    if ((!x || !r) && c->n_rows > 0) return fail(c, GSR_EINVAL, "null vector");
    cudaError_t e = cudaSetDevice(c->device);
    if (e != cudaSuccess) return cuda_fail(c, e, "cudaSetDevice");
    // the address as the runtime knows it now (a host-side lookup while the module is loaded, which
    // it is from the context's creation; never a cached pointer that a device reset would leave stale)
    float2 *xhl = nullptr;
    if ((e = static_scratch(&xhl)) != cudaSuccess) return cuda_fail(c, e, "static scratch address");
    if (c->n_rows == 0) return GSR_OK;
    const cudaStream_t s = (cudaStream_t)stream;
    // the same kernels as gsr_residual, without partial sums
    if ((e = split_launch(c, x, xhl, c->n_cols, s)) != cudaSuccess ||
        (e = residual_launch(c, xhl, c->b, r, nullptr, s, nullptr)) != cudaSuccess)
        return cuda_fail(c, e, "residual_static");
    return GSR_OK;
}
