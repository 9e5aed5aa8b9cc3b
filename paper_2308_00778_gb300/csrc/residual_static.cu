// residual_static.cu -- gsr_residual_static: the double-float residual r = b - A x
// of an FP32-stored context, computed without allocating any memory.
//
// gsr_residual needs scratch for the split copy of x and for its partial
// sums, and takes it from the context's workspace, which is allocated with
// cudaMalloc on first use. This entry point runs the same kernels but keeps
// its only scratch, the split copy of x, in a file-scope __device__ array of
// fixed size and writes no partial sums, so a call allocates nothing.
#include <mutex>

#include "gsr_internal.cuh"

#define GSR_API extern "C" __attribute__((visibility("default")))

namespace gsr {

// Capacity: 2^20 columns. The array (8 MiB) exists on every GPU that loads the
// library, from module load until the process exits.
static constexpr int64_t kStaticMaxCols = int64_t(1) << 20;
static __device__ __align__(256) float2 g_static_xhl[kStaticMaxCols];

// Device address of g_static_xhl per device ordinal. In host code the symbol
// name is only a host-side stand-in; the address a kernel can use comes from
// cudaGetSymbolAddress, called once per device with that device current.
static constexpr int kMaxDevices = 64;
static std::mutex g_static_mu;
static float2 *g_static_addr[kMaxDevices];

static cudaError_t static_scratch(int device, float2 **out)
{
    if (device < 0 || device >= kMaxDevices) return cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> lock(g_static_mu);
    if (!g_static_addr[device]) {
        void *p = nullptr;
        const cudaError_t e = cudaGetSymbolAddress(&p, g_static_xhl);
        if (e != cudaSuccess) return e;
        g_static_addr[device] = static_cast<float2 *>(p);
    }
    *out = g_static_addr[device];
    return cudaSuccess;
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
    float2 *xhl = nullptr;
    if ((e = static_scratch(c->device, &xhl)) != cudaSuccess) return cuda_fail(c, e, "static scratch address");
    if (c->n_rows == 0) return GSR_OK;
    const cudaStream_t s = (cudaStream_t)stream;
    // the same kernels as gsr_residual, without partial sums
    if ((e = split_launch(c, x, xhl, c->n_cols, s)) != cudaSuccess ||
        (e = residual_launch(c, xhl, c->b, r, nullptr, s, nullptr)) != cudaSuccess)
        return cuda_fail(c, e, "residual_static");
    return GSR_OK;
}
