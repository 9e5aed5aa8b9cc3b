// residual_static.cu -- gsr_residual_static: the double-float residual r = b - A x
// of an FP32-stored context, computed without allocating any memory.
//
// gsr_residual needs scratch for the split copies of x and b and for its
// partial sums, and takes it from the context's workspace, which is allocated
// with cudaMalloc on first use. This entry point keeps its only scratch, the
// split copy of x, in a file-scope __device__ array of fixed size, splits b
// inside the kernel, and writes no partial sums, so a call allocates nothing.
#include <mutex>

#include "dfloat.cuh"
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

__global__ void k_split_static(const double *__restrict__ x, float2 *__restrict__ out, int64_t n)
{
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        out[i] = split_double(x[i]);
}

// r = b - A x, one warp per star; x as (hi, lo) pairs, b split per row here.
__global__ void __launch_bounds__(256) k_residual_static(SysView<float> S, const float2 *__restrict__ xhl,
                                                         const double *__restrict__ b, float *__restrict__ r_out)
{
    const int lane = threadIdx.x & 31;
    const int64_t gw = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
    const float2 *__restrict__ xt = xhl + S.att0;
    const float2 *__restrict__ xi = xhl + S.instr0;
    const float2 xg = S.n_glob ? xhl[S.glob0] : make_float2(0.f, 0.f);
    for (int64_t s = gw; s < S.n_stars; s += nw) {
        const int64_t r0 = S.star_ptr[s], r1 = S.star_ptr[s + 1];
        float2 xa[NASTRO];
#pragma unroll
        for (int j = 0; j < NASTRO; ++j) xa[j] = xhl[NASTRO * s + j];
        for (int64_t r = r0 + lane; r < r1; r += 32) {
            float a[NPAR];
#pragma unroll
            for (int j = 0; j < NPAR; ++j) a[j] = __ldcs(S.val + j * S.plane + r);
            const int32_t k = __ldcs(S.knot + r);
            int32_t ic[NINSTR];
#pragma unroll
            for (int j = 0; j < NINSTR; ++j) ic[j] = __ldcs(S.instr + j * S.plane + r);
            float sh = 0.f, c = 0.f;
#pragma unroll
            for (int j = 0; j < NASTRO; ++j) acc_term(a[j], xa[j], sh, c);
#pragma unroll
            for (int ax = 0; ax < NAXES; ++ax) {
                const float2 *__restrict__ xk = xt + (int64_t)ax * S.n_dfa + k;
#pragma unroll
                for (int j = 0; j < NPARAXIS; ++j) acc_term(a[NASTRO + NPARAXIS * ax + j], xk[j], sh, c);
            }
#pragma unroll
            for (int j = 0; j < NINSTR; ++j) acc_term(a[17 + j], xi[ic[j]], sh, c);
            acc_term(a[23], xg, sh, c);
            const float2 bb = split_double(__ldcs(b + r));
            float t, e;
            two_sum(bb.x, -sh, t, e);
            const float lo = __fadd_rn(__fadd_rn(e, bb.y), -c);
            r_out[r] = __fadd_rn(t, lo);
        }
    }
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
    int64_t gsplit = (c->n_cols + 255) / 256;
    gsplit = std::min<int64_t>(std::max<int64_t>(gsplit, 1), (int64_t)c->sm_count * 4);
    k_split_static<<<(unsigned)gsplit, 256, 0, s>>>(x, xhl, c->n_cols);
    int per_sm = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_residual_static, 256, 0) != cudaSuccess || per_sm < 1)
        per_sm = 1;
    int64_t blocks = (int64_t)per_sm * c->sm_count;
    blocks = std::min<int64_t>(blocks, (c->n_stars + 7) / 8);
    blocks = std::max<int64_t>(blocks, 1);
    k_residual_static<<<(unsigned)blocks, 256, 0, s>>>(view<float>(c), xhl, c->b, r);
    if ((e = cudaGetLastError()) != cudaSuccess) return cuda_fail(c, e, "residual_static");
    return GSR_OK;
}
