// probe.cu -- the device's binary64 fused multiply-add rate, the arithmetic ceiling of the
// binary64 aprods (24 multiply-adds per row against 236 / 228 bytes: on a GPU whose binary64
// rate is a small fraction of its binary32 rate, the binary64 products bound them before HBM).
//
// Each thread runs eight independent chains a = fma(a, m, c) (no chain waits on another, so the
// pipeline stays full), on 8 resident blocks of 256 threads per SM; the rate is the best of three
// timed launches after a warm-up launch.
#include "gsr_internal.cuh"
#include "tc.cuh"

#define GSR_API extern "C" __attribute__((visibility("default")))

namespace gsr {

static __device__ double g_probe_sink;

constexpr int kProbeChains = 8;
constexpr int kProbeIters = 4096;

__global__ void __launch_bounds__(256) k_fma_probe(double m, double c, int iters)
{
    double a[kProbeChains];
#pragma unroll
    for (int q = 0; q < kProbeChains; ++q) a[q] = (double)(threadIdx.x + q);
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int q = 0; q < kProbeChains; ++q) a[q] = fma(a[q], m, c);
    }
    double s = 0.0;
#pragma unroll
    for (int q = 0; q < kProbeChains; ++q) s += a[q];
    if (s == 1234.5) g_probe_sink = s;  // keeps the chains live; m and c make it (practically) never true
}

// The tensor-core kernels' bounded wait, exercised on its timeout path: one CTA takes TMEM and an
// mbarrier that nothing will arrive on, waits limit_ns, reports whether the wait gave up, releases
// the TMEM and returns (the path a convolution takes when its MMAs do not complete in time).
__global__ void __launch_bounds__(128) k_tc_wait(uint64_t limit_ns, int32_t *timed_out)
{
    __shared__ __align__(8) uint64_t mbar;
    __shared__ uint32_t tslot;
    const int warp = threadIdx.x >> 5;
    if (warp == 0) tc::tmem_alloc(&tslot, 32);
    if (threadIdx.x == 32) tc::mbar_init(&mbar, 1);
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    const bool ok = __syncthreads_and(tc::mbar_wait(&mbar, 0, limit_ns));
    if (threadIdx.x == 0) *timed_out = ok ? 0 : 1;
    tc::fence_before_sync();
    __syncthreads();
    if (warp == 0) {
        tc::fence_after_sync();
        tc::tmem_dealloc(tslot, 32);
    }
}

}  // namespace gsr

using namespace gsr;

GSR_API gsr_status gsr_tc_wait_check(int32_t device, double limit_ms, int32_t *timed_out, double *waited_ms)
{
    if (!timed_out || !waited_ms || !(limit_ms > 0.0) || limit_ms > 2000.0) return GSR_EINVAL;
    *timed_out = -1;
    *waited_ms = 0.0;
    cudaError_t e = cudaSetDevice(device);
    int32_t *d = nullptr;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    if (e == cudaSuccess) e = cudaMalloc(&d, sizeof(int32_t));
    if (e == cudaSuccess) e = cudaMemset(d, 0xff, sizeof(int32_t));
    if (e == cudaSuccess) e = cudaEventCreate(&e0);
    if (e == cudaSuccess) e = cudaEventCreate(&e1);
    if (e == cudaSuccess) {
        cudaEventRecord(e0);
        k_tc_wait<<<1, 128>>>((uint64_t)(limit_ms * 1e6), d);
        cudaEventRecord(e1);
        e = cudaEventSynchronize(e1);
    }
    if (e == cudaSuccess) e = cudaGetLastError();
    float ms = 0.f;
    if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
    if (e == cudaSuccess) e = cudaMemcpy(timed_out, d, sizeof(int32_t), cudaMemcpyDeviceToHost);
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    if (d) cudaFree(d);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return GSR_ECUDA;
    }
    *waited_ms = ms;
    return GSR_OK;
}

GSR_API gsr_status gsr_fp64_fma_rate(int32_t device, double *tflops)
{
    if (!tflops) return GSR_EINVAL;
    *tflops = 0.0;
    int sms = 0;
    cudaError_t e = cudaSetDevice(device);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return GSR_ECUDA;
    }
    const int blocks = sms * 8, threads = 256;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    if ((e = cudaEventCreate(&e0)) == cudaSuccess) e = cudaEventCreate(&e1);
    float best = 0.f;
    if (e == cudaSuccess) {
        k_fma_probe<<<blocks, threads>>>(0.999999, 1e-7, kProbeIters);
        for (int r = 0; r < 3 && e == cudaSuccess; ++r) {
            cudaEventRecord(e0);
            k_fma_probe<<<blocks, threads>>>(0.999999, 1e-7, kProbeIters);
            cudaEventRecord(e1);
            if ((e = cudaEventSynchronize(e1)) == cudaSuccess) {
                float ms = 0.f;
                if ((e = cudaEventElapsedTime(&ms, e0, e1)) == cudaSuccess && (best == 0.f || ms < best)) best = ms;
            }
        }
        if (e == cudaSuccess) e = cudaGetLastError();
    }
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    if (e != cudaSuccess || best <= 0.f) {
        cudaGetLastError();
        return GSR_ECUDA;
    }
    const double fmas = (double)blocks * threads * kProbeIters * kProbeChains;
    *tflops = 2.0 * fmas / ((double)best * 1e-3) / 1e12;
    return GSR_OK;
}
