// probe.cu -- the device's binary64 fused multiply-add rate, the arithmetic ceiling of the
// binary64 aprods (24 multiply-adds per row against 236 / 228 bytes: on a GPU whose binary64
// rate is a small fraction of its binary32 rate, the binary64 products bound them before HBM).
//
// Each thread runs eight independent chains a = fma(a, m, c) (no chain waits on another, so the
// pipeline stays full), on 8 resident blocks of 256 threads per SM; the rate is the best of three
// timed launches after a warm-up launch.
#include "gsr_internal.cuh"

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

}  // namespace gsr

using namespace gsr;

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
