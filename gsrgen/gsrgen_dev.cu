/*
 * gsrgen_dev.cu -- device twin of the seeded synthetic-system generator.
 *
 * Writes the same rows, planted solution and noise as gsrgen_host.c straight
 * into device memory, so systems with 1e8+ rows need no host generation and no
 * host-to-device copy of the matrix. It includes the same gsrgen_core.h and is
 * compiled with -fmad=false, so every value is bit-identical to the host's.
 *
 * Row arrays are written as SoA planes: plane j of the values starts at
 * vals + j*plane_stride (gsrgen_npar planes: 24 for the standard sections),
 * plane j of the instrumental columns at instr + j*plane_stride (n_ipr planes). Row r of the chunk is at offset
 * r - star_ptr[s0] within each plane.
 */
#include "gsrgen_core.h"

#include <cuda_runtime.h>

#define GSRGEN_API extern "C" __attribute__((visibility("default")))

/* one thread per star: raw knots, then an in-place insertion sort of the
 * star's segment (segments are at most GSRGEN_MAX_OBS rows) */
__global__ void gsrgen_knots_kernel(gsrgen_cfg c, const int64_t *__restrict__ star_ptr, int64_t s0, int64_t s1,
                                    int32_t *__restrict__ knot)
{
    int64_t s = s0 + (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= s1) return;
    const int64_t base = star_ptr[s0];
    const int64_t r0 = star_ptr[s], r1 = star_ptr[s + 1];
    int32_t *kn = knot + (r0 - base);
    const int32_t n = (int32_t)(r1 - r0);
    for (int32_t i = 0; i < n; ++i) kn[i] = gsrgen_knot_raw(&c, r0 + i);
    for (int32_t i = 1; i < n; ++i) {
        int32_t v = kn[i];
        int32_t j = i - 1;
        while (j >= 0 && kn[j] > v) {
            kn[j + 1] = kn[j];
            --j;
        }
        kn[j + 1] = v;
    }
}

/* one thread per row: instrumental columns and the coefficients */
template <typename VT>
__global__ void gsrgen_rows_kernel(gsrgen_cfg c, int64_t row0, int64_t nrow, int64_t plane_stride, int32_t round32,
                                   VT *__restrict__ vals, int32_t *__restrict__ instr)
{
    int64_t o = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (o >= nrow) return;
    const int64_t r = row0 + o;
    int32_t ic[6];
    gsrgen_instr_row(&c, r, ic);
    for (int j = 0; j < c.n_ipr; ++j) instr[(int64_t)j * plane_stride + o] = ic[j];
    const int np = gsrgen_npar(&c);
    for (int j = 0; j < np; ++j) {
        double v = gsrgen_value(&c, r, j);
        if (round32) v = (double)(float)v;
        vals[(int64_t)j * plane_stride + o] = (VT)v;
    }
}

__global__ void gsrgen_xtrue_kernel(gsrgen_cfg c, int64_t col0, int64_t ncol, double *__restrict__ x)
{
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < ncol) x[i] = gsrgen_xtrue(&c, col0 + i);
}

__global__ void gsrgen_noise_kernel(gsrgen_cfg c, int64_t row0, int64_t nrow, double *__restrict__ eps)
{
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < nrow) eps[i] = gsrgen_noise(&c, row0 + i);
}

static unsigned grid_for(int64_t n, int threads)
{
    return (unsigned)((n + threads - 1) / threads);
}

/*
 * Rows of stars [s0, s1) on the device. star_ptr: device array [n_stars+1]
 * (same contents as gsrgen_host_star_ptr); star_ptr_host: the same on the host
 * (only entries s0 and s1 are read). Exactly one of vals64 / vals32 is used.
 * Returns a cudaError_t value (0 on success).
 */
GSRGEN_API int gsrgen_dev_rows(const gsrgen_cfg *cfg, const int64_t *star_ptr, const int64_t *star_ptr_host,
                               int64_t s0, int64_t s1, int32_t round32, double *vals64, float *vals32,
                               int64_t plane_stride, int32_t *knot, int32_t *instr, void *stream)
{
    cudaStream_t st = (cudaStream_t)stream;
    if (s1 <= s0) return 0;
    const int64_t row0 = star_ptr_host[s0];
    const int64_t nrow = star_ptr_host[s1] - row0;
    gsrgen_knots_kernel<<<grid_for(s1 - s0, 128), 128, 0, st>>>(*cfg, star_ptr, s0, s1, knot);
    if (nrow > 0) {
        if (vals64)
            gsrgen_rows_kernel<double><<<grid_for(nrow, 256), 256, 0, st>>>(*cfg, row0, nrow, plane_stride, round32,
                                                                            vals64, instr);
        else
            gsrgen_rows_kernel<float><<<grid_for(nrow, 256), 256, 0, st>>>(*cfg, row0, nrow, plane_stride, 1,
                                                                           vals32, instr);
    }
    return (int)cudaGetLastError();
}

GSRGEN_API int gsrgen_dev_xtrue(const gsrgen_cfg *cfg, int64_t col0, int64_t ncol, double *x, void *stream)
{
    if (ncol > 0) gsrgen_xtrue_kernel<<<grid_for(ncol, 256), 256, 0, (cudaStream_t)stream>>>(*cfg, col0, ncol, x);
    return (int)cudaGetLastError();
}

GSRGEN_API int gsrgen_dev_noise(const gsrgen_cfg *cfg, int64_t row0, int64_t nrow, double *eps, void *stream)
{
    if (nrow > 0) gsrgen_noise_kernel<<<grid_for(nrow, 256), 256, 0, (cudaStream_t)stream>>>(*cfg, row0, nrow, eps);
    return (int)cudaGetLastError();
}
