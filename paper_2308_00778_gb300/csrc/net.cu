// net.cu -- the learned warm start's network: six 1D convolution layers over the
// attitude knots (6 -> 64 -> 64 -> 64 -> 64 -> 64 -> 3 channels, kernel 5, zero
// padding 2, ReLU after the first five), trained and evaluated on the GPU.
//
// Each convolution is an implicit GEMM on the BF16 tensor cores with FP32 accumulation:
//   forward      out[p][co]   = sum_{t,ci} W[co][ci][t] in[p+t-2][ci]        M = positions, N = co, K = 5*Cin
//   backward x   dIn[p][ci]   = sum_{t,co} W[co][ci][4-t] dOut[p+t-2][co]    the same kernel, flipped weights
//   backward W   dW[co][t,ci] = sum_p dOut[p][co] in[p+t-2][ci]               M = co, N = 5*Cin, K = positions
// All three products issue tcgen05 MMAs from shared memory into a TMEM accumulator (tc.cuh): the
// forward and backward-data ones (k_conv) over 128 positions per CTA, the weight gradient
// (k_conv_wgrad) over chunks of 64 positions accumulated in TMEM.
// Activations are position-major bf16 [B][L][C] with C padded to a multiple
// of 16 (the first layer's 6 input channels and the last layer's 3 output
// channels to 16). FP32 master weights are updated with Adam and copied to
// two bf16 GEMM operands: Bf [Cout][5*Cin] (tap-major K) for the forward pass
// and Bb [Cin][5*Cout] (flipped taps) for the backward-data pass.
// Rounding points (mirrored by the oracle): weights and layer inputs in bf16
// for the forward; the output gradients fed to both backward products in bf16.
#include <cuda_bf16.h>

#include <cstdio>
#include <cstring>
#include <string>

#include "../../include/gsr_warm.h"
#include "gsr_internal.cuh"
#include "tc.cuh"

#define GSR_API extern "C" __attribute__((visibility("default")))

namespace gsr {

constexpr int NLAYER = 6;
// channel counts at layer boundaries 0..6 (true, and padded to multiples of 16, the MMA's K step)
__host__ __device__ constexpr int CH(int l) { return l == 0 ? 6 : (l == NLAYER ? 3 : 64); }
__host__ __device__ constexpr int CHP(int l) { return (l == 0 || l == NLAYER) ? 16 : 64; }
constexpr int KW = 5;                                          // kernel width

__host__ __device__ constexpr int64_t layer_wsize(int l) { return (int64_t)CH(l + 1) * CH(l) * KW; }

static int64_t total_params()
{
    int64_t n = 0;
    for (int l = 0; l < NLAYER; ++l) n += layer_wsize(l) + CH(l + 1);
    return n;
}

__device__ __forceinline__ uint32_t pack2(__nv_bfloat16 lo, __nv_bfloat16 hi)
{
    return (uint32_t)__bfloat16_as_ushort(lo) | ((uint32_t)__bfloat16_as_ushort(hi) << 16);
}

// ---------------------------------------------------------------- convolution (forward / backward-data)
enum { CONV_RELU = 0, CONV_LAST = 1, CONV_BWD = 2, CONV_RAW = 3 };

// The convolution as one tcgen05 MMA chain per CTA: M = 128 positions (one TMEM lane each), N =
// COUT, K = 5 CIN in steps of 16 (one tap and 16 input channels per MMA). The CTA stages its 132
// input rows (positions p0-2 .. p0+129, zero outside [0, L)) and the weights in shared memory as
// 8-row x 16-byte core matrices, so that the operand of tap t is the input block shifted by t rows
// (16 bytes further on): no im2col copy. One thread issues the 5 CIN/16 MMAs; their completion
// arrives on an mbarrier; every warp then reads its 32 rows of the FP32 accumulator from TMEM.
constexpr int CONV_POS = 128;               // positions per CTA: the MMA's M
constexpr uint32_t CONV_TMEM_COLS = 128;    // accumulator columns allocated (>= COUT, a power of two)
constexpr uint64_t CONV_WAIT_NS = 1000000000ull;  // the longest wait for the MMAs (1 s), then a fault

template <int CIN, int COUT>
struct ConvSmem {
    static constexpr int ROWS = CONV_POS + 4;                 // input rows p0-2 .. p0+CONV_POS+1
    static constexpr int K = KW * CIN;
    static constexpr uint32_t A_CHUNK = ROWS * 16;            // one 8-channel column of the input rows
    static constexpr uint32_t A_BYTES = (CIN / 8) * A_CHUNK;
    static constexpr uint32_t B_CHUNK = COUT * 16;            // one 8-wide K column of the weights
    static constexpr uint32_t B_BYTES = (K / 8) * B_CHUNK;
    static constexpr uint32_t B_OFF = (A_BYTES + 127) / 128 * 128;
    static constexpr uint32_t CTRL_OFF = (B_OFF + B_BYTES + 127) / 128 * 128;  // mbarrier, TMEM address
    static constexpr uint32_t USED = CTRL_OFF + 16;
    // at least 72 KB: at most 3 CTAs per SM, whose 3 x 128 TMEM columns fit the SM's 512, so the
    // allocation never waits for another CTA
    static constexpr uint32_t BYTES = USED > 73728 ? USED : 73728;
};

// in: bf16 [B][L][CIN]; Bm: bf16 [COUT][5*CIN] (tap-major K). MODE:
//   CONV_RELU: out16 = bf16(relu(acc + bias))                     [B][L][COUT]
//   CONV_LAST: out32 = acc + bias (fp32)                          [B][L][COUT]
//   CONV_BWD : v = acc * (mask > 0): out32 = v, out16 = bf16(v)   [B][L][COUT]
//   CONV_RAW : out32 = acc (fp32)                                  [B][L][COUT]
// fault: set to 1 when the MMAs did not complete within CONV_WAIT_NS (outputs of the CTA unwritten).
template <int CIN, int COUT, int MODE>
__global__ void __launch_bounds__(128) k_conv(const __nv_bfloat16 *__restrict__ in, int64_t L,
                                              const __nv_bfloat16 *__restrict__ Bm, const float *__restrict__ bias,
                                              const __nv_bfloat16 *__restrict__ mask, __nv_bfloat16 *__restrict__ out16,
                                              float *__restrict__ out32, int32_t *__restrict__ fault)
{
    using SM = ConvSmem<CIN, COUT>;
    static_assert(CIN % 16 == 0 && COUT % 16 == 0 && COUT <= (int)CONV_TMEM_COLS, "MMA shape");
    extern __shared__ __align__(1024) unsigned char conv_smem[];
    unsigned char *sA = conv_smem;
    unsigned char *sB = conv_smem + SM::B_OFF;
    uint64_t *mbar = reinterpret_cast<uint64_t *>(conv_smem + SM::CTRL_OFF);
    uint32_t *tslot = reinterpret_cast<uint32_t *>(conv_smem + SM::CTRL_OFF + 8);
    const int warp = threadIdx.x >> 5;
    const int64_t b = blockIdx.y;
    const int64_t p0 = (int64_t)blockIdx.x * CONV_POS;
    const __nv_bfloat16 *inb = in + b * L * CIN;
    if (warp == 0) tc::tmem_alloc(tslot, CONV_TMEM_COLS);
    if (threadIdx.x == 32) tc::mbar_init(mbar, 1);
    // input rows: row r (position p0 - 2 + r), channels 8j .. 8j+7 at sA + j A_CHUNK + 16 r
    constexpr int CJ = CIN / 8;
    for (int i = threadIdx.x; i < SM::ROWS * CJ; i += blockDim.x) {
        const int r = i / CJ, j = i % CJ;
        const int64_t p = p0 - 2 + r;
        uint4 v = make_uint4(0u, 0u, 0u, 0u);
        if (p >= 0 && p < L) v = *reinterpret_cast<const uint4 *>(inb + p * CIN + 8 * j);
        *reinterpret_cast<uint4 *>(sA + j * SM::A_CHUNK + r * 16) = v;
    }
    // weights: output channel n, K columns 8j .. 8j+7 at sB + j B_CHUNK + 16 n
    constexpr int KJ = SM::K / 8;
    for (int i = threadIdx.x; i < COUT * KJ; i += blockDim.x) {
        const int n = i / KJ, j = i % KJ;
        *reinterpret_cast<uint4 *>(sB + j * SM::B_CHUNK + n * 16) =
            *reinterpret_cast<const uint4 *>(Bm + (int64_t)n * SM::K + 8 * j);
    }
    tc::fence_proxy_async_smem();
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    const uint32_t tmem = *tslot;
    if (threadIdx.x == 0) {
        constexpr uint32_t idesc = tc::idesc_bf16_f32(CONV_POS, COUT);
        const uint32_t a0 = tc::smem_u32(sA), b0 = tc::smem_u32(sB);
#pragma unroll 1
        for (int t = 0; t < KW; ++t)
#pragma unroll 1
            for (int c = 0; c < CIN / 16; ++c) {
                // A: positions p0 .. p0+127 at tap t (input rows t .. t+127), channels 16c .. 16c+15
                const uint64_t ad = tc::smem_desc(a0 + 2 * c * SM::A_CHUNK + 16 * t, SM::A_CHUNK, 128);
                // B: K columns t CIN + 16c .. +15 of every output channel
                const uint64_t bd = tc::smem_desc(b0 + ((t * CIN + 16 * c) / 8) * SM::B_CHUNK, SM::B_CHUNK, 128);
                tc::mma_bf16(tmem, ad, bd, idesc, t > 0 || c > 0);
            }
        tc::mma_commit(mbar);
    }
    // the same verdict for every thread: the TMEM loads below are warp-collective
    const bool ok = __syncthreads_and(tc::mbar_wait(mbar, 0, CONV_WAIT_NS));
    tc::fence_after_sync();
    if (ok) {
        const int m = threadIdx.x;  // accumulator row = TMEM lane = position p0 + m
        const int64_t p = p0 + m;
        const int64_t o = (b * L + p) * COUT;
        const uint32_t lane_addr = tmem + ((uint32_t)(warp * 32) << 16);
#pragma unroll 1
        for (int n0 = 0; n0 < COUT; n0 += 16) {
            float v[16];
            tc::tmem_ld16(lane_addr + (uint32_t)n0, v);
            if (p >= L) continue;
            if (MODE == CONV_RELU || MODE == CONV_LAST) {
#pragma unroll
                for (int e = 0; e < 16; ++e) v[e] += bias[n0 + e];
            }
            if (MODE == CONV_BWD) {
                const uint4 *mk = reinterpret_cast<const uint4 *>(mask + o + n0);
                const uint4 mv[2] = {mk[0], mk[1]};
                const __nv_bfloat16 *mb = reinterpret_cast<const __nv_bfloat16 *>(mv);
#pragma unroll
                for (int e = 0; e < 16; ++e) v[e] = __bfloat162float(mb[e]) > 0.f ? v[e] : 0.f;
            }
            if (MODE == CONV_RELU || MODE == CONV_BWD) {
                uint4 w[2];
                uint32_t *wp = reinterpret_cast<uint32_t *>(w);
#pragma unroll
                for (int e = 0; e < 8; ++e) {
                    float lo = v[2 * e], hi = v[2 * e + 1];
                    if (MODE == CONV_RELU) {
                        lo = lo > 0.f ? lo : 0.f;
                        hi = hi > 0.f ? hi : 0.f;
                    }
                    wp[e] = pack2(__float2bfloat16_rn(lo), __float2bfloat16_rn(hi));
                }
                uint4 *dst = reinterpret_cast<uint4 *>(out16 + o + n0);
                dst[0] = w[0];
                dst[1] = w[1];
            }
            if (MODE != CONV_RELU) {
                float4 *dst = reinterpret_cast<float4 *>(out32 + o + n0);
#pragma unroll
                for (int q = 0; q < 4; ++q) dst[q] = make_float4(v[4 * q], v[4 * q + 1], v[4 * q + 2], v[4 * q + 3]);
            }
        }
    } else if (threadIdx.x == 0) {
        atomicExch(fault, 1);
    }
    tc::fence_before_sync();
    __syncthreads();
    if (warp == 0) {
        // after a timeout, give the MMAs one more bounded wait before their TMEM is released
        if (!ok) tc::mbar_wait(mbar, 0, CONV_WAIT_NS);
        tc::fence_after_sync();
        tc::tmem_dealloc(tmem, CONV_TMEM_COLS);
    }
}

// ---------------------------------------------------------------- backward weights
// dW[co][t*CIN + ci] += sum_p dout[p][co] in[p+t-2][ci] as tcgen05 MMAs: M = 128 of the 5 CIN
// (tap, channel) rows (blockIdx.y picks the M tile), N = COUT, K = positions, 64 per chunk. A CTA
// stages a chunk's input and output-gradient rows position-major, transposes them into K-major core
// matrices (A[m][k] = in[p0+k+t-2][ci], B[n][k] = dout[p0+k][n]), issues 4 MMAs of K = 16 and waits
// for them (bounded) before the next chunk; its FP32 accumulator (TMEM) is added into dW with atomics
// at the end. Positions past L have zero output gradient, so they add nothing.
constexpr int WG_POS = 64;  // positions per chunk (the MMAs' K per chunk)

template <int CIN, int COUT>
struct WgradSmem {
    static constexpr uint32_t A_CHUNK = 128 * 16;                 // one 8-position column of A
    static constexpr uint32_t A_BYTES = (WG_POS / 8) * A_CHUNK;
    static constexpr uint32_t B_CHUNK = COUT * 16;                // one 8-position column of B
    static constexpr uint32_t B_OFF = A_BYTES;
    static constexpr uint32_t B_BYTES = (WG_POS / 8) * B_CHUNK;
    static constexpr uint32_t IN_OFF = B_OFF + B_BYTES;           // input rows p0-2 .. p0+65, [pos][ch]
    static constexpr uint32_t IN_BYTES = (WG_POS + 4) * CIN * 2;
    static constexpr uint32_t D_OFF = (IN_OFF + IN_BYTES + 15) / 16 * 16;  // output-gradient rows, [pos][co]
    static constexpr uint32_t D_BYTES = WG_POS * COUT * 2;
    static constexpr uint32_t CTRL_OFF = (D_OFF + D_BYTES + 15) / 16 * 16;
    static constexpr uint32_t USED = CTRL_OFF + 16;
    static constexpr uint32_t BYTES = USED > 73728 ? USED : 73728;  // at most 3 CTAs (TMEM) per SM
};

template <int CIN, int COUT>
__global__ void __launch_bounds__(128) k_conv_wgrad(const __nv_bfloat16 *__restrict__ in,
                                                    const __nv_bfloat16 *__restrict__ dout, int64_t B, int64_t L,
                                                    float *__restrict__ dW, int32_t *__restrict__ fault)
{
    using SM = WgradSmem<CIN, COUT>;
    constexpr int K5 = KW * CIN;
    static_assert(CIN % 8 == 0 && COUT % 16 == 0 && COUT <= (int)CONV_TMEM_COLS, "MMA shape");
    extern __shared__ __align__(1024) unsigned char wg_smem[];
    unsigned char *sA = wg_smem;
    unsigned char *sB = wg_smem + SM::B_OFF;
    const __nv_bfloat16 *s_in = reinterpret_cast<const __nv_bfloat16 *>(wg_smem + SM::IN_OFF);
    const __nv_bfloat16 *s_d = reinterpret_cast<const __nv_bfloat16 *>(wg_smem + SM::D_OFF);
    uint64_t *mbar = reinterpret_cast<uint64_t *>(wg_smem + SM::CTRL_OFF);
    uint32_t *tslot = reinterpret_cast<uint32_t *>(wg_smem + SM::CTRL_OFF + 8);
    const int warp = threadIdx.x >> 5;
    const int mt = blockIdx.y;
    if (warp == 0) tc::tmem_alloc(tslot, CONV_TMEM_COLS);
    if (threadIdx.x == 32) tc::mbar_init(mbar, 1);
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    const uint32_t tmem = *tslot;
    const int64_t cps = (L + WG_POS - 1) / WG_POS;
    const int64_t n_chunks = B * cps;
    uint32_t phase = 0;
    bool any = false, ok = true;
    for (int64_t ch = blockIdx.x; ch < n_chunks; ch += gridDim.x) {
        if (any) {  // the previous chunk's MMAs read shared memory: wait for them before restaging
            ok = __syncthreads_and(tc::mbar_wait(mbar, phase, CONV_WAIT_NS));
            if (!ok) break;  // phase still names the uncompleted one, for the last wait below
            phase ^= 1u;
            tc::fence_after_sync();
        }
        const int64_t b = ch / cps;
        const int64_t p0 = (ch % cps) * WG_POS;
        // position-major staging: input rows p0-2 .. p0+WG_POS+1 and output-gradient rows p0 .. p0+63
        {
            uint4 *si = reinterpret_cast<uint4 *>(wg_smem + SM::IN_OFF);
            constexpr int CJ = CIN / 8;
            for (int i = threadIdx.x; i < (WG_POS + 4) * CJ; i += blockDim.x) {
                const int r = i / CJ, j = i % CJ;
                const int64_t p = p0 - 2 + r;
                si[i] = (p >= 0 && p < L) ? *reinterpret_cast<const uint4 *>(in + (b * L + p) * CIN + 8 * j)
                                          : make_uint4(0u, 0u, 0u, 0u);
            }
            uint4 *sd = reinterpret_cast<uint4 *>(wg_smem + SM::D_OFF);
            constexpr int NJ = COUT / 8;
            for (int i = threadIdx.x; i < WG_POS * NJ; i += blockDim.x) {
                const int r = i / NJ, j = i % NJ;
                const int64_t p = p0 + r;
                sd[i] = p < L ? *reinterpret_cast<const uint4 *>(dout + (b * L + p) * COUT + 8 * j)
                              : make_uint4(0u, 0u, 0u, 0u);
            }
        }
        __syncthreads();
        // K-major core matrices: row m (or n), 8 consecutive positions per 16 bytes
        for (int i = threadIdx.x; i < 128 * (WG_POS / 8); i += blockDim.x) {
            const int m = i % 128, j = i / 128;
            const int mg = mt * 128 + m;
            uint32_t w[4] = {0u, 0u, 0u, 0u};
            if (mg < K5) {
                const int t = mg / CIN, ci = mg % CIN;
#pragma unroll
                for (int q = 0; q < 4; ++q)
                    w[q] = pack2(s_in[(8 * j + 2 * q + t) * CIN + ci], s_in[(8 * j + 2 * q + 1 + t) * CIN + ci]);
            }
            *reinterpret_cast<uint4 *>(sA + j * SM::A_CHUNK + m * 16) = make_uint4(w[0], w[1], w[2], w[3]);
        }
        for (int i = threadIdx.x; i < COUT * (WG_POS / 8); i += blockDim.x) {
            const int n = i % COUT, j = i / COUT;
            uint32_t w[4];
#pragma unroll
            for (int q = 0; q < 4; ++q)
                w[q] = pack2(s_d[(8 * j + 2 * q) * COUT + n], s_d[(8 * j + 2 * q + 1) * COUT + n]);
            *reinterpret_cast<uint4 *>(sB + j * SM::B_CHUNK + n * 16) = make_uint4(w[0], w[1], w[2], w[3]);
        }
        tc::fence_proxy_async_smem();
        tc::fence_before_sync();
        __syncthreads();
        tc::fence_after_sync();
        if (threadIdx.x == 0) {
            constexpr uint32_t idesc = tc::idesc_bf16_f32(128, COUT);
            const uint32_t a0 = tc::smem_u32(sA), b0 = tc::smem_u32(sB);
#pragma unroll 1
            for (int j = 0; j < WG_POS / 16; ++j) {
                const uint64_t ad = tc::smem_desc(a0 + 2 * j * SM::A_CHUNK, SM::A_CHUNK, 128);
                const uint64_t bd = tc::smem_desc(b0 + 2 * j * SM::B_CHUNK, SM::B_CHUNK, 128);
                tc::mma_bf16(tmem, ad, bd, idesc, any || j > 0);
            }
            tc::mma_commit(mbar);
        }
        any = true;
    }
    if (any && ok) ok = __syncthreads_and(tc::mbar_wait(mbar, phase, CONV_WAIT_NS));
    tc::fence_after_sync();
    if (any && ok) {
        const int mg = mt * 128 + (int)threadIdx.x;  // accumulator row = TMEM lane
        const uint32_t lane_addr = tmem + ((uint32_t)(warp * 32) << 16);
#pragma unroll 1
        for (int n0 = 0; n0 < COUT; n0 += 16) {
            float v[16];
            tc::tmem_ld16(lane_addr + (uint32_t)n0, v);
            if (mg >= K5) continue;
#pragma unroll
            for (int e = 0; e < 16; ++e)
                if (v[e] != 0.f) atomicAdd(dW + (int64_t)(n0 + e) * K5 + mg, v[e]);
        }
    } else if (any && threadIdx.x == 0) {
        atomicExch(fault, 1);
    }
    tc::fence_before_sync();
    __syncthreads();
    if (warp == 0) {
        // after a timeout, give the MMAs one more bounded wait before their TMEM is released
        if (any && !ok) tc::mbar_wait(mbar, phase, CONV_WAIT_NS);
        tc::fence_after_sync();
        tc::tmem_dealloc(tmem, CONV_TMEM_COLS);
    }
}

template <int CIN, int COUT>
static void wgrad_launch(const __nv_bfloat16 *in, const __nv_bfloat16 *dout, int64_t B, int64_t L, float *dW,
                         int32_t *fault, cudaStream_t s)
{
    constexpr uint32_t smem = WgradSmem<CIN, COUT>::BYTES;
    cudaFuncSetAttribute(k_conv_wgrad<CIN, COUT>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    const int64_t n_chunks = B * ((L + WG_POS - 1) / WG_POS);
    const dim3 grid((unsigned)std::min<int64_t>(std::max<int64_t>(n_chunks, 1), 128),
                    (unsigned)((KW * CIN + 127) / 128));
    k_conv_wgrad<CIN, COUT><<<grid, 128, smem, s>>>(in, dout, B, L, dW, fault);
}

// db[co] += sum over positions of the fp32 output gradient
__global__ void k_bias_grad(const float *__restrict__ d32, int64_t n_pos, int cout, int cstride, float *__restrict__ db)
{
    extern __shared__ float sdb[];
    for (int c = threadIdx.x; c < cout; c += blockDim.x) sdb[c] = 0.f;
    __syncthreads();
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n_pos * cout;
         i += (int64_t)gridDim.x * blockDim.x) {
        const int64_t p = i / cout;
        const int c = (int)(i % cout);
        atomicAdd(sdb + c, d32[p * cstride + c]);
    }
    __syncthreads();
    for (int c = threadIdx.x; c < cout; c += blockDim.x)
        if (sdb[c] != 0.f) atomicAdd(db + c, sdb[c]);
}

// ---------------------------------------------------------------- input / output / loss
// fp32 [n][6] -> bf16 [n][16] (zero padding)
__global__ void k_pack_input(const float *__restrict__ x, int64_t n, __nv_bfloat16 *__restrict__ out)
{
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n * CHP(0);
         i += (int64_t)gridDim.x * blockDim.x) {
        const int64_t p = i / CHP(0);
        const int c = (int)(i % CHP(0));
        out[i] = __float2bfloat16_rn(c < CH(0) ? x[p * CH(0) + c] : 0.f);
    }
}

// fp32 [n][c] -> bf16 [n][cp] and (f32 non-null) fp32 [n][cp], zero padding
__global__ void k_pack_any(const float *__restrict__ x, int64_t n, int c, int cp, __nv_bfloat16 *__restrict__ out,
                           float *__restrict__ f32)
{
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n * cp; i += (int64_t)gridDim.x * blockDim.x) {
        const int64_t p = i / cp;
        const int ch = (int)(i % cp);
        const float v = ch < c ? x[p * c + ch] : 0.f;
        out[i] = __float2bfloat16_rn(v);
        if (f32) f32[i] = v;
    }
}

// fp32 [n][cp] -> fp32 [n][c]
__global__ void k_unpack_any(const float *__restrict__ y, int64_t n, int c, int cp, float *__restrict__ out)
{
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n * c; i += (int64_t)gridDim.x * blockDim.x)
        out[i] = y[(i / c) * cp + i % c];
}

// padded dW [coutp][5 cinp] (tap-major) -> W layout [cout][cin][5]
__global__ void k_unpack_dw(const float *__restrict__ dwp, int cin, int cout, int cinp, float *__restrict__ dw)
{
    const int64_t n = (int64_t)cout * cin * KW;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const int co = (int)(i / (cin * KW)), ci = (int)((i / KW) % cin), t = (int)(i % KW);
        dw[i] = dwp[(int64_t)co * (KW * cinp) + t * cinp + ci];
    }
}

__global__ void k_unpack_output(const float *__restrict__ y8, int64_t n, float *__restrict__ y3)
{
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n * CH(NLAYER);
         i += (int64_t)gridDim.x * blockDim.x)
        y3[i] = y8[(i / CH(NLAYER)) * CHP(NLAYER) + i % CH(NLAYER)];
}

// MSE over the 3 true output channels: d = 2 (y - t) / N in fp32 and bf16 [n][8]; loss partial sums
__global__ void k_mse(const float *__restrict__ y8, const float *__restrict__ t3, int64_t n,
                      float *__restrict__ d32, __nv_bfloat16 *__restrict__ d16, double *__restrict__ loss)
{
    __shared__ double sm32[32];
    const double inv = 1.0 / (double)(n * CH(NLAYER));
    double s = 0.0;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n * CHP(NLAYER);
         i += (int64_t)gridDim.x * blockDim.x) {
        const int64_t p = i / CHP(NLAYER);
        const int c = (int)(i % CHP(NLAYER));
        float d = 0.f;
        if (c < CH(NLAYER)) {
            const float e = y8[i] - t3[p * CH(NLAYER) + c];
            s += (double)e * (double)e;
            d = (float)(2.0 * (double)e * inv);
        }
        d32[i] = d;
        d16[i] = __float2bfloat16_rn(d);
    }
    const double tot = block_sum(s, sm32);
    if (threadIdx.x == 0) atomicAdd(loss, tot * inv);
}

// ---------------------------------------------------------------- Adam + operand refresh
// Per true parameter (co, ci, t) of layer l: Adam on the fp32 master and
// refresh of the two bf16 GEMM operands; bias entries follow the weights.
__global__ void k_adam_layer(float *__restrict__ w, float *__restrict__ m, float *__restrict__ v,
                             float *__restrict__ bias, float *__restrict__ mb, float *__restrict__ vb,
                             float *__restrict__ dW, float *__restrict__ db, int cin, int cout, int cinp, int coutp,
                             float lr, float b1, float b2, float eps, float c1, float c2, int update,
                             __nv_bfloat16 *__restrict__ Bf, __nv_bfloat16 *__restrict__ Bb)
{
    const int64_t nw = (int64_t)cout * cin * KW;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < nw + cout;
         i += (int64_t)gridDim.x * blockDim.x) {
        if (i < nw) {
            const int co = (int)(i / (cin * KW));
            const int ci = (int)((i / KW) % cin);
            const int t = (int)(i % KW);
            const int64_t gi = (int64_t)co * (KW * cinp) + t * cinp + ci;
            float wv = w[i];
            if (update) {
                const float gr = dW[gi];
                const float mv = b1 * m[i] + (1.f - b1) * gr;
                const float vv = b2 * v[i] + (1.f - b2) * gr * gr;
                m[i] = mv;
                v[i] = vv;
                wv = wv - lr * (mv / c1) / (sqrtf(vv / c2) + eps);
                w[i] = wv;
                dW[gi] = 0.f;
            }
            const __nv_bfloat16 h = __float2bfloat16_rn(wv);
            Bf[gi] = h;
            Bb[(int64_t)ci * (KW * coutp) + (KW - 1 - t) * coutp + co] = h;
        } else {
            const int co = (int)(i - nw);
            if (update) {
                const float gr = db[co];
                const float mv = b1 * mb[co] + (1.f - b1) * gr;
                const float vv = b2 * vb[co] + (1.f - b2) * gr * gr;
                mb[co] = mv;
                vb[co] = vv;
                bias[co] = bias[co] - lr * (mv / c1) / (sqrtf(vv / c2) + eps);
                db[co] = 0.f;
            }
        }
    }
}

}  // namespace gsr

using namespace gsr;

// ---------------------------------------------------------------- the net object
struct gsr_net {
    int device = 0;
    float *w[NLAYER] = {}, *b[NLAYER] = {}, *mw[NLAYER] = {}, *vw[NLAYER] = {}, *mb[NLAYER] = {}, *vb[NLAYER] = {};
    float *dW[NLAYER] = {}, *db[NLAYER] = {};
    __nv_bfloat16 *Bf[NLAYER] = {}, *Bb[NLAYER] = {};
    // activations for a batch of up to cap_pos positions
    int64_t cap_pos = 0;
    __nv_bfloat16 *act[NLAYER] = {};  // input of layer l, [pos][CHP(l)]
    float *y8 = nullptr;              // last layer output [pos][16] (3 used)
    float *d32 = nullptr;             // output gradient fp32 [pos][64]
    __nv_bfloat16 *d16a = nullptr, *d16b = nullptr;  // output gradients bf16 [pos][64] (ping-pong)
    double *loss = nullptr;
    // set by a convolution whose tensor-core wait ran out (mapped pinned word and its device alias);
    // read and cleared by the next call on the net, and by a solve that ran the net
    int32_t *fault_h = nullptr, *fault_d = nullptr;
    int step = 0;
    std::string err;
};

namespace gsr {

static void net_free_acts(gsr_net *n)
{
    for (int l = 0; l < NLAYER; ++l) {
        cudaFree(n->act[l]);
        n->act[l] = nullptr;
    }
    cudaFree(n->y8);
    cudaFree(n->d32);
    cudaFree(n->d16a);
    cudaFree(n->d16b);
    n->y8 = n->d32 = nullptr;
    n->d16a = n->d16b = nullptr;
    n->cap_pos = 0;
}

static cudaError_t net_reserve(gsr_net *n, int64_t pos)
{
    if (pos <= n->cap_pos) return cudaSuccess;
    net_free_acts(n);
    cudaError_t e = cudaSuccess;
    for (int l = 0; l < NLAYER && e == cudaSuccess; ++l)
        e = cudaMalloc(&n->act[l], sizeof(__nv_bfloat16) * (size_t)pos * CHP(l));
    if (e == cudaSuccess) e = cudaMalloc(&n->y8, sizeof(float) * (size_t)pos * CHP(NLAYER));
    if (e == cudaSuccess) e = cudaMalloc(&n->d32, sizeof(float) * (size_t)pos * 64);
    if (e == cudaSuccess) e = cudaMalloc(&n->d16a, sizeof(__nv_bfloat16) * (size_t)pos * 64);
    if (e == cudaSuccess) e = cudaMalloc(&n->d16b, sizeof(__nv_bfloat16) * (size_t)pos * 64);
    if (e != cudaSuccess) {
        net_free_acts(n);
        return e;
    }
    n->cap_pos = pos;
    return cudaSuccess;
}

static int grid_n(int64_t n, int threads = 256)
{
    return (int)std::max<int64_t>(1, std::min<int64_t>((n + threads - 1) / threads, 4096));
}

static cudaError_t refresh_operands(gsr_net *n, bool update, float lr, cudaStream_t s)
{
    const float b1 = 0.9f, b2 = 0.999f, eps = 1e-8f;
    const float c1 = update ? 1.f - powf(b1, (float)n->step) : 1.f;
    const float c2 = update ? 1.f - powf(b2, (float)n->step) : 1.f;
    for (int l = 0; l < NLAYER; ++l) {
        const int64_t cnt = layer_wsize(l) + CH(l + 1);
        k_adam_layer<<<grid_n(cnt), 256, 0, s>>>(n->w[l], n->mw[l], n->vw[l], n->b[l], n->mb[l], n->vb[l], n->dW[l],
                                                 n->db[l], CH(l), CH(l + 1), CHP(l), CHP(l + 1), lr, b1, b2, eps, c1,
                                                 c2, update ? 1 : 0, n->Bf[l], n->Bb[l]);
    }
    return cudaGetLastError();
}

template <int CIN, int COUT, int MODE>
static void conv_launch(dim3 grid, const __nv_bfloat16 *in, int64_t L, const __nv_bfloat16 *Bm, const float *bias,
                        const __nv_bfloat16 *mask, __nv_bfloat16 *out16, float *out32, int32_t *fault, cudaStream_t s)
{
    constexpr uint32_t smem = ConvSmem<CIN, COUT>::BYTES;
    // the opt-in above 48 KB of shared memory (per device: set on every launch)
    cudaFuncSetAttribute(k_conv<CIN, COUT, MODE>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    k_conv<CIN, COUT, MODE><<<grid, 128, smem, s>>>(in, L, Bm, bias, mask, out16, out32, fault);
}

// forward of the whole net on act[0] (already packed); fills act[1..5] and y8
static cudaError_t net_forward_packed(gsr_net *n, int64_t B, int64_t L, cudaStream_t s)
{
    const dim3 grid((unsigned)((L + CONV_POS - 1) / CONV_POS), (unsigned)B);
    conv_launch<16, 64, CONV_RELU>(grid, n->act[0], L, n->Bf[0], n->b[0], nullptr, n->act[1], nullptr, n->fault_d, s);
    for (int l = 1; l < NLAYER - 1; ++l)
        conv_launch<64, 64, CONV_RELU>(grid, n->act[l], L, n->Bf[l], n->b[l], nullptr, n->act[l + 1], nullptr, n->fault_d, s);
    conv_launch<64, 16, CONV_LAST>(grid, n->act[NLAYER - 1], L, n->Bf[NLAYER - 1], n->b[NLAYER - 1], nullptr,
                                   nullptr, n->y8, n->fault_d, s);
    return cudaGetLastError();
}

cudaError_t net_forward_dev(gsr_net *n, const float *in, int64_t B, int64_t L, float *out, cudaStream_t s)
{
    cudaError_t e = net_reserve(n, B * L);
    if (e != cudaSuccess) return e;
    k_pack_input<<<grid_n(B * L * CHP(0)), 256, 0, s>>>(in, B * L, n->act[0]);
    if ((e = net_forward_packed(n, B, L, s)) != cudaSuccess) return e;
    k_unpack_output<<<grid_n(B * L * 3), 256, 0, s>>>(n->y8, B * L, out);
    return cudaGetLastError();
}

// gradients of layer l from its output gradient (dcur bf16, d32 fp32): dW, db and,
// for l > 0, the masked gradient of the previous layer's output into dnext / d32
static void backward_layer(gsr_net *n, int l, const __nv_bfloat16 *dcur, __nv_bfloat16 *dnext, int64_t B, int64_t L,
                           cudaStream_t s)
{
    const int64_t P = B * L;
    const int cout = CHP(l + 1);
    if (l == 0)
        wgrad_launch<16, 64>(n->act[l], dcur, B, L, n->dW[l], n->fault_d, s);
    else if (l == NLAYER - 1)
        wgrad_launch<64, 16>(n->act[l], dcur, B, L, n->dW[l], n->fault_d, s);
    else
        wgrad_launch<64, 64>(n->act[l], dcur, B, L, n->dW[l], n->fault_d, s);
    k_bias_grad<<<grid_n(P * CH(l + 1)), 256, sizeof(float) * CH(l + 1), s>>>(n->d32, P, CH(l + 1), cout, n->db[l]);
    if (l > 0) {
        const dim3 grid((unsigned)((L + CONV_POS - 1) / CONV_POS), (unsigned)B);
        if (l == NLAYER - 1)
            conv_launch<16, 64, CONV_BWD>(grid, dcur, L, n->Bb[l], nullptr, n->act[l], dnext, n->d32, n->fault_d, s);
        else
            conv_launch<64, 64, CONV_BWD>(grid, dcur, L, n->Bb[l], nullptr, n->act[l], dnext, n->d32, n->fault_d, s);
    }
}

static cudaError_t net_train_dev(gsr_net *n, const float *in, const float *target, int64_t B, int64_t L, float lr,
                                 double *loss_host, cudaStream_t s)
{
    cudaError_t e = net_reserve(n, B * L);
    if (e != cudaSuccess) return e;
    const int64_t P = B * L;
    k_pack_input<<<grid_n(P * CHP(0)), 256, 0, s>>>(in, P, n->act[0]);
    if ((e = net_forward_packed(n, B, L, s)) != cudaSuccess) return e;
    if ((e = cudaMemsetAsync(n->loss, 0, sizeof(double), s)) != cudaSuccess) return e;
    k_mse<<<grid_n(P * CHP(NLAYER)), 256, 0, s>>>(n->y8, target, P, n->d32, n->d16a, n->loss);
    __nv_bfloat16 *dcur = n->d16a, *dnext = n->d16b;
    for (int l = NLAYER - 1; l >= 0; --l) {
        backward_layer(n, l, dcur, dnext, B, L, s);
        if (l > 0) std::swap(dcur, dnext);
    }
    n->step += 1;
    if ((e = refresh_operands(n, true, lr, s)) != cudaSuccess) return e;
    if (loss_host) {
        if ((e = cudaMemcpyAsync(loss_host, n->loss, sizeof(double), cudaMemcpyDeviceToHost, s)) != cudaSuccess)
            return e;
        if ((e = cudaStreamSynchronize(s)) != cudaSuccess) return e;
    }
    return cudaGetLastError();
}

// one layer on caller data (the per-layer checks of gsr_net_layer_forward / _backward)
template <int CINP, int COUTP>
static cudaError_t layer_fwd_t(gsr_net *n, int l, const float *in, int64_t B, int64_t L, float *out, cudaStream_t s)
{
    const int64_t P = B * L;
    k_pack_any<<<grid_n(P * CINP), 256, 0, s>>>(in, P, CH(l), CINP, n->act[l], nullptr);
    const dim3 grid((unsigned)((L + CONV_POS - 1) / CONV_POS), (unsigned)B);
    conv_launch<CINP, COUTP, CONV_LAST>(grid, n->act[l], L, n->Bf[l], n->b[l], nullptr, nullptr, n->d32, n->fault_d, s);
    k_unpack_any<<<grid_n(P * CH(l + 1)), 256, 0, s>>>(n->d32, P, CH(l + 1), COUTP, out);
    return cudaGetLastError();
}

template <int CINP, int COUTP>
static cudaError_t layer_bwd_t(gsr_net *n, int l, const float *in, const float *dout, int64_t B, int64_t L, float *din,
                               float *dW, float *db, cudaStream_t s)
{
    const int64_t P = B * L;
    cudaError_t e = cudaMemsetAsync(n->dW[l], 0, sizeof(float) * (size_t)COUTP * KW * CINP, s);
    if (e == cudaSuccess) e = cudaMemsetAsync(n->db[l], 0, sizeof(float) * CH(l + 1), s);
    if (e != cudaSuccess) return e;
    k_pack_any<<<grid_n(P * CINP), 256, 0, s>>>(in, P, CH(l), CINP, n->act[l], nullptr);
    // the output gradient in bf16 for both products, in fp32 for the bias gradient
    k_pack_any<<<grid_n(P * COUTP), 256, 0, s>>>(dout, P, CH(l + 1), COUTP, n->d16a, n->d32);
    wgrad_launch<CINP, COUTP>(n->act[l], n->d16a, B, L, n->dW[l], n->fault_d, s);
    k_bias_grad<<<grid_n(P * CH(l + 1)), 256, sizeof(float) * CH(l + 1), s>>>(n->d32, P, CH(l + 1), COUTP, n->db[l]);
    k_unpack_dw<<<grid_n(layer_wsize(l)), 256, 0, s>>>(n->dW[l], CH(l), CH(l + 1), CINP, dW);
    if ((e = cudaMemcpyAsync(db, n->db[l], sizeof(float) * CH(l + 1), cudaMemcpyDeviceToDevice, s)) != cudaSuccess)
        return e;
    if (din) {  // the flipped-weight product, unmasked, fp32 (after the bias gradient has read d32)
        const dim3 grid((unsigned)((L + CONV_POS - 1) / CONV_POS), (unsigned)B);
        conv_launch<COUTP, CINP, CONV_RAW>(grid, n->d16a, L, n->Bb[l], nullptr, nullptr, nullptr, n->d32, n->fault_d, s);
        k_unpack_any<<<grid_n(P * CH(l)), 256, 0, s>>>(n->d32, P, CH(l), CINP, din);
    }
    // leave the accumulators zero for training
    if ((e = cudaMemsetAsync(n->dW[l], 0, sizeof(float) * (size_t)COUTP * KW * CINP, s)) == cudaSuccess)
        e = cudaMemsetAsync(n->db[l], 0, sizeof(float) * CH(l + 1), s);
    if (e != cudaSuccess) return e;
    return cudaGetLastError();
}

static gsr_status net_fail(gsr_net *n, gsr_status st, const std::string &m)
{
    if (n) n->err = m;
    return st;
}

// true (and cleared) when a convolution launched earlier on this net found its tensor-core wait
// run out; the word is written by kernels that have finished, so a caller that synchronised after
// the launches sees all of them
bool net_take_fault(gsr_net *n)
{
    if (!n || !n->fault_h) return false;
    volatile int32_t *f = n->fault_h;
    if (*f == 0) return false;
    *f = 0;
    return true;
}

static gsr_status net_fault_status(gsr_net *n)
{
    return net_take_fault(n) ? net_fail(n, GSR_ECUDA, "an earlier call's tensor-core wait timed out") : GSR_OK;
}

}  // namespace gsr

// ---------------------------------------------------------------- C ABI
GSR_API int64_t gsr_net_num_params(void) { return total_params(); }

GSR_API const char *gsr_net_last_error(const gsr_net *n) { return n ? n->err.c_str() : "null net"; }

GSR_API gsr_status gsr_net_destroy(gsr_net *n)
{
    if (!n) return GSR_OK;
    cudaSetDevice(n->device);
    net_free_acts(n);
    for (int l = 0; l < NLAYER; ++l) {
        float *fp[] = {n->w[l], n->b[l], n->mw[l], n->vw[l], n->mb[l], n->vb[l], n->dW[l], n->db[l]};
        for (float *p : fp) cudaFree(p);
        cudaFree(n->Bf[l]);
        cudaFree(n->Bb[l]);
    }
    cudaFree(n->loss);
    cudaFreeHost(n->fault_h);
    cudaGetLastError();
    delete n;
    return GSR_OK;
}

GSR_API gsr_status gsr_net_create(gsr_net **out, int32_t device)
{
    if (!out) return GSR_EINVAL;
    *out = nullptr;
    gsr_net *n = new gsr_net();
    n->device = device;
    cudaError_t e = cudaSetDevice(device);
    for (int l = 0; l < NLAYER && e == cudaSuccess; ++l) {
        const size_t ws = sizeof(float) * (size_t)layer_wsize(l), bs = sizeof(float) * CHP(l + 1);
        const size_t gs = sizeof(float) * (size_t)CHP(l + 1) * KW * CHP(l);
        const size_t os = sizeof(__nv_bfloat16) * (size_t)CHP(l + 1) * KW * CHP(l);
        float **wp[] = {&n->w[l], &n->mw[l], &n->vw[l]};
        for (float **p : wp)
            if (e == cudaSuccess && (e = cudaMalloc(p, ws)) == cudaSuccess) e = cudaMemset(*p, 0, ws);
        float **bp[] = {&n->b[l], &n->mb[l], &n->vb[l], &n->db[l]};
        for (float **p : bp)
            if (e == cudaSuccess && (e = cudaMalloc(p, bs)) == cudaSuccess) e = cudaMemset(*p, 0, bs);
        if (e == cudaSuccess && (e = cudaMalloc(&n->dW[l], gs)) == cudaSuccess) e = cudaMemset(n->dW[l], 0, gs);
        if (e == cudaSuccess && (e = cudaMalloc(&n->Bf[l], os)) == cudaSuccess) e = cudaMemset(n->Bf[l], 0, os);
        if (e == cudaSuccess && (e = cudaMalloc(&n->Bb[l], os)) == cudaSuccess) e = cudaMemset(n->Bb[l], 0, os);
    }
    if (e == cudaSuccess) e = cudaMalloc(&n->loss, sizeof(double));
    if (e == cudaSuccess && (e = cudaHostAlloc(&n->fault_h, sizeof(int32_t), cudaHostAllocMapped)) == cudaSuccess) {
        *n->fault_h = 0;
        e = cudaHostGetDevicePointer(&n->fault_d, n->fault_h, 0);
    }
    if (e != cudaSuccess) {
        cudaGetLastError();
        gsr_net_destroy(n);
        return e == cudaErrorMemoryAllocation ? GSR_ENOMEM : GSR_ECUDA;
    }
    *out = n;
    return GSR_OK;
}

// parameters: for each layer, W [cout][cin][5] then bias [cout] (fp32); resets Adam
GSR_API gsr_status gsr_net_set_params(gsr_net *n, const float *params, int64_t count)
{
    if (!n || !params) return GSR_EINVAL;
    if (count != total_params()) return net_fail(n, GSR_EINVAL, "parameter count mismatch");
    cudaError_t e = cudaSetDevice(n->device);
    int64_t off = 0;
    for (int l = 0; l < NLAYER && e == cudaSuccess; ++l) {
        const int64_t nw = layer_wsize(l), nb = CH(l + 1);
        e = cudaMemcpy(n->w[l], params + off, sizeof(float) * nw, cudaMemcpyHostToDevice);
        if (e == cudaSuccess) e = cudaMemcpy(n->b[l], params + off + nw, sizeof(float) * nb, cudaMemcpyHostToDevice);
        if (e == cudaSuccess) e = cudaMemset(n->mw[l], 0, sizeof(float) * nw);
        if (e == cudaSuccess) e = cudaMemset(n->vw[l], 0, sizeof(float) * nw);
        if (e == cudaSuccess) e = cudaMemset(n->mb[l], 0, sizeof(float) * nb);
        if (e == cudaSuccess) e = cudaMemset(n->vb[l], 0, sizeof(float) * nb);
        off += nw + nb;
    }
    n->step = 0;
    if (e == cudaSuccess) e = refresh_operands(n, false, 0.f, nullptr);
    if (e == cudaSuccess) e = cudaDeviceSynchronize();
    if (e != cudaSuccess) {
        cudaGetLastError();
        return net_fail(n, GSR_ECUDA, std::string("set_params: ") + cudaGetErrorString(e));
    }
    return GSR_OK;
}

GSR_API gsr_status gsr_net_get_params(gsr_net *n, float *params, int64_t count)
{
    if (!n || !params) return GSR_EINVAL;
    if (count != total_params()) return net_fail(n, GSR_EINVAL, "parameter count mismatch");
    cudaError_t e = cudaSetDevice(n->device);
    if (e == cudaSuccess) e = cudaDeviceSynchronize();
    int64_t off = 0;
    for (int l = 0; l < NLAYER && e == cudaSuccess; ++l) {
        const int64_t nw = layer_wsize(l), nb = CH(l + 1);
        e = cudaMemcpy(params + off, n->w[l], sizeof(float) * nw, cudaMemcpyDeviceToHost);
        if (e == cudaSuccess) e = cudaMemcpy(params + off + nw, n->b[l], sizeof(float) * nb, cudaMemcpyDeviceToHost);
        off += nw + nb;
    }
    if (e != cudaSuccess) {
        cudaGetLastError();
        return net_fail(n, GSR_ECUDA, std::string("get_params: ") + cudaGetErrorString(e));
    }
    return GSR_OK;
}

GSR_API gsr_status gsr_net_forward(gsr_net *n, const float *in, int64_t batch, int64_t len, float *out, void *stream)
{
    if (!n || !in || !out || batch < 1 || len < 1) return GSR_EINVAL;
    if (const gsr_status f = net_fault_status(n); f != GSR_OK) return f;
    cudaError_t e = cudaSetDevice(n->device);
    if (e == cudaSuccess) e = net_forward_dev(n, in, batch, len, out, (cudaStream_t)stream);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return net_fail(n, e == cudaErrorMemoryAllocation ? GSR_ENOMEM : GSR_ECUDA,
                        std::string("forward: ") + cudaGetErrorString(e));
    }
    return GSR_OK;
}

GSR_API gsr_status gsr_net_train_step(gsr_net *n, const float *in, const float *target, int64_t batch, int64_t len,
                                      float lr, double *loss, void *stream)
{
    if (!n || !in || !target || batch < 1 || len < 1 || !(lr >= 0.f)) return GSR_EINVAL;
    if (const gsr_status f = net_fault_status(n); f != GSR_OK) return f;
    cudaError_t e = cudaSetDevice(n->device);
    if (e == cudaSuccess) e = net_train_dev(n, in, target, batch, len, lr, loss, (cudaStream_t)stream);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return net_fail(n, e == cudaErrorMemoryAllocation ? GSR_ENOMEM : GSR_ECUDA,
                        std::string("train_step: ") + cudaGetErrorString(e));
    }
    return GSR_OK;
}

// gradients of the last train step are consumed by Adam; this returns the
// gradients of one batch without updating (for checks): fp32, same layout as
// the parameters. Adam state and step count are left unchanged.
GSR_API gsr_status gsr_net_gradients(gsr_net *n, const float *in, const float *target, int64_t batch, int64_t len,
                                     float *grads, int64_t count, double *loss, void *stream)
{
    if (!n || !in || !target || !grads || batch < 1 || len < 1) return GSR_EINVAL;
    if (const gsr_status f = net_fault_status(n); f != GSR_OK) return f;
    if (count != total_params()) return net_fail(n, GSR_EINVAL, "parameter count mismatch");
    cudaStream_t s = (cudaStream_t)stream;
    cudaError_t e = cudaSetDevice(n->device);
    if (e == cudaSuccess) e = net_reserve(n, batch * len);
    const int64_t P = batch * len;
    if (e == cudaSuccess) {
        k_pack_input<<<grid_n(P * CHP(0)), 256, 0, s>>>(in, P, n->act[0]);
        e = net_forward_packed(n, batch, len, s);
    }
    if (e == cudaSuccess) e = cudaMemsetAsync(n->loss, 0, sizeof(double), s);
    if (e == cudaSuccess) {
        k_mse<<<grid_n(P * CHP(NLAYER)), 256, 0, s>>>(n->y8, target, P, n->d32, n->d16a, n->loss);
        __nv_bfloat16 *dcur = n->d16a, *dnext = n->d16b;
        for (int l = NLAYER - 1; l >= 0 && e == cudaSuccess; --l) {
            backward_layer(n, l, dcur, dnext, batch, len, s);
            if (l > 0) std::swap(dcur, dnext);
            e = cudaGetLastError();
        }
    }
    // copy out (padded dW -> true layout on the host) and clear the accumulators
    int64_t off = 0;
    for (int l = 0; l < NLAYER && e == cudaSuccess; ++l) {
        const int cin = CH(l), cout = CH(l + 1), cinp = CHP(l);
        std::vector<float> dWp((size_t)CHP(l + 1) * KW * cinp), dbv((size_t)cout);
        e = cudaMemcpyAsync(dWp.data(), n->dW[l], sizeof(float) * dWp.size(), cudaMemcpyDeviceToHost, s);
        if (e == cudaSuccess) e = cudaMemcpyAsync(dbv.data(), n->db[l], sizeof(float) * cout, cudaMemcpyDeviceToHost, s);
        if (e == cudaSuccess) e = cudaStreamSynchronize(s);
        if (e != cudaSuccess) break;
        for (int co = 0; co < cout; ++co)
            for (int ci = 0; ci < cin; ++ci)
                for (int t = 0; t < KW; ++t)
                    grads[off + ((int64_t)co * cin + ci) * KW + t] = dWp[(size_t)co * KW * cinp + t * cinp + ci];
        for (int co = 0; co < cout; ++co) grads[off + layer_wsize(l) + co] = dbv[(size_t)co];
        off += layer_wsize(l) + cout;
        e = cudaMemsetAsync(n->dW[l], 0, sizeof(float) * dWp.size(), s);
        if (e == cudaSuccess) e = cudaMemsetAsync(n->db[l], 0, sizeof(float) * cout, s);
    }
    if (e == cudaSuccess && loss) e = cudaMemcpyAsync(loss, n->loss, sizeof(double), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return net_fail(n, GSR_ECUDA, std::string("gradients: ") + cudaGetErrorString(e));
    }
    return net_fault_status(n);  // this call's own convolutions have finished
}

GSR_API gsr_status gsr_net_layer_forward(gsr_net *n, int32_t layer, const float *in, int64_t batch, int64_t len,
                                         float *out, void *stream)
{
    if (!n || !in || !out || batch < 1 || len < 1 || layer < 0 || layer >= NLAYER) return GSR_EINVAL;
    if (const gsr_status f = net_fault_status(n); f != GSR_OK) return f;
    const cudaStream_t s = (cudaStream_t)stream;
    cudaError_t e = cudaSetDevice(n->device);
    if (e == cudaSuccess) e = net_reserve(n, batch * len);
    if (e == cudaSuccess) {
        if (layer == 0)
            e = layer_fwd_t<16, 64>(n, layer, in, batch, len, out, s);
        else if (layer == NLAYER - 1)
            e = layer_fwd_t<64, 16>(n, layer, in, batch, len, out, s);
        else
            e = layer_fwd_t<64, 64>(n, layer, in, batch, len, out, s);
    }
    if (e != cudaSuccess) {
        cudaGetLastError();
        return net_fail(n, e == cudaErrorMemoryAllocation ? GSR_ENOMEM : GSR_ECUDA,
                        std::string("layer_forward: ") + cudaGetErrorString(e));
    }
    return GSR_OK;
}

GSR_API gsr_status gsr_net_layer_backward(gsr_net *n, int32_t layer, const float *in, const float *dout, int64_t batch,
                                          int64_t len, float *din, float *dW, float *db, void *stream)
{
    if (!n || !in || !dout || !dW || !db || batch < 1 || len < 1 || layer < 0 || layer >= NLAYER) return GSR_EINVAL;
    if (const gsr_status f = net_fault_status(n); f != GSR_OK) return f;
    const cudaStream_t s = (cudaStream_t)stream;
    cudaError_t e = cudaSetDevice(n->device);
    if (e == cudaSuccess) e = net_reserve(n, batch * len);
    if (e == cudaSuccess) {
        if (layer == 0)
            e = layer_bwd_t<16, 64>(n, layer, in, dout, batch, len, din, dW, db, s);
        else if (layer == NLAYER - 1)
            e = layer_bwd_t<64, 16>(n, layer, in, dout, batch, len, din, dW, db, s);
        else
            e = layer_bwd_t<64, 64>(n, layer, in, dout, batch, len, din, dW, db, s);
    }
    if (e != cudaSuccess) {
        cudaGetLastError();
        return net_fail(n, e == cudaErrorMemoryAllocation ? GSR_ENOMEM : GSR_ECUDA,
                        std::string("layer_backward: ") + cudaGetErrorString(e));
    }
    return GSR_OK;
}

GSR_API gsr_status gsr_net_apply_gradients(gsr_net *n, const float *grads, int64_t count, float lr, void *stream)
{
    if (!n || !grads || !(lr >= 0.f)) return GSR_EINVAL;
    if (count != total_params()) return net_fail(n, GSR_EINVAL, "parameter count mismatch");
    const cudaStream_t s = (cudaStream_t)stream;
    cudaError_t e = cudaSetDevice(n->device);
    // host layout [cout][cin][5] + bias -> the padded accumulators the Adam kernel reads
    int64_t off = 0;
    for (int l = 0; l < NLAYER && e == cudaSuccess; ++l) {
        const int cin = CH(l), cout = CH(l + 1), cinp = CHP(l);
        std::vector<float> dWp((size_t)CHP(l + 1) * KW * cinp, 0.f);
        for (int co = 0; co < cout; ++co)
            for (int ci = 0; ci < cin; ++ci)
                for (int t = 0; t < KW; ++t)
                    dWp[(size_t)co * KW * cinp + t * cinp + ci] = grads[off + ((int64_t)co * cin + ci) * KW + t];
        e = cudaMemcpy(n->dW[l], dWp.data(), sizeof(float) * dWp.size(), cudaMemcpyHostToDevice);
        if (e == cudaSuccess)
            e = cudaMemcpy(n->db[l], grads + off + layer_wsize(l), sizeof(float) * cout, cudaMemcpyHostToDevice);
        off += layer_wsize(l) + cout;
    }
    if (e == cudaSuccess) {
        n->step += 1;
        e = refresh_operands(n, true, lr, s);
    }
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return net_fail(n, GSR_ECUDA, std::string("apply_gradients: ") + cudaGetErrorString(e));
    }
    return GSR_OK;
}

GSR_API gsr_status gsr_net_save(gsr_net *n, const char *path)
{
    if (!n || !path) return GSR_EINVAL;
    std::vector<float> p((size_t)total_params());
    gsr_status st = gsr_net_get_params(n, p.data(), (int64_t)p.size());
    if (st != GSR_OK) return st;
    FILE *f = fopen(path, "wb");
    if (!f) return net_fail(n, GSR_EINVAL, std::string("cannot write ") + path);
    const char magic[8] = {'G', 'S', 'R', 'N', 'E', 'T', '0', '1'};
    const int64_t cnt = (int64_t)p.size();
    const bool ok = fwrite(magic, 1, 8, f) == 8 && fwrite(&cnt, sizeof(cnt), 1, f) == 1 &&
                    fwrite(p.data(), sizeof(float), p.size(), f) == p.size();
    fclose(f);
    return ok ? GSR_OK : net_fail(n, GSR_EINVAL, std::string("short write ") + path);
}

GSR_API gsr_status gsr_net_load(gsr_net *n, const char *path)
{
    if (!n || !path) return GSR_EINVAL;
    FILE *f = fopen(path, "rb");
    if (!f) return net_fail(n, GSR_EINVAL, std::string("cannot read ") + path);
    char magic[8];
    int64_t cnt = 0;
    std::vector<float> p((size_t)total_params());
    const bool ok = fread(magic, 1, 8, f) == 8 && memcmp(magic, "GSRNET01", 8) == 0 &&
                    fread(&cnt, sizeof(cnt), 1, f) == 1 && cnt == (int64_t)p.size() &&
                    fread(p.data(), sizeof(float), p.size(), f) == p.size();
    fclose(f);
    if (!ok) return net_fail(n, GSR_EINVAL, std::string("not a weights file of this network: ") + path);
    return gsr_net_set_params(n, p.data(), cnt);
}
