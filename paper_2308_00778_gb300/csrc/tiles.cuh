// tiles.cuh -- the tiled row layout of the coefficient matrix and its device accessors.
//
// Rows are stored in tiles of T = 32*R consecutive rows (R = 16 / sizeof(value):
// 4 rows per lane for binary32, 2 for binary64). One tile is one contiguous
// record of 31 planes:
//   24 value planes   (T values each = 512 bytes)   slots: 0-4 astro, 5-16 attitude, 17-22 instr, 23 global
//    1 knot plane     (T int32)
//    6 instr planes   (T instrumental indices in [0, n_instr): 16-bit when n_instr <= 65536,
//                      else 32-bit; SysView::iw16 says which, SysView::tile_bytes the record size)
// A section variant (Sec. 2: n_astro 0..5, n_ipr 0..6, n_glob 0..NGLOB_MAX)
// stores only its planes: n_astro + 12 + n_ipr + n_glob value planes in that
// order, the knot plane, n_ipr instrumental planes (Sec<true> below).
// Lane l of a warp owns rows [l*R, l*R + R) of a tile and reads each value plane
// with one 16-byte load, so a warp reads a tile as one contiguous block and
// warps working on consecutive tiles stream consecutive memory (measured:
// 7.1 TB/s for a pure 31-plane tile stream vs 5.0-5.4 TB/s for 32-row warp
// steps scattered one star apart).
//
// The knot-ordered attitude copy (layout.cu) uses the same scheme with 13
// planes per tile: 12 attitude value planes and the row permutation.
#pragma once

#include "gsr_internal.cuh"

namespace gsr {

// Ask L2 to fetch bytes at p (16-byte aligned, a multiple of 16 bytes) ahead of their use: one bulk
// prefetch by the warp's lane 0, nothing returned and nothing to wait for.
__device__ __forceinline__ void prefetch_l2(const void *p, int64_t bytes)
{
    if ((threadIdx.x & 31) == 0) asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(p), "r"((uint32_t)bytes));
}

// One 32-byte read-only load (p 32-byte aligned): two consecutive float4 in one request, where two
// 16-byte loads of the same sector would make two.
__device__ __forceinline__ void ldg_v8(const float4 *p, float4 &a, float4 &b)
{
    asm("ld.global.nc.v8.f32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];"
        : "=f"(a.x), "=f"(a.y), "=f"(a.z), "=f"(a.w), "=f"(b.x), "=f"(b.y), "=f"(b.z), "=f"(b.w)
        : "l"(p));
}

// A row's three attitude windows from the knot-major window copy (64 bytes per knot: axes 0 and 1 in
// one 32-byte load, axis 2 in a 16-byte one: two requests instead of three)
__device__ __forceinline__ void att_window_load(const float4 *__restrict__ xw, int32_t k, float4 (&w)[3])
{
    ldg_v8(xw + 4 * (int64_t)k, w[0], w[1]);
    w[2] = __ldg(xw + 4 * (int64_t)k + 2);
}

template <typename VT>
struct Tile {
    static constexpr int R = 16 / (int)sizeof(VT);                   // rows per lane
    static constexpr int T = 32 * R;                                  // rows per tile
    static constexpr int64_t VBLK = (int64_t)T * sizeof(VT);          // 512 bytes
    static constexpr int64_t IBLK = (int64_t)T * sizeof(int32_t);     // int32 plane
    static constexpr int64_t ABYTES = NAXES * NPARAXIS * VBLK + IBLK;  // knot-ordered attitude tile
    // bytes of a star-ordered tile record with 16- or 32-bit instrumental planes
    static constexpr int64_t bytes(bool iw16) { return bytes(NPAR, NINSTR, iw16); }
    // ... with npl value planes and ni instrumental planes (a section variant)
    static constexpr int64_t bytes(int npl, int ni, bool iw16)
    {
        return npl * VBLK + IBLK + (int64_t)ni * T * (iw16 ? 2 : 4);
    }
};

// Section geometry of a tile record. SV = false: the paper's standard row,
// compile-time constants (the code every standard system runs). SV = true: a
// section variant, read from the view at run time; MAXG register slots hold
// its global coefficients. Kernels keep a row's coefficients in register slots
// of the standard row (A_ATT, A_INS, A_GLOB) and load them from planes
// p_att / p_ins / p_glob.
template <bool SV>
struct Sec {
    static constexpr int MAXG = SV ? NGLOB_MAX : 1;
    int na, ni, ng, p_att, p_ins, p_glob, npl;
    template <typename VT>
    __device__ __forceinline__ explicit Sec(const SysView<VT> &S)
        : na(SV ? S.na : NASTRO), ni(SV ? S.ni : NINSTR), ng(S.n_glob), p_att(SV ? S.p_att : A_ATT),
          p_ins(SV ? S.p_ins : A_INS), p_glob(SV ? S.p_glob : A_GLOB), npl(SV ? S.npl : NPAR)
    {
    }
};

template <typename VT>
struct Vec16;
template <>
struct Vec16<float> {
    using type = float4;
    __device__ static __forceinline__ void unpack(const float4 &v, float (&o)[4])
    {
        o[0] = v.x;
        o[1] = v.y;
        o[2] = v.z;
        o[3] = v.w;
    }
};
template <>
struct Vec16<double> {
    using type = double2;
    __device__ static __forceinline__ void unpack(const double2 &v, double (&o)[2])
    {
        o[0] = v.x;
        o[1] = v.y;
    }
};

// value plane j of tile t, this lane's R rows, converted to AT
template <typename VT, typename AT>
__device__ __forceinline__ void load_vals(const uint8_t *__restrict__ tile, int j, AT (&out)[Tile<VT>::R])
{
    using V = typename Vec16<VT>::type;
    const V *p = reinterpret_cast<const V *>(tile + (int64_t)j * Tile<VT>::VBLK) + (threadIdx.x & 31);
    VT v[Tile<VT>::R];
    Vec16<VT>::unpack(__ldcs(p), v);
#pragma unroll
    for (int i = 0; i < Tile<VT>::R; ++i) out[i] = (AT)v[i];
}

// int32 plane q of a tile whose int planes start at `ints`, this lane's R entries
template <int R>
__device__ __forceinline__ void load_ints(const uint8_t *__restrict__ ints, int q, int32_t (&out)[R])
{
    const int lane = threadIdx.x & 31;
    if constexpr (R == 4) {
        const int4 v = __ldcs(reinterpret_cast<const int4 *>(ints + (int64_t)q * 32 * R * 4) + lane);
        out[0] = v.x;
        out[1] = v.y;
        out[2] = v.z;
        out[3] = v.w;
    } else {
        const int2 v = __ldcs(reinterpret_cast<const int2 *>(ints + (int64_t)q * 32 * R * 4) + lane);
        out[0] = v.x;
        out[1] = v.y;
    }
}

// instrumental-column plane j (0..5) of the tile record at tb (npl value planes), this lane's R entries
template <typename VT>
__device__ __forceinline__ void load_instr(const uint8_t *__restrict__ tb, int npl, bool iw16, int j,
                                           int32_t (&out)[Tile<VT>::R])
{
    constexpr int R = Tile<VT>::R;
    constexpr int T = Tile<VT>::T;
    const int lane = threadIdx.x & 31;
    const uint8_t *p = tb + (int64_t)npl * Tile<VT>::VBLK + Tile<VT>::IBLK;  // the first instrumental plane
    if (iw16) {
        p += (int64_t)j * T * 2;
        if constexpr (R == 4) {
            const uint2 v = __ldcs(reinterpret_cast<const uint2 *>(p) + lane);
            out[0] = (int32_t)(v.x & 0xffffu);
            out[1] = (int32_t)(v.x >> 16);
            out[2] = (int32_t)(v.y & 0xffffu);
            out[3] = (int32_t)(v.y >> 16);
        } else {
            const uint32_t v = __ldcs(reinterpret_cast<const uint32_t *>(p) + lane);
            out[0] = (int32_t)(v & 0xffffu);
            out[1] = (int32_t)(v >> 16);
        }
    } else {
        load_ints<R>(p + (int64_t)j * T * 4, 0, out);
    }
}

// For the run-time geometry of a section variant: instrumental plane j when j < ni, else a
// same-width read of the record's knot plane (always present), so that the load is
// unconditional and can be scheduled with the others; the caller masks what an absent plane
// would gather.
template <typename VT>
__device__ __forceinline__ void load_instr_or_knot(const uint8_t *__restrict__ tb, int npl, int ni, bool iw16, int j,
                                                   int32_t (&out)[Tile<VT>::R])
{
    constexpr int R = Tile<VT>::R;
    constexpr int T = Tile<VT>::T;
    const int lane = threadIdx.x & 31;
    const uint8_t *knot = tb + (int64_t)npl * Tile<VT>::VBLK;
    const uint8_t *p = j < ni ? knot + Tile<VT>::IBLK + (int64_t)j * T * (iw16 ? 2 : 4) : knot;
    if (iw16) {
        if constexpr (R == 4) {
            const uint2 v = __ldcs(reinterpret_cast<const uint2 *>(p) + lane);
            out[0] = (int32_t)(v.x & 0xffffu);
            out[1] = (int32_t)(v.x >> 16);
            out[2] = (int32_t)(v.y & 0xffffu);
            out[3] = (int32_t)(v.y >> 16);
        } else {
            const uint32_t v = __ldcs(reinterpret_cast<const uint32_t *>(p) + lane);
            out[0] = (int32_t)(v & 0xffffu);
            out[1] = (int32_t)(v >> 16);
        }
    } else {
        load_ints<R>(p, 0, out);
    }
}

// the same for the standard row's 24 value planes
template <typename VT>
__device__ __forceinline__ void load_instr(const uint8_t *__restrict__ tb, bool iw16, int j,
                                           int32_t (&out)[Tile<VT>::R])
{
    load_instr<VT>(tb, NPAR, iw16, j, out);
}

// write instrumental index v of row i (0..T-1) into plane j of the tile record at tb (npl value planes)
template <typename VT>
__device__ __forceinline__ void store_instr(uint8_t *__restrict__ tb, int npl, bool iw16, int j, int i, int32_t v)
{
    constexpr int T = Tile<VT>::T;
    uint8_t *p = tb + (int64_t)npl * Tile<VT>::VBLK + Tile<VT>::IBLK;
    if (iw16)
        reinterpret_cast<uint16_t *>(p + (int64_t)j * T * 2)[i] = (uint16_t)v;
    else
        reinterpret_cast<int32_t *>(p + (int64_t)j * T * 4)[i] = v;
}

// The star of row r of tile t: the largest s in [first_star[t], first_star[t+1]]
// with star_ptr[s] <= r (rows past the end map to the last star of the range).
__device__ __forceinline__ int64_t star_of_row(const int64_t *__restrict__ star_ptr,
                                               const int32_t *__restrict__ first_star, int64_t t, int64_t r)
{
    int64_t lo = first_star[t], hi = first_star[t + 1];
    while (lo < hi) {
        const int64_t mid = (lo + hi + 1) >> 1;
        if (__ldg(star_ptr + mid) <= r)
            lo = mid;
        else
            hi = mid - 1;
    }
    return lo;
}

// stars of this lane's R consecutive rows starting at r0
template <int R>
__device__ __forceinline__ void stars_of_rows(const int64_t *__restrict__ star_ptr,
                                              const int32_t *__restrict__ first_star, int64_t t, int64_t r0,
                                              int64_t (&s)[R])
{
    const int64_t hi = first_star[t + 1];
    int64_t c = star_of_row(star_ptr, first_star, t, r0);
    s[0] = c;
#pragma unroll
    for (int i = 1; i < R; ++i) {
        while (c < hi && __ldg(star_ptr + c + 1) <= r0 + i) ++c;
        s[i] = c;
    }
}

}  // namespace gsr
