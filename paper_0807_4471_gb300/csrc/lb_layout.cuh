// lb_layout.cuh -- lattice constants, storage formats and the shared-memory
// layout of the step kernels; included by the kernels and by the host code
// that sizes launches.
#pragma once

#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include "lb_internal.h"

namespace lbgb {

// ------------------------------------------------------------- lattice
// D2Q9 order: rest, +x, +y, -x, -y, (+1,+1), (-1,+1), (-1,-1), (+1,-1).
__host__ __device__ constexpr int cx(int i) {
    return (i == 1 || i == 5 || i == 8) ? 1 : ((i == 3 || i == 6 || i == 7) ? -1 : 0);
}
__host__ __device__ constexpr int cy(int i) {
    return (i == 2 || i == 5 || i == 6) ? 1 : ((i == 4 || i == 7 || i == 8) ? -1 : 0);
}
__host__ __device__ constexpr int opp(int i) {
    return i == 0 ? 0 : (i <= 4 ? ((i + 1) % 4) + 1 : ((i - 3) % 4) + 5);
}
template <typename C>
__device__ __forceinline__ C wgt(int i) {
    return i == 0 ? C(4) / C(9) : (i <= 4 ? C(1) / C(9) : C(1) / C(36));
}
// One representative d of each +-d pair of the 24-neighbour stencil; the
// first four are the first belt (also the pairs of the cross term).
__host__ __device__ constexpr int rdx(int k) {
    return k == 0 ? 1 : k == 1 ? 0 : k == 2 ? 1 : k == 3 ? -1 : k == 4 ? 2 : k == 5 ? 0
         : k == 6 ? 2 : k == 7 ? 1 : k == 8 ? -1 : k == 9 ? -2 : k == 10 ? 2 : -2;
}
__host__ __device__ constexpr int rdy(int k) {
    return k == 0 ? 0 : k == 1 ? 1 : k == 2 ? 1 : k == 3 ? 1 : k == 4 ? 0 : k == 5 ? 2
         : k == 6 ? 1 : k == 7 ? 2 : k == 8 ? 2 : k == 9 ? 1 : k == 10 ? 2 : 2;
}

// ------------------------------------------------------- storage formats
// In HBM and in shared memory the two species of one direction are stored
// as an interleaved pair (A, B), so that one vector access serves both.
// T: stored scalar, T2: stored pair, C: compute scalar, C2: compute pair.
template <int P> struct Prec;
// TX: tile width, chosen so that a deviation row with its 2-cell halo,
// TX + 4, is a multiple of 32 (one cell per thread); NB: ring slots of
// 8-row population blocks in the step kernel.
template <> struct Prec<LB_FP64> {
    typedef double T; typedef double2 T2; typedef double C; typedef double2 C2;
    static constexpr int GX = 4, TX = 28, TY = 8, NB = 3;
};
template <> struct Prec<LB_FP32> {
    typedef float T; typedef float2 T2; typedef float C; typedef float2 C2;
    static constexpr int GX = 4, TX = 60, TY = 8, NB = 4;
};
template <> struct Prec<LB_FP16_OFFSET> {
    typedef __half T; typedef __half2 T2; typedef float C; typedef float2 C2;
    static constexpr int GX = 8, TX = 60, TY = 8, NB = 4;
};
template <> struct Prec<LB_BF16_OFFSET> {
    typedef __nv_bfloat16 T; typedef __nv_bfloat162 T2; typedef float C; typedef float2 C2;
    static constexpr int GX = 8, TX = 60, TY = 8, NB = 4;
};

// Stored values are offsets h_i = f_i - w_i rho_ref from the lattice weights
// (all precisions).  The codecs only convert between storage and compute type.
__device__ __forceinline__ double2 dec2(double2 v) { return v; }
__device__ __forceinline__ float2 dec2(float2 v) { return v; }
__device__ __forceinline__ float2 dec2(__half2 v) { return __half22float2(v); }
__device__ __forceinline__ float2 dec2(__nv_bfloat162 v) { return __bfloat1622float2(v); }

template <typename T2, typename C> __device__ __forceinline__ T2 enc2(C a, C b);
template <> __device__ __forceinline__ double2 enc2<double2, double>(double a, double b) {
    return make_double2(a, b);
}
template <> __device__ __forceinline__ float2 enc2<float2, float>(float a, float b) {
    return make_float2(a, b);
}
template <> __device__ __forceinline__ __half2 enc2<__half2, float>(float a, float b) {
    return __floats2half2_rn(a, b);
}
template <> __device__ __forceinline__ __nv_bfloat162 enc2<__nv_bfloat162, float>(float a, float b) {
    return __floats2bfloat162_rn(a, b);
}
// Encoding of offsets computed in double (initialisation).
template <typename T2> __device__ __forceinline__ T2 encd2(double a, double b);
template <> __device__ __forceinline__ double2 encd2<double2>(double a, double b) {
    return make_double2(a, b);
}
template <> __device__ __forceinline__ float2 encd2<float2>(double a, double b) {
    return make_float2((float)a, (float)b);
}
template <> __device__ __forceinline__ __half2 encd2<__half2>(double a, double b) {
    return __halves2half2(__double2half(a), __double2half(b));
}
template <> __device__ __forceinline__ __nv_bfloat162 encd2<__nv_bfloat162>(double a, double b) {
    return __halves2bfloat162(__double2bfloat16(a), __double2bfloat16(b));
}

// Correctly rounded reciprocal (no division slow path in FP32).
__device__ __forceinline__ double recip(double v) { return 1.0 / v; }
__device__ __forceinline__ float recip(float v) { return __frcp_rn(v); }

__device__ __forceinline__ double cexpm1(double v) { return expm1(v); }
__device__ __forceinline__ float cexpm1(float v) { return expm1f(v); }
__device__ __forceinline__ double csin(double v) { return sin(v); }
__device__ __forceinline__ float csin(float v) { return sinf(v); }

template <int P>
struct Layout {
    typedef typename Prec<P>::T T;
    typedef typename Prec<P>::T2 T2;
    typedef typename Prec<P>::C C;
    typedef typename Prec<P>::C2 C2;
    static constexpr int TX = Prec<P>::TX, TY = Prec<P>::TY;
    static constexpr int GX = Prec<P>::GX;
    static constexpr int BX = TX + 2 * GX;            // box columns (sites)
    static constexpr int BY = TY + 2 * kGY;           // observe box rows
    static constexpr int RX = TX + 4, RY = TY + 4;    // rho/Psi tile (2-cell halo)
    // threads: one per deviation cell of a tile's 8 new rows; in the site
    // phase thread (lx, ly) = (tid % RX, tid / RX) updates site lx < TX
    static constexpr int NT = RX * TY;
    static constexpr int TYB = 8;                     // rows of a step-kernel block
    static constexpr int NB = Prec<P>::NB;            // ring slots of blocks
    static constexpr int RING = 16;                   // rho/Psi ring rows (>= TY + 4 + TY/2)
    // step kernel: NB block slots, the rho and Psi rings, the staging tile
    static constexpr int SLOT_BYTES = 9 * TYB * BX * (int)sizeof(T2);
    static constexpr int RING_OFF = NB * SLOT_BYTES;
    static constexpr int RING_BYTES = 2 * RING * RX * (int)sizeof(C2);
    static constexpr int STAGE_OFF = RING_OFF + RING_BYTES;
    static constexpr int STAGE_BYTES = 9 * TY * TX * (int)sizeof(T2);
    static constexpr int SMEM = STAGE_OFF + STAGE_BYTES + 128;
    // observe kernel: one tile box and the rho/Psi tile
    static constexpr int BOX_BYTES = 9 * BY * BX * (int)sizeof(T2);
    static constexpr int BOX_STRIDE = (BOX_BYTES + 127) / 128 * 128;
    static constexpr int RHOPSI = (2 * RX * RY * (int)sizeof(C2) + 127) / 128 * 128;
    static constexpr int SMEM_OBS = BOX_STRIDE + RHOPSI + 128;
    static_assert(TY == TYB, "a tile spans one block plus the halo of the next");
    static_assert(RX % 32 == 0, "deviation rows are whole warps");
    static_assert((2 * TX * sizeof(T)) % 16 == 0 && (2 * (TX + GX) * sizeof(T)) % 16 == 0,
                  "TMA x coordinates of tiles stay 16-byte aligned");
    static_assert(SLOT_BYTES % 128 == 0 && RING_BYTES % 128 == 0 && STAGE_BYTES % 128 == 0,
                  "128-byte alignment of the shared-memory regions");
    static_assert((BX * sizeof(T2)) % 16 == 0, "TMA box rows must be 16-byte multiples");
    static_assert(2 * BX <= 256 && 2 * TX <= 256 && BY <= 256, "TMA box extent");
    static_assert(GX >= 3 && (GX * sizeof(T)) % 16 == 0, "ghost width");
    static_assert(SMEM <= 227 * 1024 - 1024 && SMEM_OBS <= 227 * 1024, "shared memory");
};

}  // namespace lbgb
