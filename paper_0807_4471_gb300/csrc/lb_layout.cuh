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
template <int P> struct Prec;
template <> struct Prec<LB_FP64> {
    typedef double T; typedef double C;
    static constexpr int GX = 4, TX = 32, TY = 8;
};
template <> struct Prec<LB_FP32> {
    typedef float T; typedef float C;
    static constexpr int GX = 4, TX = 64, TY = 8;
};
template <> struct Prec<LB_FP16_OFFSET> {
    typedef __half T; typedef float C;
    static constexpr int GX = 8, TX = 64, TY = 8;
};
template <> struct Prec<LB_BF16_OFFSET> {
    typedef __nv_bfloat16 T; typedef float C;
    static constexpr int GX = 8, TX = 64, TY = 8;
};

// Stored values are offsets h_i = f_i - w_i rho_ref from the lattice weights
// (all precisions).  The codecs only convert between storage and compute type.
__device__ __forceinline__ double dec(double v) { return v; }
__device__ __forceinline__ float dec(float v) { return v; }
__device__ __forceinline__ float dec(__half v) { return __half2float(v); }
__device__ __forceinline__ float dec(__nv_bfloat16 v) { return __bfloat162float(v); }

template <typename T> __device__ __forceinline__ T encf(double v);
template <> __device__ __forceinline__ double encf<double>(double v) { return v; }
template <typename T> __device__ __forceinline__ T encf(float v);
template <> __device__ __forceinline__ float encf<float>(float v) { return v; }
template <> __device__ __forceinline__ __half encf<__half>(float v) { return __float2half_rn(v); }
template <> __device__ __forceinline__ __nv_bfloat16 encf<__nv_bfloat16>(float v) {
    return __float2bfloat16_rn(v);
}
// Encoding of an offset computed in double (initialisation).
template <typename T> __device__ __forceinline__ T encd(double v);
template <> __device__ __forceinline__ double encd<double>(double v) { return v; }
template <> __device__ __forceinline__ float encd<float>(double v) { return (float)v; }
template <> __device__ __forceinline__ __half encd<__half>(double v) { return __double2half(v); }
template <> __device__ __forceinline__ __nv_bfloat16 encd<__nv_bfloat16>(double v) {
    return __double2bfloat16(v);
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
    typedef typename Prec<P>::C C;
    static constexpr int TX = Prec<P>::TX, TY = Prec<P>::TY, NT = TX * TY;   // one site per thread
    static constexpr int GX = Prec<P>::GX;
    static constexpr int BX = TX + 2 * GX;            // box columns
    static constexpr int BY = TY + 2 * kGY;           // box rows
    static constexpr int SPEC = 9 * BX * BY;          // elements per species box
    static constexpr int SPEC_BYTES = SPEC * (int)sizeof(T);
    static constexpr int SPEC_STRIDE = (SPEC_BYTES + 127) / 128 * 128;
    static constexpr int RX = TX + 4, RY = TY + 4;    // rho/Psi tile (2-cell halo)
    static constexpr int RHOPSI = (4 * RX * RY * (int)sizeof(C) + 127) / 128 * 128;
    static constexpr int STAGE_SPEC = 9 * TY * TX * (int)sizeof(T);  // output tile, one species
    static constexpr int STAGE_OFF = 4 * SPEC_STRIDE + RHOPSI;
    static constexpr int SMEM = STAGE_OFF + 2 * STAGE_SPEC + 128;     // step: 2 boxes + staging
    static constexpr int SMEM_OBS = 2 * SPEC_STRIDE + RHOPSI + 128;   // observe: 1 box
    static_assert(STAGE_SPEC % 128 == 0, "staging alignment");
    static_assert((BX * sizeof(T)) % 16 == 0, "TMA box rows must be 16-byte multiples");
    static_assert(GX >= 3 && (GX * sizeof(T)) % 16 == 0, "ghost width");
    static_assert(SMEM <= 227 * 1024, "shared memory");
};

}  // namespace lbgb
