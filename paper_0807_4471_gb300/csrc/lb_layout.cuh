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
// ------------------------------------------------------- storage formats
// In HBM and in shared memory the two species of one direction are stored
// as an interleaved pair (A, B), so that one vector access serves both.
// T: stored scalar, T2: stored pair, C: compute scalar, C2: compute pair.
template <int P> struct Prec;
// TX: tile width, chosen so that a deviation row with its 2-cell halo,
// TX + 4, is a multiple of 32 (one cell per thread); NB: ring slots of
// 8-row population blocks in the step kernel with 8-row tiles, NB2 with
// 16-row tiles (0: no 16-row tile for this precision).  SCALE_LOG2: the
// stored value is the offset times 2^SCALE_LOG2 (FP16: 2^10, which keeps
// offsets down to 2^-24 in binary16's normal range, where rounding has its
// full 11 bits; the largest storable offset becomes 64).
template <> struct Prec<LB_FP64> {
    typedef double T; typedef double2 T2; typedef double C; typedef double2 C2;
    static constexpr int GX = 4, TX = 28, TY = 8, NB = 3, NB2 = 0, SCALE_LOG2 = 0;
};
template <> struct Prec<LB_FP32> {
    typedef float T; typedef float2 T2; typedef float C; typedef float2 C2;
    static constexpr int GX = 4, TX = 60, TY = 8, NB = 4, NB2 = 5, SCALE_LOG2 = 0;
};
template <> struct Prec<LB_FP16_OFFSET> {
    typedef __half T; typedef __half2 T2; typedef float C; typedef float2 C2;
    static constexpr int GX = 8, TX = 60, TY = 8, NB = 4, NB2 = 6, SCALE_LOG2 = 10;
};
template <> struct Prec<LB_BF16_OFFSET> {
    typedef __nv_bfloat16 T; typedef __nv_bfloat162 T2; typedef float C; typedef float2 C2;
    static constexpr int GX = 8, TX = 60, TY = 8, NB = 4, NB2 = 6, SCALE_LOG2 = 0;
};
// The storage scale of precision P and its inverse, in the compute type.
template <int P> __host__ __device__ constexpr typename Prec<P>::C scale_of() {
    return typename Prec<P>::C(1 << Prec<P>::SCALE_LOG2);
}
template <int P> __host__ __device__ constexpr typename Prec<P>::C inv_scale_of() {
    return typename Prec<P>::C(1) / typename Prec<P>::C(1 << Prec<P>::SCALE_LOG2);
}

// Stored values are offsets h_i = f_i - w_i rho_ref from the lattice weights
// (all precisions), times the storage scale of the precision.  The codecs
// only convert between storage and compute type; the kernels work on the
// scaled offsets and fold the scale into their constants.
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
// Stochastic rounding of an FP32 pair to a 16-bit format by the conversion
// instruction of sm_100 and later (cvt.rs), which rounds each value to one of
// its two neighbours with probability given by its distance to them, drawing
// on the 32 random bits r.
template <typename T2> __device__ __forceinline__ T2 enc2_sr(float2 v, uint32_t r);
template <> __device__ __forceinline__ __half2 enc2_sr<__half2>(float2 v, uint32_t r) {
    uint32_t d;
    asm("cvt.rs.f16x2.f32 %0, %1, %2, %3;" : "=r"(d) : "f"(v.y), "f"(v.x), "r"(r));   // high half = y
    return *reinterpret_cast<const __half2*>(&d);
}
template <> __device__ __forceinline__ __nv_bfloat162 enc2_sr<__nv_bfloat162>(float2 v, uint32_t r) {
    uint32_t d;
    asm("cvt.rs.bf16x2.f32 %0, %1, %2, %3;" : "=r"(d) : "f"(v.y), "f"(v.x), "r"(r));
    return *reinterpret_cast<const __nv_bfloat162*>(&d);
}

// 32-bit integer hash (the "lowbias32" finaliser of C. Wellons: two
// multiply-xorshift rounds).  The nine random words of a site are the
// site's hash times nine odd constants (a bijection each, so every word is
// uniform; only their mutual independence is approximate, which does not
// bias the rounding).
__device__ __forceinline__ uint32_t hash32(uint32_t x) {
    x ^= x >> 16;
    x *= 0x7feb352du;
    x ^= x >> 15;
    x *= 0x846ca68bu;
    x ^= x >> 16;
    return x;
}
__host__ __device__ constexpr uint32_t sr_mult(int i) {
    return i == 0 ? 0x9e3779b1u : i == 1 ? 0x85ebca77u : i == 2 ? 0xc2b2ae3du
         : i == 3 ? 0x27d4eb2fu : i == 4 ? 0x165667b1u : i == 5 ? 0xd3a2646du
         : i == 6 ? 0xfd7046c5u : i == 7 ? 0xb55a4f09u : 0x6a09e667u;
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

// Arithmetic on the (A, B) pair of a site.  FP32: the packed two-lane
// instructions of sm_100 and later (one instruction for both species, each
// lane rounded to nearest like the scalar operation); FP64: two scalar ones.
__device__ __forceinline__ float2 padd(float2 a, float2 b) { return __fadd2_rn(a, b); }
__device__ __forceinline__ float2 pmul(float2 a, float2 b) { return __fmul2_rn(a, b); }
__device__ __forceinline__ float2 pfma(float2 a, float2 b, float2 c) { return __ffma2_rn(a, b, c); }
__device__ __forceinline__ float2 psub(float2 a, float2 b) {
    unsigned long long d;
    asm("sub.rn.f32x2 %0, %1, %2;"
        : "=l"(d)
        : "l"(*reinterpret_cast<const unsigned long long*>(&a)),
          "l"(*reinterpret_cast<const unsigned long long*>(&b)));
    return *reinterpret_cast<const float2*>(&d);
}
__device__ __forceinline__ double2 padd(double2 a, double2 b) { return make_double2(a.x + b.x, a.y + b.y); }
__device__ __forceinline__ double2 psub(double2 a, double2 b) { return make_double2(a.x - b.x, a.y - b.y); }
__device__ __forceinline__ double2 pmul(double2 a, double2 b) { return make_double2(a.x * b.x, a.y * b.y); }
__device__ __forceinline__ double2 pfma(double2 a, double2 b, double2 c) {
    return make_double2(fma(a.x, b.x, c.x), fma(a.y, b.y, c.y));
}
__device__ __forceinline__ float2 pset(float v) { return make_float2(v, v); }
__device__ __forceinline__ double2 pset(double v) { return make_double2(v, v); }
__device__ __forceinline__ float2 pair(float a, float b) { return make_float2(a, b); }
__device__ __forceinline__ double2 pair(double a, double b) { return make_double2(a, b); }

// Reciprocal: correctly rounded in FP64; in FP32 the hardware approximation
// (rcp.approx.ftz, within 1 ulp), which has no slow path or branch.
__device__ __forceinline__ double recip(double v) { return 1.0 / v; }
__device__ __forceinline__ float recip(float v) {
    float r;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(v));
    return r;
}

// exp(x) - 1 of a pair.  FP64: the library function.  FP32: branch-free, by the
// Cody-Waite reduction x = k ln2 + r (|r| <= ln2 / 2, ln2 split into a
// 16-bit head and a tail so that k * head is exact) and
// expm1(x) = 2^k expm1(r) + (2^k - 1), with expm1(r) from its Taylor series
// through r^7 / 7! (truncation below 1.6e-8 relative on |r| <= ln2 / 2).
// Relative error about 2 ulp; a NaN argument gives NaN.  k is the integer
// nearest x / ln2, for x clamped to [-87, 88] (so that 2^k is a normal
// number, k in [-126, 127]): adding 1.5 2^23 to x log2(e) rounds it to an
// integer held in the low mantissa bits, which also give 2^k's exponent
// field by one shift.
__device__ __forceinline__ double2 pexpm1(double2 v) { return make_double2(expm1(v.x), expm1(v.y)); }
__device__ __forceinline__ float2 pexpm1(float2 x) {
    const float2 xc = make_float2(fminf(fmaxf(x.x, -87.0f), 88.0f), fminf(fmaxf(x.y, -87.0f), 88.0f));
    const float2 kt = pfma(xc, pset(1.44269504088896341f), pset(12582912.0f));
    const float2 k = padd(kt, pset(-12582912.0f));
    float2 r = pfma(k, pset(-0.693145751953125f), x);
    r = pfma(k, pset(-1.42860676533018700e-06f), r);
    float2 t = pset(1.0f / 5040.0f);
    t = pfma(t, r, pset(1.0f / 720.0f));
    t = pfma(t, r, pset(1.0f / 120.0f));
    t = pfma(t, r, pset(1.0f / 24.0f));
    t = pfma(t, r, pset(1.0f / 6.0f));
    t = pfma(t, r, pset(0.5f));
    t = pfma(t, r, pset(1.0f));
    const float2 p = pmul(t, r);
    // kt's bits are those of 1.5 2^23 plus k, and 1.5 2^23 << 23 vanishes
    // in 32 bits: (kt << 23) + (127 << 23) is the exponent field of 2^k
    const float2 s = make_float2(__uint_as_float((__float_as_uint(kt.x) << 23) + 0x3F800000u),
                                 __uint_as_float((__float_as_uint(kt.y) << 23) + 0x3F800000u));
    return pfma(s, p, padd(s, pset(-1.0f)));
}
__device__ __forceinline__ double csin(double v) { return sin(v); }
__device__ __forceinline__ float csin(float v) { return sinf(v); }

// Shared-memory layout and thread mapping of the step kernel for precision P
// and SPT sites per thread: SPT = 1, tiles of TX x 8 sites, one site per
// thread, leaving through a staging tile and a TMA bulk store; SPT = 2,
// tiles of TX x 16 sites, each thread updating two vertically adjacent
// sites (sharing their stencil rows) and storing them to global memory
// directly.  Both walk the same 8-row population blocks.
template <int P, int SPT = 1>
struct Layout {
    typedef typename Prec<P>::T T;
    typedef typename Prec<P>::T2 T2;
    typedef typename Prec<P>::C C;
    typedef typename Prec<P>::C2 C2;
    static constexpr int TX = Prec<P>::TX;
    static constexpr int TYB = Prec<P>::TY;           // rows of a population block (8)
    static constexpr int TY = TYB * SPT;              // tile rows
    static constexpr int GX = Prec<P>::GX;
    static constexpr int BX = TX + 2 * GX;            // box columns (sites)
    static constexpr int BY = TYB + 2 * kGY;          // observe box rows
    static constexpr int RX = TX + 4, RY = TYB + 4;   // rho/Psi tile (2-cell halo), observe
    // threads: one per deviation column and block row; in the site phase
    // thread (lx, j) = (tid % RX, tid / RX) updates sites (lx, SPT j + s), lx < TX
    static constexpr int NT = RX * TYB;
    static constexpr int NB = SPT == 1 ? Prec<P>::NB : Prec<P>::NB2;   // ring slots of blocks
    // rho/Psi deviation window of a tile: rows y0 - 2 .. y0 + TY + 1
    static constexpr int WIN = TY + 4;
    // step kernel: NB block slots, the rho and Psi windows, and -- where it
    // fits -- the staging tile of the bulk tensor stores, [TY / 8][9][8][TX]
    // (8-row halves, each one box of the 8-row store descriptor); without it
    // (FP32 with 16-row tiles) the threads store to global memory directly
    static constexpr int SLOT_BYTES = 9 * TYB * BX * (int)sizeof(T2);
    static constexpr int WIN_OFF = NB * SLOT_BYTES;
    static constexpr int WIN_BYTES = 2 * WIN * RX * (int)sizeof(C2);
    static constexpr int STAGE_OFF = WIN_OFF + WIN_BYTES;
    static constexpr int STAGE_FULL = 9 * TY * TX * (int)sizeof(T2);
    static constexpr bool STAGED = STAGE_OFF + STAGE_FULL + 128 <= 227 * 1024 - 1024;
    static constexpr int STAGE_BYTES = STAGED ? STAGE_FULL : 0;
    static constexpr int SMEM = STAGE_OFF + STAGE_BYTES + 128;
    // staging slot (plane 0) of tile row ly, column lx: planes of a half are
    // 8 TX pairs apart
    static __host__ __device__ constexpr int stage_off(int ly, int lx) {
        return ((ly >> 3) * 9) * TYB * TX + (ly & (TYB - 1)) * TX + lx;
    }
    // observe kernel: one tile box and the rho/Psi tile
    static constexpr int BOX_BYTES = 9 * BY * BX * (int)sizeof(T2);
    static constexpr int BOX_STRIDE = (BOX_BYTES + 127) / 128 * 128;
    static constexpr int RHOPSI = (2 * RX * RY * (int)sizeof(C2) + 127) / 128 * 128;
    static constexpr int SMEM_OBS = BOX_STRIDE + RHOPSI + 128;
    static_assert(SPT == 1 || SPT == 2, "one or two sites per thread");
    static_assert(SPT == 1 || STAGED || sizeof(T2) == 8, "direct stores: FP32 pairs only");
    static_assert(NB >= SPT + 2, "the ring holds a tile's blocks and at least one more");
    static_assert(RX % 32 == 0, "deviation rows are whole warps");
    static_assert((2 * TX * sizeof(T)) % 16 == 0 && (2 * (TX + GX) * sizeof(T)) % 16 == 0,
                  "TMA x coordinates of tiles stay 16-byte aligned");
    static_assert(SLOT_BYTES % 128 == 0 && WIN_BYTES % 128 == 0 && STAGE_BYTES % 128 == 0,
                  "128-byte alignment of the shared-memory regions");
    static_assert((BX * sizeof(T2)) % 16 == 0, "TMA box rows must be 16-byte multiples");
    static_assert(2 * BX <= 256 && 2 * TX <= 256 && BY <= 256, "TMA box extent");
    static_assert(GX >= 3 && (GX * sizeof(T)) % 16 == 0, "ghost width");
    static_assert(SMEM <= 227 * 1024 - 1024 && SMEM_OBS <= 227 * 1024, "shared memory");
};

}  // namespace lbgb
