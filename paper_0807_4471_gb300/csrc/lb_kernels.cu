// lb_kernels.cu -- sm_103a kernels of the two-species multi-range
// pseudo-potential lattice Boltzmann step (Benzi, Chibbaro & Succi,
// arXiv:0807.4471, Eqs. (1)-(2)).
//
// One launch of k_step advances every site of the lattice by one time step.
// Layout in HBM: structure of arrays, 18 planes (species s, direction i), each
// a ghost-padded [ny + 6][pitch] array of the storage type T.  The buffer read
// by a step holds the post-collision populations f*(t-1) of the previous
// step; streaming is done by pulling, f_i(r, t) = f*_i(r - c_i, t - 1).
//
// Per CTA (a TX x TY tile of sites):
//  1. TMA: two 3-D box loads (one per species, 9 planes each) bring f* on the
//     tile plus a 3-cell halo into shared memory.  The ghost columns/rows of
//     the padded planes hold periodic copies, so a box never wraps.
//  2. rho_s and Psi_s(rho_s) on the tile plus a 2-cell halo, from the pulled
//     populations (halfway bounce-back rows at Couette walls; rho mirrored
//     about a wall beyond it).
//  3. per site: moments, the force of Eq. (2) from the shared rho/Psi tile
//     (12 antisymmetric pairs of the 24-neighbour stencil, 4 pairs of the
//     cross term), the forced BGK relaxation of Eq. (1), and the write of
//     f*(t) into the other buffer together with its periodic ghost copies.
//  4. FP64 block reductions (wall momentum exchange, or mass/momentum in the
//     observe pass) into per-CTA slots; the last CTA to finish sums the slots
//     in a fixed order and advances the device step counter.
// There is no dense contraction anywhere, so no tensor cores are used.
#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include <cstdint>

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
    static constexpr int GX = 4, TX = 32, TY = 8, NT = 256;
};
template <> struct Prec<LB_FP32> {
    typedef float T; typedef float C;
    static constexpr int GX = 4, TX = 64, TY = 8, NT = 256;
};
template <> struct Prec<LB_FP16_OFFSET> {
    typedef __half T; typedef float C;
    static constexpr int GX = 8, TX = 64, TY = 8, NT = 256;
};
template <> struct Prec<LB_BF16_OFFSET> {
    typedef __nv_bfloat16 T; typedef float C;
    static constexpr int GX = 8, TX = 64, TY = 8, NT = 256;
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

__device__ __forceinline__ double cexpm1(double v) { return expm1(v); }
__device__ __forceinline__ float cexpm1(float v) { return expm1f(v); }
__device__ __forceinline__ double csin(double v) { return sin(v); }
__device__ __forceinline__ float csin(float v) { return sinf(v); }

template <int P>
struct Layout {
    typedef typename Prec<P>::T T;
    typedef typename Prec<P>::C C;
    static constexpr int TX = Prec<P>::TX, TY = Prec<P>::TY, NT = Prec<P>::NT;
    static constexpr int GX = Prec<P>::GX;
    static constexpr int BX = TX + 2 * GX;            // box columns
    static constexpr int BY = TY + 2 * kGY;           // box rows
    static constexpr int SPEC = 9 * BX * BY;          // elements per species box
    static constexpr int SPEC_BYTES = SPEC * (int)sizeof(T);
    static constexpr int SPEC_STRIDE = (SPEC_BYTES + 127) / 128 * 128;
    static constexpr int RX = TX + 4, RY = TY + 4;    // rho/Psi tile (2-cell halo)
    static constexpr int RHO_OFF = 2 * SPEC_STRIDE;
    static constexpr int SMEM = RHO_OFF + 4 * RX * RY * (int)sizeof(C) + 128;
    static_assert((BX * sizeof(T)) % 16 == 0, "TMA box rows must be 16-byte multiples");
    static_assert(GX >= 3 && (GX * sizeof(T)) % 16 == 0, "ghost width");
    static_assert(SMEM <= 227 * 1024, "shared memory");
};

// ------------------------------------------------------------ PTX helpers
__device__ __forceinline__ uint32_t smem_u32(const void* p) {
    return (uint32_t)__cvta_generic_to_shared(p);
}
__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count)
                 : "memory");
}
__device__ __forceinline__ void fence_mbar_init() {
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)),
                 "r"(bytes)
                 : "memory");
}
__device__ __forceinline__ void tma_load_3d(void* dst, const CUtensorMap* map, int x, int y,
                                            int z, uint64_t* bar) {
    asm volatile(
        "cp.async.bulk.tensor.3d.shared::cluster.global.mbarrier::complete_tx::bytes"
        " [%0], [%1, {%2, %3, %4}], [%5];" ::"r"(smem_u32(dst)),
        "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(z), "r"(smem_u32(bar))
        : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
        " selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}
// Bounded wait: each try_wait suspends for a hardware-chosen interval, so the
// bound is a few seconds at most.
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t* bar, uint32_t parity) {
    for (int it = 0; it < (1 << 22); ++it)
        if (mbar_try_wait(bar, parity)) return true;
    return false;
}

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

__device__ __forceinline__ uint64_t mix64(uint64_t z) {
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
    return z ^ (z >> 31);
}

// ---------------------------------------------------------- site helpers
// Write one value of plane q at site (x, y) and its periodic ghost copies.
template <typename T>
__device__ __forceinline__ void put(T* base, const Geom& g, int q, int x, int y, T v) {
    T* pl = base + (long long)q * g.plane;
    const int X = x + g.gx, Y = y + kGY;
    int X2 = -1, Y2 = -1;
    if (x < 3) X2 = X + g.nx;
    else if (x >= g.nx - 3) X2 = X - g.nx;
    if (g.periodic) {
        if (y < 3) Y2 = Y + g.ny;
        else if (y >= g.ny - 3) Y2 = Y - g.ny;
    }
    pl[(long long)Y * g.pitch + X] = v;
    if (X2 >= 0) pl[(long long)Y * g.pitch + X2] = v;
    if (Y2 >= 0) {
        pl[(long long)Y2 * g.pitch + X] = v;
        if (X2 >= 0) pl[(long long)Y2 * g.pitch + X2] = v;
    }
}

// The offsets h_i(r, t) = f_i(r, t) - w_i rho_ref of one species at lattice
// site (x, y), whose box coordinates are (sx, sy).  pull = 1: streamed from
// h*(r - c_i, t - 1), with halfway bounce-back at the Couette walls:
// f_i = f*_opp(i)(r) + 6 w_i rho_w (c_i . u_w), where rho_w is the
// pre-streaming density of the boundary node, rho_ref + sum_j h*_j(r).
template <int P>
__device__ __forceinline__ void load_site(const typename Prec<P>::T* sf, int sx, int sy, int y,
                                          const StepArgs<typename Prec<P>::C>& a,
                                          typename Prec<P>::C h[9]) {
    typedef Layout<P> L;
    typedef typename Prec<P>::C C;
    if (a.pull) {
#pragma unroll
        for (int i = 0; i < 9; ++i) h[i] = dec(sf[(i * L::BY + sy - cy(i)) * L::BX + sx - cx(i)]);
        if (!a.g.periodic && (y == 0 || y == a.g.ny - 1)) {
            C dr = C(0);
#pragma unroll
            for (int j = 0; j < 9; ++j) dr += dec(sf[(j * L::BY + sy) * L::BX + sx]);
            const C rw = a.k.rho_ref + dr;
            const int up = (y == 0);                 // links arriving upward
            const C uw = up ? -a.k.u_wall : a.k.u_wall;
#pragma unroll
            for (int i = 0; i < 9; ++i) {
                if ((up && cy(i) == 1) || (!up && cy(i) == -1))
                    h[i] = dec(sf[(opp(i) * L::BY + sy) * L::BX + sx]) +
                           C(6) * wgt<C>(i) * rw * (C(cx(i)) * uw);
            }
        }
    } else {
#pragma unroll
        for (int i = 0; i < 9; ++i) h[i] = dec(sf[(i * L::BY + sy) * L::BX + sx]);
    }
}

// Deviation of the pseudo-potential from Psi(rho_ref):
// Psi(rho_ref + d) - Psi(rho_ref) = -P exp(-rho_ref/rho0) expm1(-d/rho0).
template <typename C>
__device__ __forceinline__ C dpsi_of(C d, const Coef<C>& k) {
    return -k.psi_scale * cexpm1(-d * k.inv_rho0);
}

// ------------------------------------------------------------ step kernel
template <int P>
__global__ void __launch_bounds__(Prec<P>::NT)
    k_step(const __grid_constant__ CUtensorMap tin,
           const __grid_constant__ StepArgs<typename Prec<P>::C> a) {
    typedef Layout<P> L;
    typedef typename L::T T;
    typedef typename L::C C;
    extern __shared__ unsigned char smem_raw[];
    unsigned char* smem =
        reinterpret_cast<unsigned char*>((reinterpret_cast<uintptr_t>(smem_raw) + 127) & ~uintptr_t(127));
    T* sfA = reinterpret_cast<T*>(smem);
    T* sfB = reinterpret_cast<T*>(smem + L::SPEC_STRIDE);
    C* srho = reinterpret_cast<C*>(smem + L::RHO_OFF);   // [2][RY][RX]
    C* spsi = srho + 2 * L::RX * L::RY;                   // [2][RY][RX]
    __shared__ __align__(8) uint64_t bar;
    __shared__ int s_ok;
    __shared__ double s_red[L::NT / 32][4];
    __shared__ int s_last;

    const int tid = threadIdx.x;
    const int x0 = blockIdx.x * L::TX, y0 = blockIdx.y * L::TY;
    const Geom& g = a.g;
    const int nblocks = gridDim.x * gridDim.y;
    const long long t = *((volatile long long*)&a.st->t);

    // 1. stage f* on the tile + 3-cell halo.  Box origin in padded
    // coordinates: column x0 (= x0 - gx + gx), row y0 (= y0 - 3 + kGY).
    if (tid == 0) {
        s_ok = 1;
        mbar_init(&bar, 1);
        fence_mbar_init();
    }
    __syncthreads();
    if (tid == 0) {
        mbar_expect_tx(&bar, 2u * L::SPEC_BYTES);
        tma_load_3d(sfA, &tin, x0, y0, 0, &bar);
        tma_load_3d(sfB, &tin, x0, y0, 9, &bar);
    }
    if (!mbar_wait_bounded(&bar, 0)) s_ok = 0;
    __syncthreads();
    if (tid == 0 && !s_ok) {
        atomicOr(&a.st->err, ERR_TIMEOUT);
        mbar_wait_bounded(&bar, 0);   // give copies in flight a last chance to land
    }
    const bool ok = s_ok != 0;

    double red[4] = {0.0, 0.0, 0.0, 0.0};
    if (ok) {
        // 2. density and pseudo-potential deviations d_rho = rho - rho_ref,
        // d_Psi = Psi(rho) - Psi(rho_ref) on the tile + 2-cell halo.
        for (int c = tid; c < L::RX * L::RY; c += L::NT) {
            const int lx = c % L::RX, ly = c / L::RX;
            const int y = y0 - 2 + ly;
            if (!g.periodic && (y < 0 || y >= g.ny)) continue;
            const int sx = lx - 2 + L::GX, sy = ly - 2 + kGY;
            C h[9];
#pragma unroll
            for (int s = 0; s < 2; ++s) {
                load_site<P>(s ? sfB : sfA, sx, sy, y, a, h);
                C r = C(0);
#pragma unroll
                for (int i = 0; i < 9; ++i) r += h[i];
                srho[(s * L::RY + ly) * L::RX + lx] = r;
                spsi[(s * L::RY + ly) * L::RX + lx] = dpsi_of(r, a.k);
            }
        }
        __syncthreads();
        if (!g.periodic) {   // mirror the deviations about the halfway walls
            for (int c = tid; c < L::RX * L::RY; c += L::NT) {
                const int lx = c % L::RX, ly = c / L::RX;
                const int y = y0 - 2 + ly;
                int ym;
                if (y < 0) ym = -1 - y;
                else if (y >= g.ny) ym = 2 * g.ny - 1 - y;
                else continue;
                const int lm = ym - (y0 - 2);
                if (lm < 0 || lm >= L::RY) continue;
#pragma unroll
                for (int s = 0; s < 2; ++s) {
                    srho[(s * L::RY + ly) * L::RX + lx] = srho[(s * L::RY + lm) * L::RX + lx];
                    spsi[(s * L::RY + ly) * L::RX + lx] = spsi[(s * L::RY + lm) * L::RX + lx];
                }
            }
            __syncthreads();
        }

        // 3. per-site moments, forces, collision, write-back.
        T* fout = reinterpret_cast<T*>(a.fout);
        const long long N = (long long)g.nx * g.ny;
        bool bad = false;
        for (int c = tid; c < L::TX * L::TY; c += L::NT) {
            const int lx = c % L::TX, ly = c / L::TX;
            const int x = x0 + lx, y = y0 + ly;
            if (x >= g.nx || y >= g.ny) continue;
            const int sx = lx + L::GX, sy = ly + kGY;
            const int rx = lx + 2, ry = ly + 2;
            C h[2][9];
            load_site<P>(sfA, sx, sy, y, a, h[0]);
            load_site<P>(sfB, sx, sy, y, a, h[1]);
            C drho[2], rho[2], jx[2], jy[2];
#pragma unroll
            for (int s = 0; s < 2; ++s) {
                C r = C(0), mx = C(0), my = C(0);
#pragma unroll
                for (int i = 0; i < 9; ++i) r += h[s][i];
#pragma unroll
                for (int i = 0; i < 9; ++i) {   // sum_i w_i c_i = 0: offsets carry all of j
                    if (cx(i) == 1) mx += h[s][i];
                    if (cx(i) == -1) mx -= h[s][i];
                    if (cy(i) == 1) my += h[s][i];
                    if (cy(i) == -1) my -= h[s][i];
                }
                drho[s] = r;
                rho[s] = a.k.rho_ref + r;
                jx[s] = mx;
                jy[s] = my;
            }
            if (!(isfinite(rho[0]) && isfinite(rho[1]))) bad = true;

            // Eq. (2): F_s = -Psi_s(r) sum_d K_s(d) d [Psi_s(r+d) - Psi_s(r-d)]
            //               - (G_X/rho0) rho_s(r) sum_d w(d) d [rho_s'(r+d) - rho_s'(r-d)]
            // (the reference values cancel in the differences).
            C Fx[2], Fy[2];
#pragma unroll
            for (int s = 0; s < 2; ++s) {
                const C* ps = spsi + s * L::RX * L::RY;
                const C* ro = srho + (1 - s) * L::RX * L::RY;
                C ax = C(0), ay = C(0);
#pragma unroll
                for (int k = 0; k < 12; ++k) {
                    const int dx = rdx(k), dy = rdy(k);
                    const C diff = ps[(ry + dy) * L::RX + rx + dx] - ps[(ry - dy) * L::RX + rx - dx];
                    if (dx != 0) ax += (a.k.K[s][k] * C(dx)) * diff;
                    if (dy != 0) ay += (a.k.K[s][k] * C(dy)) * diff;
                }
                C qx = C(0), qy = C(0);
#pragma unroll
                for (int k = 0; k < 4; ++k) {
                    const int dx = rdx(k), dy = rdy(k);
                    const C diff = ro[(ry + dy) * L::RX + rx + dx] - ro[(ry - dy) * L::RX + rx - dx];
                    if (dx != 0) qx += (a.k.W[k] * C(dx)) * diff;
                    if (dy != 0) qy += (a.k.W[k] * C(dy)) * diff;
                }
                const C pc = a.k.psi_ref + ps[ry * L::RX + rx];
                Fx[s] = -pc * ax - a.k.gx_rho0 * rho[s] * qx;
                Fy[s] = -pc * ay - a.k.gx_rho0 * rho[s] * qy;
            }
            if (a.k.has_accel) {
                C acc = a.k.g_x;
                if (a.k.kolmo_amp != C(0)) acc += a.k.kolmo_amp * csin(a.k.kolmo_w * C(y));
                Fx[0] += rho[0] * acc;
                Fx[1] += rho[1] * acc;
            }

            if (a.obs == OBS_NONE) {
                // Eq. (1): forced BGK relaxation of the offsets,
                // h*_i = h_i - omega (h_i - heq_i), heq_i = f^eq_i - w_i rho_ref
                //      = w_i [d_rho + rho (3 c.u + 4.5 (c.u)^2 - 1.5 u^2)].
                const C den = rho[0] * a.k.omega[0] + rho[1] * a.k.omega[1];
                C upx = C(0), upy = C(0);
                if (den != C(0)) {
                    upx = (jx[0] * a.k.omega[0] + jx[1] * a.k.omega[1]) / den;
                    upy = (jy[0] * a.k.omega[0] + jy[1] * a.k.omega[1]) / den;
                }
#pragma unroll
                for (int s = 0; s < 2; ++s) {
                    C ux = upx, uy = upy;
                    if (!a.k.source && rho[s] != C(0)) {
                        const C tr = a.k.tau[s] / rho[s];
                        ux += tr * Fx[s];
                        uy += tr * Fy[s];
                    }
                    const C usq = C(1.5) * (ux * ux + uy * uy);
                    const C om = a.k.omega[s];
                    C dr = C(0);
                    C hs[9];
#pragma unroll
                    for (int i = 0; i < 9; ++i) {
                        const C cu = C(cx(i)) * ux + C(cy(i)) * uy;
                        const C heq = wgt<C>(i) * (drho[s] + rho[s] * (C(3) * cu + C(4.5) * cu * cu - usq));
                        C v = h[s][i] - om * (h[s][i] - heq);
                        if (a.k.source) v += wgt<C>(i) * C(3) * (C(cx(i)) * Fx[s] + C(cy(i)) * Fy[s]);
                        const T e = encf<T>(v);
                        put<T>(fout, g, s * 9 + i, x, y, e);
                        hs[i] = dec(e);
                        dr += hs[i];
                    }
                    if (!g.periodic && (y == 0 || y == g.ny - 1)) {
                        // x-momentum handed to the wall by the links that will
                        // bounce back at the next streaming: c_x (f*_i + f_opp),
                        // f_opp = f*_i - 6 w_i rho_w (c_i . u_w).
                        const int down = (y == 0);
                        const C uw = down ? -a.k.u_wall : a.k.u_wall;
                        const C rw = a.k.rho_ref + dr;
#pragma unroll
                        for (int i = 0; i < 9; ++i) {
                            if ((down && cy(i) == -1) || (!down && cy(i) == 1)) {
                                const C fi = hs[i] + wgt<C>(i) * a.k.rho_ref;
                                const C back = fi - C(6) * wgt<C>(i) * rw * (C(cx(i)) * uw);
                                const double dp = (double)(C(cx(i)) * (fi + back));
                                if (down) red[0] += dp; else red[1] += dp;
                            }
                        }
                    }
                }
            } else {
                const long long idx = (long long)y * g.nx + x;
                const double rA = (double)a.k.rho_ref + (double)drho[0];
                const double rB = (double)a.k.rho_ref + (double)drho[1];
                const double tot = rA + rB;
                const double mx = (double)jx[0] + (double)jx[1] + 0.5 * ((double)Fx[0] + (double)Fx[1]);
                const double my = (double)jy[0] + (double)jy[1] + 0.5 * ((double)Fy[0] + (double)Fy[1]);
                if (a.obs == OBS_FIELDS) {
                    a.obs_out[idx] = rA;
                    a.obs_out[N + idx] = rB;
                    a.obs_out[2 * N + idx] = tot != 0.0 ? mx / tot : 0.0;
                    a.obs_out[3 * N + idx] = tot != 0.0 ? my / tot : 0.0;
                } else if (a.obs == OBS_POPS) {
#pragma unroll
                    for (int q = 0; q < 18; ++q)
                        if (q >= a.q0 && q < a.q1)
                            a.obs_out[(long long)(q - a.q0) * N + idx] =
                                (double)h[q / 9][q % 9] + wgt<double>(q % 9) * (double)a.k.rho_ref;
                }
                red[0] += rA;
                red[1] += rB;
                red[2] += mx;
                red[3] += my;
            }
        }
        if (bad) atomicOr(&a.st->err, ERR_NONFINITE);
    }

    // 4. FP64 block reduction into per-CTA slots, then the last CTA sums them.
    const bool walls = (a.obs == OBS_NONE) && !g.periodic;
    const bool want = walls || a.obs != OBS_NONE;
    if (want) {
        const int lane = tid & 31, warp = tid >> 5;
#pragma unroll
        for (int k = 0; k < 4; ++k) red[k] = warp_sum(red[k]);
        if (lane == 0) {
#pragma unroll
            for (int k = 0; k < 4; ++k) s_red[warp][k] = red[k];
        }
        __syncthreads();
        if (tid == 0) {
            double v[4] = {0.0, 0.0, 0.0, 0.0};
            for (int w = 0; w < L::NT / 32; ++w)
#pragma unroll
                for (int k = 0; k < 4; ++k) v[k] += s_red[w][k];
            if (walls) {
                if (blockIdx.y == 0) a.slots[2 * blockIdx.x] = v[0];
                if (blockIdx.y == gridDim.y - 1) a.slots[2 * blockIdx.x + 1] = v[1];
            } else {
                const int b = blockIdx.y * gridDim.x + blockIdx.x;
#pragma unroll
                for (int k = 0; k < 4; ++k) a.slots[4 * b + k] = v[k];
            }
        }
    }
    __threadfence();
    __syncthreads();
    if (tid == 0) {
        const unsigned int tk = atomicAdd(&a.st->ticket, 1u);
        s_last = (tk == (unsigned int)(nblocks - 1));
    }
    __syncthreads();
    if (!s_last) return;
    __threadfence();
    const volatile double* vs = a.slots;
    if (walls) {
        double v0 = 0.0, v1 = 0.0;
        for (int b = tid; b < (int)gridDim.x; b += L::NT) { v0 += vs[2 * b]; v1 += vs[2 * b + 1]; }
        red[0] = v0; red[1] = v1; red[2] = 0.0; red[3] = 0.0;
    } else if (a.obs != OBS_NONE) {
        double v[4] = {0.0, 0.0, 0.0, 0.0};
        for (int b = tid; b < nblocks; b += L::NT)
#pragma unroll
            for (int k = 0; k < 4; ++k) v[k] += vs[4 * b + k];
#pragma unroll
        for (int k = 0; k < 4; ++k) red[k] = v[k];
    }
    if (want) {
        const int lane = tid & 31, warp = tid >> 5;
        __syncthreads();
#pragma unroll
        for (int k = 0; k < 4; ++k) red[k] = warp_sum(red[k]);
        if (lane == 0) {
#pragma unroll
            for (int k = 0; k < 4; ++k) s_red[warp][k] = red[k];
        }
        __syncthreads();
    }
    if (tid == 0) {
        double v[4] = {0.0, 0.0, 0.0, 0.0};
        if (want)
            for (int w = 0; w < L::NT / 32; ++w)
#pragma unroll
                for (int k = 0; k < 4; ++k) v[k] += s_red[w][k];
        if (a.obs == OBS_NONE) {
            if (walls) {
                const long long every = a.stress_every > 0 ? a.stress_every : 1;
                if (t >= a.stress_t0 && ((t - a.stress_t0) % every) == 0) {
                    a.st->sum_bot += v[0] / g.nx;
                    a.st->sum_top += v[1] / g.nx;
                    a.st->samples += 1;
                }
            }
            a.st->t = t + 1;
        } else {
#pragma unroll
            for (int k = 0; k < 4; ++k) a.st->totals[k] = v[k];
        }
        a.st->ticket = 0u;
        __threadfence();
    }
}

// ------------------------------------------------------------ init kernels
// f(r, 0) = f^eq(rho_s, u) in place (the first step reads it unshifted).
// mode 0: rho_s from the counter generator; mode 1: FP64 fields [4][ny][nx].
template <int P>
__global__ void k_init(Geom g, Coef<typename Prec<P>::C> k, typename Prec<P>::T* fout, int mode,
                       const double* fields, double rho0, double amp, double u_wall, int init_shear,
                       unsigned long long seed) {
    typedef typename Prec<P>::T T;
    const long long N = (long long)g.nx * g.ny;
    for (long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x; idx < N;
         idx += (long long)gridDim.x * blockDim.x) {
        const int x = (int)(idx % g.nx), y = (int)(idx / g.nx);
        double r[2], ux, uy;
        if (mode == 0) {
            for (int s = 0; s < 2; ++s) {
                const uint64_t ctr = ((uint64_t)s * g.ny + y) * g.nx + x;
                const uint64_t z = mix64(seed ^ mix64(ctr + 0x9E3779B97F4A7C15ULL));
                const double u = (double)(z >> 11) * (1.0 / 9007199254740992.0);
                r[s] = rho0 * (1.0 + amp * (2.0 * u - 1.0));
            }
            ux = init_shear ? u_wall * (2.0 * y + 1.0 - g.ny) / (double)g.ny : 0.0;
            uy = 0.0;
        } else {
            r[0] = fields[idx];
            r[1] = fields[N + idx];
            ux = fields[2 * N + idx];
            uy = fields[3 * N + idx];
        }
        const double usq = ux * ux + uy * uy;
        const double rref = (double)k.rho_ref;
        for (int s = 0; s < 2; ++s)
#pragma unroll
            for (int i = 0; i < 9; ++i) {
                const double cu = cx(i) * ux + cy(i) * uy;
                // f^eq_i - w_i rho_ref
                const double h = wgt<double>(i) * ((r[s] - rref) + r[s] * (3.0 * cu + 4.5 * cu * cu - 1.5 * usq));
                put<T>(fout, g, s * 9 + i, x, y, encd<T>(h));
            }
    }
}

// ------------------------------------------------------------- launchers
template <int P>
static cudaError_t step_t(const CUtensorMap* tin, const void* args, dim3 grid, cudaStream_t s) {
    typedef Layout<P> L;
    typedef typename L::C C;
    static int configured[64] = {0};
    int dev = 0;
    cudaGetDevice(&dev);
    if (dev < 64 && !configured[dev]) {
        cudaError_t e = cudaFuncSetAttribute(k_step<P>, cudaFuncAttributeMaxDynamicSharedMemorySize, L::SMEM);
        if (e != cudaSuccess) return e;
        configured[dev] = 1;
    }
    k_step<P><<<grid, L::NT, L::SMEM, s>>>(*tin, *reinterpret_cast<const StepArgs<C>*>(args));
    return cudaGetLastError();
}

cudaError_t launch_step(int precision, const CUtensorMap* tin, const void* args, dim3 grid,
                        cudaStream_t s) {
    switch (precision) {
        case LB_FP64: return step_t<LB_FP64>(tin, args, grid, s);
        case LB_FP32: return step_t<LB_FP32>(tin, args, grid, s);
        case LB_FP16_OFFSET: return step_t<LB_FP16_OFFSET>(tin, args, grid, s);
        case LB_BF16_OFFSET: return step_t<LB_BF16_OFFSET>(tin, args, grid, s);
    }
    return cudaErrorInvalidValue;
}

template <int P>
static cudaError_t init_t(const Geom& g, const void* coef, void* fout, int mode, const double* fields,
                          double rho0, double amp, double u_wall, int init_shear,
                          unsigned long long seed, cudaStream_t s) {
    typedef typename Prec<P>::C C;
    typedef typename Prec<P>::T T;
    const long long N = (long long)g.nx * g.ny;
    long long blocks = (N + 255) / 256;
    if (blocks > 152 * 64) blocks = 152 * 64;
    k_init<P><<<(unsigned)blocks, 256, 0, s>>>(g, *reinterpret_cast<const Coef<C>*>(coef),
                                               reinterpret_cast<T*>(fout), mode, fields, rho0, amp,
                                               u_wall, init_shear, seed);
    return cudaGetLastError();
}

cudaError_t launch_init_seeded(int precision, const Geom& g, const void* coef, void* fout,
                               double rho0, double amp, double u_wall, int init_shear,
                               unsigned long long seed, cudaStream_t s) {
    switch (precision) {
        case LB_FP64: return init_t<LB_FP64>(g, coef, fout, 0, nullptr, rho0, amp, u_wall, init_shear, seed, s);
        case LB_FP32: return init_t<LB_FP32>(g, coef, fout, 0, nullptr, rho0, amp, u_wall, init_shear, seed, s);
        case LB_FP16_OFFSET: return init_t<LB_FP16_OFFSET>(g, coef, fout, 0, nullptr, rho0, amp, u_wall, init_shear, seed, s);
        case LB_BF16_OFFSET: return init_t<LB_BF16_OFFSET>(g, coef, fout, 0, nullptr, rho0, amp, u_wall, init_shear, seed, s);
    }
    return cudaErrorInvalidValue;
}

cudaError_t launch_init_fields(int precision, const Geom& g, const void* coef, void* fout,
                               const double* fields, cudaStream_t s) {
    switch (precision) {
        case LB_FP64: return init_t<LB_FP64>(g, coef, fout, 1, fields, 0, 0, 0, 0, 0, s);
        case LB_FP32: return init_t<LB_FP32>(g, coef, fout, 1, fields, 0, 0, 0, 0, 0, s);
        case LB_FP16_OFFSET: return init_t<LB_FP16_OFFSET>(g, coef, fout, 1, fields, 0, 0, 0, 0, 0, s);
        case LB_BF16_OFFSET: return init_t<LB_BF16_OFFSET>(g, coef, fout, 1, fields, 0, 0, 0, 0, 0, s);
    }
    return cudaErrorInvalidValue;
}

int kernel_smem_bytes(int p) {
    switch (p) {
        case LB_FP64: return Layout<LB_FP64>::SMEM;
        case LB_FP32: return Layout<LB_FP32>::SMEM;
        case LB_FP16_OFFSET: return Layout<LB_FP16_OFFSET>::SMEM;
        case LB_BF16_OFFSET: return Layout<LB_BF16_OFFSET>::SMEM;
    }
    return 0;
}
int kernel_tile_x(int p) {
    return p == LB_FP64 ? Prec<LB_FP64>::TX : p == LB_FP32 ? Prec<LB_FP32>::TX : Prec<LB_FP16_OFFSET>::TX;
}
int kernel_tile_y(int p) {
    return p == LB_FP64 ? Prec<LB_FP64>::TY : p == LB_FP32 ? Prec<LB_FP32>::TY : Prec<LB_FP16_OFFSET>::TY;
}
int kernel_ghost_x(int p) {
    return p == LB_FP64 ? Prec<LB_FP64>::GX : p == LB_FP32 ? Prec<LB_FP32>::GX : Prec<LB_FP16_OFFSET>::GX;
}
int kernel_elem_bytes(int p) { return p == LB_FP64 ? 8 : p == LB_FP32 ? 4 : 2; }

}  // namespace lbgb
