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
#include "lb_layout.cuh"

namespace lbgb {

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
__device__ __forceinline__ void fence_proxy_async() {
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
// Bulk tensor store of a shared-memory box to global memory (bulk group).
__device__ __forceinline__ void tma_store_3d(const CUtensorMap* map, const void* src, int x, int y,
                                             int z) {
    asm volatile(
        "cp.async.bulk.tensor.3d.global.shared::cta.bulk_group [%0, {%2, %3, %4}], [%1];" ::"l"(
            reinterpret_cast<uint64_t>(map)),
        "r"(smem_u32(src)), "r"(x), "r"(y), "r"(z)
        : "memory");
}
__device__ __forceinline__ void bulk_commit() { asm volatile("cp.async.bulk.commit_group;" ::: "memory"); }
// Wait until the committed bulk stores have finished reading shared memory.
__device__ __forceinline__ void bulk_wait_read() {
    asm volatile("cp.async.bulk.wait_group.read 0;" ::: "memory");
}
// Wait until the committed bulk stores have completed.
__device__ __forceinline__ void bulk_wait_all() { asm volatile("cp.async.bulk.wait_group 0;" ::: "memory"); }

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
template <int P, bool PER>
__device__ __forceinline__ void load_site(const typename Prec<P>::T* sf, int sx, int sy, int y,
                                          const StepArgs<typename Prec<P>::C>& a,
                                          typename Prec<P>::C h[9]) {
    typedef Layout<P> L;
    typedef typename Prec<P>::C C;
    if (a.pull) {
#pragma unroll
        for (int i = 0; i < 9; ++i) h[i] = dec(sf[(i * L::BY + sy - cy(i)) * L::BX + sx - cx(i)]);
        if (!PER && (y == 0 || y == a.g.ny - 1)) {
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

// ------------------------------------------------------------- tile body
// Phases 2-3 for one TX x TY tile whose f* box (tile + 3-cell halo, both
// species) is in shared memory.  One site per thread in phase 3.
// OBS = false: collision and write-back of f*(t) (+ wall momentum into red).
// OBS = true : fields / populations / totals of the current state (red =
//              mass_A, mass_B, mom_x, mom_y).
// V: bit 0 = periodic in y (else Couette walls); bit 1 = general forcing
// (additive source term or body acceleration checked at run time).
template <int P, bool OBS, int V>
__device__ __forceinline__ void tile_body(const typename Prec<P>::T* __restrict__ sfA,
                                          const typename Prec<P>::T* __restrict__ sfB,
                                          typename Prec<P>::C* __restrict__ srho,
                                          typename Prec<P>::C* __restrict__ spsi, int x0, int y0,
                                          const StepArgs<typename Prec<P>::C>& a, double red[4],
                                          bool& bad, typename Prec<P>::T* __restrict__ stage) {
    typedef Layout<P> L;
    typedef typename L::T T;
    typedef typename L::C C;
    constexpr bool PER = (V & 1) != 0;
    constexpr bool GEN = (V & 2) != 0;
    const int tid = threadIdx.x;
    const Geom& g = a.g;

    // 2. density and pseudo-potential deviations d_rho = rho - rho_ref,
    // d_Psi = Psi(rho) - Psi(rho_ref) on the tile + 2-cell halo.
    for (int c = tid; c < L::RX * L::RY; c += L::NT) {
        const int ly = c / L::RX, lx = c - ly * L::RX;
        const int y = y0 - 2 + ly;
        if (!PER && (y < 0 || y >= g.ny)) continue;
        const int sx = lx - 2 + L::GX, sy = ly - 2 + kGY;
        C h[9];
#pragma unroll
        for (int s = 0; s < 2; ++s) {
            load_site<P, PER>(s ? sfB : sfA, sx, sy, y, a, h);
            C r = C(0);
#pragma unroll
            for (int i = 0; i < 9; ++i) r += h[i];
            srho[(s * L::RY + ly) * L::RX + lx] = r;
            spsi[(s * L::RY + ly) * L::RX + lx] = dpsi_of(r, a.k);
        }
    }
    if (!PER) {   // mirror the deviations about the halfway walls
        __syncthreads();
        for (int c = tid; c < L::RX * L::RY; c += L::NT) {
            const int ly = c / L::RX, lx = c - ly * L::RX;
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
    }
    // the previous tile's bulk store must have read the staging tile
    if (stage != nullptr && tid == 0) bulk_wait_read();
    __syncthreads();

    // 3. one site per thread: moments, forces, collision, write-back.
    const int lx = tid % L::TX, ly = tid / L::TX;
    const int x = x0 + lx, y = y0 + ly;
    if (x >= g.nx || y >= g.ny) return;
    const int sx = lx + L::GX, sy = ly + kGY;
    const int rx = lx + 2, ry = ly + 2;
    C h[2][9];
    load_site<P, PER>(sfA, sx, sy, y, a, h[0]);
    load_site<P, PER>(sfB, sx, sy, y, a, h[1]);
    C drho[2], rho[2], jx[2], jy[2];
#pragma unroll
    for (int s = 0; s < 2; ++s) {
        C r = C(0), mx = C(0), my = C(0);
#pragma unroll
        for (int i = 0; i < 9; ++i) r += h[s][i];
        // sum_i w_i c_i = 0, so the offsets carry all of j
        mx = (h[s][1] - h[s][3]) + ((h[s][5] - h[s][7]) + (h[s][8] - h[s][6]));
        my = (h[s][2] - h[s][4]) + ((h[s][5] - h[s][7]) + (h[s][6] - h[s][8]));
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
        const C* ps = spsi + s * L::RX * L::RY + ry * L::RX + rx;
        const C* ro = srho + (1 - s) * L::RX * L::RY + ry * L::RX + rx;
        C ax = C(0), ay = C(0);
#pragma unroll
        for (int k = 0; k < 12; ++k) {
            const int dx = rdx(k), dy = rdy(k);
            const C diff = ps[dy * L::RX + dx] - ps[-dy * L::RX - dx];
            if (dx != 0) ax += (a.k.K[s][k] * C(dx)) * diff;
            if (dy != 0) ay += (a.k.K[s][k] * C(dy)) * diff;
        }
        C qx = C(0), qy = C(0);
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            const int dx = rdx(k), dy = rdy(k);
            const C diff = ro[dy * L::RX + dx] - ro[-dy * L::RX - dx];
            if (dx != 0) qx += (a.k.W[k] * C(dx)) * diff;
            if (dy != 0) qy += (a.k.W[k] * C(dy)) * diff;
        }
        const C pc = a.k.psi_ref + ps[0];
        Fx[s] = -pc * ax - a.k.gx_rho0 * rho[s] * qx;
        Fy[s] = -pc * ay - a.k.gx_rho0 * rho[s] * qy;
    }
    if (GEN && a.k.has_accel) {
        C acc = a.k.g_x;
        if (a.k.kolmo_amp != C(0)) acc += a.k.kolmo_amp * csin(a.k.kolmo_w * C(y));
        Fx[0] += rho[0] * acc;
        Fx[1] += rho[1] * acc;
    }

    if (OBS) {
        const long long N = (long long)g.nx * g.ny;
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
        return;
    }

    // Eq. (1): forced BGK relaxation of the offsets,
    // h*_i = h_i + omega (heq_i - h_i), heq_i = f^eq_i - w_i rho_ref
    //      = w_i [d_rho + rho (3 c.u + 4.5 (c.u)^2 - 1.5 u^2)].
    const C den = rho[0] * a.k.omega[0] + rho[1] * a.k.omega[1];
    C upx = C(0), upy = C(0);
    if (den != C(0)) {
        const C inv = recip(den);
        upx = (jx[0] * a.k.omega[0] + jx[1] * a.k.omega[1]) * inv;
        upy = (jy[0] * a.k.omega[0] + jy[1] * a.k.omega[1]) * inv;
    }
    // Store address of plane 0 at (x, y) and the periodic ghost copies.
    T* __restrict__ out = reinterpret_cast<T*>(a.fout) + (long long)(y + kGY) * g.pitch + (x + g.gx);
    const long long PL = g.plane;
    const int dX = (x < 3) ? g.nx : ((x >= g.nx - 3) ? -g.nx : 0);
    long long dY = 0;
    if (PER) dY = (y < 3) ? (long long)g.ny * g.pitch : ((y >= g.ny - 3) ? -(long long)g.ny * g.pitch : 0);
    const bool ghost = (dX != 0) || (dY != 0);
    const bool wall = !PER && (y == 0 || y == g.ny - 1);
    // Full tiles go through the staging tile and a bulk tensor store.
    const bool staged = stage != nullptr && x0 + L::TX <= g.nx && y0 + L::TY <= g.ny;
    const bool source = GEN && a.k.source;
#pragma unroll
    for (int s = 0; s < 2; ++s) {
        C ux = upx, uy = upy;
        if (!source && rho[s] != C(0)) {
            const C tr = a.k.tau[s] * recip(rho[s]);
            ux += tr * Fx[s];
            uy += tr * Fy[s];
        }
        const C usq = C(1.5) * (ux * ux + uy * uy);
        const C om = a.k.omega[s];
        T e[9];
#pragma unroll
        for (int i = 0; i < 9; ++i) {
            const C cu = C(cx(i)) * ux + C(cy(i)) * uy;
            const C heq = wgt<C>(i) * (drho[s] + rho[s] * (cu * (C(3) + C(4.5) * cu) - usq));
            C v = h[s][i] + om * (heq - h[s][i]);
            if (source) v += wgt<C>(i) * C(3) * (C(cx(i)) * Fx[s] + C(cy(i)) * Fy[s]);
            e[i] = encf<T>(v);
            if (staged)
                stage[((s * 9 + i) * L::TY + ly) * L::TX + lx] = e[i];
            else
                out[(s * 9 + i) * PL] = e[i];
        }
        if (ghost) {
#pragma unroll
            for (int i = 0; i < 9; ++i) {
                T* o = out + (s * 9 + i) * PL;
                if (dX) o[dX] = e[i];
                if (dY) {
                    o[dY] = e[i];
                    if (dX) o[dY + dX] = e[i];
                }
            }
        }
        if (wall) {
            // x-momentum handed to the wall by the links that will bounce
            // back at the next streaming: c_x (f*_i + f_opp),
            // f_opp = f*_i - 6 w_i rho_w (c_i . u_w).
            const int down = (y == 0);
            const C uw = down ? -a.k.u_wall : a.k.u_wall;
            C hs[9];
            C dr = C(0);
#pragma unroll
            for (int i = 0; i < 9; ++i) {
                hs[i] = dec(e[i]);
                dr += hs[i];
            }
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
    if (staged) fence_proxy_async();   // staging writes before the bulk store reads them
}

// FP64 block reduction of red[0..3] (all threads), result valid in thread 0.
template <int NT>
__device__ __forceinline__ void block_sum4(double red[4], double (*s_red)[4]) {
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
#pragma unroll
    for (int k = 0; k < 4; ++k) red[k] = warp_sum(red[k]);
    __syncthreads();
    if (lane == 0)
#pragma unroll
        for (int k = 0; k < 4; ++k) s_red[warp][k] = red[k];
    __syncthreads();
    if (tid == 0) {
        double v[4] = {0.0, 0.0, 0.0, 0.0};
        for (int w = 0; w < NT / 32; ++w)
#pragma unroll
            for (int k = 0; k < 4; ++k) v[k] += s_red[w][k];
#pragma unroll
        for (int k = 0; k < 4; ++k) red[k] = v[k];
    }
}

// Last-CTA pattern: every CTA has written its slot (thread 0); the CTA that
// arrives last sums the `nslots` slots of `width` doubles in a fixed order.
// Returns true in the last CTA, with the sums in red (valid in thread 0).
template <int NT>
__device__ __forceinline__ bool last_cta_sum(DevStats* st,
                                             const double* slots, int nslots, int width,
                                             double red[4], double (*s_red)[4], int* s_last) {
    const int tid = threadIdx.x;
    if (tid == 0) {
        __threadfence();
        const unsigned int tk = atomicAdd(&st->ticket, 1u);
        *s_last = (tk == gridDim.x * gridDim.y - 1) ? 1 : 0;
    }
    __syncthreads();
    if (!*s_last) return false;
    __threadfence();
    const volatile double* vs = slots;
    double v[4] = {0.0, 0.0, 0.0, 0.0};
    for (int b = tid; b < nslots; b += NT)
        for (int k = 0; k < width; ++k) v[k] += vs[width * b + k];
#pragma unroll
    for (int k = 0; k < 4; ++k) red[k] = v[k];
    block_sum4<NT>(red, s_red);
    return true;
}

// ------------------------------------------------------------ step kernel
// Persistent: one CTA per SM walks the tiles tile = blockIdx.x + k gridDim.x
// (row-major tile order, so the CTAs in flight cover a narrow band of rows and
// the halo overlap between tile rows is served by L2).  The box of the next
// tile is loaded by TMA into the second buffer while the current tile is
// computed.
template <int P, int V>
__global__ void __launch_bounds__(Layout<P>::NT, 1)
    k_step(const __grid_constant__ CUtensorMap tin, const __grid_constant__ CUtensorMap tout,
           const __grid_constant__ StepArgs<typename Prec<P>::C> a) {
    typedef Layout<P> L;
    typedef typename L::T T;
    typedef typename L::C C;
    extern __shared__ unsigned char smem_raw[];
    // 128-byte aligned base, derived from the shared array by indexing so
    // that every access below compiles to shared-memory instructions.
    unsigned char* smem = smem_raw + ((128u - (smem_u32(smem_raw) & 127u)) & 127u);
    // box b (b = 0, 1) holds both species: A at +0, B at +SPEC_STRIDE bytes
    auto box = [&](int b) { return reinterpret_cast<T*>(smem + b * (2 * L::SPEC_STRIDE)); };
    C* srho = reinterpret_cast<C*>(smem + 4 * L::SPEC_STRIDE);   // [2][RY][RX]
    C* spsi = srho + 2 * L::RX * L::RY;                           // [2][RY][RX]
    T* stage = reinterpret_cast<T*>(smem + L::STAGE_OFF);         // [18][TY][TX]
    __shared__ __align__(8) uint64_t bars[2];
    __shared__ int s_fail, s_last;
    __shared__ double s_red[L::NT / 32][4];

    const int tid = threadIdx.x;
    const Geom& g = a.g;
    const int ntx = (g.nx + L::TX - 1) / L::TX;
    const int ntiles = ntx * ((g.ny + L::TY - 1) / L::TY);

    if (tid == 0) {
        s_fail = 0;
        mbar_init(&bars[0], 1);
        mbar_init(&bars[1], 1);
        fence_mbar_init();
    }
    __syncthreads();
    // Box origin in padded coordinates: column x0 (= x0 - gx + gx), row y0
    // (= y0 - 3 + kGY).
    auto issue = [&](int tile, int b) {
        const int x0 = (tile % ntx) * L::TX, y0 = (tile / ntx) * L::TY;
        mbar_expect_tx(&bars[b], 2u * L::SPEC_BYTES);
        tma_load_3d(box(b), &tin, x0, y0, 0, &bars[b]);
        tma_load_3d(box(b) + L::SPEC_STRIDE / sizeof(T), &tin, x0, y0, 9, &bars[b]);
    };
    if (tid == 0 && (int)blockIdx.x < ntiles) issue(blockIdx.x, 0);

    double red[4] = {0.0, 0.0, 0.0, 0.0};
    bool bad = false;
    int k = 0;
    for (int tile = blockIdx.x; tile < ntiles; tile += gridDim.x, ++k) {
        const int b = k & 1;
        if (tid == 0 && tile + (int)gridDim.x < ntiles) {
            fence_proxy_async();   // earlier generic reads of box[b^1] before the async write
            issue(tile + gridDim.x, b ^ 1);
        }
        if (!mbar_wait_bounded(&bars[b], (k >> 1) & 1)) s_fail = 1;
        __syncthreads();
        if (s_fail) break;
        const int x0 = (tile % ntx) * L::TX, y0 = (tile / ntx) * L::TY;
        tile_body<P, false, V>(box(b), box(b) + L::SPEC_STRIDE / sizeof(T), srho, spsi, x0, y0,
                               a, red, bad, stage);
        __syncthreads();
        if (tid == 0 && x0 + L::TX <= g.nx && y0 + L::TY <= g.ny) {
            // padded coordinates of site (x0, y0): column x0 + gx, row y0 + kGY
            tma_store_3d(&tout, stage, x0 + L::GX, y0 + kGY, 0);
            tma_store_3d(&tout, stage + L::STAGE_SPEC / sizeof(T), x0 + L::GX, y0 + kGY, 9);
            bulk_commit();
        }
    }
    if (tid == 0) bulk_wait_all();
    if (s_fail) {
        if (tid == 0) {
            atomicOr(&a.st->err, ERR_TIMEOUT);
            // let copies in flight land before the CTA exits
            mbar_wait_bounded(&bars[k & 1], (k >> 1) & 1);
            mbar_wait_bounded(&bars[(k + 1) & 1], ((k + 1) >> 1) & 1);
        }
    }
    if (bad) atomicOr(&a.st->err, ERR_NONFINITE);
    if (V & 1) return;   // periodic: no wall sums; the host keeps the step count

    // Couette: wall momentum of this step, then the last CTA samples it.
    const long long t = *((volatile long long*)&a.st->t);
    block_sum4<L::NT>(red, s_red);
    if (tid == 0) {
        a.slots[2 * blockIdx.x] = red[0];
        a.slots[2 * blockIdx.x + 1] = red[1];
    }
    if (!last_cta_sum<L::NT>(a.st, a.slots, gridDim.x, 2, red, s_red, &s_last)) return;
    if (tid == 0) {
        const long long every = a.stress_every > 0 ? a.stress_every : 1;
        if (t >= a.stress_t0 && ((t - a.stress_t0) % every) == 0) {
            a.st->sum_bot += red[0] / g.nx;
            a.st->sum_top += red[1] / g.nx;
            a.st->samples += 1;
        }
        a.st->t = t + 1;
        a.st->ticket = 0u;
        __threadfence();
    }
}

// --------------------------------------------------------- observe kernel
// One CTA per tile: fields, populations or totals of the current state.
template <int P, int V>
__global__ void __launch_bounds__(Layout<P>::NT)
    k_observe(const __grid_constant__ CUtensorMap tin,
              const __grid_constant__ StepArgs<typename Prec<P>::C> a) {
    typedef Layout<P> L;
    typedef typename L::T T;
    typedef typename L::C C;
    extern __shared__ unsigned char smem_raw[];
    // 128-byte aligned base, derived from the shared array by indexing so
    // that every access below compiles to shared-memory instructions.
    unsigned char* smem = smem_raw + ((128u - (smem_u32(smem_raw) & 127u)) & 127u);
    T* sfA = reinterpret_cast<T*>(smem);
    C* srho = reinterpret_cast<C*>(smem + 2 * L::SPEC_STRIDE);
    C* spsi = srho + 2 * L::RX * L::RY;
    __shared__ __align__(8) uint64_t bar;
    __shared__ int s_fail, s_last;
    __shared__ double s_red[L::NT / 32][4];
    const int tid = threadIdx.x;
    const int x0 = blockIdx.x * L::TX, y0 = blockIdx.y * L::TY;
    if (tid == 0) {
        s_fail = 0;
        mbar_init(&bar, 1);
        fence_mbar_init();
        mbar_expect_tx(&bar, 2u * L::SPEC_BYTES);
        tma_load_3d(sfA, &tin, x0, y0, 0, &bar);
        tma_load_3d(sfA + L::SPEC_STRIDE / sizeof(T), &tin, x0, y0, 9, &bar);
    }
    __syncthreads();
    if (!mbar_wait_bounded(&bar, 0)) s_fail = 1;
    __syncthreads();
    double red[4] = {0.0, 0.0, 0.0, 0.0};
    bool bad = false;
    if (!s_fail) {
        tile_body<P, true, V>(sfA, sfA + L::SPEC_STRIDE / sizeof(T), srho, spsi, x0, y0, a, red,
                              bad, nullptr);
    } else if (tid == 0) {
        atomicOr(&a.st->err, ERR_TIMEOUT);
        mbar_wait_bounded(&bar, 0);
    }
    if (bad) atomicOr(&a.st->err, ERR_NONFINITE);
    block_sum4<L::NT>(red, s_red);
    const int bid = blockIdx.y * gridDim.x + blockIdx.x;
    if (tid == 0)
#pragma unroll
        for (int q = 0; q < 4; ++q) a.slots[4 * bid + q] = red[q];
    if (!last_cta_sum<L::NT>(a.st, a.slots, gridDim.x * gridDim.y, 4, red, s_red, &s_last))
        return;
    if (tid == 0) {
#pragma unroll
        for (int q = 0; q < 4; ++q) a.st->totals[q] = red[q];
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
template <int P, typename KS, typename KO>
static cudaError_t configure(KS ks, KO ko) {
    typedef Layout<P> L;
    cudaError_t e = cudaFuncSetAttribute(ks, cudaFuncAttributeMaxDynamicSharedMemorySize, L::SMEM);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(ko, cudaFuncAttributeMaxDynamicSharedMemorySize, L::SMEM_OBS);
    return e;
}

template <int P>
cudaError_t launch_step_prec(const CUtensorMap* tin, const CUtensorMap* tout, const void* args,
                             int obs, dim3 grid, cudaStream_t s) {
    typedef Layout<P> L;
    typedef typename L::C C;
    static int configured[64] = {0};
    int dev = 0;
    cudaGetDevice(&dev);
    if (dev < 64 && !configured[dev]) {
        cudaError_t e = configure<P>(k_step<P, 0>, k_observe<P, 2>);
        if (e == cudaSuccess) e = configure<P>(k_step<P, 1>, k_observe<P, 3>);
        if (e == cudaSuccess) e = configure<P>(k_step<P, 2>, k_observe<P, 2>);
        if (e == cudaSuccess) e = configure<P>(k_step<P, 3>, k_observe<P, 3>);
        if (e != cudaSuccess) return e;
        configured[dev] = 1;
    }
    const StepArgs<C>& a = *reinterpret_cast<const StepArgs<C>*>(args);
    const int v = (a.g.periodic ? 1 : 0) | ((a.k.source || a.k.has_accel) ? 2 : 0);
    if (obs == OBS_NONE) {
        switch (v) {
            case 0: k_step<P, 0><<<grid, L::NT, L::SMEM, s>>>(*tin, *tout, a); break;
            case 1: k_step<P, 1><<<grid, L::NT, L::SMEM, s>>>(*tin, *tout, a); break;
            case 2: k_step<P, 2><<<grid, L::NT, L::SMEM, s>>>(*tin, *tout, a); break;
            default: k_step<P, 3><<<grid, L::NT, L::SMEM, s>>>(*tin, *tout, a); break;
        }
    } else if (a.g.periodic) {
        k_observe<P, 3><<<grid, L::NT, L::SMEM_OBS, s>>>(*tin, a);
    } else {
        k_observe<P, 2><<<grid, L::NT, L::SMEM_OBS, s>>>(*tin, a);
    }
    return cudaGetLastError();
}

template <int P>
cudaError_t launch_init_prec(const Geom& g, const void* coef, void* fout, int mode,
                             const double* fields, double rho0, double amp, double u_wall,
                             int init_shear, unsigned long long seed, cudaStream_t s) {
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

#ifndef LB_PREC
#error "compile lb_kernels.cu once per storage precision with -DLB_PREC=0..3"
#endif
template cudaError_t launch_step_prec<LB_PREC>(const CUtensorMap*, const CUtensorMap*, const void*,
                                               int, dim3, cudaStream_t);
template cudaError_t launch_init_prec<LB_PREC>(const Geom&, const void*, void*, int, const double*,
                                               double, double, double, int, unsigned long long,
                                               cudaStream_t);

}  // namespace lbgb
