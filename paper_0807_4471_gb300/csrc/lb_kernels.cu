// lb_kernels.cu -- sm_103a kernels of the two-species multi-range
// pseudo-potential lattice Boltzmann step (Benzi, Chibbaro & Succi,
// arXiv:0807.4471, Eqs. (1)-(2)).
//
// One launch of k_step advances every site of the lattice by one time step.
// Layout in HBM: 9 direction planes, each a ghost-padded [ny + 6][pitch]
// array of interleaved (A, B) pairs of the storage type, holding offsets
// h_i = f_i - w_i rho_ref.  The buffer read by a step holds the
// post-collision populations f*(t-1) of the previous step; streaming is a
// pull, f_i(r, t) = f*_i(r - c_i, t - 1).
//
// k_step is persistent: one CTA per SM walks the TX x TY tiles.  Per tile:
//  1. TMA: one 3-D box load brings f* on the tile plus a 3-cell halo (both
//     species, 9 planes) into shared memory; the next tile's box loads into
//     the second buffer meanwhile.  The ghost columns/rows of the padded
//     planes hold periodic copies, so a box never wraps.
//  2. density and pseudo-potential deviations on the tile plus a 2-cell halo
//     (halfway bounce-back at Couette walls; mirrored beyond a wall).
//  3. one site per thread: moments, the force of Eq. (2) from the shared
//     tiles (12 antisymmetric pairs of the 24-neighbour stencil, 4 pairs of
//     the cross term), the forced BGK relaxation of Eq. (1) into a staging
//     tile, written back by a TMA bulk tensor store (plus ghost copies).
//  4. Couette: FP64 wall-momentum sums, per-CTA slots, last CTA samples.
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
// Pair (A, B) of plane i at site (x, y) in the padded global buffer, in
// units of pairs: row stride `pitch`, plane stride rows * pitch.
template <typename T2>
__device__ __forceinline__ void put2(T2* base, const Geom& g, int i, int x, int y, T2 v) {
    const long long pl = (long long)g.rows * g.pitch;
    T2* p = base + i * pl + (long long)(y + kGY) * g.pitch + (x + g.gx);
    const int dX = (x < 3) ? g.nx : ((x >= g.nx - 3) ? -g.nx : 0);
    long long dY = 0;
    if (g.periodic) dY = (y < 3) ? (long long)g.ny * g.pitch : ((y >= g.ny - 3) ? -(long long)g.ny * g.pitch : 0);
    p[0] = v;
    if (dX) p[dX] = v;
    if (dY) {
        p[dY] = v;
        if (dX) p[dY + dX] = v;
    }
}

template <typename C>
__device__ __forceinline__ C sum9(const C h[9]) {
    return ((h[0] + h[1]) + (h[2] + h[3])) + ((h[4] + h[5]) + (h[6] + h[7])) + h[8];
}

// The offsets h_i(r, t) of both species at lattice site (x, y), whose box
// coordinates are (sx, sy).  pull = 1: streamed from h*(r - c_i, t - 1), with
// halfway bounce-back at the Couette walls: f_i = f*_opp(i)(r)
// + 6 w_i rho_w (c_i . u_w), rho_w the pre-streaming density of the
// boundary node, rho_ref + sum_j h*_j(r).
template <int P, bool PER>
__device__ __forceinline__ void load_site(const typename Prec<P>::T2* box, int sx, int sy, int y,
                                          const StepArgs<typename Prec<P>::C>& a,
                                          typename Prec<P>::C hA[9], typename Prec<P>::C hB[9]) {
    typedef Layout<P> L;
    typedef typename Prec<P>::C C;
    typedef typename Prec<P>::C2 C2;
    if (a.pull) {
#pragma unroll
        for (int i = 0; i < 9; ++i) {
            const C2 v = dec2(box[(i * L::BY + sy - cy(i)) * L::BX + sx - cx(i)]);
            hA[i] = v.x;
            hB[i] = v.y;
        }
        if (!PER && (y == 0 || y == a.g.ny - 1)) {
            C sA[9], sB[9];
#pragma unroll
            for (int j = 0; j < 9; ++j) {
                const C2 v = dec2(box[(j * L::BY + sy) * L::BX + sx]);
                sA[j] = v.x;
                sB[j] = v.y;
            }
            const C rwA = a.k.rho_ref + sum9(sA), rwB = a.k.rho_ref + sum9(sB);
            const int up = (y == 0);                 // links arriving upward
            const C uw = up ? -a.k.u_wall : a.k.u_wall;
#pragma unroll
            for (int i = 0; i < 9; ++i) {
                if ((up && cy(i) == 1) || (!up && cy(i) == -1)) {
                    const C m = C(6) * wgt<C>(i) * (C(cx(i)) * uw);
                    hA[i] = sA[opp(i)] + m * rwA;
                    hB[i] = sB[opp(i)] + m * rwB;
                }
            }
        }
    } else {
#pragma unroll
        for (int i = 0; i < 9; ++i) {
            const C2 v = dec2(box[(i * L::BY + sy) * L::BX + sx]);
            hA[i] = v.x;
            hB[i] = v.y;
        }
    }
}

// Deviation of the pseudo-potential from Psi(rho_ref):
// Psi(rho_ref + d) - Psi(rho_ref) = -P exp(-rho_ref/rho0) expm1(-d/rho0).
template <typename C>
__device__ __forceinline__ C dpsi_of(C d, const Coef<C>& k) {
    return -k.psi_scale * cexpm1(-d * k.inv_rho0);
}

// Post-collision offsets of one species (Eq. (1), BGK toward the
// equilibrium at velocity (ux, uy)):
// h*_i = h_i + omega (heq_i - h_i) [+ 3 w_i c_i . F for the source scheme],
// heq_i = f^eq_i - w_i rho_ref = w_i [d_rho + rho (3 c.u + 4.5 (c.u)^2 - 1.5 u^2)],
// evaluated per pair (i, opp(i)), whose c.u differ only in sign:
// heq = E +- O with E = w (d_rho - 1.5 rho u^2 + 4.5 rho (c.u)^2), O = 3 w rho c.u.
template <typename C, bool SRC>
__device__ __forceinline__ void collide(const C h[9], C out[9], C drho, C rho, C ux, C uy,
                                        C om, C Fx, C Fy) {
    const C Q = drho - rho * (C(1.5) * (ux * ux + uy * uy));
    out[0] = h[0] + om * (wgt<C>(0) * Q - h[0]);
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        const int i = k == 0 ? 1 : (k == 1 ? 2 : (k == 2 ? 5 : 6));   // c.u = ux, uy, ux+uy, uy-ux
        const int j = opp(i);
        const C cu = C(cx(i)) * ux + C(cy(i)) * uy;
        const C w = wgt<C>(i);
        const C rcu = rho * cu;
        const C E = w * (Q + C(4.5) * cu * rcu);
        const C O = (C(3) * w) * rcu;
        out[i] = h[i] + om * ((E + O) - h[i]);
        out[j] = h[j] + om * ((E - O) - h[j]);
        if (SRC) {
            const C S = (C(3) * w) * (C(cx(i)) * Fx + C(cy(i)) * Fy);
            out[i] += S;
            out[j] -= S;
        }
    }
}

// ------------------------------------------------------------- tile body
// Phases 2-3 for one TX x TY tile whose f* box is in shared memory.
// OBS = false: collision and write-back of f*(t) (+ wall momentum into red).
// OBS = true : fields / populations / totals of the current state (red =
//              mass_A, mass_B, mom_x, mom_y).
// V: bit 0 = periodic in y (else Couette walls); bit 1 = general forcing
// (additive source term or body acceleration checked at run time).
template <int P, bool OBS, int V>
__device__ __forceinline__ void tile_body(const typename Prec<P>::T2* __restrict__ box,
                                          typename Prec<P>::C2* __restrict__ srho,
                                          typename Prec<P>::C2* __restrict__ spsi, int x0, int y0,
                                          const StepArgs<typename Prec<P>::C>& a, double red[4],
                                          bool& bad, typename Prec<P>::T2* __restrict__ stage) {
    typedef Layout<P> L;
    typedef typename L::T2 T2;
    typedef typename L::C C;
    typedef typename L::C2 C2;
    constexpr bool PER = (V & 1) != 0;
    constexpr bool GEN = (V & 2) != 0;
    const int tid = threadIdx.x;
    const Geom& g = a.g;

    // 2. density and pseudo-potential deviations d_rho = rho - rho_ref,
    // d_Psi = Psi(rho) - Psi(rho_ref), on the tile + 2-cell halo.
    for (int c = tid; c < L::RX * L::RY; c += L::NT) {
        const int ly = c / L::RX, lx = c - ly * L::RX;
        const int y = y0 - 2 + ly;
        if (!PER && (y < 0 || y >= g.ny)) continue;
        C hA[9], hB[9];
        load_site<P, PER>(box, lx - 2 + L::GX, ly - 2 + kGY, y, a, hA, hB);
        const C rA = sum9(hA), rB = sum9(hB);
        C2 r, q;
        r.x = rA;
        r.y = rB;
        q.x = dpsi_of(rA, a.k);
        q.y = dpsi_of(rB, a.k);
        srho[ly * L::RX + lx] = r;
        spsi[ly * L::RX + lx] = q;
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
            srho[ly * L::RX + lx] = srho[lm * L::RX + lx];
            spsi[ly * L::RX + lx] = spsi[lm * L::RX + lx];
        }
    }
    // the previous tile's bulk store must have read the staging tile
    if (stage != nullptr && tid == 0) bulk_wait_read();
    __syncthreads();

    // 3. one site per thread: moments, forces, collision, write-back.
    const int lx = tid % L::TX, ly = tid / L::TX;
    const int x = x0 + lx, y = y0 + ly;
    if (x >= g.nx || y >= g.ny) return;
    C h[2][9];
    load_site<P, PER>(box, lx + L::GX, ly + kGY, y, a, h[0], h[1]);
    C drho[2], rho[2], jx[2], jy[2];
#pragma unroll
    for (int s = 0; s < 2; ++s) {
        drho[s] = sum9(h[s]);
        rho[s] = a.k.rho_ref + drho[s];
        // sum_i w_i c_i = 0, so the offsets carry all of j
        const C d57 = h[s][5] - h[s][7], d68 = h[s][6] - h[s][8];
        jx[s] = (h[s][1] - h[s][3]) + (d57 - d68);
        jy[s] = (h[s][2] - h[s][4]) + (d57 + d68);
    }
    if (!(isfinite(rho[0]) && isfinite(rho[1]))) bad = true;

    // Eq. (2): F_s = -Psi_s(r) sum_d K_s(d) d [Psi_s(r+d) - Psi_s(r-d)]
    //               - (G_X/rho0) rho_s(r) sum_d w(d) d [rho_s'(r+d) - rho_s'(r-d)]
    // over one representative d of each +-d pair (the reference values cancel
    // in the differences); belt-1 and belt-2 pairs accumulate separately.
    const int c0 = (ly + 2) * L::RX + (lx + 2);
    C axA1 = C(0), ayA1 = C(0), axB1 = C(0), ayB1 = C(0);
    C axA2 = C(0), ayA2 = C(0), axB2 = C(0), ayB2 = C(0);
#pragma unroll
    for (int k = 0; k < 12; ++k) {
        const int dx = rdx(k), dy = rdy(k);
        const C2 pp = spsi[c0 + dy * L::RX + dx], pm = spsi[c0 - dy * L::RX - dx];
        const C dA = pp.x - pm.x, dB = pp.y - pm.y;
        C& axA = k < 4 ? axA1 : axA2;
        C& ayA = k < 4 ? ayA1 : ayA2;
        C& axB = k < 4 ? axB1 : axB2;
        C& ayB = k < 4 ? ayB1 : ayB2;
        if (dx != 0) {
            axA += (a.k.K[0][k] * C(dx)) * dA;
            axB += (a.k.K[1][k] * C(dx)) * dB;
        }
        if (dy != 0) {
            ayA += (a.k.K[0][k] * C(dy)) * dA;
            ayB += (a.k.K[1][k] * C(dy)) * dB;
        }
    }
    C qxA = C(0), qyA = C(0), qxB = C(0), qyB = C(0);
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        const int dx = rdx(k), dy = rdy(k);
        const C2 rp = srho[c0 + dy * L::RX + dx], rm = srho[c0 - dy * L::RX - dx];
        const C dB = rp.y - rm.y, dA = rp.x - rm.x;   // A feels rho_B, B feels rho_A
        if (dx != 0) {
            qxA += (a.k.W[k] * C(dx)) * dB;
            qxB += (a.k.W[k] * C(dx)) * dA;
        }
        if (dy != 0) {
            qyA += (a.k.W[k] * C(dy)) * dB;
            qyB += (a.k.W[k] * C(dy)) * dA;
        }
    }
    const C2 pc = spsi[c0];
    const C pcA = a.k.psi_ref + pc.x, pcB = a.k.psi_ref + pc.y;
    C Fx[2], Fy[2];
    Fx[0] = -pcA * (axA1 + axA2) - a.k.gx_rho0 * rho[0] * qxA;
    Fy[0] = -pcA * (ayA1 + ayA2) - a.k.gx_rho0 * rho[0] * qyA;
    Fx[1] = -pcB * (axB1 + axB2) - a.k.gx_rho0 * rho[1] * qxB;
    Fy[1] = -pcB * (ayB1 + ayB2) - a.k.gx_rho0 * rho[1] * qyB;
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

    // Eq. (1): forced BGK relaxation.  Common velocity
    // u' = sum_s (j_s/tau_s) / sum_s (rho_s/tau_s); shift u_s = u' + tau_s F_s/rho_s.
    const C den = rho[0] * a.k.omega[0] + rho[1] * a.k.omega[1];
    C upx = C(0), upy = C(0);
    if (den != C(0)) {
        const C inv = recip(den);
        upx = (jx[0] * a.k.omega[0] + jx[1] * a.k.omega[1]) * inv;
        upy = (jy[0] * a.k.omega[0] + jy[1] * a.k.omega[1]) * inv;
    }
    const bool source = GEN && a.k.source;
    C hs[2][9];
#pragma unroll
    for (int s = 0; s < 2; ++s) {
        C ux = upx, uy = upy;
        if (!source && rho[s] != C(0)) {
            const C tr = a.k.tau[s] * recip(rho[s]);
            ux += tr * Fx[s];
            uy += tr * Fy[s];
        }
        if (source)
            collide<C, true>(h[s], hs[s], drho[s], rho[s], ux, uy, a.k.omega[s], Fx[s], Fy[s]);
        else
            collide<C, false>(h[s], hs[s], drho[s], rho[s], ux, uy, a.k.omega[s], Fx[s], Fy[s]);
    }
    T2 e[9];
#pragma unroll
    for (int i = 0; i < 9; ++i) e[i] = enc2<T2, C>(hs[0][i], hs[1][i]);

    // Full tiles go through the staging tile and a bulk tensor store; ragged
    // tiles and periodic ghost copies use plain stores.
    const bool staged = stage != nullptr && x0 + L::TX <= g.nx && y0 + L::TY <= g.ny;
    const int dX = (x < 3) ? g.nx : ((x >= g.nx - 3) ? -g.nx : 0);
    long long dY = 0;
    if (PER) dY = (y < 3) ? (long long)g.ny * g.pitch : ((y >= g.ny - 3) ? -(long long)g.ny * g.pitch : 0);
    if (staged) {
#pragma unroll
        for (int i = 0; i < 9; ++i) stage[(i * L::TY + ly) * L::TX + lx] = e[i];
    }
    if (!staged || dX != 0 || dY != 0) {
        const long long PL = (long long)g.rows * g.pitch;
        T2* __restrict__ out =
            reinterpret_cast<T2*>(a.fout) + (long long)(y + kGY) * g.pitch + (x + g.gx);
#pragma unroll
        for (int i = 0; i < 9; ++i) {
            T2* o = out + i * PL;
            if (!staged) o[0] = e[i];
            if (dX) o[dX] = e[i];
            if (dY) {
                o[dY] = e[i];
                if (dX) o[dY + dX] = e[i];
            }
        }
    }
    if (!PER && (y == 0 || y == g.ny - 1)) {
        // x-momentum handed to the wall by the links that will bounce back
        // at the next streaming: c_x (f*_i + f_opp), f_opp = f*_i - 6 w_i
        // rho_w (c_i . u_w), from the stored (rounded) values.
        const int down = (y == 0);
        const C uw = down ? -a.k.u_wall : a.k.u_wall;
        C sA[9], sB[9];
#pragma unroll
        for (int i = 0; i < 9; ++i) {
            const C2 v = dec2(e[i]);
            sA[i] = v.x;
            sB[i] = v.y;
        }
        const C rw[2] = {a.k.rho_ref + sum9(sA), a.k.rho_ref + sum9(sB)};
#pragma unroll
        for (int i = 0; i < 9; ++i) {
            if ((down && cy(i) == -1) || (!down && cy(i) == 1)) {
#pragma unroll
                for (int s = 0; s < 2; ++s) {
                    const C fi = (s ? sB[i] : sA[i]) + wgt<C>(i) * a.k.rho_ref;
                    const C back = fi - C(6) * wgt<C>(i) * rw[s] * (C(cx(i)) * uw);
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
__device__ __forceinline__ bool last_cta_sum(DevStats* st, const double* slots, int nslots,
                                             int width, double red[4], double (*s_red)[4],
                                             int* s_last) {
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
// computed; full tiles are written back by bulk tensor stores.
template <int P, int V>
__global__ void __launch_bounds__(Layout<P>::NT, 1)
    k_step(const __grid_constant__ CUtensorMap tin, const __grid_constant__ CUtensorMap tout,
           const __grid_constant__ StepArgs<typename Prec<P>::C> a) {
    typedef Layout<P> L;
    typedef typename L::T2 T2;
    typedef typename L::C2 C2;
    extern __shared__ unsigned char smem_raw[];
    // 128-byte aligned base, derived from the shared array by indexing so
    // that every access below compiles to shared-memory instructions.
    unsigned char* smem = smem_raw + ((128u - (smem_u32(smem_raw) & 127u)) & 127u);
    auto box = [&](int b) { return reinterpret_cast<T2*>(smem + b * L::BOX_STRIDE); };
    C2* srho = reinterpret_cast<C2*>(smem + 2 * L::BOX_STRIDE);   // [RY][RX]
    C2* spsi = srho + L::RX * L::RY;                              // [RY][RX]
    T2* stage = reinterpret_cast<T2*>(smem + L::STAGE_OFF);       // [9][TY][TX]
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
    // Box origin in padded coordinates: site column x0 (= x0 - gx + gx), i.e.
    // element 2 x0 of the interleaved rows, and row y0 (= y0 - 3 + kGY).
    auto issue = [&](int tile, int b) {
        const int x0 = (tile % ntx) * L::TX, y0 = (tile / ntx) * L::TY;
        mbar_expect_tx(&bars[b], (uint32_t)L::BOX_BYTES);
        tma_load_3d(box(b), &tin, 2 * x0, y0, 0, &bars[b]);
    };
    if (tid == 0 && (int)blockIdx.x < ntiles) issue(blockIdx.x, 0);

    double red[4] = {0.0, 0.0, 0.0, 0.0};
    bool bad = false;
    int k = 0;
    for (int tile = blockIdx.x; tile < ntiles; tile += gridDim.x, ++k) {
        const int b = k & 1;
        if (tid == 0 && tile + (int)gridDim.x < ntiles) {
            fence_proxy_async();   // earlier generic reads of box b^1 before the async write
            issue(tile + gridDim.x, b ^ 1);
        }
        if (!mbar_wait_bounded(&bars[b], (k >> 1) & 1)) s_fail = 1;
        __syncthreads();
        if (s_fail) break;
        const int x0 = (tile % ntx) * L::TX, y0 = (tile / ntx) * L::TY;
        tile_body<P, false, V>(box(b), srho, spsi, x0, y0, a, red, bad, stage);
        __syncthreads();
        if (tid == 0 && x0 + L::TX <= g.nx && y0 + L::TY <= g.ny) {
            // padded coordinates of site (x0, y0): pair column x0 + gx, row y0 + kGY
            tma_store_3d(&tout, stage, 2 * (x0 + L::GX), y0 + kGY, 0);
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
    typedef typename L::T2 T2;
    typedef typename L::C2 C2;
    extern __shared__ unsigned char smem_raw[];
    unsigned char* smem = smem_raw + ((128u - (smem_u32(smem_raw) & 127u)) & 127u);
    T2* box = reinterpret_cast<T2*>(smem);
    C2* srho = reinterpret_cast<C2*>(smem + L::BOX_STRIDE);
    C2* spsi = srho + L::RX * L::RY;
    __shared__ __align__(8) uint64_t bar;
    __shared__ int s_fail, s_last;
    __shared__ double s_red[L::NT / 32][4];
    const int tid = threadIdx.x;
    const int x0 = blockIdx.x * L::TX, y0 = blockIdx.y * L::TY;
    if (tid == 0) {
        s_fail = 0;
        mbar_init(&bar, 1);
        fence_mbar_init();
        mbar_expect_tx(&bar, (uint32_t)L::BOX_BYTES);
        tma_load_3d(box, &tin, 2 * x0, y0, 0, &bar);
    }
    __syncthreads();
    if (!mbar_wait_bounded(&bar, 0)) s_fail = 1;
    __syncthreads();
    double red[4] = {0.0, 0.0, 0.0, 0.0};
    bool bad = false;
    if (!s_fail) {
        tile_body<P, true, V>(box, srho, spsi, x0, y0, a, red, bad, nullptr);
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
__global__ void k_init(Geom g, Coef<typename Prec<P>::C> k, typename Prec<P>::T2* fout, int mode,
                       const double* fields, double rho0, double amp, double u_wall, int init_shear,
                       unsigned long long seed) {
    typedef typename Prec<P>::T2 T2;
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
#pragma unroll
        for (int i = 0; i < 9; ++i) {
            const double cu = cx(i) * ux + cy(i) * uy;
            const double e = 3.0 * cu + 4.5 * cu * cu - 1.5 * usq;
            // f^eq_i - w_i rho_ref for both species
            const double hA = wgt<double>(i) * ((r[0] - rref) + r[0] * e);
            const double hB = wgt<double>(i) * ((r[1] - rref) + r[1] * e);
            put2<T2>(fout, g, i, x, y, encd2<T2>(hA, hB));
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
    typedef typename Prec<P>::T2 T2;
    const long long N = (long long)g.nx * g.ny;
    long long blocks = (N + 255) / 256;
    if (blocks > 152 * 64) blocks = 152 * 64;
    k_init<P><<<(unsigned)blocks, 256, 0, s>>>(g, *reinterpret_cast<const Coef<C>*>(coef),
                                               reinterpret_cast<T2*>(fout), mode, fields, rho0, amp,
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
