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

// The offsets h_i(r, t) of both species at lattice row y.  bm, b0, bp point
// at the site's pair in the staged rows y-1, y, y+1 of plane 0 (plane i is
// PS pairs further).  pull = 1: streamed from h*(r - c_i, t - 1), with
// halfway bounce-back at the Couette walls: f_i = f*_opp(i)(r)
// + 6 w_i rho_w (c_i . u_w), rho_w the pre-streaming density of the
// boundary node, rho_ref + sum_j h*_j(r).  pull = 0: the state in place.
template <int P, int PS>
__device__ __forceinline__ void load_site(const typename Prec<P>::T2* bm,
                                          const typename Prec<P>::T2* b0,
                                          const typename Prec<P>::T2* bp, int y, bool per,
                                          int pull, const Geom& g,
                                          const LatVals<typename Prec<P>::C>& v,
                                          typename Prec<P>::C hA[9], typename Prec<P>::C hB[9]) {
    typedef typename Prec<P>::C C;
    typedef typename Prec<P>::C2 C2;
    if (pull) {
#pragma unroll
        for (int i = 0; i < 9; ++i) {
            const typename Prec<P>::T2* r = cy(i) == 1 ? bm : (cy(i) == -1 ? bp : b0);
            const C2 q = dec2(r[i * PS - cx(i)]);
            hA[i] = q.x;
            hB[i] = q.y;
        }
        if (!per && (y == 0 || y == g.ny - 1)) {
            C sA[9], sB[9];
#pragma unroll
            for (int j = 0; j < 9; ++j) {
                const C2 q = dec2(b0[j * PS]);
                sA[j] = q.x;
                sB[j] = q.y;
            }
            const C rwA = v.rho_ref + sum9(sA), rwB = v.rho_ref + sum9(sB);
            const int up = (y == 0);                 // links arriving upward
            const C uw = up ? -v.u_wall : v.u_wall;
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
            const C2 q = dec2(b0[i * PS]);
            hA[i] = q.x;
            hB[i] = q.y;
        }
    }
}

// Deviation of the pseudo-potential from Psi(rho_ref):
// Psi(rho_ref + d) - Psi(rho_ref) = -P exp(-rho_ref/rho0) expm1(-d/rho0).
template <typename C>
__device__ __forceinline__ C dpsi_of(C d, const LatVals<C>& v) {
    return -v.psi_scale * cexpm1(-d * v.inv_rho0);
}

// Density and pseudo-potential deviations (rho - rho_ref, Psi - Psi(rho_ref))
// of both species at one site.
template <int P, int PS>
__device__ __forceinline__ void cell_dev(const typename Prec<P>::T2* bm,
                                         const typename Prec<P>::T2* b0,
                                         const typename Prec<P>::T2* bp, int y, bool per, int pull,
                                         const Geom& g, const LatVals<typename Prec<P>::C>& v,
                                         typename Prec<P>::C2& r, typename Prec<P>::C2& q) {
    typedef typename Prec<P>::C C;
    C hA[9], hB[9];
    load_site<P, PS>(bm, b0, bp, y, per, pull, g, v, hA, hB);
    r.x = sum9(hA);
    r.y = sum9(hB);
    q.x = dpsi_of(r.x, v);
    q.y = dpsi_of(r.y, v);
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

// Where a site update sends its result.
template <typename T2>
struct SiteOut {
    T2* stage;             // staging tile slot of the site (full tiles), or null
    T2* fout;              // output buffer (ragged tiles and ghost copies)
    int obs;               // ObsKind (observe kernel) or OBS_NONE
    double* obs_out;
    int q0, q1;
};

// One lattice site: moments, the force of Eq. (2) from the staged deviation
// rows, and either the forced BGK collision and write-back (OBS = false) or
// the observables (OBS = true).  ps[k] / rr[k]: Psi / rho deviation rows
// y + k - 2, pointing at the site's column.  red accumulates the bottom/top
// wall momentum (step) or mass_A, mass_B, mom_x, mom_y (observe).
template <int P, bool OBS, bool GEN, int PS>
__device__ __forceinline__ void site_update(
    const typename Prec<P>::T2* bm, const typename Prec<P>::T2* b0,
    const typename Prec<P>::T2* bp, const typename Prec<P>::C2* const ps[5],
    const typename Prec<P>::C2* const rr[5], int x, int y, bool per, int pull, const Geom& g,
    const LatVals<typename Prec<P>::C>& v, const Coef<typename Prec<P>::C>& k,
    const SiteOut<typename Prec<P>::T2>& o, double red[4], bool& bad) {
    typedef typename Prec<P>::T2 T2;
    typedef typename Prec<P>::C C;
    typedef typename Prec<P>::C2 C2;
    C h[2][9];
    load_site<P, PS>(bm, b0, bp, y, per, pull, g, v, h[0], h[1]);
    C drho[2], rho[2], jx[2], jy[2];
#pragma unroll
    for (int s = 0; s < 2; ++s) {
        drho[s] = sum9(h[s]);
        rho[s] = v.rho_ref + drho[s];
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
    C axA1 = C(0), ayA1 = C(0), axB1 = C(0), ayB1 = C(0);
    C axA2 = C(0), ayA2 = C(0), axB2 = C(0), ayB2 = C(0);
#pragma unroll
    for (int q = 0; q < 12; ++q) {
        const int dx = rdx(q), dy = rdy(q);
        const C2 pp = ps[2 + dy][dx], pm = ps[2 - dy][-dx];
        const C dA = pp.x - pm.x, dB = pp.y - pm.y;
        C& axA = q < 4 ? axA1 : axA2;
        C& ayA = q < 4 ? ayA1 : ayA2;
        C& axB = q < 4 ? axB1 : axB2;
        C& ayB = q < 4 ? ayB1 : ayB2;
        if (dx != 0) {
            axA += (k.K[0][q] * C(dx)) * dA;
            axB += (k.K[1][q] * C(dx)) * dB;
        }
        if (dy != 0) {
            ayA += (k.K[0][q] * C(dy)) * dA;
            ayB += (k.K[1][q] * C(dy)) * dB;
        }
    }
    C qxA = C(0), qyA = C(0), qxB = C(0), qyB = C(0);
#pragma unroll
    for (int q = 0; q < 4; ++q) {
        const int dx = rdx(q), dy = rdy(q);
        const C2 rp = rr[2 + dy][dx], rm = rr[2 - dy][-dx];
        const C dB = rp.y - rm.y, dA = rp.x - rm.x;   // A feels rho_B, B feels rho_A
        if (dx != 0) {
            qxA += (k.W[q] * C(dx)) * dB;
            qxB += (k.W[q] * C(dx)) * dA;
        }
        if (dy != 0) {
            qyA += (k.W[q] * C(dy)) * dB;
            qyB += (k.W[q] * C(dy)) * dA;
        }
    }
    const C2 pc = ps[2][0];
    const C pcA = v.psi_ref + pc.x, pcB = v.psi_ref + pc.y;
    C Fx[2], Fy[2];
    Fx[0] = -pcA * (axA1 + axA2) - v.gx_rho0 * rho[0] * qxA;
    Fy[0] = -pcA * (ayA1 + ayA2) - v.gx_rho0 * rho[0] * qyA;
    Fx[1] = -pcB * (axB1 + axB2) - v.gx_rho0 * rho[1] * qxB;
    Fy[1] = -pcB * (ayB1 + ayB2) - v.gx_rho0 * rho[1] * qyB;
    if (GEN && k.has_accel) {
        C acc = k.g_x;
        if (k.kolmo_amp != C(0)) acc += k.kolmo_amp * csin(k.kolmo_w * C(y));
        Fx[0] += rho[0] * acc;
        Fx[1] += rho[1] * acc;
    }

    if (OBS) {
        const long long N = (long long)g.nx * g.ny;
        const long long idx = (long long)y * g.nx + x;
        const double rA = (double)v.rho_ref + (double)drho[0];
        const double rB = (double)v.rho_ref + (double)drho[1];
        const double tot = rA + rB;
        const double mx = (double)jx[0] + (double)jx[1] + 0.5 * ((double)Fx[0] + (double)Fx[1]);
        const double my = (double)jy[0] + (double)jy[1] + 0.5 * ((double)Fy[0] + (double)Fy[1]);
        if (o.obs == OBS_FIELDS) {
            o.obs_out[idx] = rA;
            o.obs_out[N + idx] = rB;
            o.obs_out[2 * N + idx] = tot != 0.0 ? mx / tot : 0.0;
            o.obs_out[3 * N + idx] = tot != 0.0 ? my / tot : 0.0;
        } else if (o.obs == OBS_POPS) {
#pragma unroll
            for (int q = 0; q < 18; ++q)
                if (q >= o.q0 && q < o.q1)
                    o.obs_out[(long long)(q - o.q0) * N + idx] =
                        (double)h[q / 9][q % 9] + wgt<double>(q % 9) * (double)v.rho_ref;
        }
        red[0] += rA;
        red[1] += rB;
        red[2] += mx;
        red[3] += my;
        return;
    }

    // Eq. (1): forced BGK relaxation.  Common velocity
    // u' = sum_s (j_s/tau_s) / sum_s (rho_s/tau_s); shift u_s = u' + tau_s F_s/rho_s.
    const C den = rho[0] * k.omega[0] + rho[1] * k.omega[1];
    C upx = C(0), upy = C(0);
    if (den != C(0)) {
        const C inv = recip(den);
        upx = (jx[0] * k.omega[0] + jx[1] * k.omega[1]) * inv;
        upy = (jy[0] * k.omega[0] + jy[1] * k.omega[1]) * inv;
    }
    const bool source = GEN && k.source;
    C hs[2][9];
#pragma unroll
    for (int s = 0; s < 2; ++s) {
        C ux = upx, uy = upy;
        if (!source && rho[s] != C(0)) {
            const C tr = k.tau[s] * recip(rho[s]);
            ux += tr * Fx[s];
            uy += tr * Fy[s];
        }
        if (source)
            collide<C, true>(h[s], hs[s], drho[s], rho[s], ux, uy, k.omega[s], Fx[s], Fy[s]);
        else
            collide<C, false>(h[s], hs[s], drho[s], rho[s], ux, uy, k.omega[s], Fx[s], Fy[s]);
    }
    T2 e[9];
#pragma unroll
    for (int i = 0; i < 9; ++i) e[i] = enc2<T2, C>(hs[0][i], hs[1][i]);

    // Full tiles go through the staging tile and a bulk tensor store; ragged
    // tiles and periodic ghost copies use plain stores.
    constexpr int TX = Prec<P>::TX, TY = Prec<P>::TY;
    const int dX = (x < 3) ? g.nx : ((x >= g.nx - 3) ? -g.nx : 0);
    long long dY = 0;
    if (per) dY = (y < 3) ? (long long)g.ny * g.pitch : ((y >= g.ny - 3) ? -(long long)g.ny * g.pitch : 0);
    if (o.stage != nullptr) {
#pragma unroll
        for (int i = 0; i < 9; ++i) o.stage[i * TY * TX] = e[i];
    }
    if (o.stage == nullptr || dX != 0 || dY != 0) {
        const long long PL = (long long)g.rows * g.pitch;
        T2* __restrict__ out = o.fout + (long long)(y + kGY) * g.pitch + (x + g.gx);
#pragma unroll
        for (int i = 0; i < 9; ++i) {
            T2* d = out + i * PL;
            if (o.stage == nullptr) d[0] = e[i];
            if (dX) d[dX] = e[i];
            if (dY) {
                d[dY] = e[i];
                if (dX) d[dY + dX] = e[i];
            }
        }
    }
    if (!per && (y == 0 || y == g.ny - 1)) {
        // x-momentum handed to the wall by the links that will bounce back
        // at the next streaming: c_x (f*_i + f_opp), f_opp = f*_i - 6 w_i
        // rho_w (c_i . u_w), from the stored (rounded) values.
        const int down = (y == 0);
        const C uw = down ? -v.u_wall : v.u_wall;
        C sA[9], sB[9];
#pragma unroll
        for (int i = 0; i < 9; ++i) {
            const C2 q = dec2(e[i]);
            sA[i] = q.x;
            sB[i] = q.y;
        }
        const C rw[2] = {v.rho_ref + sum9(sA), v.rho_ref + sum9(sB)};
#pragma unroll
        for (int i = 0; i < 9; ++i) {
            if ((down && cy(i) == -1) || (!down && cy(i) == 1)) {
#pragma unroll
                for (int s = 0; s < 2; ++s) {
                    const C fi = (s ? sB[i] : sA[i]) + wgt<C>(i) * v.rho_ref;
                    const C back = fi - C(6) * wgt<C>(i) * rw[s] * (C(cx(i)) * uw);
                    const double dp = (double)(C(cx(i)) * (fi + back));
                    if (down) red[0] += dp; else red[1] += dp;
                }
            }
        }
    }
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

// ------------------------------------------------------------ step kernel
// Persistent and multi-lattice.  The work items of a launch are segments of
// TX-wide column strips, `seg` tiles (TY rows each) long, over all lattices
// (segment-major within a lattice, so that the CTAs in flight cover a band
// of rows and halo columns are shared through L2).  CTA b takes items
// b, b + gridDim.x, ...  Walking down a strip, a CTA keeps the 8-row blocks
// of f* (TMA-loaded into a ring of NB slots, one block ahead of use and
// across item boundaries) and the density/Psi deviation rows (a ring of 16
// rows), so each block is loaded and each deviation row computed once per
// strip; only the x halo (4 of 72 columns) is redundant.  Full tiles are
// written back by TMA bulk tensor stores.  The last CTA to finish advances
// every lattice's step counter and buffer parity and takes the Couette wall
// samples.
// V: bit 0 = every lattice periodic (no wall code); bit 1 = general forcing.
template <int P, int V>
__global__ void __launch_bounds__(Layout<P>::NT, 1)
    k_step(const __grid_constant__ BatchArgs<typename Prec<P>::C> a) {
    typedef Layout<P> L;
    typedef typename L::T2 T2;
    typedef typename L::C C;
    typedef typename L::C2 C2;
    constexpr bool ALLPER = (V & 1) != 0;
    constexpr bool GEN = (V & 2) != 0;
    constexpr int PS = L::TYB * L::BX;   // plane stride in a block slot (pairs)
    extern __shared__ unsigned char smem_raw[];
    // 128-byte aligned base, derived from the shared array by indexing so
    // that every access below compiles to shared-memory instructions.
    unsigned char* smem = smem_raw + ((128u - (smem_u32(smem_raw) & 127u)) & 127u);
    C2* ring_r = reinterpret_cast<C2*>(smem + L::RING_OFF);   // [RING][RX]
    C2* ring_p = ring_r + L::RING * L::RX;                    // [RING][RX]
    T2* stage = reinterpret_cast<T2*>(smem + L::STAGE_OFF);   // [9][TY][TX]
    __shared__ __align__(8) uint64_t bars[L::NB];
    __shared__ int s_fail, s_last;
    __shared__ double s_red[L::NT / 32][4];

    const int tid = threadIdx.x;
    const int G = gridDim.x;
    auto slot = [&](int pos) { return reinterpret_cast<T2*>(smem + (pos % L::NB) * L::SLOT_BYTES); };
    // descriptor of the lattice that owns work item it (descriptors sorted by item0)
    auto find = [&](int it) {
        int lo = 0, hi = a.nlat - 1;
        while (lo < hi) {
            const int mid = (lo + hi + 1) >> 1;
            if (a.lat[mid].item0 <= it) lo = mid; else hi = mid - 1;
        }
        return &a.lat[lo];
    };

    if (tid == 0) {
        s_fail = 0;
        for (int b = 0; b < L::NB; ++b) mbar_init(&bars[b], 1);
        fence_mbar_init();
    }
    __syncthreads();

    // Producer (thread 0): the blocks of this CTA's items, in order.  Item
    // tiles [ty_a, ty_b) need blocks ty_a .. ty_b (block j = padded rows
    // [8j, 8j + 8)); consecutive items' blocks follow each other.
    int p_item = blockIdx.x, p_j = 0, p_pos = 0;
    // cached geometry of the producer's current item
    const CUtensorMap* p_map = nullptr;
    int p_x0 = 0, p_ty_a = 0, p_nblk = 0;
    auto p_load = [&]() {
        if (p_item >= a.nitems) return;
        const LatDesc<C>* d = find(p_item);
        const int local = p_item - d->item0;
        p_x0 = (local % d->nstrips) * L::TX;
        p_ty_a = (local / d->nstrips) * d->seg;
        p_nblk = min(p_ty_a + d->seg, d->ntiles_y) - p_ty_a + 1;
        p_map = &d->tin[*((volatile int*)&d->st->cur)];
    };
    auto issue_next = [&]() -> bool {
        if (p_item >= a.nitems) return false;
        uint64_t* bar = &bars[p_pos % L::NB];
        mbar_expect_tx(bar, (uint32_t)L::SLOT_BYTES);
        // box origin: pair column x0 (= x0 - gx + gx) -> element 2 x0; padded row 8j
        tma_load_3d(slot(p_pos), p_map, 2 * p_x0, L::TYB * (p_ty_a + p_j), 0, bar);
        ++p_pos;
        if (++p_j == p_nblk) {
            p_j = 0;
            p_item += G;
            p_load();
        }
        return true;
    };
    if (tid == 0) p_load();
    if (tid == 0)
        while (p_pos < L::NB && issue_next()) {}

    double red[4] = {0.0, 0.0, 0.0, 0.0};
    bool bad = false;
    int c_pos = 0;   // ring position of the current item's first block
    for (int it = blockIdx.x; it < a.nitems && !s_fail; it += G) {
        const LatDesc<C>* d = find(it);
        const int local = it - d->item0;
        const int x0 = (local % d->nstrips) * L::TX;
        const int ty_a = (local / d->nstrips) * d->seg;
        const int ty_b = min(ty_a + d->seg, d->ntiles_y);
        const Geom g = d->g;
        const LatVals<C> v = d->v;
        const bool per = ALLPER || g.periodic;
        const int cur = *((volatile int*)&d->st->cur);
        const int pull = *((volatile int*)&d->st->pull);
        T2* fout = reinterpret_cast<T2*>(d->fbuf[cur ^ 1]);
        auto rrow = [&](C2* ring, int y) { return ring + ((y + L::RING) & (L::RING - 1)) * L::RX; };
        double wall[2] = {0.0, 0.0};
        for (int ty = ty_a; ty < ty_b; ++ty) {
            const int q = c_pos + (ty - ty_a);   // this tile uses blocks q and q + 1
            // each thread sees the blocks land itself; a timeout is acted on
            // after the next barrier (garbage read meanwhile is harmless)
            if (!mbar_wait_bounded(&bars[q % L::NB], (q / L::NB) & 1) ||
                !mbar_wait_bounded(&bars[(q + 1) % L::NB], ((q + 1) / L::NB) & 1))
                s_fail = 1;
            const int y0 = ty * L::TY;
            // The tile's padded rows [8 ty, 8 ty + 16) are blocks q (slot s0) and
            // q + 1 (slot s1); row pointers address plane 0.
            const T2* s0 = slot(q);
            const T2* s1 = slot(q + 1);
            auto brow = [&](int R, int c) {
                const int r = R - L::TYB * ty;
                return (r < L::TYB ? s0 + r * L::BX : s1 + (r - L::TYB) * L::BX) + c;
            };

            // Phase 2: deviation rows new to this tile (all 12 at an item's start).
            const int r_lo = (ty == ty_a) ? y0 - 2 : y0 + 2;
            const int ncell = (y0 + L::TY + 2 - r_lo) * L::RX;
            for (int c = tid; c < ncell; c += L::NT) {
                const int ly = c / L::RX, lx = c - ly * L::RX;
                const int y = r_lo + ly;
                if (!per && (y < 0 || y >= g.ny)) continue;
                const int bc = lx - 2 + L::GX;   // pair column in the block
                const int R = y + kGY;
                C2 r, p;
                cell_dev<P, PS>(brow(R - 1, bc), brow(R, bc), brow(R + 1, bc), y, per, pull, g, v,
                                r, p);
                rrow(ring_r, y)[lx] = r;
                rrow(ring_p, y)[lx] = p;
            }
            if (!per) {   // mirror the deviations about the halfway walls
                __syncthreads();
                for (int c = tid; c < ncell; c += L::NT) {
                    const int ly = c / L::RX, lx = c - ly * L::RX;
                    const int y = r_lo + ly;
                    int ym;
                    if (y < 0) ym = -1 - y;
                    else if (y >= g.ny && y <= g.ny + 1) ym = 2 * g.ny - 1 - y;
                    else continue;
                    rrow(ring_r, y)[lx] = rrow(ring_r, ym)[lx];
                    rrow(ring_p, y)[lx] = rrow(ring_p, ym)[lx];
                }
            }
            if (tid == 0) bulk_wait_read();   // previous bulk store has read the staging tile
            __syncthreads();
            if (s_fail) break;

            // Phase 3: one site per thread (lx < TX).
            const bool full = x0 + L::TX <= g.nx && y0 + L::TY <= g.ny;
            {
                const int lx = tid % L::RX, ly = tid / L::RX;
                const int x = x0 + lx, y = y0 + ly;
                if (lx < L::TX && x < g.nx && y < g.ny) {
                    const int bc = lx + L::GX;
                    const int R = y + kGY;
                    const C2* ps[5];
                    const C2* rr[5];
#pragma unroll
                    for (int k2 = 0; k2 < 5; ++k2) {
                        ps[k2] = rrow(ring_p, y + k2 - 2) + lx + 2;
                        rr[k2] = rrow(ring_r, y + k2 - 2) + lx + 2;
                    }
                    SiteOut<T2> o;
                    o.stage = full ? stage + ly * L::TX + lx : nullptr;
                    o.fout = fout;
                    o.obs = OBS_NONE;
                    double wr[4] = {0.0, 0.0, 0.0, 0.0};
                    site_update<P, false, GEN, PS>(brow(R - 1, bc), brow(R, bc), brow(R + 1, bc),
                                                   ps, rr, x, y, per, pull, g, v, a.k, o, wr, bad);
                    wall[0] += wr[0];
                    wall[1] += wr[1];
                    if (full) fence_proxy_async();   // staging writes before the bulk store
                }
            }
            __syncthreads();
            if (tid == 0) {
                if (full) {
                    // site (x0, y0) in padded coordinates: pair column x0 + gx, row y0 + kGY
                    tma_store_3d(&d->tout[cur ^ 1], stage, 2 * (x0 + L::GX), y0 + kGY, 0);
                    bulk_commit();
                }
                // blocks before the next tile's first block are free
                const int released = (ty + 1 < ty_b) ? q + 1 : q + 2;
                fence_proxy_async();   // generic reads of freed slots before async writes
                while (p_pos < released + L::NB && issue_next()) {}
            }
        }
        if (bad) {   // a density of this lattice went non-finite
            atomicOr(&d->st->err, ERR_NONFINITE);
            bad = false;
        }
        if (s_fail) break;
        c_pos += (ty_b - ty_a) + 1;
        if (!per) {   // wall momentum of this item (zero unless it holds a wall row)
            red[0] = wall[0];
            red[1] = wall[1];
            red[2] = red[3] = 0.0;
            block_sum4<L::NT>(red, s_red);
            if (tid == 0) {
                a.slots[2 * it] = red[0];
                a.slots[2 * it + 1] = red[1];
            }
        }
    }
    if (tid == 0) bulk_wait_all();
    if (s_fail && tid == 0) {
        // let copies in flight land before the CTA exits
        for (int b = 0; b < L::NB; ++b) mbar_wait_bounded(&bars[b], 0), mbar_wait_bounded(&bars[b], 1);
    }
    if (s_fail && tid == 0)   // report on every lattice of the launch
        for (int l = 0; l < a.nlat; ++l) atomicOr(&a.lat[l].st->err, ERR_TIMEOUT);

    // The last CTA advances every lattice and takes the wall samples.
    if (tid == 0) {
        __threadfence();
        s_last = atomicAdd(a.ticket, 1u) == (unsigned int)(G - 1);
    }
    __syncthreads();
    if (!s_last) return;
    __threadfence();
    for (int l = tid; l < a.nlat; l += L::NT) {
        const LatDesc<C>* d = &a.lat[l];
        DevStats* st = d->st;
        const long long t = st->t;
        if (!ALLPER && !d->g.periodic) {
            const int n = d->nstrips * ((d->ntiles_y + d->seg - 1) / d->seg);
            const volatile double* vs = a.slots + 2 * d->item0;
            double sb = 0.0, stp = 0.0;
            for (int i = 0; i < n; ++i) {
                sb += vs[2 * i];
                stp += vs[2 * i + 1];
            }
            const long long every = d->stress_every > 0 ? d->stress_every : 1;
            if (t >= d->stress_t0 && ((t - d->stress_t0) % every) == 0) {
                st->sum_bot += sb / d->g.nx;
                st->sum_top += stp / d->g.nx;
                st->samples += 1;
            }
        }
        st->t = t + 1;
        st->cur ^= 1;
        st->pull = 1;
    }
    __threadfence();
    if (tid == 0) *a.ticket = 0u;
}

// --------------------------------------------------------- observe kernel
// One CTA per tile of one lattice: fields, populations or totals of the
// current state, with the same site arithmetic as the step.
template <int P, int V>
__global__ void __launch_bounds__(Layout<P>::NT)
    k_observe(const __grid_constant__ CUtensorMap tin,
              const __grid_constant__ StepArgs<typename Prec<P>::C> a) {
    typedef Layout<P> L;
    typedef typename L::T2 T2;
    typedef typename L::C C;
    typedef typename L::C2 C2;
    constexpr bool GEN = (V & 2) != 0;
    constexpr int PS = L::BY * L::BX;    // plane stride in the tile box (pairs)
    extern __shared__ unsigned char smem_raw[];
    unsigned char* smem = smem_raw + ((128u - (smem_u32(smem_raw) & 127u)) & 127u);
    T2* box = reinterpret_cast<T2*>(smem);                    // [9][BY][BX]
    C2* srho = reinterpret_cast<C2*>(smem + L::BOX_STRIDE);   // [RY][RX]
    C2* spsi = srho + L::RX * L::RY;
    __shared__ __align__(8) uint64_t bar;
    __shared__ int s_fail, s_last;
    __shared__ double s_red[L::NT / 32][4];
    const int tid = threadIdx.x;
    const int x0 = blockIdx.x * L::TX, y0 = blockIdx.y * L::TY;
    const Geom& g = a.g;
    const bool per = g.periodic != 0;
    LatVals<C> v;
    v.rho_ref = a.k.rho_ref;
    v.psi_ref = a.k.psi_ref;
    v.psi_scale = a.k.psi_scale;
    v.inv_rho0 = a.k.inv_rho0;
    v.gx_rho0 = a.k.gx_rho0;
    v.u_wall = a.k.u_wall;
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
        // box row of lattice row y: y - y0 + kGY; deviation tile row: y - y0 + 2
        for (int c = tid; c < L::RX * L::RY; c += L::NT) {
            const int ly = c / L::RX, lx = c - ly * L::RX;
            const int y = y0 - 2 + ly;
            if (!per && (y < 0 || y >= g.ny)) continue;
            const T2* b0 = box + (ly + 1) * L::BX + lx - 2 + L::GX;
            C2 r, p;
            cell_dev<P, PS>(b0 - L::BX, b0, b0 + L::BX, y, per, a.pull, g, v, r, p);
            srho[ly * L::RX + lx] = r;
            spsi[ly * L::RX + lx] = p;
        }
        if (!per) {
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
        __syncthreads();
        const int lx = tid % L::RX, ly = tid / L::RX;
        const int x = x0 + lx, y = y0 + ly;
        if (lx < L::TX && x < g.nx && y < g.ny) {
            const T2* b0 = box + (ly + kGY) * L::BX + lx + L::GX;
            const C2* ps[5];
            const C2* rr[5];
#pragma unroll
            for (int k2 = 0; k2 < 5; ++k2) {
                ps[k2] = spsi + (ly + k2) * L::RX + lx + 2;
                rr[k2] = srho + (ly + k2) * L::RX + lx + 2;
            }
            SiteOut<T2> o;
            o.stage = nullptr;
            o.fout = nullptr;
            o.obs = a.obs;
            o.obs_out = a.obs_out;
            o.q0 = a.q0;
            o.q1 = a.q1;
            site_update<P, true, GEN, PS>(b0 - L::BX, b0, b0 + L::BX, ps, rr, x, y, per, a.pull, g,
                                          v, a.k, o, red, bad);
        }
    } else if (tid == 0) {
        atomicOr(&a.st->err, ERR_TIMEOUT);
        mbar_wait_bounded(&bar, 0);
    }
    if (bad) atomicOr(&a.st->err, ERR_NONFINITE);
    block_sum4<L::NT>(red, s_red);
    const int bid = blockIdx.y * gridDim.x + blockIdx.x;
    if (tid == 0) {
#pragma unroll
        for (int q = 0; q < 4; ++q) a.slots[4 * bid + q] = red[q];
        __threadfence();
        s_last = atomicAdd(&a.st->ticket, 1u) == gridDim.x * gridDim.y - 1;
    }
    __syncthreads();
    if (!s_last) return;
    __threadfence();
    const int nb = gridDim.x * gridDim.y;
    const volatile double* vs = a.slots;
    double w[4] = {0.0, 0.0, 0.0, 0.0};
    for (int b = tid; b < nb; b += L::NT)
#pragma unroll
        for (int q = 0; q < 4; ++q) w[q] += vs[4 * b + q];
#pragma unroll
    for (int q = 0; q < 4; ++q) red[q] = w[q];
    block_sum4<L::NT>(red, s_red);
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

// Restore directions [i0, i1) of a saved state: pops holds FP64 populations
// f_is(r) of those directions as [i1 - i0][2][ny][nx]; the offsets
// f - w_i rho_ref are encoded to the storage format (plus ghost copies).
template <int P>
__global__ void k_load_pops(Geom g, typename Prec<P>::C rho_ref, typename Prec<P>::T2* fout,
                            const double* pops, int i0, int i1) {
    typedef typename Prec<P>::T2 T2;
    const long long N = (long long)g.nx * g.ny;
    const double rref = (double)rho_ref;
    for (long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x; idx < N;
         idx += (long long)gridDim.x * blockDim.x) {
        const int x = (int)(idx % g.nx), y = (int)(idx / g.nx);
        for (int i = i0; i < i1; ++i) {
            const double* src = pops + (long long)(i - i0) * 2 * N;
            const double off = wgt<double>(i) * rref;
            put2<T2>(fout, g, i, x, y, encd2<T2>(src[idx] - off, src[N + idx] - off));
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

// Opt every kernel of this precision into its dynamic shared memory, once
// per device.
template <int P>
static cudaError_t ensure_configured() {
    static int configured[64] = {0};
    int dev = 0;
    cudaGetDevice(&dev);
    if (dev >= 0 && dev < 64 && configured[dev]) return cudaSuccess;
    cudaError_t e = configure<P>(k_step<P, 0>, k_observe<P, 2>);
    if (e == cudaSuccess) e = configure<P>(k_step<P, 1>, k_observe<P, 3>);
    if (e == cudaSuccess) e = configure<P>(k_step<P, 2>, k_observe<P, 2>);
    if (e == cudaSuccess) e = configure<P>(k_step<P, 3>, k_observe<P, 3>);
    if (e == cudaSuccess && dev >= 0 && dev < 64) configured[dev] = 1;
    return e;
}

template <int P>
cudaError_t launch_step_prec(const void* args, int variant, dim3 grid, cudaStream_t s) {
    typedef Layout<P> L;
    typedef typename L::C C;
    cudaError_t e = ensure_configured<P>();
    if (e != cudaSuccess) return e;
    const BatchArgs<C>& a = *reinterpret_cast<const BatchArgs<C>*>(args);
    switch (variant & 3) {
        case 0: k_step<P, 0><<<grid, L::NT, L::SMEM, s>>>(a); break;
        case 1: k_step<P, 1><<<grid, L::NT, L::SMEM, s>>>(a); break;
        case 2: k_step<P, 2><<<grid, L::NT, L::SMEM, s>>>(a); break;
        default: k_step<P, 3><<<grid, L::NT, L::SMEM, s>>>(a); break;
    }
    return cudaGetLastError();
}

template <int P>
cudaError_t launch_observe_prec(const CUtensorMap* tin, const void* args, dim3 grid,
                                cudaStream_t s) {
    typedef Layout<P> L;
    typedef typename L::C C;
    cudaError_t e = ensure_configured<P>();
    if (e != cudaSuccess) return e;
    const StepArgs<C>& a = *reinterpret_cast<const StepArgs<C>*>(args);
    if (a.g.periodic)
        k_observe<P, 3><<<grid, L::NT, L::SMEM_OBS, s>>>(*tin, a);
    else
        k_observe<P, 2><<<grid, L::NT, L::SMEM_OBS, s>>>(*tin, a);
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
template <int P>
cudaError_t configure_prec() {
    return ensure_configured<P>();
}

template cudaError_t configure_prec<LB_PREC>();
template cudaError_t launch_step_prec<LB_PREC>(const void*, int, dim3, cudaStream_t);
template cudaError_t launch_observe_prec<LB_PREC>(const CUtensorMap*, const void*, dim3,
                                                  cudaStream_t);
template <int P>
cudaError_t launch_load_pops_prec(const Geom& g, const void* coef, void* fout, const double* pops,
                                  int i0, int i1, cudaStream_t s) {
    typedef typename Prec<P>::C C;
    typedef typename Prec<P>::T2 T2;
    const long long N = (long long)g.nx * g.ny;
    long long blocks = (N + 255) / 256;
    if (blocks > 152 * 64) blocks = 152 * 64;
    k_load_pops<P><<<(unsigned)blocks, 256, 0, s>>>(
        g, reinterpret_cast<const Coef<C>*>(coef)->rho_ref, reinterpret_cast<T2*>(fout), pops, i0, i1);
    return cudaGetLastError();
}

template cudaError_t launch_load_pops_prec<LB_PREC>(const Geom&, const void*, void*, const double*,
                                                    int, int, cudaStream_t);
template cudaError_t launch_init_prec<LB_PREC>(const Geom&, const void*, void*, int, const double*,
                                               double, double, double, int, unsigned long long,
                                               cudaStream_t);

}  // namespace lbgb
