// lb_kernels.cu -- sm_103a kernels of the two-species multi-range
// pseudo-potential lattice Boltzmann step (Benzi, Chibbaro & Succi,
// arXiv:0807.4471, Eqs. (1)-(2)).
//
// One launch of k_step advances every site of a set of lattices by one time
// step.  Layout in HBM: 9 direction planes, each a ghost-padded
// [ny + 6][pitch] array of interleaved (A, B) pairs of the storage type,
// holding offsets h_i = f_i - w_i rho_ref.  The buffer read by a step holds
// the post-collision populations f*(t-1) of the previous step; streaming is
// a pull, f_i(r, t) = f*_i(r - c_i, t - 1).
//
// k_step is persistent: one CTA per SM walks its work items (a lattice's
// strip of TX x TY tiles, one after the other).  Per tile:
//  1. TMA: 3-D box loads bring f* in 8-row blocks (both species, 9 planes,
//     the strip plus its ghost columns) into a ring of shared-memory slots,
//     several blocks ahead.  The ghost columns/rows of the padded planes
//     hold periodic copies, so a box never wraps.
//  2. density phase: density and pseudo-potential deviations on the tile
//     plus a 2-row halo (halfway bounce-back at Couette walls; mirrored
//     beyond a wall), and at tau = 1 the momenta of the tile's sites.
//  3. site phase, one or two sites per thread: the force of Eq. (2) from the
//     shared deviation window (row sums of the 24-neighbour stencil and of
//     the cross term), the forced BGK relaxation of Eq. (1), the write-back
//     (staging tile + TMA bulk tensor store, or direct stores) and the
//     periodic ghost copies.
//  4. Couette: the wall sites' momentum exchange, summed per strip in FP64
//     after the tile loop; the last CTA takes the wall samples.
// There is no dense contraction anywhere, so no tensor cores are used.
#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include <cstdint>
#include <cstdlib>
#include <type_traits>

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
// The same box load, and the bulk tensor store of a shared-memory box to
// global memory (bulk group), with an L2 cache policy (createpolicy).
__device__ __forceinline__ void tma_load_3d_hint(void* dst, const CUtensorMap* map, int x, int y,
                                                 int z, uint64_t* bar, uint64_t policy) {
    asm volatile(
        "cp.async.bulk.tensor.3d.shared::cluster.global.mbarrier::complete_tx::bytes.L2::cache_hint"
        " [%0], [%1, {%2, %3, %4}], [%5], %6;" ::"r"(smem_u32(dst)),
        "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(z), "r"(smem_u32(bar)),
        "l"(policy)
        : "memory");
}
__device__ __forceinline__ void tma_store_3d_hint(const CUtensorMap* map, const void* src, int x,
                                                  int y, int z, uint64_t policy) {
    asm volatile(
        "cp.async.bulk.tensor.3d.global.shared::cta.bulk_group.L2::cache_hint"
        " [%0, {%2, %3, %4}], [%1], %5;" ::"l"(reinterpret_cast<uint64_t>(map)),
        "r"(smem_u32(src)), "r"(x), "r"(y), "r"(z), "l"(policy)
        : "memory");
}
__device__ __forceinline__ uint64_t policy_evict_last() {
    uint64_t p;
    asm volatile("createpolicy.fractional.L2::evict_last.b64 %0, 1.0;" : "=l"(p));
    return p;
}
__device__ __forceinline__ uint64_t policy_evict_first() {
    uint64_t p;
    asm volatile("createpolicy.fractional.L2::evict_first.b64 %0, 1.0;" : "=l"(p));
    return p;
}
__device__ __forceinline__ uint64_t policy_evict_normal() {
    uint64_t p;
    asm volatile("createpolicy.fractional.L2::evict_normal.b64 %0, 1.0;" : "=l"(p));
    return p;
}
__device__ __forceinline__ void bulk_commit() { asm volatile("cp.async.bulk.commit_group;" ::: "memory"); }
// Wait until the committed bulk stores have finished reading shared memory.
__device__ __forceinline__ void bulk_wait_read() {
    asm volatile("cp.async.bulk.wait_group.read 0;" ::: "memory");
}
// Wait until the committed bulk stores have completed.
__device__ __forceinline__ void bulk_wait_all() { asm volatile("cp.async.bulk.wait_group 0;" ::: "memory"); }
// Programmatic dependent launch: wait for the grids this one depends on to
// complete (their writes visible), and let this grid's dependents be
// scheduled onto SMs as this grid's CTAs retire.  Both are no-ops when the
// launch carries no programmatic dependency.
__device__ __forceinline__ void griddep_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
__device__ __forceinline__ void griddep_launch_dependents() {
    asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
}

// Arrival at a launch's CTA counter: the old count, with release semantics
// for this CTA's writes (made ordered before by a CTA barrier) and acquire
// semantics for those of the CTAs that arrived before, at GPU scope.
__device__ __forceinline__ unsigned int ticket_arrive(unsigned int* ticket) {
    unsigned int old;
    asm volatile("atom.add.acq_rel.gpu.u32 %0, [%1], 1;" : "=r"(old) : "l"(ticket) : "memory");
    return old;
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
// default bound is a few seconds at most.
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t* bar, uint32_t parity,
                                                  int limit = 1 << 22) {
    for (int it = 0; it < limit; ++it)
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

// ((h0 + h1) + (h2 + h3)) + ((h4 + h5) + (h6 + h7)) + h8, per species.
template <typename C2>
__device__ __forceinline__ C2 sum9(const C2 h[9]) {
    return padd(padd(padd(padd(h[0], h[1]), padd(h[2], h[3])), padd(padd(h[4], h[5]), padd(h[6], h[7]))),
                h[8]);
}

// The offsets h_i(r, t) of both species at lattice row y, as (A, B) pairs,
// in the storage scale of precision P.
// bm, b0, bp point at the site's pair in the staged rows y-1, y, y+1 of
// plane 0 (plane i is PS pairs further).  pull = 1: streamed from
// h*(r - c_i, t - 1), with halfway bounce-back at the Couette walls:
// f_i = f*_opp(i)(r) + 6 w_i rho_w (c_i . u_w), rho_w the pre-streaming
// density of the boundary node, rho_ref + sum_j h*_j(r).  pull = 0: the
// state in place.
template <int P, int PS>
__device__ __forceinline__ void load_site(const typename Prec<P>::T2* bm,
                                          const typename Prec<P>::T2* b0,
                                          const typename Prec<P>::T2* bp, int y, bool per,
                                          int pull, const Geom& g,
                                          const LatVals<typename Prec<P>::C>& v,
                                          typename Prec<P>::C2 h[9]) {
    typedef typename Prec<P>::C C;
    typedef typename Prec<P>::C2 C2;
    if (pull) {
#pragma unroll
        for (int i = 0; i < 9; ++i) {
            const typename Prec<P>::T2* r = cy(i) == 1 ? bm : (cy(i) == -1 ? bp : b0);
            h[i] = dec2(r[i * PS - cx(i)]);
        }
        if (!per && (y == 0 || y == g.ny - 1)) {
            C2 sv[9];
#pragma unroll
            for (int j = 0; j < 9; ++j) sv[j] = dec2(b0[j * PS]);
            const C2 rw = pfma(sum9(sv), pset(inv_scale_of<P>()), pset(v.rho_ref));
            const int up = (y == 0);                 // links arriving upward
            const C uw = up ? -v.u_wall : v.u_wall;
#pragma unroll
            for (int i = 0; i < 9; ++i) {
                if ((up && cy(i) == 1) || (!up && cy(i) == -1)) {
                    const C m = scale_of<P>() * C(6) * wgt<C>(i) * (C(cx(i)) * uw);
                    h[i] = pfma(pset(m), rw, sv[opp(i)]);
                }
            }
        }
    } else {
#pragma unroll
        for (int i = 0; i < 9; ++i) h[i] = dec2(b0[i * PS]);
    }
}

// Deviation of the pseudo-potential from Psi(rho_ref), both species:
// Psi(rho_ref + d) - Psi(rho_ref) = -P exp(-rho_ref/rho0) expm1(-d/rho0).
template <typename C, typename C2>
__device__ __forceinline__ C2 dpsi_of(C2 d, const LatVals<C>& v) {
    return pmul(pset(-v.psi_scale), pexpm1(pmul(d, pset(-v.inv_rho0))));
}

// Momentum j = sum_i c_i f_i of both species from the offsets (sum_i w_i c_i
// = 0, so the offsets carry all of j), in the compute scale.
// SCALED = false: left in the storage scale (the caller folds the scale,
// a power of two, into a later factor).
template <int P, bool SCALED = true>
__device__ __forceinline__ void moments(const typename Prec<P>::C2 h[9], typename Prec<P>::C2& jx,
                                        typename Prec<P>::C2& jy) {
    typedef typename Prec<P>::C2 C2;
    const C2 d57 = psub(h[5], h[7]), d68 = psub(h[6], h[8]);
    jx = padd(psub(h[1], h[3]), psub(d57, d68));
    jy = padd(psub(h[2], h[4]), padd(d57, d68));
    if constexpr (SCALED && Prec<P>::SCALE_LOG2 != 0) {
        jx = pmul(jx, pset(inv_scale_of<P>()));
        jy = pmul(jy, pset(inv_scale_of<P>()));
    }
}

// Density and pseudo-potential deviations (rho - rho_ref, Psi - Psi(rho_ref))
// of both species at one site; with J, also the site's momentum, in the
// storage scale.
template <int P, int PS, bool J = false>
__device__ __forceinline__ void cell_dev(const typename Prec<P>::T2* bm,
                                         const typename Prec<P>::T2* b0,
                                         const typename Prec<P>::T2* bp, int y, bool per, int pull,
                                         const Geom& g, const LatVals<typename Prec<P>::C>& v,
                                         typename Prec<P>::C2& r, typename Prec<P>::C2& q,
                                         typename Prec<P>::C2* j = nullptr) {
    typename Prec<P>::C2 h[9];
    load_site<P, PS>(bm, b0, bp, y, per, pull, g, v, h);
    r = sum9(h);
    if constexpr (Prec<P>::SCALE_LOG2 != 0) r = pmul(r, pset(inv_scale_of<P>()));
    q = dpsi_of(r, v);
    if constexpr (J) moments<P, false>(h, j[0], j[1]);
}

// Post-collision offsets of both species (Eq. (1), BGK toward the
// equilibrium at velocity u, per species), written with v = 3u:
//   h*_i = (1 - omega) h_i + omega heq_i [+ 3 w_i c_i . F for the source scheme],
//   heq_i = f^eq_i - w_i rho_ref = w_i [d_rho + rho (3 c.u + 4.5 (c.u)^2 - 1.5 u^2)]
//         = w_i [Q + rho (c.v) + rho (c.v)^2 / 2],  Q = d_rho - rho v^2 / 6,
// evaluated per pair (i, opp(i)), whose c.v differ only in sign:
// heq = w (g +- rho c.v) with g = Q + rho (c.v)^2 / 2.  h and out are in
// the storage scale SC (a power of two); k.omw holds omega SC w per class
// of |c|^2 and k.omm = 1 - omega.
// TAU1: omega = 1 for both species, where h*_i = heq_i and h is not read.
//
// TAU1 (omega = 1): h*_i = heq_i, taken per class c of |c_i|^2 as
//   h*_{i, opp(i)} = E +- kv,  E = T_c + kv (c.v) / 2,  kv = K_c (c.v),
// with T_c = omega S w_c Q and K_c = omega S w_c rho per site; h is not read.
template <typename C, typename C2, bool SRC, bool TAU1 = false>
__device__ __forceinline__ void collide(const C2 h[9], C2 out[9], C2 drho, C2 rho, C2 vx, C2 vy,
                                        const Coef<C>& k, C2 Fx, C2 Fy, C SC) {
    const C2 Q = pfma(pmul(rho, pset(C(-1) / C(6))), pfma(vx, vx, pmul(vy, vy)), drho);
    out[0] = TAU1 ? pmul(k.omw[0], Q) : pfma(k.omw[0], Q, pmul(k.omm, h[0]));
    C2 T[2], K[2];
    if (TAU1) {
        T[0] = pmul(k.omw[1], Q);
        T[1] = pmul(k.omw[2], Q);
        K[0] = pmul(k.omw[1], rho);
        K[1] = pmul(k.omw[2], rho);
    }
#pragma unroll
    for (int q = 0; q < 4; ++q) {
        const int i = q == 0 ? 1 : (q == 1 ? 2 : (q == 2 ? 5 : 6));   // c.v = vx, vy, vx+vy, vy-vx
        const int j = opp(i);
        const C2 cv = q == 0 ? vx : (q == 1 ? vy : (q == 2 ? padd(vx, vy) : psub(vy, vx)));
        if (TAU1) {
            const C2 kv = pmul(K[q >> 1], cv);
            const C2 E = pfma(kv, pmul(cv, pset(C(0.5))), T[q >> 1]);
            out[i] = padd(E, kv);
            out[j] = psub(E, kv);
        } else {
            const C2 ow = k.omw[q < 2 ? 1 : 2];
            const C2 rv = pmul(rho, cv);
            const C2 g = pfma(rv, pmul(cv, pset(C(0.5))), Q);
            out[i] = pfma(ow, padd(g, rv), pmul(k.omm, h[i]));
            out[j] = pfma(ow, psub(g, rv), pmul(k.omm, h[j]));
        }
        if (SRC) {
            const C w3 = C(3) * SC * wgt<C>(i);
            const C2 S = pmul(pset(w3), pfma(pset(C(cx(i))), Fx, pmul(pset(C(cy(i))), Fy)));
            out[i] = padd(out[i], S);
            out[j] = psub(out[j], S);
        }
    }
}

// ------------------------------------------------------- force of Eq. (2)
// The stencil sums of Eq. (2) are taken row by row.  For the stencil row at
// vertical offset dy of a site, with the row's deviations q(dx), dx = -2..2
// (Psi for the like-species terms, rho for the cross term), and weights
// K(d) that depend on |d|^2 = dx^2 + dy^2 only:
//   sum_dx K(d) d_x q(dx) = K(1,|dy|) [q(1) - q(-1)] + 2 K(2,|dy|) [q(2) - q(-2)],
//   sum_dx K(d) d_y q(dx) = dy [K(0,|dy|) q(0) + K(1,|dy|) (q(1) + q(-1))
//                              + K(2,|dy|) (q(2) + q(-2))].
// (The reference values of Psi and rho drop out: sum_d K(d) d = 0.)  The
// differences and sums of a row are shared by every site whose stencil
// holds the row; each site adds its rows in a fixed order (x: dy = -2 .. 2;
// y: the rows above minus the rows below, each part in the order of dy), so
// a site's force is the same whether it shares rows with another or not.

// The shared quantities of one stencil row, p at the site's column.
template <typename C2>
struct Row5 {
    C2 d1, d2, s1, s2, q0;
};
template <typename C2>
__device__ __forceinline__ Row5<C2> row5(const C2* p) {
    const C2 m2 = p[-2], m1 = p[-1], q0 = p[0], p1 = p[1], p2 = p[2];
    Row5<C2> r;
    r.d1 = psub(p1, m1);
    r.d2 = psub(p2, m2);
    r.s1 = padd(p1, m1);
    r.s2 = padd(p2, m2);
    r.q0 = q0;
    return r;
}
template <typename C2>
struct Row3 {
    C2 e, t, q0;
};
template <typename C2>
__device__ __forceinline__ Row3<C2> row3(const C2* p) {
    const C2 m1 = p[-1], q0 = p[0], p1 = p[1];
    Row3<C2> r;
    r.e = psub(p1, m1);
    r.t = padd(p1, m1);
    r.q0 = q0;
    return r;
}

// Like-species row at offset dy (|dy| <= 2) into the x and y sums, with the
// weights KC = {K(1), K(2), K(5), 2K(4), 2K(5), 2K(8)}: x takes
// K(1,|dy|) = K(1), K(2), K(5) and 2K(2,|dy|) = 2K(4), 2K(5), 2K(8) for
// |dy| = 0, 1, 2; y takes {K(1), K(2), K(5)} for |dy| = 1 and
// {2K(4), 2K(5), 2K(8)} for |dy| = 2.  The y sum is kept as two chains,
// rows below the site (fyn: dy = -2, -1) and above it (fyp: dy = 1, 2),
// each started by its first row; fy = fyp - fyn.
template <typename C, typename C2>
__device__ __forceinline__ void like_row(int dy, const Row5<C2>& r, const Coef<C>& k, C2& fx,
                                         C2& fyp, C2& fyn) {
    const int a = dy < 0 ? -dy : dy;
    fx = pfma(a == 0 ? k.KC[0] : (a == 1 ? k.KC[1] : k.KC[2]), r.d1, fx);
    fx = pfma(a == 0 ? k.KC[3] : (a == 1 ? k.KC[4] : k.KC[5]), r.d2, fx);
    if (a != 0) {
        C2& t = dy > 0 ? fyp : fyn;
        const C2 K0 = a == 1 ? k.KC[0] : k.KC[3];
        t = (dy == -2 || dy == 1) ? pmul(K0, r.q0) : pfma(K0, r.q0, t);
        t = pfma(a == 1 ? k.KC[1] : k.KC[4], r.s1, t);
        t = pfma(a == 1 ? k.KC[2] : k.KC[5], r.s2, t);
    }
}
// Cross-species row at offset dy (|dy| <= 1), D2Q9 weights WC = {w(1), w(2)};
// qy is taken as qyp - qyn, the rows above and below.
template <typename C, typename C2>
__device__ __forceinline__ void cross_row(int dy, const Row3<C2>& r, const Coef<C>& k, C2& qx,
                                          C2& qyp, C2& qyn) {
    qx = pfma(dy == 0 ? k.WC[0] : k.WC[1], r.e, qx);
    if (dy != 0) {
        C2& u = dy > 0 ? qyp : qyn;
        u = pfma(k.WC[1], r.t, pmul(k.WC[0], r.q0));
    }
}

// Stencil sums of NS vertically adjacent sites.  ps, rr: the Psi and rho
// deviation rows (row stride RXS) at the sites' column, starting two rows
// above the first site.  Out, per site s: fx, fy = sum_d K_s(d) d Psi_s(r+d),
// qx, qy = sum_d w(d) d rho_s(r+d) (species not yet swapped), and the site's
// own Psi and rho deviations.
template <int NS, int RXS, typename C, typename C2>
__device__ __forceinline__ void force_sums(const C2* ps, const C2* rr, const Coef<C>& k, C2 fx[NS],
                                           C2 fy[NS], C2 qx[NS], C2 qy[NS], C2 dpsi[NS],
                                           C2 drho[NS]) {
    const C2 z = pset(C(0));
    C2 fyp[NS], fyn[NS], qyp[NS], qyn[NS];
#pragma unroll
    for (int s = 0; s < NS; ++s) fx[s] = qx[s] = z;
#pragma unroll
    for (int r = 0; r < NS + 4; ++r) {
        const Row5<C2> w = row5(ps + r * RXS);
#pragma unroll
        for (int s = 0; s < NS; ++s) {
            const int dy = r - 2 - s;
            if (dy >= -2 && dy <= 2) like_row(dy, w, k, fx[s], fyp[s], fyn[s]);
            if (dy == 0) dpsi[s] = w.q0;
        }
    }
#pragma unroll
    for (int r = 1; r < NS + 3; ++r) {
        const Row3<C2> w = row3(rr + r * RXS);
#pragma unroll
        for (int s = 0; s < NS; ++s) {
            const int dy = r - 2 - s;
            if (dy >= -1 && dy <= 1) cross_row(dy, w, k, qx[s], qyp[s], qyn[s]);
            if (dy == 0) drho[s] = w.q0;
        }
    }
#pragma unroll
    for (int s = 0; s < NS; ++s) {
        fy[s] = psub(fyp[s], fyn[s]);
        qy[s] = psub(qyp[s], qyn[s]);
    }
}

// Plain global stores of a stored pair, with an L2 cache policy.
__device__ __forceinline__ void st_pair(float2* p, float2 v, uint64_t pol) {
    asm volatile("st.global.L2::cache_hint.v2.f32 [%0], {%1, %2}, %3;" ::"l"(p), "f"(v.x), "f"(v.y),
                 "l"(pol));
}
__device__ __forceinline__ void st_pair(double2* p, double2 v, uint64_t pol) {
    asm volatile("st.global.L2::cache_hint.v2.f64 [%0], {%1, %2}, %3;" ::"l"(p), "d"(v.x), "d"(v.y),
                 "l"(pol));
}
template <typename T2>
__device__ __forceinline__ void st_pair(T2* p, T2 v, uint64_t pol) {   // 16-bit pairs
    static_assert(sizeof(T2) == 4, "a pair of 16-bit values");
    asm volatile("st.global.L2::cache_hint.b32 [%0], %1, %2;" ::"l"(p),
                 "r"(*reinterpret_cast<const uint32_t*>(&v)), "l"(pol));
}

// Random word of site (x, y) for the stochastic rounding of its stored
// pairs, from key, the hash of the lattice's step: sites (x, 2m) and
// (x, 2m + 1) share one hash of (x, 2m) -- the second site takes it times an
// odd constant (a bijection, so each word is uniform) -- whichever thread
// updates them.
__device__ __forceinline__ uint32_t sr_hash(uint32_t key, int x, int y, int nx) {
    return hash32(key ^ (uint32_t)((y & ~1) * nx + x));
}
__device__ __forceinline__ uint32_t sr_word(uint32_t h, int y) {
    return (y & 1) ? h * 0x2c1b3c6du : h;
}

// Where a site update sends its result.
enum SiteSink : int { SINK_STAGE = 0, SINK_GLOBAL = 1 };
template <typename T2>
struct SiteOut {
    T2* stage;             // SINK_STAGE: staging tile slot of the site (plane 0)
    T2* gout;              // SINK_GLOBAL: the site's pair in plane 0 of the output buffer
    long long plane;       // SINK_GLOBAL: plane stride (pairs)
    long long gdy;         // SINK_GLOBAL: offset of the periodic image in y (0: none)
    int gdx;               // SINK_GLOBAL: offset of the periodic image in x (0: none)
    uint64_t pol;          // SINK_GLOBAL: L2 policy of the stores
    uint32_t rbits;        // stochastic rounding: the site's random word (sr_word)
    int valid;             // 0: a site beyond the lattice, computed only to keep
                           // the site updates of a thread free of branches:
                           // its global stores and non-finite flag are dropped
    int obs;               // ObsKind (observe kernel) or OBS_NONE
    void* wallx;           // step: the lattice's wall-momentum pairs, [2][nx] compute type
    double* obs_out;
    int q0, q1;
};

// One lattice site, given its force sums: moments from its pulled
// populations, the force of Eq. (2), and either the forced BGK collision and
// write-back (OBS = false) or the observables (OBS = true).  Both species are
// carried as (A, B) pairs throughout.  TAU1 (omega = 1 for both species,
// OBS = false): the collision needs the populations only through j, which the
// caller passes in jg = {jx, jy} (in the storage scale); bm, b0 and bp are
// not read.  Non-finite densities: the step (OBS = false) accumulates
// 0 * rho into *nf, which turns NaN at an inf or NaN density and stays zero
// otherwise; the observables set `bad`.
template <int P, bool OBS, bool GEN, int PS, int SINK, bool TAU1 = false>
__device__ __forceinline__ void site_update(
    const typename Prec<P>::T2* bm, const typename Prec<P>::T2* b0,
    const typename Prec<P>::T2* bp, typename Prec<P>::C2 fxl, typename Prec<P>::C2 fyl,
    typename Prec<P>::C2 qx, typename Prec<P>::C2 qy, typename Prec<P>::C2 dpsi,
    typename Prec<P>::C2 drho, int x, int y, bool per, int pull, const Geom& g,
    const LatVals<typename Prec<P>::C>& v, const Coef<typename Prec<P>::C>& k,
    const SiteOut<typename Prec<P>::T2>& o, double red[4], bool& bad,
    typename Prec<P>::C2* nf = nullptr, const typename Prec<P>::C2* jg = nullptr) {
    typedef typename Prec<P>::T2 T2;
    typedef typename Prec<P>::C C;
    typedef typename Prec<P>::C2 C2;
    static_assert(!(TAU1 && OBS), "the observables read the populations");
    C2 h[9];
    C2 jx, jy;
    if constexpr (TAU1) {
        jx = jg[0];
        jy = jg[1];
    } else {
        load_site<P, PS>(bm, b0, bp, y, per, pull, g, v, h);
        moments<P>(h, jx, jy);
    }
    const C2 rho = padd(pset(v.rho_ref), drho);
    if constexpr (OBS) {
        if (o.valid && !(isfinite(rho.x) && isfinite(rho.y))) bad = true;
    } else if (o.valid) {
        *nf = pfma(rho, pset(C(0)), *nf);   // stays zero unless a density is inf or NaN
    }

    // Eq. (2): F_s = -Psi_s(r) sum_d K_s(d) d Psi_s(r + d)
    //               - (G_X/rho0) rho_s(r) sum_d w(d) d rho_s'(r + d);
    // species A feels rho_B, so the cross sums are used swapped.
    const C2 npc = psub(pset(-v.psi_ref), dpsi);          // -Psi_s(r)
    const C2 ng = pmul(pset(-v.gx_rho0), rho);             // -(G_X/rho0) rho_s
    C2 Fx = pfma(npc, fxl, pmul(ng, pair(qx.y, qx.x)));
    C2 Fy = pfma(npc, fyl, pmul(ng, pair(qy.y, qy.x)));
    if (GEN && k.has_accel) {
        C acc = k.g_x;
        if (k.kolmo_amp != C(0)) acc += k.kolmo_amp * csin(v.kolmo_w * C(y));
        Fx = pfma(rho, pset(acc), Fx);
    }

    if (OBS) {
        const long long N = (long long)g.nx * g.ny;
        const long long idx = (long long)y * g.nx + x;
        const double rA = (double)v.rho_ref + (double)drho.x;
        const double rB = (double)v.rho_ref + (double)drho.y;
        const double tot = rA + rB;
        const double mx = (double)jx.x + (double)jx.y + 0.5 * ((double)Fx.x + (double)Fx.y);
        const double my = (double)jy.x + (double)jy.y + 0.5 * ((double)Fy.x + (double)Fy.y);
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
                        (double)(q < 9 ? h[q % 9].x : h[q % 9].y) * (double)inv_scale_of<P>() +
                        wgt<double>(q % 9) * (double)v.rho_ref;
        }
        red[0] += rA;
        red[1] += rB;
        red[2] += mx;
        red[3] += my;
        return;
    }

    // Eq. (1): forced BGK relaxation.  Common velocity
    // u' = sum_s (j_s/tau_s) / sum_s (rho_s/tau_s); shift u_s = u' + tau_s F_s/rho_s;
    // carried as v = 3u.  (Selects, not branches: an empty site has u' = 0
    // and no shift.)
    // (TAU1: omega = 1 exactly, and the products are the values themselves)
    const C2 om = pair(k.omega[0], k.omega[1]);
    const C2 ro = TAU1 ? rho : pmul(rho, om), jxo = TAU1 ? jx : pmul(jx, om),
             jyo = TAU1 ? jy : pmul(jy, om);
    const C den = ro.x + ro.y;
    // 3 / den, times the storage scale's inverse where j is taken in the
    // storage scale (TAU1; both factors exact powers of two apart)
    const C inv3 = den != C(0) ? (TAU1 ? C(3) * inv_scale_of<P>() : C(3)) * recip(den) : C(0);
    const C2 vp = pair((jxo.x + jxo.y) * inv3, (jyo.x + jyo.y) * inv3);
    const bool source = GEN && k.source;
    C2 vx = pset(vp.x), vy = pset(vp.y);
    if (!source) {
        const C2 tr = pair(rho.x != C(0) ? k.tau3[0] * recip(rho.x) : C(0),
                           rho.y != C(0) ? k.tau3[1] * recip(rho.y) : C(0));
        vx = pfma(tr, Fx, vx);
        vy = pfma(tr, Fy, vy);
    }
    C2 hs[9];
    if (source)
        collide<C, C2, true, TAU1>(h, hs, drho, rho, vx, vy, k, Fx, Fy, scale_of<P>());
    else
        collide<C, C2, false, TAU1>(h, hs, drho, rho, vx, vy, k, Fx, Fy, scale_of<P>());
    T2 e[9];
    if constexpr (sizeof(T2) == 4) {
        if (k.sr) {   // half formats: random bits from (site, step), one word per pair
            const uint32_t r = o.rbits;
#pragma unroll
            for (int i = 0; i < 9; ++i) e[i] = enc2_sr<T2>(hs[i], r * sr_mult(i));
        } else {
#pragma unroll
            for (int i = 0; i < 9; ++i) e[i] = enc2<T2, C>(hs[i].x, hs[i].y);
        }
    } else {
#pragma unroll
        for (int i = 0; i < 9; ++i) e[i] = enc2<T2, C>(hs[i].x, hs[i].y);
    }

    if constexpr (SINK == SINK_STAGE) {
        // The staging tile leaves by a bulk tensor store (clipped at the
        // lattice edge); the periodic ghost copies follow by the plain
        // stores of write_edges after the tile's barrier.
        constexpr int TX = Prec<P>::TX, TY = Prec<P>::TY;
#pragma unroll
        for (int i = 0; i < 9; ++i) o.stage[i * TY * TX] = e[i];
    } else {
        // Straight to the output buffer, and to the periodic images of a
        // site within three sites of an edge (ghost columns, and ghost rows
        // when periodic in y).
        if (o.valid) {
#pragma unroll
            for (int i = 0; i < 9; ++i) st_pair(o.gout + i * o.plane, e[i], o.pol);
        }
        if (o.valid && (o.gdx != 0 || o.gdy != 0)) {
#pragma unroll
            for (int i = 0; i < 9; ++i) {
                T2* d = o.gout + i * o.plane;
                if (o.gdx) st_pair(d + o.gdx, e[i], o.pol);
                if (o.gdy) {
                    st_pair(d + o.gdy, e[i], o.pol);
                    if (o.gdx) st_pair(d + o.gdy + o.gdx, e[i], o.pol);
                }
            }
        }
    }
    if (!per && (y == 0 || y == g.ny - 1)) {
        // x-momentum handed to the wall by the links that will bounce back
        // at the next streaming, from the stored (rounded) values:
        // sum_i c_ix (f*_i + f_opp), f_opp = f*_i - 6 w_i rho_w (c_i . u_w),
        // over the three links i leaving through the wall, which is
        // 2 (f*_a - f*_b) - 6 rho_w u_w (w_a + w_b) = 2 (f*_a - f*_b) - rho_w u_w / 3
        // with (a, b) = (8, 7) at the bottom wall and (5, 6) at the top
        // (c_ax = 1, c_bx = -1; w_a = w_b, so the offsets' difference is the
        // populations').  One compute-type value per site and species, kept
        // in the lattice's wall columns for the sums after the tile loop.
        const int down = (y == 0);
        const C uw = down ? -v.u_wall : v.u_wall;
        C2 sv[9];
#pragma unroll
        for (int i = 0; i < 9; ++i) sv[i] = dec2(e[i]);
        const C2 rw2 = pfma(sum9(sv), pset(inv_scale_of<P>()), pset(v.rho_ref));
        const C2 dd = pmul(down ? psub(sv[8], sv[7]) : psub(sv[5], sv[6]), pset(inv_scale_of<P>()));
        const C2 m = psub(pmul(pset(C(2)), dd), pmul(rw2, pset(uw * (C(1) / C(3)))));
        if (o.valid) reinterpret_cast<C2*>(o.wallx)[(down ? 0 : g.nx) + x] = m;
    }
}

// Wall momentum of one CTA's items that hold a wall row, in FP64: the
// wall-site values the site phase left in the lattice's wall columns, summed
// over the item's strip in a fixed order (lane l takes columns l, l + 32,
// ..., then the butterfly), one warp per item -- so the sums do not depend
// on the partition or the tile shape.
template <int P, int SPT>
__device__ __forceinline__ void wall_sums(const BatchArgs<typename Prec<P>::C>& a, int it0, int it_end,
                                       int tid) {
    typedef Layout<P, SPT> L;
    typedef typename L::C C;
    typedef typename L::C2 C2;
    const int lane = tid & 31, warp = tid >> 5;
    int n = 0;
    for (int it = it0; it < it_end; ++it) {
        const int4 w = a.items[it];
        const LatDesc<C>* d = &a.lat[w.x];
        const bool bot = w.z == 0, top = w.w == d->ntiles_y;
        if (d->g.periodic || !(bot || top)) continue;
        if (n++ % (L::NT / 32) != warp) continue;
        const int nx = d->g.nx;
        const int xe = min(w.y * L::TX + L::TX, nx);
        const C2* wx = reinterpret_cast<const C2*>(d->wallx);
        double sb = 0.0, st = 0.0;
        for (int x = w.y * L::TX + lane; x < xe; x += 32) {
            if (bot) sb += (double)wx[x].x + (double)wx[x].y;
            if (top) st += (double)wx[nx + x].x + (double)wx[nx + x].y;
        }
        sb = warp_sum(sb);
        st = warp_sum(st);
        if (lane == 0) {
            if (bot) d->wsum[w.y] = sb;
            if (top) d->wsum[d->nstrips + w.y] = st;
        }
    }
}

// The last CTA of a step launch: the Couette wall samples, one warp per
// lattice, then every lattice's step counter and buffer parity, one thread
// per lattice.  t0, cur0: the step counter and buffer of lattice tid,
// loaded by every CTA before its arrival (they change only between
// launches), so the counters take no load on the launch's tail.
template <int P, bool ALLPER, int NT>
__device__ __forceinline__ void advance_lattices(const BatchArgs<typename Prec<P>::C>& a, int tid,
                                                 long long t0, int cur0) {
    typedef typename Prec<P>::C C;
    if constexpr (!ALLPER) {
        // Strip sums in a fixed order -- lane l adds strips l, l + 32, ...,
        // then a butterfly over the lanes -- so they do not depend on the
        // partition; FP64 has a long latency on this GPU, so no serial chain
        // runs over the strips.  Sampled steps: stress_t0 + k stress_every,
        // tracked by next_sample (no 64-bit remainder: it would compile to a
        // call, which burdens the whole kernel's register allocation).
        const int lane = tid & 31;
        for (int l = tid >> 5; l < a.nlat; l += NT / 32) {
            const LatDesc<C>* d = &a.lat[l];
            if (d->g.periodic) continue;
            DevStats* st = d->st;
            const int ns = d->nstrips;
            const volatile double* ws = d->wsum;
            double sb = 0.0, stp = 0.0;
            for (int i = lane; i < ns; i += 32) {
                sb += ws[i];
                stp += ws[ns + i];
            }
            sb = warp_sum(sb);
            stp = warp_sum(stp);
            const long long t = st->t;
            if (lane == 0 && t == st->next_sample) {
                st->sum_bot += sb * d->inv_nx;
                st->sum_top += stp * d->inv_nx;
                st->samples += 1;
                st->next_sample = t + (d->stress_every > 0 ? d->stress_every : 1);
            }
        }
        __syncthreads();   // the samples have read the step counters
    }
    for (int l = tid; l < a.nlat; l += NT) {
        DevStats* st = a.lat[l].st;
        const long long t = l == tid ? t0 : st->t;
        const int cur = l == tid ? cur0 : st->cur;
        st->t = t + 1;
        st->cur = cur ^ 1;
        st->pull = 1;
    }
}

// Periodic images of one tile's edge sites, from the staging tile into the
// ghost columns (x within 3 of either edge) and, when the lattice is
// periodic in y, the ghost rows (y within 3 of either edge) and corners, and
// the sites themselves in the last lattice columns the bulk store leaves
// out (x >= x_tail, within 3 of the right edge); by
// all NT threads of the CTA, one (site, plane) copy each in turn, with
// consecutive threads on consecutive sites of a plane.  The first copies go
// to warps 2 and up: warps 0 and 1 have just issued the tile's loads and
// store, and every warp waits for the last one at the next barrier.  Kept
// out of the site update, whose register allocation it would otherwise
// burden.  L: the step kernel's layout (tile rows TY, staging layout).
template <int P, class L>
__device__ __forceinline__ void write_edges(const typename Prec<P>::T2* stage,
                                            typename Prec<P>::T2* fout, const Geom& g, int x0,
                                            int y0, bool per, int tid) {
    typedef typename Prec<P>::T2 T2;
    constexpr int TX = L::TX, TY = L::TY, NT = L::NT;
    const int w = min(TX, g.nx - x0), h = min(TY, g.ny - y0);   // valid part of the tile
    // source columns [0, nca) and [cb0, w), rows [0, na) and [rb0, h); the
    // two ranges of each never meet since nx, ny >= 8
    const int nca = max(0, min(3 - x0, w)), cb0 = max(g.nx - 3 - x0, 0), ncb = max(w - cb0, 0);
    const int na = per ? max(0, min(3 - y0, h)) : 0;
    const int rb0 = max(g.ny - 3 - y0, 0), nb = per ? max(h - rb0, 0) : 0;
    const int nrow = na + nb;                 // ghost-source rows: every column
    const int mid0 = na, mid1 = nb > 0 ? rb0 : h;   // other rows: the edge columns only
    const int ncol = nca + ncb;
    const int nA = nrow * w, nB = max(mid1 - mid0, 0) * ncol, n = nA + nB;
    if (n == 0) return;
    const long long PL = (long long)g.rows * g.pitch;
    const long long SY = (long long)g.ny * g.pitch;
    for (int u = tid >= 64 ? tid - 64 : tid + NT - 64; u < 9 * n; u += NT) {
        const int i = u / n, k = u - i * n;
        int lx, ly;
        if (k < nA) {
            const int r = k / w;
            lx = k - r * w;
            ly = r < na ? r : rb0 + (r - na);
        } else {
            const int kb = k - nA, r = kb / ncol, c = kb - r * ncol;
            ly = mid0 + r;
            lx = c < nca ? c : cb0 + (c - nca);
        }
        const int dX = lx < nca ? g.nx : (ncb > 0 && lx >= cb0 ? -g.nx : 0);
        const long long dY = ly < na ? SY : (nb > 0 && ly >= rb0 ? -SY : 0);
        const T2 e = stage[L::stage_off(ly, lx) + i * L::TYB * TX];
        T2* d = fout + i * PL + (long long)(y0 + ly + kGY) * g.pitch + (x0 + lx + g.gx);
        if (x0 + lx >= g.x_tail) d[0] = e;
        if (dX) d[dX] = e;
        if (dY) {
            d[dY] = e;
            if (dX) d[dY + dX] = e;
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
// Persistent and multi-lattice.  The work items of a launch are runs of
// tiles (TY = 8 SPT rows each) down TX-wide column strips, over all
// lattices; CTA b takes the items a.items[a.cta_items[b] .. a.cta_items[b + 1])
// of a table the host builds (segments dealt by estimated work in band
// order, or one contiguous run per CTA).  Walking down a strip, a CTA keeps
// the 8-row blocks of f* (TMA-loaded into a ring of NB slots, ahead of use
// and across item boundaries) and a window of the density/Psi deviation rows
// y0 - 2 .. y0 + TY + 1 of the current tile, whose last four rows are
// carried forward as the next tile's first four; so each block is loaded
// and each deviation row computed once per strip, and only the x halo (4 of
// 64 columns) is redundant.  Every thread keeps one column and SPT rows of
// the window (its own sites' cells, see t_m and t_w), so all its
// shared-memory addresses within a slot are fixed.  SPT = 2: each thread
// updates two vertically adjacent
// sites, which share four of their six stencil rows.  Tiles leave through a
// staging tile by TMA bulk tensor stores (one per 8 rows), clipped at the
// lattice edge, and tiles near an edge then write the periodic ghost
// copies; where the staging tile does not fit beside the ring (FP32 with
// 16-row tiles) the threads store their sites and ghost copies to global
// memory themselves.  The last CTA to finish advances every lattice's step
// counter and buffer parity and takes the Couette wall samples.
// V: bit 0 = every lattice periodic (no wall code); bit 1 = general forcing;
// bit 2 = omega = 1 for both species (the site phase reads no populations).
template <int P, int V, int SPT>
__global__ void __launch_bounds__(Layout<P, SPT>::NT, 1)
    k_step(const __grid_constant__ BatchArgs<typename Prec<P>::C> a) {
    typedef Layout<P, SPT> L;
    typedef typename L::T2 T2;
    typedef typename L::C C;
    typedef typename L::C2 C2;
    constexpr bool ALLPER = (V & 1) != 0;
    constexpr bool GEN = (V & 2) != 0;
    // omega = 1 for both species: the site phase needs the populations only
    // through j, which the density phase computes beside rho and Psi
    constexpr bool TAU1 = (V & 4) != 0;
    constexpr bool STAGED = L::STAGED;   // output through the staging tile
    constexpr int PS = L::TYB * L::BX;   // plane stride in a block slot (pairs)
    extern __shared__ unsigned char smem_raw[];
    // 128-byte aligned base, derived from the shared array by indexing so
    // that every access below compiles to shared-memory instructions.
    unsigned char* smem = smem_raw + ((128u - (smem_u32(smem_raw) & 127u)) & 127u);
    C2* win_r = reinterpret_cast<C2*>(smem + L::WIN_OFF);     // [WIN][RX]
    C2* win_p = win_r + L::WIN * L::RX;                       // [WIN][RX]
    T2* stage = reinterpret_cast<T2*>(smem + L::STAGE_OFF);   // staging tile (STAGED)
    __shared__ __align__(8) uint64_t bars[L::NB];
    __shared__ int s_fail, s_last;
    __shared__ uint64_t s_pol[2];   // L2 policies of the block loads and the tile stores

    const int tid = threadIdx.x;
    const int G = gridDim.x;
    // thread 0 issues the block loads; this thread (warp 1) the bulk stores
    // of the staging tile and the waits on them (STAGED)
    constexpr int kStoreThread = 32;
    // When one buffer of every lattice of the launch fits in L2 together, the
    // step's output stays there for the next step (evict last) and the input,
    // dead once read, goes first; otherwise both keep the normal priority.
    // The two policies are made once, by thread 0, and kept in shared memory
    // (held in registers through the tile loop, or made at each issue, they
    // cost the large lattices 1-3 %).
    // window column and block row of this thread (both phases)
    const int t_lx = tid % L::RX, t_j = tid / L::RX;
    static_assert(L::NT == L::RX * L::TYB && L::TY >= 4, "one window column per thread and block row");
    // Rows of the density phase: thread row t_j computes the new window rows
    // 4 + SPT t_m + c, c < SPT, which hold its own sites (window rows
    // 2 + SPT t_j + c) for t_j >= 2 / SPT; the first 2 / SPT thread rows,
    // whose sites sit in the two rows carried over from the previous tile,
    // compute the last two rows -- the next tile's first sites, theirs again.
    // So every thread's sites were computed by the thread itself, in this
    // tile or (first thread rows) in the previous one, and their momenta stay
    // with it (TAU1): in registers, and for the first thread rows across the
    // tile boundary in a small shared buffer of their own.
    constexpr int kCarry = 2 / SPT;   // thread rows whose sites are carried rows
    static_assert(2 % SPT == 0, "two carried rows per tile");
    const int t_m = (t_j + L::TYB - kCarry) % L::TYB;
    const bool t_carry = t_j < kCarry;
    // Columns likewise: window column w holds lattice column x0 - 2 + w and
    // site column lx is window column lx + 2, so thread t_lx computes window
    // column (t_lx + 2) mod RX -- its own site column, and for the RX - TX
    // threads without a site the halo columns.
    const int t_w = (t_lx + 2) % L::RX;
    // TAU1: momenta (jx, jy) of the first thread rows' new cells, kept for
    // the next tile, whose first sites they are; jc: this thread's entries
    __shared__ __align__(16) C2 s_jcarry[kCarry * L::RX * SPT * 2];
    C2* const jc = s_jcarry + ((t_carry ? t_j : 0) * L::RX + t_lx) * (SPT * 2);
    auto slot = [&](int pos) { return reinterpret_cast<T2*>(smem + (pos % L::NB) * L::SLOT_BYTES); };
    const int it_end = a.cta_items[blockIdx.x + 1];

    if (tid == 0) {
        s_fail = 0;
        for (int b = 0; b < L::NB; ++b) mbar_init(&bars[b], 1);
        fence_mbar_init();
        s_pol[0] = a.l2_resident ? policy_evict_first() : policy_evict_normal();
        s_pol[1] = a.l2_resident ? policy_evict_last() : policy_evict_normal();
    }
    __syncthreads();
    // Up to here only shared memory and the host-built item tables were
    // touched; the lattice state (DevStats, populations) written by the
    // previous step is read after the wait.  The next step's CTAs may then
    // take each SM as soon as this CTA leaves it (one CTA fills an SM).
    griddep_wait();
    griddep_launch_dependents();

    // Producer (thread 0): the blocks of this CTA's items, in order.  Item
    // tiles [ty_a, ty_b) need blocks SPT ty_a .. SPT ty_b (block j = padded
    // rows [8j, 8j + 8)); consecutive items' blocks follow each other.
    int p_item = a.cta_items[blockIdx.x], p_j = 0, p_pos = 0;
    // cached geometry of the producer's current item
    const CUtensorMap* p_map = nullptr;
    int p_x0 = 0, p_ty_a = 0, p_nblk = 0;
    auto p_load = [&]() {
        if (p_item >= it_end) return;
        const int4 w = a.items[p_item];
        const LatDesc<C>* d = &a.lat[w.x];
        p_x0 = w.y * L::TX;
        p_ty_a = w.z;
        p_nblk = SPT * (w.w - w.z) + 1;
        p_map = &d->tin[*((volatile int*)&d->st->cur)];
    };
    auto issue_next = [&]() -> bool {
        if (p_item >= it_end) return false;
        uint64_t* bar = &bars[p_pos % L::NB];
        mbar_expect_tx(bar, (uint32_t)L::SLOT_BYTES);
        // box origin: pair column x0 (= x0 - gx + gx) -> element 2 x0; padded row 8j
        tma_load_3d_hint(slot(p_pos), p_map, 2 * p_x0, L::TYB * (SPT * p_ty_a + p_j), 0, bar,
                         s_pol[0]);
        ++p_pos;
        if (++p_j == p_nblk) {
            p_j = 0;
            ++p_item;
            p_load();
        }
        return true;
    };
    if (tid == 0) p_load();
    if (tid == 0)
        while (p_pos < L::NB && issue_next()) {}
    int ty_b = 0, ty = 0;   // the consumer's item end and tile (read by release)
    // Producer: the tile whose first block is at position q is done with
    // its blocks before the next tile's first one (all of them at an item's
    // last tile): refill those slots.
    auto release = [&](int q) {
        const int released = (ty + 1 < ty_b) ? q + SPT : q + SPT + 1;
        fence_proxy_async();   // generic reads of freed slots before async writes
        while (p_pos < released + L::NB && issue_next()) {}
    };

    bool bad_unused = false;   // (the observables' flag; the step uses nf)
    int c_pos = 0;   // ring position of the current item's first block
    for (int it = a.cta_items[blockIdx.x]; it < it_end && !s_fail; ++it) {
        const int4 w = a.items[it];
        const LatDesc<C>* d = &a.lat[w.x];
        const int x0 = w.y * L::TX;
        const int ty_a = w.z;
        ty_b = w.w;
        const Geom g = d->g;
        const LatVals<C> v = d->v;
        const bool per_lat = ALLPER || g.periodic;
        const int cur = *((volatile int*)&d->st->cur);
        const int pull = *((volatile int*)&d->st->pull);
        // the step counter advances only after every CTA of the launch is done
        const uint32_t key = hash32((uint32_t)*((volatile long long*)&d->st->t) * 0x9e3779b9u);
        T2* fout = reinterpret_cast<T2*>(d->fbuf[cur ^ 1]);
        C2 nf = pset(C(0));   // 0 * rho over the item's sites: NaN at a non-finite density
        // ring slot and phase parity of the tile's first block, kept as the
        // tiles advance
        int qm = c_pos % L::NB, qph = (c_pos / L::NB) & 1;
        for (ty = ty_a; ty < ty_b; ++ty) {
            const int q = c_pos + SPT * (ty - ty_a);   // this tile uses blocks q .. q + SPT
            // Each thread sees the blocks land itself (the first block of a
            // tile after an item's first was seen as the previous tile's
            // last); a timeout is acted on after the next barrier (garbage
            // read meanwhile is harmless).
            int sl[SPT + 1];
#pragma unroll
            for (int b = 0; b <= SPT; ++b) {
                int sb = qm + b, ph = qph;
                if (sb >= L::NB) {
                    sb -= L::NB;
                    ph ^= 1;
                }
                sl[b] = sb;
                if ((b > 0 || ty == ty_a) && !mbar_wait_bounded(&bars[sb], ph)) s_fail = 1;
            }
            const int y0 = ty * L::TY;
            // The tile's padded rows [y0, y0 + 8 (SPT + 1)) are blocks q ..
            // q + SPT; brow(r, c): padded row y0 + r, pair column c, plane 0.
            const T2* s0 = reinterpret_cast<const T2*>(smem + sl[0] * L::SLOT_BYTES);
            const T2* s1 = reinterpret_cast<const T2*>(smem + sl[1] * L::SLOT_BYTES);
            const T2* s2 = reinterpret_cast<const T2*>(smem + sl[SPT] * L::SLOT_BYTES);
            auto brow = [&](int r, int c) {
                const T2* base = r < L::TYB ? s0 : (SPT == 1 || r < 2 * L::TYB ? s1 : s2);
                return base + (r & (L::TYB - 1)) * L::BX + c;
            };

            // The tile's two phases, with or without the wall code: a tile
            // whose deviation window (rows y0 - 2 .. y0 + TY + 1) keeps clear
            // of the walls and of the periodic ghost rows runs the periodic
            // code, which is exact there, so only the tiles at a wall pay for
            // the wall logic.  Returns false when a block wait gave up.
            auto tile_body = [&](auto wall_tag) -> bool {
                constexpr bool W = decltype(wall_tag)::value;
                const bool per = !W || per_lat;
                C2 jn[SPT][2];   // TAU1: momenta of this thread's new rows
                // Phase 2: window row k holds lattice row y0 - 2 + k (padded row
                // y0 + 1 + k).  Rows 4 .. TY + 3 are new: thread (t_lx, t_j)
                // computes rows 4 + SPT t_m + c, c < SPT, of window column t_w
                // (the thread's own sites, see t_m).  Rows 0 .. 3 are the previous
                // tile's rows TY .. TY + 3, carried forward by the threads that
                // own those before they overwrite them, or at an item's first
                // tile computed from block q.  No other thread touches these
                // cells in this phase.
                {
                    const int bc = t_w - 2 + L::GX;   // pair column in the block
                    // rows 0 .. 3: carried forward, or computed at an item's first
                    // tile, before this thread's new rows overwrite their sources
                    // (rows 2 and 3, at an item's first tile, by the thread rows
                    // whose sites they are: their momenta start the carry)
    #pragma unroll
                    for (int c = 0; c < SPT; ++c) {
                        const int k = 4 + SPT * t_m + c;
                        const int kk = k - L::TY;
                        if (kk >= 0) {
                            if (ty == ty_a) {
                                C2 r, p, jt[2];
                                cell_dev<P, PS, TAU1>(brow(kk, bc), brow(kk + 1, bc), brow(kk + 2, bc),
                                                      y0 - 2 + kk, per, pull, g, v, r, p, jt);
                                win_r[kk * L::RX + t_w] = r;
                                win_p[kk * L::RX + t_w] = p;
                                if (TAU1 && t_carry) {   // rows 2 and 3: this thread's sites
                                    jc[2 * c] = jt[0];
                                    jc[2 * c + 1] = jt[1];
                                }
                            } else {
                                win_r[kk * L::RX + t_w] = win_r[k * L::RX + t_w];
                                win_p[kk * L::RX + t_w] = win_p[k * L::RX + t_w];
                            }
                        }
                    }
                    // The new rows, without a branch between the cells.  Rows
                    // outside the lattice (beyond a wall, or below a ragged last
                    // tile) are computed from whatever the slots hold there (the
                    // TMA fill or ghost rows): no site reads them -- the wall
                    // mirror below overwrites the two rows past each wall.
    #pragma unroll
                    for (int c = 0; c < SPT; ++c) {
                        const int k = 4 + SPT * t_m + c;
                        C2 r, p;
                        cell_dev<P, PS, TAU1>(brow(k, bc), brow(k + 1, bc), brow(k + 2, bc), y0 - 2 + k,
                                              per, pull, g, v, r, p, jn[c]);
                        win_r[k * L::RX + t_w] = r;
                        win_p[k * L::RX + t_w] = p;
                    }
                    // The first thread rows (whole warps) swap their new cells'
                    // momenta, the next tile's, for their sites', kept from the
                    // previous tile; jn then holds every thread's sites'.
                    if (TAU1 && t_carry) {
    #pragma unroll
                        for (int c = 0; c < SPT; ++c) {
                            const C2 px = jc[2 * c], py = jc[2 * c + 1];
                            jc[2 * c] = jn[c][0];
                            jc[2 * c + 1] = jn[c][1];
                            jn[c][0] = px;
                            jn[c][1] = py;
                        }
                    }
                }
                // mirror the deviations about the halfway walls, in the tiles whose
                // window rows y0 - 2 .. y0 + TY + 1 reach past a wall (uniform)
                if (!per && (y0 < 2 || y0 + L::TY + 1 >= g.ny)) {
                    __syncthreads();
                    for (int c = tid; c < L::WIN * L::RX; c += L::NT) {
                        const int k = c / L::RX, lx = c - k * L::RX;
                        const int y = y0 - 2 + k;
                        int ym;
                        if (y < 0) ym = -1 - y;
                        else if (y >= g.ny && y <= g.ny + 1) ym = 2 * g.ny - 1 - y;
                        else continue;
                        const int km = ym - (y0 - 2);   // in [0, WIN): see the wall cases
                        win_r[k * L::RX + lx] = win_r[km * L::RX + lx];
                        win_p[k * L::RX + lx] = win_p[km * L::RX + lx];
                    }
                }
                if (STAGED && tid == kStoreThread) bulk_wait_read();   // previous bulk store has read the staging tile
                __syncthreads();
                if (s_fail) return false;
                if constexpr (TAU1) {
                    // The site phase reads no populations: the tile's blocks
                    // before the next tile's first one are free already.
                    if (a.early_release && tid == 0) release(q);
                }

                // Phase 3: SPT sites per thread (lx < TX): sites (x0 + t_lx,
                // y0 + SPT t_j + s), whose stencil rows y - 2 .. y + 2 are window
                // rows SPT t_j + s .. SPT t_j + s + 4 and whose populations sit in
                // padded rows y0 + SPT t_j + s + 2 .. + 4.
                {
                    const int lx = t_lx, ly = SPT * t_j;
                    const int x = x0 + lx, y = y0 + ly;
                    if (lx < L::TX && x < g.nx && y < g.ny) {
                        C2 fx[SPT], fy[SPT], qx[SPT], qy[SPT], dp[SPT], dr[SPT];
                        force_sums<SPT, L::RX>(win_p + ly * L::RX + lx + 2,
                                               win_r + ly * L::RX + lx + 2, a.k, fx, fy, qx, qy, dp, dr);
                        SiteOut<T2> o;
                        o.rbits = 0u;
                        [[maybe_unused]] uint32_t srh = 0u;   // the shared hash of this thread's sites
                        if constexpr (sizeof(T2) == 4) srh = sr_hash(key, x, y, g.nx);
                        o.obs = OBS_NONE;
                        o.valid = 1;
                        o.wallx = d->wallx;
                        if constexpr (!STAGED) {
                            o.plane = g.plane;
                            o.gdx = x < 3 ? g.nx : (x >= g.nx - 3 ? -g.nx : 0);
                            o.pol = s_pol[1];
                        }
                        // Both sites are updated without a branch between them (a
                        // site below the lattice's last row, in a ragged tile, is
                        // computed and dropped), so their work can interleave.
    #pragma unroll
                        for (int s = 0; s < SPT; ++s) {
                            const int ys = y + s;
                            o.valid = s == 0 || ys < g.ny;
                            if constexpr (sizeof(T2) == 4) {
                                // SPT = 2: y is even (tile rows are multiples of 16)
                                o.rbits = sr_word(SPT == 2 ? srh : sr_hash(key, x, ys, g.nx), ys);
                            }
                            if constexpr (STAGED) {
                                o.stage = stage + L::stage_off(ly + s, lx);
                            } else {
                                o.gout = fout + (long long)(ys + kGY) * g.pitch + (x + g.gx);
                                o.gdy = !per ? 0
                                        : ys < 3 ? (long long)g.ny * g.pitch
                                        : (ys >= g.ny - 3 ? -(long long)g.ny * g.pitch : 0);
                            }
                            double wr[4];   // (observables only)
                            if constexpr (TAU1) {
                                site_update<P, false, GEN, PS, STAGED ? SINK_STAGE : SINK_GLOBAL, true>(
                                    nullptr, nullptr, nullptr, fx[s], fy[s], qx[s], qy[s], dp[s], dr[s],
                                    x, ys, per, pull, g, v, a.k, o, wr, bad_unused, &nf, jn[s]);
                            } else {
                                const int bc = lx + L::GX;
                                site_update<P, false, GEN, PS, STAGED ? SINK_STAGE : SINK_GLOBAL>(
                                    brow(ly + s + 2, bc), brow(ly + s + 3, bc), brow(ly + s + 4, bc),
                                    fx[s], fy[s], qx[s], qy[s], dp[s], dr[s], x, ys, per, pull, g, v,
                                    a.k, o, wr, bad_unused, &nf);
                            }
                        }
                        if constexpr (STAGED) fence_proxy_async();   // staging writes before the bulk store
                    }
                }
                return true;
            };
            bool ok;
            if constexpr (ALLPER)
                ok = tile_body(std::false_type{});
            else if (per_lat || (y0 >= 3 && y0 + L::TY + 3 <= g.ny))
                ok = tile_body(std::false_type{});
            else
                ok = tile_body(std::true_type{});
            if (!ok) break;
            __syncthreads();
            if constexpr (STAGED) {
                // The bulk stores and the next loads are issued by two threads
                // of different warps, side by side.
                if (tid == kStoreThread) {
                    // site (x0, y0 + 8h) in padded coordinates: pair column
                    // x0 + gx, row y0 + 8h + kGY; a ragged tile's store is
                    // clipped at x = nx, y = ny (no box starts below the lattice)
#pragma unroll
                    for (int h = 0; h < SPT; ++h)
                        if (h == 0 || y0 + h * L::TYB < g.ny)
                            tma_store_3d_hint(&d->tout[cur ^ 1], stage + L::stage_off(h * L::TYB, 0),
                                              2 * (x0 + L::GX), y0 + h * L::TYB + kGY, 0, s_pol[1]);
                    bulk_commit();
                }
            }
            if (!(TAU1 && a.early_release) && tid == 0) release(q);
            if constexpr (STAGED) {
                // only tiles within 3 sites of an edge write periodic ghost copies
                const bool edge = x0 < 3 || x0 + L::TX > g.nx - 3 ||
                                  (per_lat && (y0 < 3 || y0 + L::TY > g.ny - 3));
                if (edge) write_edges<P, L>(stage, fout, g, x0, y0, per_lat, tid);
            }
            qm += SPT;
            if (qm >= L::NB) {
                qm -= L::NB;
                qph ^= 1;
            }
        }
        if (!(nf.x == C(0) && nf.y == C(0)))   // a density of this lattice went non-finite
            atomicOr(&d->st->err, ERR_NONFINITE);
        if (s_fail) break;
        c_pos += SPT * (ty_b - ty_a) + 1;
    }
    // Wall momentum of this CTA's items that hold a wall row, in FP64: the
    // wall-site values the site phase left in the lattice's wall columns,
    // summed over the item's strip in a fixed order (lane l takes columns
    // l, l + 32, ..., then the butterfly), one warp per item -- so the sums
    // do not depend on the partition or the tile shape.  Kept out of the
    // tile loop: a per-item reduction there (barriers, FP64 shuffles) cost
    // the generic variant 1-4 % even on periodic lattices, which skip it.
    if constexpr (!ALLPER) {
        __syncthreads();   // this CTA's wall-site values are written
        if (!s_fail) wall_sums<P, SPT>(a, a.cta_items[blockIdx.x], it_end, tid);
    }   // (the barrier before the arrival orders the sums before it)
    if (STAGED && tid == kStoreThread) bulk_wait_all();
    if (s_fail && tid == 0) {
        // Let copies in flight land before the CTA exits.  No slot is
        // re-armed once a wait has failed, so the last NB positions issued
        // are each slot's latest arm, and every earlier one has landed; wait
        // on each of those once, with its own phase parity (a position that
        // has landed returns at once).
        for (int pos = p_pos > L::NB ? p_pos - L::NB : 0; pos < p_pos; ++pos)
            mbar_wait_bounded(&bars[pos % L::NB], (pos / L::NB) & 1);
    }
    if (s_fail && tid == 0)   // report on every lattice of the launch
        for (int l = 0; l < a.nlat; ++l) atomicOr(&a.lat[l].st->err, ERR_TIMEOUT);

    // The last CTA advances every lattice and takes the wall samples.  Its
    // step counters are loaded by every CTA now, off the launch's tail.
    long long t0 = 0;
    int cur0 = 0;
    if (tid < a.nlat) {
        const DevStats* st = a.lat[tid].st;
        t0 = *((volatile const long long*)&st->t);
        cur0 = *((volatile const int*)&st->cur);
    }
    __syncthreads();   // this CTA's writes (wall sums, timeout flags) precede its arrival
    if (tid == 0) s_last = ticket_arrive(a.ticket) == (unsigned int)(G - 1);
    __syncthreads();
    if (!s_last) return;
    advance_lattices<P, ALLPER, L::NT>(a, tid, t0, cur0);
    // no other CTA of the launch touches the ticket again; the next launch
    // reads it after this one has completed
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
    v.kolmo_w = a.k.kolmo_w;
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
            C2 fx[1], fy[1], qx[1], qy[1], dp[1], dr[1];
            force_sums<1, L::RX>(spsi + ly * L::RX + lx + 2, srho + ly * L::RX + lx + 2, a.k, fx, fy,
                                 qx, qy, dp, dr);
            SiteOut<T2> o;
            o.stage = nullptr;
            o.rbits = 0u;
            o.valid = 1;
            o.obs = a.obs;
            o.obs_out = a.obs_out;
            o.q0 = a.q0;
            o.q1 = a.q1;
            site_update<P, true, GEN, PS, SINK_STAGE>(b0 - L::BX, b0, b0 + L::BX, fx[0], fy[0], qx[0],
                                                      qy[0], dp[0], dr[0], x, y, per, a.pull, g, v,
                                                      a.k, o, red, bad);
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
            const double sc = (double)scale_of<P>();
            const double hA = sc * wgt<double>(i) * ((r[0] - rref) + r[0] * e);
            const double hB = sc * wgt<double>(i) * ((r[1] - rref) + r[1] * e);
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
            const double off = wgt<double>(i) * rref, sc = (double)scale_of<P>();
            put2<T2>(fout, g, i, x, y, encd2<T2>(sc * (src[idx] - off), sc * (src[N + idx] - off)));
        }
    }
}

// ------------------------------------------------------ wait self-test
// One CTA arms an mbarrier that no copy will ever complete and waits on it
// with the step kernel's bounded wait (bound `limit`); the wait gives up, the
// kernel latches ERR_TIMEOUT in *err and returns, leaving the context usable.
// (Compiled in the FP32 translation unit only.)
#if LB_PREC == 1
// ------------------------------------------------------ FP32 math probe
// The step kernel's FP32 exp(x) - 1 and reciprocal on caller values, next
// to the CUDA library's expm1f: out[3k] = pexpm1(x[k]), out[3k + 1] =
// expm1f(x[k]), out[3k + 2] = recip(x[k]) (x[k] taken in pairs, as the
// kernel does; an odd tail element is paired with itself).
__global__ void k_math_probe(const float* __restrict__ x, float* __restrict__ out, long long n) {
    for (long long k = 2 * (blockIdx.x * (long long)blockDim.x + threadIdx.x); k < n;
         k += 2LL * gridDim.x * blockDim.x) {
        const float a = x[k], b = k + 1 < n ? x[k + 1] : a;
        const float2 e = pexpm1(make_float2(a, b));
        out[3 * k] = e.x;
        out[3 * k + 1] = expm1f(a);
        out[3 * k + 2] = recip(a);
        if (k + 1 < n) {
            out[3 * k + 3] = e.y;
            out[3 * k + 4] = expm1f(b);
            out[3 * k + 5] = recip(b);
        }
    }
}

__global__ void k_wait_selftest(unsigned int* err, int limit) {
    __shared__ __align__(8) uint64_t bar;
    if (threadIdx.x == 0) {
        mbar_init(&bar, 1);
        fence_mbar_init();
    }
    __syncthreads();
    if (threadIdx.x == 0 && !mbar_wait_bounded(&bar, 0, limit)) atomicOr(err, ERR_TIMEOUT);
}
#endif

// ------------------------------------------------------------- launchers
// Step kernels of precision P (8-row tiles; 16-row tiles where the
// precision has them) and the observe kernels, variant by variant.
template <int P>
static cudaError_t configure_all() {
    typedef Layout<P> L;
    cudaError_t e = cudaSuccess;
    auto opt = [&](auto kern, int bytes) {
        if (e == cudaSuccess) e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
    };
    opt(k_step<P, 0, 1>, L::SMEM);
    opt(k_step<P, 1, 1>, L::SMEM);
    opt(k_step<P, 2, 1>, L::SMEM);
    opt(k_step<P, 3, 1>, L::SMEM);
    opt(k_step<P, 4, 1>, L::SMEM);
    opt(k_step<P, 5, 1>, L::SMEM);
    opt(k_step<P, 6, 1>, L::SMEM);
    opt(k_step<P, 7, 1>, L::SMEM);
    if constexpr (Prec<P>::NB2 > 0) {
        typedef Layout<P, 2> L2;
        opt(k_step<P, 0, 2>, L2::SMEM);
        opt(k_step<P, 1, 2>, L2::SMEM);
        opt(k_step<P, 2, 2>, L2::SMEM);
        opt(k_step<P, 3, 2>, L2::SMEM);
        opt(k_step<P, 4, 2>, L2::SMEM);
        opt(k_step<P, 5, 2>, L2::SMEM);
        opt(k_step<P, 6, 2>, L2::SMEM);
        opt(k_step<P, 7, 2>, L2::SMEM);
    }
    opt(k_observe<P, 2>, L::SMEM_OBS);
    opt(k_observe<P, 3>, L::SMEM_OBS);
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
    cudaError_t e = configure_all<P>();
    if (e == cudaSuccess && dev >= 0 && dev < 64) configured[dev] = 1;
    return e;
}

// LB_PDL=0 in the environment turns the programmatic launches off (A/B
// timing); read once per process.
static bool pdl_enabled() {
    static const bool on = [] {
        const char* v = getenv("LB_PDL");
        return !(v && v[0] == '0');
    }();
    return on;
}

template <int P, int SPT>
static cudaError_t launch_step_shape(const BatchArgs<typename Prec<P>::C>& a, int variant, dim3 grid,
                                     cudaStream_t s) {
    typedef Layout<P, SPT> L;
    // Consecutive steps on a stream overlap the next launch's set-up with the
    // previous launch's last CTAs (programmatic stream serialization); the
    // kernel waits for the previous grid before it reads the lattice state.
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    at[0].val.programmaticStreamSerializationAllowed = 1;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = grid;
    cfg.blockDim = dim3(L::NT, 1, 1);
    cfg.dynamicSmemBytes = L::SMEM;
    cfg.stream = s;
    cfg.attrs = at;
    cfg.numAttrs = pdl_enabled() ? 1 : 0;
    cudaError_t e;
    switch (variant & 7) {
        case 0: e = cudaLaunchKernelEx(&cfg, k_step<P, 0, SPT>, a); break;
        case 1: e = cudaLaunchKernelEx(&cfg, k_step<P, 1, SPT>, a); break;
        case 2: e = cudaLaunchKernelEx(&cfg, k_step<P, 2, SPT>, a); break;
        case 3: e = cudaLaunchKernelEx(&cfg, k_step<P, 3, SPT>, a); break;
        case 4: e = cudaLaunchKernelEx(&cfg, k_step<P, 4, SPT>, a); break;
        case 5: e = cudaLaunchKernelEx(&cfg, k_step<P, 5, SPT>, a); break;
        case 6: e = cudaLaunchKernelEx(&cfg, k_step<P, 6, SPT>, a); break;
        default: e = cudaLaunchKernelEx(&cfg, k_step<P, 7, SPT>, a); break;
    }
    return e != cudaSuccess ? e : cudaGetLastError();
}

template <int P>
cudaError_t launch_step_prec(const void* args, int variant, int spt, dim3 grid, cudaStream_t s) {
    typedef typename Prec<P>::C C;
    cudaError_t e = ensure_configured<P>();
    if (e != cudaSuccess) return e;
    const BatchArgs<C>& a = *reinterpret_cast<const BatchArgs<C>*>(args);
    if (spt == 1) return launch_step_shape<P, 1>(a, variant, grid, s);
    if constexpr (Prec<P>::NB2 > 0)
        if (spt == 2) return launch_step_shape<P, 2>(a, variant, grid, s);
    return cudaErrorInvalidValue;
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
template cudaError_t launch_step_prec<LB_PREC>(const void*, int, int, dim3, cudaStream_t);
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

#if LB_PREC == 1
namespace lbgb {
cudaError_t launch_wait_selftest(unsigned int* err, int limit, cudaStream_t s) {
    k_wait_selftest<<<1, 32, 0, s>>>(err, limit);
    return cudaGetLastError();
}
cudaError_t launch_math_probe(const float* x, float* out, long long n, cudaStream_t s) {
    long long blocks = (n + 511) / 512;
    if (blocks > 152 * 16) blocks = 152 * 16;
    k_math_probe<<<(unsigned)(blocks > 0 ? blocks : 1), 256, 0, s>>>(x, out, n);
    return cudaGetLastError();
}
}  // namespace lbgb
#endif
