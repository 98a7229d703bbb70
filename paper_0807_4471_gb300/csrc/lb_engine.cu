// lb_engine.cu -- host-side engine shared by the single-lattice ABI and the
// lattice pool: parameter validation, device regions, TMA descriptors,
// model coefficients, lattice descriptors, the work partition and launch of
// the persistent step kernel, and the observe/initialise helpers.  Every
// step of the model runs in the kernels of lb_kernels.cu.
#include "lb_engine.h"

#include <algorithm>
#include <cmath>
#include <cstring>
#include <functional>
#include <queue>
#include <utility>

namespace lbgb {

constexpr size_t kAlign = 256;
size_t align_up(size_t v, size_t a) { return (v + a - 1) / a * a; }

// Multi-range weights p(|d|^2) (8th-order isotropic, second moment 1/3) and
// the D2Q9 weights w(|d|^2), for the 12 pair representatives used by the
// kernels: (1,0) (0,1) (1,1) (-1,1) (2,0) (0,2) (2,1) (1,2) (-1,2) (-2,1)
// (2,2) (-2,2).
static double p_weight(int c2) {
    switch (c2) {
        case 1: return 4.0 / 63.0;
        case 2: return 4.0 / 135.0;
        case 4: return 1.0 / 180.0;
        case 5: return 2.0 / 945.0;
        case 8: return 1.0 / 15120.0;
    }
    return 0.0;
}
static double w_weight(int c2) { return c2 == 1 ? 1.0 / 9.0 : c2 == 2 ? 1.0 / 36.0 : 0.0; }

lb_status validate_params(const lb_params* p) {
    if (!p) return LB_ERR_INVALID;
    if (p->nx < 8 || p->ny < 8 || p->nx > (1 << 20) || p->ny > (1 << 19)) return LB_ERR_INVALID;
    if (p->boundary != LB_PERIODIC && p->boundary != LB_COUETTE) return LB_ERR_INVALID;
    if (p->precision < LB_FP64 || p->precision > LB_BF16_OFFSET) return LB_ERR_INVALID;
    if (p->psi_form != LB_PSI_SQRT_RHO0 && p->psi_form != LB_PSI_RHO0) return LB_ERR_INVALID;
    if (p->force_scheme != LB_FORCE_SHIFT && p->force_scheme != LB_FORCE_SOURCE) return LB_ERR_INVALID;
    if (!(p->tau_A > 0.5) || !(p->tau_B > 0.5) || !(p->rho0 > 0.0)) return LB_ERR_INVALID;
    if (p->stress_every < 1 || p->stress_t0 < 0) return LB_ERR_INVALID;
    if (p->rounding != LB_ROUND_NEAREST && p->rounding != LB_ROUND_STOCHASTIC) return LB_ERR_INVALID;
    if (p->tile_rows != 0 && p->tile_rows != 8 && p->tile_rows != 16) return LB_ERR_INVALID;
    if (p->tile_rows == 16 && p->precision == LB_FP64) return LB_ERR_INVALID;
    const double vals[] = {p->tau_A, p->tau_B, p->G_A1, p->G_A2, p->G_B1, p->G_B2, p->G_X,
                           p->rho0, p->u_wall, p->init_amp, p->rho_ref, p->g_x, p->kolmo_amp,
                           p->kolmo_k};
    for (double v : vals)
        if (!std::isfinite(v)) return LB_ERR_INVALID;
    if (p->init_amp < 0.0 || p->init_amp >= 1.0 || p->rho_ref < 0.0) return LB_ERR_INVALID;
    return LB_OK;
}

lb_status cuda_status(cudaError_t e) {
    if (e == cudaSuccess) return LB_OK;
    cudaGetLastError();
    if (e == cudaErrorMemoryAllocation) return LB_ERR_NOMEM;
    return LB_ERR_CUDA;
}

int device_sms(int device) {
    int sms = 0;
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device) != cudaSuccess || sms < 1)
        sms = 1;
    return sms;
}

// L2 bytes of the current device (0 if unknown).
static long long device_l2_bytes() {
    int dev = 0, l2 = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&l2, cudaDevAttrL2CacheSize, dev) != cudaSuccess)
        return 0;
    return l2;
}

static Geom make_geom(const lb_params* p) {
    Geom g;
    const int prec = p->precision;
    const int es = kernel_elem_bytes(prec);
    const int gx = kernel_ghost_x(prec);
    // a row of pairs is 2 * pitch * es bytes: keep pitch * es a multiple of 16
    const int align_pairs = 16 / es;
    const int box_w = kernel_tile_x(prec) + 2 * gx;
    int pitch = (int)align_up((size_t)(p->nx + 2 * gx), (size_t)align_pairs);
    if (pitch < box_w) pitch = box_w;
    g.nx = p->nx;
    g.ny = p->ny;
    g.pitch = pitch;
    g.rows = p->ny + 2 * kGY;
    g.plane = (long long)g.rows * g.pitch;
    g.gx = gx;
    g.periodic = p->boundary == LB_PERIODIC ? 1 : 0;
    // the tile stores end at the last 16-byte boundary of a row's lattice part
    const int pair_bytes = 2 * es;
    g.x_tail = (p->nx + gx) * pair_bytes / 16 * 16 / pair_bytes - gx;
    return g;
}

// Device region of one lattice: stats, observe slots, wall columns, two
// buffers.
struct Region {
    size_t stats, slots, wallx, wsum, f0, f1, total, fbytes;
};
static Region region_layout(const lb_params* p) {
    Geom g = make_geom(p);
    const int tx = kernel_tile_x(p->precision), ty = kernel_tile_y(p->precision);
    const size_t ntiles = (size_t)((p->nx + tx - 1) / tx) * (size_t)((p->ny + ty - 1) / ty);
    Region r;
    size_t off = 0;
    r.stats = off;
    off = align_up(off + sizeof(DevStats), kAlign);
    r.slots = off;
    off = align_up(off + sizeof(double) * 4 * ntiles, kAlign);
    // the step's wall-momentum pair of every wall site (bottom row, then top
    // row), in the compute precision (at most two doubles)
    r.wallx = off;
    off = align_up(off + (size_t)2 * (size_t)p->nx * 2 * sizeof(double), kAlign);
    // their sums per strip (at most nx strips), bottom then top
    r.wsum = off;
    off = align_up(off + (size_t)2 * (size_t)p->nx * sizeof(double), kAlign);
    r.fbytes = align_up((size_t)18 * (size_t)g.plane * (size_t)kernel_elem_bytes(p->precision), kAlign);
    r.f0 = off;
    off += r.fbytes;
    r.f1 = off;
    off += r.fbytes;
    r.total = off;
    return r;
}

size_t lattice_bytes(const lb_params* p) { return region_layout(p).total; }

template <typename C>
static void fill_coef(Coef<C>& k, const lb_params* p) {
    const double Ga[2] = {p->G_A1, p->G_B1};
    const double Gr[2] = {p->G_A2, p->G_B2};
    // K(|d|^2) per species: attraction on the first belt (|d|^2 = 1, 2) with
    // the D2Q9 weights, repulsion on both belts with the weights p; the row
    // sums use K(1), K(2), K(5) and 2 K(4), 2 K(5), 2 K(8) (doubling is exact)
    const int c2s[6] = {1, 2, 5, 4, 5, 8};
    for (int r = 0; r < 6; ++r) {
        const int c2 = c2s[r];
        C K[2];
        for (int s = 0; s < 2; ++s)
            K[s] = (C)((c2 <= 2 ? Ga[s] * w_weight(c2) : 0.0) + Gr[s] * p_weight(c2));
        const C f = r < 3 ? C(1) : C(2);
        k.KC[r].x = K[0] * f;
        k.KC[r].y = K[1] * f;
    }
    k.WC[0].x = k.WC[0].y = (C)w_weight(1);
    k.WC[1].x = k.WC[1].y = (C)w_weight(2);
    // Offsets are taken from rho_ref rounded to the compute precision, so that
    // rho = rho_ref + sum_i h_i holds with the same rho_ref on every path.
    const double rref = (double)(C)(p->rho_ref > 0.0 ? p->rho_ref : p->rho0);
    const double pref = p->psi_form == LB_PSI_RHO0 ? p->rho0 : std::sqrt(p->rho0);
    k.gx_rho0 = (C)(p->G_X / p->rho0);
    k.rho_ref = (C)rref;
    k.psi_ref = (C)(pref * (1.0 - std::exp(-rref / p->rho0)));
    k.psi_scale = (C)(pref * std::exp(-rref / p->rho0));
    k.inv_rho0 = (C)(1.0 / p->rho0);
    k.tau3[0] = (C)(3.0 * p->tau_A);
    k.tau3[1] = (C)(3.0 * p->tau_B);
    k.omega[0] = (C)(1.0 / p->tau_A);
    k.omega[1] = (C)(1.0 / p->tau_B);
    // omega w times the storage scale (a power of two: exact), per class of
    // |c_i|^2; the products are rounded once, in the compute precision
    const double sc = std::ldexp(1.0, kernel_scale_log2(p->precision));
    const double wc[3] = {4.0 / 9.0, 1.0 / 9.0, 1.0 / 36.0};
    for (int c = 0; c < 3; ++c) {
        k.omw[c].x = (C)(sc * wc[c] / p->tau_A);
        k.omw[c].y = (C)(sc * wc[c] / p->tau_B);
    }
    k.omm.x = (C)(1.0 - 1.0 / p->tau_A);
    k.omm.y = (C)(1.0 - 1.0 / p->tau_B);
    k.u_wall = (C)p->u_wall;
    k.g_x = (C)p->g_x;
    k.kolmo_amp = (C)p->kolmo_amp;
    k.kolmo_w = (C)(2.0 * M_PI * p->kolmo_k / p->ny);
    k.sr = (p->rounding == LB_ROUND_STOCHASTIC &&
            (p->precision == LB_FP16_OFFSET || p->precision == LB_BF16_OFFSET)) ? 1 : 0;
    k.source = p->force_scheme == LB_FORCE_SOURCE ? 1 : 0;
    k.has_accel = (p->g_x != 0.0 || p->kolmo_amp != 0.0) ? 1 : 0;
}

template <typename C>
static LatVals<C> vals_of(const Coef<C>& k) {
    LatVals<C> v;
    v.rho_ref = k.rho_ref;
    v.psi_ref = k.psi_ref;
    v.psi_scale = k.psi_scale;
    v.inv_rho0 = k.inv_rho0;
    v.gx_rho0 = k.gx_rho0;
    v.u_wall = k.u_wall;
    v.kolmo_w = k.kolmo_w;
    return v;
}

typedef CUresult (*EncodeTiledFn)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*,
                                  const cuuint64_t*, const cuuint64_t*, const cuuint32_t*,
                                  const cuuint32_t*, CUtensorMapInterleave, CUtensorMapSwizzle,
                                  CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

static EncodeTiledFn encode_fn() {
    static EncodeTiledFn fn = nullptr;
    if (!fn) {
        void* ptr = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &ptr, 12000, cudaEnableDefault,
                                             &q) != cudaSuccess ||
            q != cudaDriverEntryPointSuccess)
            return nullptr;
        fn = reinterpret_cast<EncodeTiledFn>(ptr);
    }
    return fn;
}

// TMA descriptor of one population buffer: 9 direction planes of interleaved
// (A, B) pairs, a row holding 2 * pitch elements.  Box: cols pairs x rows x
// 9 planes.  The descriptor spans the first ext_pairs pairs of each of the
// first ext_rows rows (all of the padded plane when 0): a store clips what
// falls outside.
static lb_status make_tmap(CUtensorMap* m, int precision, const Geom& g, void* base, int cols,
                           int rows, int ext_pairs = 0, int ext_rows = 0) {
    EncodeTiledFn fn = encode_fn();
    if (!fn) return LB_ERR_CUDA;
    const int es = kernel_elem_bytes(precision);
    CUtensorMapDataType dt = precision == LB_FP64   ? CU_TENSOR_MAP_DATA_TYPE_FLOAT64
                             : precision == LB_FP32 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT32
                                                    : CU_TENSOR_MAP_DATA_TYPE_UINT16;
    cuuint64_t dims[3] = {(cuuint64_t)(2 * (ext_pairs > 0 ? ext_pairs : g.pitch)),
                          (cuuint64_t)(ext_rows > 0 ? ext_rows : g.rows), 9};
    cuuint64_t strides[2] = {(cuuint64_t)(2 * g.pitch) * es,
                             (cuuint64_t)g.rows * (cuuint64_t)(2 * g.pitch) * es};
    cuuint32_t box[3] = {(cuuint32_t)(2 * cols), (cuuint32_t)rows, 9};
    cuuint32_t estr[3] = {1, 1, 1};
    CUresult r = fn(m, dt, 3, base, dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                    CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                    CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    return r == CUDA_SUCCESS ? LB_OK : LB_ERR_CUDA;
}

lb_status lattice_setup(Lattice& L, const lb_params* p, char* region) {
    L.p = *p;
    L.g = make_geom(p);
    Region r = region_layout(p);
    L.region = region;
    L.st = reinterpret_cast<DevStats*>(region + r.stats);
    L.slots = reinterpret_cast<double*>(region + r.slots);
    L.wallx = region + r.wallx;
    L.wsum = reinterpret_cast<double*>(region + r.wsum);
    L.fbuf[0] = region + r.f0;
    L.fbuf[1] = region + r.f1;
    L.fbytes = r.fbytes;
    L.cur = 0;
    L.pull = 0;
    L.inited = false;
    L.t = 0;
    L.err_latched = 0;
    const int tx = kernel_tile_x(p->precision), ty = kernel_tile_y(p->precision);
    L.nstrips = (p->nx + tx - 1) / tx;
    L.ntiles_y = (p->ny + ty - 1) / ty;
    L.seg = 1;
    fill_coef(L.kd, p);
    fill_coef(L.kf, p);
    const int bx = tx + 2 * L.g.gx;
    lb_status s = LB_OK;
    for (int b = 0; b < 2 && s == LB_OK; ++b) {
        s = make_tmap(&L.tblock[b], p->precision, L.g, L.fbuf[b], bx, kernel_block_rows(p->precision));
        // Tile stores end at the lattice's last row and at the last 16-byte
        // boundary of its rows (x_tail): a clipped bulk store writes up to a
        // 16-byte boundary, which would reach into the ghost column beside
        // an unaligned last lattice column and race with the plain stores
        // of the ghost copies.  Columns x_tail .. nx - 1 get plain stores.
        if (s == LB_OK)
            s = make_tmap(&L.ttile[b], p->precision, L.g, L.fbuf[b], tx, ty, L.g.x_tail + L.g.gx,
                          p->ny + kGY);
        if (s == LB_OK) s = make_tmap(&L.tobs[b], p->precision, L.g, L.fbuf[b], bx, ty + 2 * kGY);
    }
    return s;
}

// Load-balance model of the persistent step kernel: items are segments of
// `seg` tiles of the column strips; CTA b takes items b, b + G, ...  A CTA's
// cost is its tiles plus a quarter tile per item (the first tile of an item
// computes 12 rather than 8 deviation rows).  Returns the seg in [1, 64]
// minimising the most loaded CTA (ties: longer segments).
int choose_seg(const int* nstrips, const int* ntiles_y, int nlat, int G) {
    int best_seg = 1;
    double best = 1e300;
    std::vector<double> cost;
    for (int seg = 1; seg <= 64; ++seg) {
        long long items = 0;
        for (int l = 0; l < nlat; ++l) items += (long long)nstrips[l] * ((ntiles_y[l] + seg - 1) / seg);
        const int g = items < G ? (int)items : G;
        if (g <= 0) continue;
        cost.assign((size_t)g, 0.0);
        long long it = 0;
        for (int l = 0; l < nlat; ++l) {
            const int nseg = (ntiles_y[l] + seg - 1) / seg;
            for (int sg = 0; sg < nseg; ++sg) {
                const int size = (sg + 1) * seg <= ntiles_y[l] ? seg : ntiles_y[l] - sg * seg;
                for (int sx = 0; sx < nstrips[l]; ++sx, ++it) cost[(size_t)(it % g)] += size + 0.25;
            }
        }
        double mx = 0.0;
        for (double c : cost) mx = c > mx ? c : mx;
        if (mx <= best) {
            best = mx;
            best_seg = seg;
        }
    }
    return best_seg;
}

int max_spt(int precision) { return precision == LB_FP64 ? 1 : 2; }
int default_spt(int precision) { return max_spt(precision); }
int tiles_y(const Lattice& L, int spt) {
    const int ty = kernel_tile_y(L.p.precision) * spt;
    return (L.p.ny + ty - 1) / ty;
}

template <typename C>
static void fill_desc(LatDesc<C>& d, const Lattice& L, const Coef<C>& k, int ntiles) {
    memset(&d, 0, sizeof(d));
    for (int b = 0; b < 2; ++b) {
        d.tin[b] = L.tblock[b];
        d.tout[b] = L.ttile[b];
        d.fbuf[b] = L.fbuf[b];
    }
    d.g = L.g;
    d.v = vals_of(k);
    d.st = L.st;
    d.wallx = L.wallx;
    d.wsum = L.wsum;
    d.nstrips = L.nstrips;
    d.ntiles_y = ntiles;
    d.stress_every = L.p.stress_every;
    d.stress_t0 = L.p.stress_t0;
    d.inv_nx = 1.0 / L.p.nx;
}

size_t launch_area_doubles(size_t tiles, size_t strips, int sms) {
    // items (int4, at most one per tile and strip) | CTA offsets
    return 2 * (tiles + strips) + ((size_t)sms + 2) / 2 + 8;
}

namespace {

struct Item {
    int lat, strip, ty_a, ty_b;
};

// seg > 0: segments of seg tiles, numbered lattice by lattice, segment row by
// segment row, strip by strip; CTA b takes items b, b + G, ...
// seg < 0: the tiles of all lattices in strip order (lattice, strip, tile
// row) cut into G contiguous runs of equal estimated cost, each run cut
// again at strip boundaries: every CTA walks one or two strips.
void partition(Lattice* const* lats, int nlat, int seg, int spt, int sms, std::vector<Item>& items,
               std::vector<int>& cta, int* grid) {
    items.clear();
    cta.clear();
    std::vector<int> nty((size_t)nlat);
    long long tiles = 0;
    for (int l = 0; l < nlat; ++l) {
        nty[(size_t)l] = tiles_y(*lats[l], spt);
        tiles += (long long)lats[l]->nstrips * nty[(size_t)l];
    }
    // Tile costs relative to a full interior tile, fitted on GB300 to the
    // per-CTA times of single steps (5 x 512^2 sweeps, periodic and Couette,
    // FP32 and FP16, 16-row tiles): tiles writing periodic ghost columns
    // +0.21; ghost rows +0.25 where they leave through the staging tile, +0.02
    // where the threads store them directly; Couette tiles holding a wall row
    // (mirror, bounce-back, wall momentum) 1.38; ragged tiles 1.07; and an
    // item's start (its block ring fills, it computes four more deviation
    // rows) 0.8 of a tile.
    auto cost = [&](int l, int sx, int ty) {
        const Lattice& L = *lats[l];
        const int tx = kernel_tile_x(L.p.precision), tyy = kernel_tile_y(L.p.precision) * spt;
        const int x0 = sx * tx, y0 = ty * tyy;
        const bool full = x0 + tx <= L.p.nx && y0 + tyy <= L.p.ny;
        if (!full) return 1.07;
        const bool per = L.g.periodic != 0;
        if (!per && (y0 == 0 || y0 + tyy >= L.p.ny)) return 1.38;
        double c = 1.0;
        if (x0 < 3 || x0 + tx > L.p.nx - 3) c += 0.21;
        if (per && (y0 < 3 || y0 + tyy > L.p.ny - 3)) c += kernel_staged(L.p.precision, spt) ? 0.25 : 0.02;
        return c;
    };
    const double kItemStart = 0.8;
    if (seg > 0) {
        // Segments in band order (all strips of a segment row, row after row),
        // each given to the CTA with the least work so far (the lowest index
        // among equals): round-robin dealing when costs are equal, while the
        // CTAs that draw the costlier edge segments take fewer of them.
        std::vector<Item> all;
        for (int l = 0; l < nlat; ++l) {
            const int ns = lats[l]->nstrips, nt = nty[(size_t)l];
            for (int a = 0; a < nt; a += seg)
                for (int sx = 0; sx < ns; ++sx) all.push_back({l, sx, a, std::min(a + seg, nt)});
        }
        const int G = (int)std::min<long long>((long long)all.size(), sms);
        std::vector<std::vector<int>> mine((size_t)G);
        typedef std::pair<double, int> Load;   // (work so far, CTA): smallest first
        std::priority_queue<Load, std::vector<Load>, std::greater<Load>> heap;
        for (int b = 0; b < G; ++b) heap.push({0.0, b});
        for (size_t k = 0; k < all.size(); ++k) {
            const Load top = heap.top();
            heap.pop();
            double w = kItemStart;
            for (int ty = all[k].ty_a; ty < all[k].ty_b; ++ty) w += cost(all[k].lat, all[k].strip, ty);
            mine[(size_t)top.second].push_back((int)k);
            heap.push({top.first + w, top.second});
        }
        for (int b = 0; b < G; ++b) {
            cta.push_back((int)items.size());
            for (int k : mine[(size_t)b]) items.push_back(all[(size_t)k]);
        }
        cta.push_back((int)items.size());
        *grid = G;
        return;
    }
    // Contiguous runs over the tiles in order (lattice, strip, tile row); a
    // run pays an item start where it begins and where it crosses into the
    // next strip.  The runs minimise the largest run cost: the smallest bound
    // B for which runs filled greedily (a run takes the next tile while its
    // cost stays within B) number at most sms, found by bisection -- at most
    // one tile above the mean, where cutting at equal cumulative cost lets
    // some runs overshoot by a whole tile.
    std::vector<double> tc;
    std::vector<char> sbeg;   // tile begins a strip
    tc.reserve((size_t)tiles);
    sbeg.reserve((size_t)tiles);
    double sum = 0.0, cmax = 0.0;
    for (int l = 0; l < nlat; ++l)
        for (int sx = 0; sx < lats[l]->nstrips; ++sx)
            for (int ty = 0; ty < nty[(size_t)l]; ++ty) {
                tc.push_back(cost(l, sx, ty));
                sbeg.push_back(ty == 0 ? 1 : 0);
                sum += tc.back() + (ty == 0 ? kItemStart : 0.0);
                cmax = std::max(cmax, tc.back());
            }
    // runs needed under bound B; with starts, the first tile of each run
    auto runs_for = [&](double B, std::vector<long long>* starts) -> long long {
        long long n = 0;
        double acc = 0.0;
        for (long long k = 0; k < tiles; ++k) {
            const double add = tc[(size_t)k] + (sbeg[(size_t)k] ? kItemStart : 0.0);
            if (n > 0 && acc + add <= B) {
                acc += add;
            } else {
                ++n;
                if (starts) starts->push_back(k);
                acc = tc[(size_t)k] + kItemStart;
            }
        }
        return n;
    };
    double lo = cmax + kItemStart, hi = sum + kItemStart * (double)sms;
    if (runs_for(lo, nullptr) > sms)
        for (int it = 0; it < 60 && hi - lo > 1e-6 * hi; ++it) {
            const double mid = 0.5 * (lo + hi);
            if (runs_for(mid, nullptr) <= sms) hi = mid; else lo = mid;
        }
    else
        hi = lo;
    std::vector<long long> starts;
    runs_for(hi, &starts);
    const int G = (int)starts.size();
    starts.push_back(tiles);
    // tile k -> (lattice, strip, tile row), walking the same order
    int l = 0, sx = 0, ty = 0;
    for (int b = 0; b < G; ++b) {
        cta.push_back((int)items.size());
        long long k = starts[(size_t)b];
        while (k < starts[(size_t)b + 1]) {
            const int nt = nty[(size_t)l];
            const int take = (int)std::min<long long>(nt - ty, starts[(size_t)b + 1] - k);
            items.push_back({l, sx, ty, ty + take});
            k += take;
            ty += take;
            if (ty == nt) {
                ty = 0;
                if (++sx == lats[l]->nstrips) {
                    sx = 0;
                    ++l;
                }
            }
        }
    }
    cta.push_back((int)items.size());
    *grid = G;
}

}  // namespace

// Default partition: cost-balanced contiguous runs while each CTA has up to
// ~40 tiles of 8 rows (measured faster on 512^2-1024^2 lattices), the
// load-balance model's dealt segments beyond (their CTAs sweep a band of
// rows together, which keeps the halo columns in L2 on large lattices);
// `tiles` counts tiles of 8 spt rows.
static int default_seg(long long tiles, int spt, const int* ns, const int* nt, int nlat, int sms) {
    return tiles * spt <= 40LL * sms ? -1 : choose_seg(ns, nt, nlat, sms);
}

// Host-only plan of a launch's work items (lb_plan_partition).
lb_status plan_partition(const lb_params* ps, int nlat, int seg, int tile_rows, int sms,
                         int32_t* items, int32_t* nitems, int32_t* cta, int32_t* grid,
                         int32_t* seg_used) {
    if (!ps || nlat < 1 || sms < 1 || !nitems || !grid || !seg_used) return LB_ERR_INVALID;
    std::vector<Lattice> lv((size_t)nlat);
    std::vector<Lattice*> lp((size_t)nlat);
    std::vector<int> ns((size_t)nlat), nt((size_t)nlat);
    if (validate_params(&ps[0]) != LB_OK) return LB_ERR_INVALID;
    const int ty8 = kernel_tile_y(ps[0].precision);
    if (tile_rows != 0 && tile_rows != ty8 && tile_rows != 2 * ty8) return LB_ERR_INVALID;
    const int spt = tile_rows == 0 ? 1 : tile_rows / ty8;
    if (spt > max_spt(ps[0].precision)) return LB_ERR_INVALID;
    long long tiles = 0;
    for (int l = 0; l < nlat; ++l) {
        if (validate_params(&ps[l]) != LB_OK || ps[l].precision != ps[0].precision)
            return LB_ERR_INVALID;
        Lattice& L = lv[(size_t)l];
        L.p = ps[l];
        L.g = make_geom(&ps[l]);
        const int tx = kernel_tile_x(ps[l].precision);
        L.nstrips = (ps[l].nx + tx - 1) / tx;
        L.ntiles_y = tiles_y(L, 1);
        lp[(size_t)l] = &L;
        ns[(size_t)l] = L.nstrips;
        nt[(size_t)l] = tiles_y(L, spt);
        tiles += (long long)L.nstrips * nt[(size_t)l];
    }
    const int s = seg != 0 ? seg : default_seg(tiles, spt, ns.data(), nt.data(), nlat, sms);
    std::vector<Item> it;
    std::vector<int> c;
    int G = 0;
    partition(lp.data(), nlat, s, spt, sms, it, c, &G);
    const int cap_items = *nitems, cap_cta = *grid;
    *nitems = (int32_t)it.size();
    *grid = G;
    *seg_used = s;
    if (cap_items < (int)it.size() || cap_cta < G + 1 || !items || !cta) return LB_ERR_INVALID;
    for (size_t k = 0; k < it.size(); ++k) {
        items[4 * k] = it[k].lat;
        items[4 * k + 1] = it[k].strip;
        items[4 * k + 2] = it[k].ty_a;
        items[4 * k + 3] = it[k].ty_b;
    }
    for (int b = 0; b <= G; ++b) cta[b] = c[(size_t)b];
    return LB_OK;
}

lb_status launch_build(Launch& Ln, Lattice* const* lats, int nlat, void* descs, double* slots,
                       unsigned int* ticket, int sms, cudaStream_t stream, void* host_scratch,
                       int forced_seg, int spt) {
    if (nlat < 1) return LB_ERR_INVALID;
    const int prec = lats[0]->p.precision;
    if (spt < 1 || spt > max_spt(prec)) return LB_ERR_INVALID;
    std::vector<int> ns((size_t)nlat), nt((size_t)nlat);
    bool allper = true, gen = false, tau1 = true;
    long long tiles = 0, strips = 0;
    for (int l = 0; l < nlat; ++l) {
        ns[(size_t)l] = lats[l]->nstrips;
        nt[(size_t)l] = tiles_y(*lats[l], spt);
        allper = allper && lats[l]->g.periodic;
        gen = gen || lats[l]->kd.source || lats[l]->kd.has_accel;
        // 1 - omega rounds to zero in the compute precision for both species:
        // the collision does not read the populations (kernel variant bit 4)
        tau1 = tau1 && (prec == LB_FP64
                            ? (lats[l]->kd.omm.x == 0.0 && lats[l]->kd.omm.y == 0.0)
                            : (lats[l]->kf.omm.x == 0.0f && lats[l]->kf.omm.y == 0.0f));
        tiles += (long long)lats[l]->nstrips * nt[(size_t)l];
        strips += lats[l]->nstrips;
    }
    const int seg = forced_seg != 0 ? forced_seg : default_seg(tiles, spt, ns.data(), nt.data(), nlat, sms);
    std::vector<Item> items;
    std::vector<int> cta;
    int grid = 0;
    partition(lats, nlat, seg, spt, sms, items, cta, &grid);
    const int nitems = (int)items.size();
    const size_t dsz = prec == LB_FP64 ? sizeof(LatDesc<double>) : sizeof(LatDesc<float>);
    char* hs = reinterpret_cast<char*>(host_scratch);
    for (int l = 0; l < nlat; ++l) {
        lats[l]->seg = seg;
        if (prec == LB_FP64)
            fill_desc(*reinterpret_cast<LatDesc<double>*>(hs + l * dsz), *lats[l], lats[l]->kd,
                      nt[(size_t)l]);
        else
            fill_desc(*reinterpret_cast<LatDesc<float>*>(hs + l * dsz), *lats[l], lats[l]->kf,
                      nt[(size_t)l]);
    }
    // device tables: items (16-byte aligned), CTA offsets
    int4* d_items = reinterpret_cast<int4*>(slots);
    int* d_cta = reinterpret_cast<int*>(d_items + nitems);
    static_assert(sizeof(Item) == sizeof(int4), "item layout");
    cudaError_t e = cudaMemcpyAsync(descs, hs, dsz * nlat, cudaMemcpyHostToDevice, stream);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(d_items, items.data(), sizeof(int4) * (size_t)nitems, cudaMemcpyHostToDevice, stream);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(d_cta, cta.data(), sizeof(int) * cta.size(), cudaMemcpyHostToDevice, stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(stream);   // host buffers are reused
    if (e != cudaSuccess) return cuda_status(e);
    Ln.precision = prec;
    Ln.variant = (allper ? 1 : 0) | (gen ? 2 : 0) | (tau1 ? 4 : 0);
    Ln.spt = spt;
    Ln.grid = dim3((unsigned)grid, 1, 1);
    Ln.nitems = nitems;
    Ln.seg = seg;
    // One buffer of every lattice within 80 % of L2: the step's output can
    // stay in L2 for the next step, next to the input streaming through.
    long long buf = 0;
    for (int l = 0; l < nlat; ++l) buf += (long long)lats[l]->fbytes;
    const int l2_resident = buf * 5 <= device_l2_bytes() * 4 ? 1 : 0;
    // With the collision free of the populations (tau = 1), a tile's ring
    // slots can be refilled as soon as its density phase is done.  Measured
    // on GB300: that deeper prefetch pays where the step's input comes
    // largely from L2 (one buffer of every lattice within L2) and for the
    // 16-bit formats (issue-bound), but costs FP32 lattices streaming from
    // DRAM (4096^2, 16-row tiles: 39.2 against 42.3 GLUPS), which keep the
    // refill after the site phase.
    const int early_release = tau1 && (l2_resident || prec == LB_FP16_OFFSET || prec == LB_BF16_OFFSET) ? 1 : 0;
    if (prec == LB_FP64) {
        BatchArgs<double>& a = Ln.ad;
        a.k = lats[0]->kd;
        a.lat = reinterpret_cast<const LatDesc<double>*>(descs);
        a.nlat = nlat;
        a.nitems = nitems;
        a.items = d_items;
        a.cta_items = d_cta;
        a.ticket = ticket;
        a.l2_resident = l2_resident;
        a.early_release = early_release;
    } else {
        BatchArgs<float>& a = Ln.af;
        a.k = lats[0]->kf;
        a.lat = reinterpret_cast<const LatDesc<float>*>(descs);
        a.nlat = nlat;
        a.nitems = nitems;
        a.items = d_items;
        a.cta_items = d_cta;
        a.ticket = ticket;
        a.l2_resident = l2_resident;
        a.early_release = early_release;
    }
    return LB_OK;
}

lb_status launch_run(const Launch& Ln, cudaStream_t s) {
    const void* args = Ln.precision == LB_FP64 ? (const void*)&Ln.ad : (const void*)&Ln.af;
    return cuda_status(launch_step(Ln.precision, args, Ln.variant, Ln.spt, Ln.grid, s));
}

static lb_status lattice_observe_pull(Lattice& L, int obs, double* out, int q0, int q1, int pull,
                                      cudaStream_t s);
lb_status lattice_observe(Lattice& L, int obs, double* out, int q0, int q1, cudaStream_t s) {
    return lattice_observe_pull(L, obs, out, q0, q1, L.pull, s);
}

static lb_status lattice_observe_pull(Lattice& L, int obs, double* out, int q0, int q1, int pull,
                                      cudaStream_t s) {
    const int tx = kernel_tile_x(L.p.precision), ty = kernel_tile_y(L.p.precision);
    dim3 grid((unsigned)((L.p.nx + tx - 1) / tx), (unsigned)((L.p.ny + ty - 1) / ty), 1);
    cudaError_t e;
    if (L.p.precision == LB_FP64) {
        StepArgs<double> a;
        memset(&a, 0, sizeof(a));
        a.g = L.g;
        a.k = L.kd;
        a.st = L.st;
        a.slots = L.slots;
        a.pull = pull;
        a.obs = obs;
        a.obs_out = out;
        a.q0 = q0;
        a.q1 = q1;
        e = launch_observe(L.p.precision, &L.tobs[L.cur], &a, grid, s);
    } else {
        StepArgs<float> a;
        memset(&a, 0, sizeof(a));
        a.g = L.g;
        a.k = L.kf;
        a.st = L.st;
        a.slots = L.slots;
        a.pull = pull;
        a.obs = obs;
        a.obs_out = out;
        a.q0 = q0;
        a.q1 = q1;
        e = launch_observe(L.p.precision, &L.tobs[L.cur], &a, grid, s);
    }
    return cuda_status(e);
}

lb_status lattice_read_stats(Lattice& L, DevStats* out, cudaStream_t s) {
    cudaError_t e = cudaMemcpyAsync(out, L.st, sizeof(DevStats), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return cuda_status(e);
    L.err_latched |= out->err;
    if (L.err_latched & ERR_TIMEOUT) return LB_ERR_TIMEOUT;
    if (L.err_latched & ERR_NONFINITE) return LB_ERR_NONFINITE;
    return LB_OK;
}

// The first step >= t at which the wall momentum is sampled:
// stress_t0 + k stress_every, k >= 0.
static long long first_sample(const lb_params& p, long long t) {
    if (t <= p.stress_t0) return p.stress_t0;
    const long long every = p.stress_every > 0 ? p.stress_every : 1;
    return p.stress_t0 + (t - p.stress_t0 + every - 1) / every * every;
}

static lb_status lattice_reset(Lattice& L, cudaStream_t s) {
    cudaError_t e = cudaMemsetAsync(L.st, 0, sizeof(DevStats), s);   // t = 0, cur = 0, pull = 0
    L.next_sample = first_sample(L.p, 0);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(&L.st->next_sample, &L.next_sample, sizeof(long long), cudaMemcpyHostToDevice, s);
    if (e != cudaSuccess) return cuda_status(e);
    L.t = 0;
    L.cur = 0;
    L.pull = 0;
    L.inited = true;
    L.err_latched = 0;
    return LB_OK;
}

static void* coef_ptr(Lattice& L) {
    return L.p.precision == LB_FP64 ? (void*)&L.kd : (void*)&L.kf;
}

lb_status lattice_init_seeded(Lattice& L, uint64_t seed, cudaStream_t s) {
    lb_status st = lattice_reset(L, s);
    if (st != LB_OK) return st;
    return cuda_status(launch_init_seeded(L.p.precision, L.g, coef_ptr(L), L.fbuf[0], L.p.rho0,
                                          L.p.init_amp, L.p.u_wall, L.p.init_shear,
                                          (unsigned long long)seed, s));
}

lb_status lattice_init_fields(Lattice& L, const double* rho_A, const double* rho_B,
                              const double* ux, const double* uy, cudaStream_t s) {
    lb_status st = lattice_reset(L, s);
    if (st != LB_OK) return st;
    const size_t n = (size_t)L.p.nx * L.p.ny;
    // Stage the four FP64 fields in buffer 1 (its size, 18 planes of at least
    // 2 bytes per padded site, always exceeds 32 bytes per site).
    double* stage = reinterpret_cast<double*>(L.fbuf[1]);
    cudaError_t e = cudaMemcpyAsync(stage, rho_A, n * 8, cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(stage + n, rho_B, n * 8, cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess)
        e = ux ? cudaMemcpyAsync(stage + 2 * n, ux, n * 8, cudaMemcpyHostToDevice, s)
               : cudaMemsetAsync(stage + 2 * n, 0, n * 8, s);
    if (e == cudaSuccess)
        e = uy ? cudaMemcpyAsync(stage + 3 * n, uy, n * 8, cudaMemcpyHostToDevice, s)
               : cudaMemsetAsync(stage + 3 * n, 0, n * 8, s);
    if (e != cudaSuccess) return cuda_status(e);
    e = launch_init_fields(L.p.precision, L.g, coef_ptr(L), L.fbuf[0], stage, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    return cuda_status(e);
}

lb_status lattice_load_populations(Lattice& L, const double* f, long long t, int pulled,
                                   cudaStream_t s) {
    if (t < 0 || (pulled != 0 && pulled != 1) || (pulled && t < 1)) return LB_ERR_INVALID;
    lb_status st = lattice_reset(L, s);
    if (st != LB_OK) return st;
    const size_t n = (size_t)L.p.nx * L.p.ny;
    // Stage whole directions (both species, 16 bytes per site) in buffer 1.
    int per = (int)(L.fbytes / (n * 16));
    if (per < 1) return LB_ERR_UNSUPPORTED;
    double* stage = reinterpret_cast<double*>(L.fbuf[1]);
    cudaError_t e = cudaSuccess;
    for (int i0 = 0; i0 < 9 && e == cudaSuccess; i0 += per) {
        const int i1 = i0 + per < 9 ? i0 + per : 9;
        for (int i = i0; i < i1 && e == cudaSuccess; ++i)
            for (int sp = 0; sp < 2 && e == cudaSuccess; ++sp)
                e = cudaMemcpyAsync(stage + ((size_t)(i - i0) * 2 + sp) * n,
                                    f + ((size_t)sp * 9 + i) * n, n * 8, cudaMemcpyHostToDevice, s);
        if (e == cudaSuccess) e = launch_load_pops(L.p.precision, L.g, coef_ptr(L), L.fbuf[0], stage, i0, i1, s);
        if (e == cudaSuccess) e = cudaStreamSynchronize(s);   // the stage is reused
    }
    if (e == cudaSuccess) e = cudaMemcpyAsync(&L.st->t, &t, sizeof(long long), cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(&L.st->pull, &pulled, sizeof(int), cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);   // the reset's copy has read next_sample
    L.next_sample = first_sample(L.p, t);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(&L.st->next_sample, &L.next_sample, sizeof(long long), cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return cuda_status(e);
    L.t = t;
    L.pull = pulled;
    return LB_OK;
}

void lattice_advanced(Lattice& L, long long n) {
    if (n <= 0) return;
    L.t += n;
    L.cur ^= (int)(n & 1);
    L.pull = 1;
}

lb_status lattice_fields(Lattice& L, double* rho_A, double* rho_B, double* ux, double* uy,
                         cudaStream_t s) {
    const size_t n = (size_t)L.p.nx * L.p.ny;
    double* out = reinterpret_cast<double*>(L.fbuf[1 - L.cur]);
    lb_status st = lattice_observe(L, OBS_FIELDS, out, 0, 0, s);
    if (st != LB_OK) return st;
    double* dst[4] = {rho_A, rho_B, ux, uy};
    for (int k = 0; k < 4; ++k)
        if (dst[k]) {
            cudaError_t e = cudaMemcpyAsync(dst[k], out + k * n, n * 8, cudaMemcpyDeviceToHost, s);
            if (e != cudaSuccess) return cuda_status(e);
        }
    DevStats ds;
    return lattice_read_stats(L, &ds, s);
}

lb_status lattice_populations(Lattice& L, double* f, cudaStream_t s, int raw) {
    const size_t n = (size_t)L.p.nx * L.p.ny;
    double* out = reinterpret_cast<double*>(L.fbuf[1 - L.cur]);
    int per = (int)(L.fbytes / (n * 8));
    if (per < 1) return LB_ERR_UNSUPPORTED;
    if (per > 18) per = 18;
    for (int q0 = 0; q0 < 18; q0 += per) {
        const int q1 = q0 + per < 18 ? q0 + per : 18;
        lb_status st = lattice_observe_pull(L, OBS_POPS, out, q0, q1, raw ? 0 : L.pull, s);
        if (st != LB_OK) return st;
        cudaError_t e = cudaMemcpyAsync(f + (size_t)q0 * n, out, (size_t)(q1 - q0) * n * 8,
                                        cudaMemcpyDeviceToHost, s);
        if (e == cudaSuccess) e = cudaStreamSynchronize(s);
        if (e != cudaSuccess) return cuda_status(e);
    }
    DevStats ds;
    return lattice_read_stats(L, &ds, s);
}

lb_status lattice_stress(Lattice& L, lb_stress_out* out, cudaStream_t s) {
    lb_status st = lattice_observe(L, OBS_TOTALS, nullptr, 0, 0, s);
    if (st != LB_OK) return st;
    DevStats ds;
    st = lattice_read_stats(L, &ds, s);
    memset(out, 0, sizeof(*out));
    out->mass_A = ds.totals[0];
    out->mass_B = ds.totals[1];
    out->mom_x = ds.totals[2];
    out->mom_y = ds.totals[3];
    out->samples = ds.samples;
    out->step = L.t;
    if (ds.samples > 0) {
        out->sigma_bot = ds.sum_bot / (double)ds.samples;
        out->sigma_top = ds.sum_top / (double)ds.samples;
        out->sigma_mean = 0.5 * (out->sigma_bot - out->sigma_top);
    }
    const double rate = 2.0 * L.p.u_wall / L.p.ny;
    const double mass = ds.totals[0] + ds.totals[1];
    const double rho_mean = mass / ((double)L.p.nx * L.p.ny);
    if (L.p.boundary == LB_COUETTE && rate != 0.0 && rho_mean > 0.0 && ds.samples > 0) {
        out->nu_eff = out->sigma_mean / (rate * rho_mean);
        const double tau = mass > 0.0 ? (L.p.tau_A * ds.totals[0] + L.p.tau_B * ds.totals[1]) / mass
                                      : L.p.tau_A;
        const double nu0 = (tau - 0.5) / 3.0;
        out->response_R = out->nu_eff != 0.0 ? nu0 / out->nu_eff : 0.0;
    }
    return st;
}

}  // namespace lbgb
