// lb_api.cu -- host side of the C ABI declared in include/lb.h.
//
// Owns parameter validation, the device workspace layout, the TMA tensor
// descriptors, the model coefficients handed to the kernels, and the
// host<->device copies of the synchronising calls.  Every step of the model
// runs in the kernels of lb_kernels.cu.
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <new>

#include "lb_internal.h"

using namespace lbgb;

struct lb_handle {
    lb_params p;
    Geom g;
    cudaStream_t stream;
    int device;
    bool owns;             // workspace allocated here with cudaMalloc
    char* ws;
    size_t ws_bytes;
    DevStats* st;
    double* slots;
    char* fbuf[2];
    size_t fbuf_bytes;
    CUtensorMap tmap[2];   // load descriptors (tile + halo boxes) of buffers 0, 1
    CUtensorMap smap[2];   // store descriptors (tile boxes) of buffers 0, 1
    int cur;               // index of the buffer holding the current state
    int pull;              // 1: cur holds post-collision f*(t-1); 0: f(t) in place
    bool inited;
    long long t;
    dim3 grid;             // observe kernel: one CTA per tile
    dim3 grid_step;        // persistent step kernel: one CTA per SM (at most one per tile)
    Coef<double> kd;
    Coef<float> kf;
    unsigned int err_latched;
};

namespace {

constexpr size_t kAlign = 256;
size_t align_up(size_t v, size_t a) { return (v + a - 1) / a * a; }

// Multi-range weights p(|d|^2) (8th-order isotropic, second moment 1/3) and
// the D2Q9 weights w(|d|^2), for the 12 pair representatives used by the
// kernels: (1,0) (0,1) (1,1) (-1,1) (2,0) (0,2) (2,1) (1,2) (-1,2) (-2,1)
// (2,2) (-2,2).
const int kRepC2[12] = {1, 1, 2, 2, 4, 4, 5, 5, 5, 5, 8, 8};
double p_weight(int c2) {
    switch (c2) {
        case 1: return 4.0 / 63.0;
        case 2: return 4.0 / 135.0;
        case 4: return 1.0 / 180.0;
        case 5: return 2.0 / 945.0;
        case 8: return 1.0 / 15120.0;
    }
    return 0.0;
}
double w_weight(int c2) { return c2 == 1 ? 1.0 / 9.0 : c2 == 2 ? 1.0 / 36.0 : 0.0; }

lb_status validate(const lb_params* p) {
    if (!p) return LB_ERR_INVALID;
    if (p->nx < 8 || p->ny < 8 || p->nx > (1 << 20) || p->ny > (1 << 19)) return LB_ERR_INVALID;
    if (p->boundary != LB_PERIODIC && p->boundary != LB_COUETTE) return LB_ERR_INVALID;
    if (p->precision < LB_FP64 || p->precision > LB_BF16_OFFSET) return LB_ERR_INVALID;
    if (p->psi_form != LB_PSI_SQRT_RHO0 && p->psi_form != LB_PSI_RHO0) return LB_ERR_INVALID;
    if (p->force_scheme != LB_FORCE_SHIFT && p->force_scheme != LB_FORCE_SOURCE) return LB_ERR_INVALID;
    if (!(p->tau_A > 0.5) || !(p->tau_B > 0.5) || !(p->rho0 > 0.0)) return LB_ERR_INVALID;
    if (p->stress_every < 1 || p->stress_t0 < 0) return LB_ERR_INVALID;
    const double vals[] = {p->tau_A, p->tau_B, p->G_A1, p->G_A2, p->G_B1, p->G_B2, p->G_X,
                           p->rho0, p->u_wall, p->init_amp, p->rho_ref, p->g_x, p->kolmo_amp,
                           p->kolmo_k};
    for (double v : vals)
        if (!std::isfinite(v)) return LB_ERR_INVALID;
    if (p->init_amp < 0.0 || p->init_amp >= 1.0) return LB_ERR_INVALID;
    return LB_OK;
}

Geom make_geom(const lb_params* p) {
    Geom g;
    const int prec = p->precision;
    const int es = kernel_elem_bytes(prec);
    const int gx = kernel_ghost_x(prec);
    const int align_elems = 16 / es;
    const int box_w = kernel_tile_x(prec) + 2 * gx;
    int pitch = (int)align_up((size_t)(p->nx + 2 * gx), (size_t)align_elems);
    if (pitch < box_w) pitch = box_w;
    g.nx = p->nx;
    g.ny = p->ny;
    g.pitch = pitch;
    g.rows = p->ny + 2 * kGY;
    g.plane = (long long)g.rows * g.pitch;
    g.gx = gx;
    g.periodic = p->boundary == LB_PERIODIC ? 1 : 0;
    return g;
}

dim3 make_grid(const lb_params* p) {
    const int tx = kernel_tile_x(p->precision), ty = kernel_tile_y(p->precision);
    return dim3((unsigned)((p->nx + tx - 1) / tx), (unsigned)((p->ny + ty - 1) / ty), 1);
}

struct WsLayout {
    size_t stats, slots, f0, f1, total, fbytes;
};
WsLayout layout(const lb_params* p) {
    Geom g = make_geom(p);
    dim3 gr = make_grid(p);
    WsLayout L;
    size_t off = 0;
    L.stats = off;
    off = align_up(off + sizeof(DevStats), kAlign);
    L.slots = off;
    off = align_up(off + sizeof(double) * 4 * (size_t)gr.x * gr.y, kAlign);
    L.fbytes = align_up((size_t)18 * (size_t)g.plane * (size_t)kernel_elem_bytes(p->precision), kAlign);
    L.f0 = off;
    off += L.fbytes;
    L.f1 = off;
    off += L.fbytes;
    L.total = off;
    return L;
}

template <typename C>
void fill_coef(Coef<C>& k, const lb_params* p) {
    const double Ga[2] = {p->G_A1, p->G_B1};
    const double Gr[2] = {p->G_A2, p->G_B2};
    for (int s = 0; s < 2; ++s)
        for (int r = 0; r < 12; ++r) {
            const int c2 = kRepC2[r];
            const double v = (r < 4 ? Ga[s] * w_weight(c2) : 0.0) + Gr[s] * p_weight(c2);
            k.K[s][r] = (C)v;
        }
    for (int r = 0; r < 4; ++r) k.W[r] = (C)w_weight(kRepC2[r]);
    k.gx_rho0 = (C)(p->G_X / p->rho0);
    // Offsets are taken from rho_ref rounded to the compute precision, so that
    // rho = rho_ref + sum_i h_i holds with the same rho_ref on every path.
    const double rref = (double)(C)(p->rho_ref > 0.0 ? p->rho_ref : p->rho0);
    const double pref = p->psi_form == LB_PSI_RHO0 ? p->rho0 : std::sqrt(p->rho0);
    k.rho_ref = (C)rref;
    k.psi_ref = (C)(pref * (1.0 - std::exp(-rref / p->rho0)));
    k.psi_scale = (C)(pref * std::exp(-rref / p->rho0));
    k.inv_rho0 = (C)(1.0 / p->rho0);
    k.tau[0] = (C)p->tau_A;
    k.tau[1] = (C)p->tau_B;
    k.omega[0] = (C)(1.0 / p->tau_A);
    k.omega[1] = (C)(1.0 / p->tau_B);
    k.u_wall = (C)p->u_wall;
    k.g_x = (C)p->g_x;
    k.kolmo_amp = (C)p->kolmo_amp;
    k.kolmo_w = (C)(2.0 * M_PI * p->kolmo_k / p->ny);
    k.source = p->force_scheme == LB_FORCE_SOURCE ? 1 : 0;
    k.has_accel = (p->g_x != 0.0 || p->kolmo_amp != 0.0) ? 1 : 0;
}

typedef CUresult (*EncodeTiledFn)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*,
                                  const cuuint64_t*, const cuuint64_t*, const cuuint32_t*,
                                  const cuuint32_t*, CUtensorMapInterleave, CUtensorMapSwizzle,
                                  CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

EncodeTiledFn encode_fn() {
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

lb_status make_tmap(CUtensorMap* m, const lb_params* p, const Geom& g, void* base, bool store) {
    EncodeTiledFn fn = encode_fn();
    if (!fn) return LB_ERR_CUDA;
    const int es = kernel_elem_bytes(p->precision);
    CUtensorMapDataType dt = p->precision == LB_FP64   ? CU_TENSOR_MAP_DATA_TYPE_FLOAT64
                             : p->precision == LB_FP32 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT32
                                                       : CU_TENSOR_MAP_DATA_TYPE_UINT16;
    // 9 direction planes of interleaved (A, B) pairs: a row holds 2 * pitch
    // elements.
    cuuint64_t dims[3] = {(cuuint64_t)(2 * g.pitch), (cuuint64_t)g.rows, 9};
    cuuint64_t strides[2] = {(cuuint64_t)(2 * g.pitch) * es,
                             (cuuint64_t)g.rows * (cuuint64_t)(2 * g.pitch) * es};
    cuuint32_t box[3] = {(cuuint32_t)(2 * (kernel_tile_x(p->precision) + (store ? 0 : 2 * g.gx))),
                         (cuuint32_t)(kernel_tile_y(p->precision) + (store ? 0 : 2 * kGY)), 9};
    cuuint32_t estr[3] = {1, 1, 1};
    CUresult r = fn(m, dt, 3, base, dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                    CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                    CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    return r == CUDA_SUCCESS ? LB_OK : LB_ERR_CUDA;
}

lb_status cuda_status(cudaError_t e) {
    if (e == cudaSuccess) return LB_OK;
    if (e == cudaErrorMemoryAllocation) return LB_ERR_NOMEM;
    return LB_ERR_CUDA;
}

void* coef_ptr(lb_handle* h) {
    return h->p.precision == LB_FP64 ? (void*)&h->kd : (void*)&h->kf;
}

template <typename C>
void fill_args(StepArgs<C>& a, lb_handle* h, const Coef<C>& k) {
    memset(&a, 0, sizeof(a));
    a.g = h->g;
    a.k = k;
    a.st = h->st;
    a.slots = h->slots;
    a.pull = h->pull;
    a.stress_t0 = h->p.stress_t0;
    a.stress_every = h->p.stress_every;
}

// One launch of the step kernel in step (obs = OBS_NONE) or observe mode.
lb_status launch(lb_handle* h, int obs, double* obs_out, int q0, int q1) {
    cudaError_t e;
    if (h->p.precision == LB_FP64) {
        StepArgs<double> a;
        fill_args(a, h, h->kd);
        a.obs = obs;
        a.obs_out = obs_out;
        a.q0 = q0;
        a.q1 = q1;
        a.fout = obs == OBS_NONE ? h->fbuf[1 - h->cur] : nullptr;
        e = launch_step(h->p.precision, &h->tmap[h->cur], &h->smap[1 - h->cur], &a, obs,
                        obs == OBS_NONE ? h->grid_step : h->grid, h->stream);
    } else {
        StepArgs<float> a;
        fill_args(a, h, h->kf);
        a.obs = obs;
        a.obs_out = obs_out;
        a.q0 = q0;
        a.q1 = q1;
        a.fout = obs == OBS_NONE ? h->fbuf[1 - h->cur] : nullptr;
        e = launch_step(h->p.precision, &h->tmap[h->cur], &h->smap[1 - h->cur], &a, obs,
                        obs == OBS_NONE ? h->grid_step : h->grid, h->stream);
    }
    return cuda_status(e);
}

lb_status read_stats(lb_handle* h, DevStats* out) {
    cudaError_t e = cudaMemcpyAsync(out, h->st, sizeof(DevStats), cudaMemcpyDeviceToHost, h->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
    if (e != cudaSuccess) return cuda_status(e);
    h->err_latched |= out->err;
    if (h->err_latched & ERR_TIMEOUT) return LB_ERR_TIMEOUT;
    if (h->err_latched & ERR_NONFINITE) return LB_ERR_NONFINITE;
    return LB_OK;
}

lb_status reset_state(lb_handle* h) {
    cudaError_t e = cudaMemsetAsync(h->st, 0, sizeof(DevStats), h->stream);
    if (e != cudaSuccess) return cuda_status(e);
    h->t = 0;
    h->pull = 0;
    h->inited = true;
    h->err_latched = 0;
    return LB_OK;
}

}  // namespace

extern "C" {

void lb_params_default(lb_params* p) {
    if (!p) return;
    memset(p, 0, sizeof(*p));
    p->nx = 128;
    p->ny = 128;
    p->boundary = LB_PERIODIC;
    p->precision = LB_FP32;
    p->psi_form = LB_PSI_SQRT_RHO0;
    p->force_scheme = LB_FORCE_SHIFT;
    p->stress_every = 1;
    p->tau_A = 1.0;
    p->tau_B = 1.0;
    p->G_A1 = -12.55;
    p->G_A2 = 11.70;
    p->G_B1 = -11.80;
    p->G_B2 = 10.95;
    p->G_X = 0.58;
    p->rho0 = 0.70;
    p->init_amp = 0.03;
}

lb_status lb_workspace_size(const lb_params* p, size_t* bytes) {
    lb_status s = validate(p);
    if (s != LB_OK) return s;
    if (!bytes) return LB_ERR_INVALID;
    *bytes = layout(p).total;
    return LB_OK;
}

static lb_status create_common(const lb_params* p, void* stream, void* ws, size_t bytes, bool owns,
                               lb_handle** out) {
    lb_handle* h = new (std::nothrow) lb_handle();
    if (!h) return LB_ERR_NOMEM;
    h->p = *p;
    h->g = make_geom(p);
    h->grid = make_grid(p);
    h->stream = reinterpret_cast<cudaStream_t>(stream);
    cudaGetDevice(&h->device);
    int sms = 0;
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, h->device) != cudaSuccess || sms < 1)
        sms = 1;
    const unsigned ntiles = h->grid.x * h->grid.y;
    h->grid_step = dim3(ntiles < (unsigned)sms ? ntiles : (unsigned)sms, 1, 1);
    h->owns = owns;
    h->ws = reinterpret_cast<char*>(ws);
    h->ws_bytes = bytes;
    WsLayout L = layout(p);
    h->st = reinterpret_cast<DevStats*>(h->ws + L.stats);
    h->slots = reinterpret_cast<double*>(h->ws + L.slots);
    h->fbuf[0] = h->ws + L.f0;
    h->fbuf[1] = h->ws + L.f1;
    h->fbuf_bytes = L.fbytes;
    h->cur = 0;
    h->pull = 0;
    h->inited = false;
    h->t = 0;
    h->err_latched = 0;
    fill_coef(h->kd, p);
    fill_coef(h->kf, p);
    lb_status s = make_tmap(&h->tmap[0], p, h->g, h->fbuf[0], false);
    if (s == LB_OK) s = make_tmap(&h->tmap[1], p, h->g, h->fbuf[1], false);
    if (s == LB_OK) s = make_tmap(&h->smap[0], p, h->g, h->fbuf[0], true);
    if (s == LB_OK) s = make_tmap(&h->smap[1], p, h->g, h->fbuf[1], true);
    if (s == LB_OK) s = cuda_status(cudaMemsetAsync(h->ws, 0, L.total, h->stream));
    if (s != LB_OK) {
        if (owns) cudaFree(ws);
        delete h;
        return s;
    }
    *out = h;
    return LB_OK;
}

lb_status lb_create(const lb_params* p, void* stream, lb_handle** out) {
    if (!out) return LB_ERR_INVALID;
    *out = nullptr;
    lb_status s = validate(p);
    if (s != LB_OK) return s;
    const size_t bytes = layout(p).total;
    void* ws = nullptr;
    cudaError_t e = cudaMalloc(&ws, bytes);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return e == cudaErrorMemoryAllocation ? LB_ERR_NOMEM : LB_ERR_CUDA;
    }
    return create_common(p, stream, ws, bytes, true, out);
}

lb_status lb_create_in(const lb_params* p, void* stream, void* workspace, size_t bytes,
                       lb_handle** out) {
    if (!out) return LB_ERR_INVALID;
    *out = nullptr;
    lb_status s = validate(p);
    if (s != LB_OK) return s;
    if (!workspace || (reinterpret_cast<uintptr_t>(workspace) % kAlign) != 0) return LB_ERR_INVALID;
    if (bytes < layout(p).total) return LB_ERR_NOMEM;
    return create_common(p, stream, workspace, bytes, false, out);
}

lb_status lb_init_seeded(lb_handle* h, uint64_t seed) {
    if (!h) return LB_ERR_INVALID;
    lb_status s = reset_state(h);
    if (s != LB_OK) return s;
    h->cur = 0;
    return cuda_status(launch_init_seeded(h->p.precision, h->g, coef_ptr(h), h->fbuf[0], h->p.rho0,
                                          h->p.init_amp, h->p.u_wall, h->p.init_shear,
                                          (unsigned long long)seed, h->stream));
}

lb_status lb_init_fields(lb_handle* h, const double* rho_A, const double* rho_B, const double* ux,
                         const double* uy) {
    if (!h || !rho_A || !rho_B) return LB_ERR_INVALID;
    lb_status s = reset_state(h);
    if (s != LB_OK) return s;
    const size_t n = (size_t)h->p.nx * h->p.ny;
    // Stage the four FP64 fields in buffer 1 (its size, 18 planes of at least
    // 2 bytes per padded site, always exceeds 32 bytes per site).
    double* stage = reinterpret_cast<double*>(h->fbuf[1]);
    cudaError_t e = cudaMemcpyAsync(stage, rho_A, n * 8, cudaMemcpyHostToDevice, h->stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(stage + n, rho_B, n * 8, cudaMemcpyHostToDevice, h->stream);
    if (e == cudaSuccess)
        e = ux ? cudaMemcpyAsync(stage + 2 * n, ux, n * 8, cudaMemcpyHostToDevice, h->stream)
               : cudaMemsetAsync(stage + 2 * n, 0, n * 8, h->stream);
    if (e == cudaSuccess)
        e = uy ? cudaMemcpyAsync(stage + 3 * n, uy, n * 8, cudaMemcpyHostToDevice, h->stream)
               : cudaMemsetAsync(stage + 3 * n, 0, n * 8, h->stream);
    if (e != cudaSuccess) return cuda_status(e);
    h->cur = 0;
    e = launch_init_fields(h->p.precision, h->g, coef_ptr(h), h->fbuf[0], stage, h->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
    return cuda_status(e);
}

lb_status lb_step(lb_handle* h, int64_t n) {
    if (!h || n < 0) return LB_ERR_INVALID;
    if (!h->inited) return LB_ERR_STATE;
    for (int64_t k = 0; k < n; ++k) {
        lb_status s = launch(h, OBS_NONE, nullptr, 0, 0);
        if (s != LB_OK) return s;
        h->cur ^= 1;
        h->pull = 1;
        h->t += 1;
    }
    return LB_OK;
}

lb_status lb_fields(lb_handle* h, double* rho_A, double* rho_B, double* ux, double* uy) {
    if (!h) return LB_ERR_INVALID;
    if (!h->inited) return LB_ERR_STATE;
    const size_t n = (size_t)h->p.nx * h->p.ny;
    double* out = reinterpret_cast<double*>(h->fbuf[1 - h->cur]);
    lb_status s = launch(h, OBS_FIELDS, out, 0, 0);
    if (s != LB_OK) return s;
    double* dst[4] = {rho_A, rho_B, ux, uy};
    for (int k = 0; k < 4; ++k)
        if (dst[k]) {
            cudaError_t e = cudaMemcpyAsync(dst[k], out + k * n, n * 8, cudaMemcpyDeviceToHost, h->stream);
            if (e != cudaSuccess) return cuda_status(e);
        }
    DevStats st;
    return read_stats(h, &st);
}

lb_status lb_populations(lb_handle* h, double* f) {
    if (!h || !f) return LB_ERR_INVALID;
    if (!h->inited) return LB_ERR_STATE;
    const size_t n = (size_t)h->p.nx * h->p.ny;
    double* out = reinterpret_cast<double*>(h->fbuf[1 - h->cur]);
    int per = (int)(h->fbuf_bytes / (n * 8));
    if (per < 1) return LB_ERR_UNSUPPORTED;
    if (per > 18) per = 18;
    for (int q0 = 0; q0 < 18; q0 += per) {
        const int q1 = q0 + per < 18 ? q0 + per : 18;
        lb_status s = launch(h, OBS_POPS, out, q0, q1);
        if (s != LB_OK) return s;
        cudaError_t e = cudaMemcpyAsync(f + (size_t)q0 * n, out, (size_t)(q1 - q0) * n * 8,
                                        cudaMemcpyDeviceToHost, h->stream);
        if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
        if (e != cudaSuccess) return cuda_status(e);
    }
    DevStats st;
    return read_stats(h, &st);
}

lb_status lb_stress(lb_handle* h, lb_stress_out* out) {
    if (!h || !out) return LB_ERR_INVALID;
    if (!h->inited) return LB_ERR_STATE;
    lb_status s = launch(h, OBS_TOTALS, nullptr, 0, 0);
    if (s != LB_OK) return s;
    DevStats st;
    s = read_stats(h, &st);
    memset(out, 0, sizeof(*out));
    out->mass_A = st.totals[0];
    out->mass_B = st.totals[1];
    out->mom_x = st.totals[2];
    out->mom_y = st.totals[3];
    out->samples = st.samples;
    out->step = h->t;
    if (st.samples > 0) {
        out->sigma_bot = st.sum_bot / (double)st.samples;
        out->sigma_top = st.sum_top / (double)st.samples;
        out->sigma_mean = 0.5 * (out->sigma_bot - out->sigma_top);
    }
    const double rate = 2.0 * h->p.u_wall / h->p.ny;
    const double mass = st.totals[0] + st.totals[1];
    const double rho_mean = mass / ((double)h->p.nx * h->p.ny);
    if (h->p.boundary == LB_COUETTE && rate != 0.0 && rho_mean > 0.0 && st.samples > 0) {
        out->nu_eff = out->sigma_mean / (rate * rho_mean);
        const double tau = mass > 0.0 ? (h->p.tau_A * st.totals[0] + h->p.tau_B * st.totals[1]) / mass
                                      : h->p.tau_A;
        const double nu0 = (tau - 0.5) / 3.0;
        out->response_R = out->nu_eff != 0.0 ? nu0 / out->nu_eff : 0.0;
    }
    return s;
}

lb_status lb_sync(lb_handle* h) {
    if (!h) return LB_ERR_INVALID;
    DevStats st;
    return read_stats(h, &st);
}

int64_t lb_time(const lb_handle* h) { return h ? h->t : -1; }

lb_status lb_destroy(lb_handle* h) {
    if (!h) return LB_OK;
    cudaError_t e = cudaStreamSynchronize(h->stream);
    if (h->owns) {
        cudaError_t e2 = cudaFree(h->ws);
        if (e == cudaSuccess) e = e2;
    }
    delete h;
    return cuda_status(e);
}

const char* lb_status_string(lb_status s) {
    switch (s) {
        case LB_OK: return "ok";
        case LB_ERR_INVALID: return "invalid argument";
        case LB_ERR_NOMEM: return "out of device memory or workspace too small";
        case LB_ERR_CUDA: return "CUDA runtime error";
        case LB_ERR_NONFINITE: return "a density became non-finite";
        case LB_ERR_TIMEOUT: return "a bounded device-side wait timed out";
        case LB_ERR_STATE: return "call out of order (initialise the lattice first)";
        case LB_ERR_UNSUPPORTED: return "configuration not supported";
    }
    return "unknown status";
}

}  // extern "C"
