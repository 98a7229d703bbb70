// lb_api.cu -- the single-lattice C ABI declared in include/lb.h: a handle is
// one lattice region plus the step-launch area (arrival counter, lattice
// descriptor, item tables) in one workspace.  The engine in
// lb_engine.cu does the work; every step of the model runs in the kernels.
#include <cstring>
#include <new>

#include <nvtx3/nvToolsExt.h>

#include "lb_engine.h"

using namespace lbgb;

struct lb_handle {
    Lattice lat;
    cudaStream_t stream;
    int device;
    bool owns;             // workspace allocated here with cudaMalloc
    char* ws;
    size_t ws_bytes;
    Launch launch;         // the single-lattice step launch
};

namespace {

constexpr size_t kAlign = 256;

// Handle workspace: the lattice region, then the step-launch area.
struct HandleLayout {
    size_t lattice, ticket, desc, slots, total;
};
HandleLayout handle_layout(const lb_params* p) {
    HandleLayout H;
    const int tx = kernel_tile_x(p->precision), ty = kernel_tile_y(p->precision);
    const size_t nstrips = (size_t)((p->nx + tx - 1) / tx);
    const size_t ntiles = nstrips * (size_t)((p->ny + ty - 1) / ty);
    size_t off = 0;
    H.lattice = off;
    off = align_up(off + lattice_bytes(p), kAlign);
    H.ticket = off;
    off = align_up(off + sizeof(unsigned int), kAlign);
    H.desc = off;
    off = align_up(off + sizeof(LatDesc<double>), kAlign);
    H.slots = off;
    // item tables (items <= tiles + strips; up to 1024 CTAs)
    off = align_up(off + sizeof(double) * launch_area_doubles(ntiles, nstrips, 1024), kAlign);
    H.total = off;
    return H;
}

lb_status create_common(const lb_params* p, void* stream, void* ws, size_t bytes, bool owns,
                        lb_handle** out) {
    lb_handle* h = new (std::nothrow) lb_handle();
    if (!h) return LB_ERR_NOMEM;
    h->stream = reinterpret_cast<cudaStream_t>(stream);
    cudaGetDevice(&h->device);
    h->owns = owns;
    h->ws = reinterpret_cast<char*>(ws);
    h->ws_bytes = bytes;
    HandleLayout H = handle_layout(p);
    lb_status s = cuda_status(cudaMemsetAsync(h->ws, 0, H.total, h->stream));
    if (s == LB_OK) s = lattice_setup(h->lat, p, h->ws + H.lattice);
    if (s == LB_OK) {
        Lattice* one = &h->lat;
        alignas(128) unsigned char scratch[sizeof(LatDesc<double>)];
        const int spt = p->tile_rows == 0 ? default_spt(p->precision)
                                           : p->tile_rows / kernel_tile_y(p->precision);
        s = launch_build(h->launch, &one, 1, h->ws + H.desc,
                         reinterpret_cast<double*>(h->ws + H.slots),
                         reinterpret_cast<unsigned int*>(h->ws + H.ticket), device_sms(h->device),
                         h->stream, scratch, 0, spt);
    }
    if (s != LB_OK) {
        if (owns) cudaFree(ws);
        delete h;
        return s;
    }
    *out = h;
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
    p->rounding = LB_ROUND_STOCHASTIC;
}

lb_status lb_workspace_size(const lb_params* p, size_t* bytes) {
    lb_status s = validate_params(p);
    if (s != LB_OK) return s;
    if (!bytes) return LB_ERR_INVALID;
    *bytes = handle_layout(p).total;
    return LB_OK;
}

lb_status lb_create(const lb_params* p, void* stream, lb_handle** out) {
    if (!out) return LB_ERR_INVALID;
    *out = nullptr;
    lb_status s = validate_params(p);
    if (s != LB_OK) return s;
    const size_t bytes = handle_layout(p).total;
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
    lb_status s = validate_params(p);
    if (s != LB_OK) return s;
    if (!workspace || (reinterpret_cast<uintptr_t>(workspace) % kAlign) != 0) return LB_ERR_INVALID;
    if (bytes < handle_layout(p).total) return LB_ERR_NOMEM;
    return create_common(p, stream, workspace, bytes, false, out);
}

lb_status lb_init_seeded(lb_handle* h, uint64_t seed) {
    if (!h) return LB_ERR_INVALID;
    return lattice_init_seeded(h->lat, seed, h->stream);
}

lb_status lb_init_fields(lb_handle* h, const double* rho_A, const double* rho_B, const double* ux,
                         const double* uy) {
    if (!h || !rho_A || !rho_B) return LB_ERR_INVALID;
    return lattice_init_fields(h->lat, rho_A, rho_B, ux, uy, h->stream);
}

lb_status lb_init_populations(lb_handle* h, const double* f, int64_t t) {
    if (!h || !f) return LB_ERR_INVALID;
    return lattice_load_populations(h->lat, f, t, 0, h->stream);
}

lb_status lb_checkpoint(lb_handle* h, double* state, int64_t* t, int32_t* pulled) {
    if (!h || !state || !t || !pulled) return LB_ERR_INVALID;
    if (!h->lat.inited) return LB_ERR_STATE;
    lb_status s = lattice_populations(h->lat, state, h->stream, 1);
    *t = h->lat.t;
    *pulled = h->lat.pull;
    return s;
}

lb_status lb_restore(lb_handle* h, const double* state, int64_t t, int32_t pulled) {
    if (!h || !state) return LB_ERR_INVALID;
    return lattice_load_populations(h->lat, state, t, pulled, h->stream);
}

lb_status lb_step(lb_handle* h, int64_t n) {
    if (!h || n < 0) return LB_ERR_INVALID;
    if (!h->lat.inited) return LB_ERR_STATE;
    nvtxRangePushA("lb_step");   // a profiler range around the launches (free without a tool)
    lb_status s = LB_OK;
    for (int64_t k = 0; k < n && s == LB_OK; ++k) {
        s = launch_run(h->launch, h->stream);
        if (s == LB_OK) lattice_advanced(h->lat, 1);
    }
    nvtxRangePop();
    return s;
}

lb_status lb_fields(lb_handle* h, double* rho_A, double* rho_B, double* ux, double* uy) {
    if (!h) return LB_ERR_INVALID;
    if (!h->lat.inited) return LB_ERR_STATE;
    return lattice_fields(h->lat, rho_A, rho_B, ux, uy, h->stream);
}

lb_status lb_populations(lb_handle* h, double* f) {
    if (!h || !f) return LB_ERR_INVALID;
    if (!h->lat.inited) return LB_ERR_STATE;
    return lattice_populations(h->lat, f, h->stream);
}

lb_status lb_stress(lb_handle* h, lb_stress_out* out) {
    if (!h || !out) return LB_ERR_INVALID;
    if (!h->lat.inited) return LB_ERR_STATE;
    return lattice_stress(h->lat, out, h->stream);
}

lb_status lb_sync(lb_handle* h) {
    if (!h) return LB_ERR_INVALID;
    DevStats st;
    return lattice_read_stats(h->lat, &st, h->stream);
}

int64_t lb_time(const lb_handle* h) { return h ? h->lat.t : -1; }

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

lb_status lb_selftest_wait(void* stream, int32_t limit) {
    if (limit < 1) return LB_ERR_INVALID;
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    unsigned int* err = nullptr;
    cudaError_t e = cudaMalloc(&err, sizeof(unsigned int));
    if (e != cudaSuccess) {
        cudaGetLastError();
        return e == cudaErrorMemoryAllocation ? LB_ERR_NOMEM : LB_ERR_CUDA;
    }
    unsigned int h = 0;
    e = cudaMemsetAsync(err, 0, sizeof(unsigned int), s);
    if (e == cudaSuccess) e = launch_wait_selftest(err, limit, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(&h, err, sizeof(unsigned int), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    cudaFree(err);
    if (e != cudaSuccess) return cuda_status(e);
    return (h & ERR_TIMEOUT) ? LB_ERR_TIMEOUT : LB_OK;
}

lb_status lb_selftest_math(const float* x, float* out, int64_t n, void* stream) {
    if (n < 0 || (n > 0 && (!x || !out))) return LB_ERR_INVALID;
    if (n == 0) return LB_OK;
    return cuda_status(launch_math_probe(x, out, (long long)n, reinterpret_cast<cudaStream_t>(stream)));
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

lb_status lb_plan_partition(const lb_params* ps, int32_t nlat, int32_t seg, int32_t tile_rows,
                            int32_t sms, int32_t* items, int32_t* nitems, int32_t* cta,
                            int32_t* grid, int32_t* seg_used) {
    return lbgb::plan_partition(ps, nlat, seg, tile_rows, sms, items, nitems, cta, grid, seg_used);
}

}  // extern "C"
