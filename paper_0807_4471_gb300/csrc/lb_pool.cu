// lb_pool.cu -- the lattice pool of include/lb.h: many resident lattices in
// one device arena, stepped together by one persistent launch per time step.
//
// Native runtime pieces: a first-fit arena allocator (one cudaMalloc at
// creation), admission by footprint, the active-set bookkeeping, CUDA-graph
// capture and replay of step chunks, and a measured autotuner of the step
// kernel's tile shape and work partition, cached per member-set signature.
#include <algorithm>
#include <cstdlib>
#include <cstring>
#include <map>
#include <new>
#include <string>
#include <vector>

#include <nvtx3/nvToolsExt.h>

#include "lb_engine.h"

using namespace lbgb;

namespace {

constexpr size_t kAlign = 256;
constexpr int kGraphChunk = 16;   // steps per captured graph
constexpr int kTuneSteps = 6;     // timed steps per candidate (tile shape, partition)
// A new member set is tuned only if it runs at least kTuneShare times the
// steps that timing all candidates takes: a short-lived set (a server's
// quantum between arrivals) keeps the load-balance model's partition.
constexpr int kTuneShare = 8;

// First-fit allocator over [0, size) with kAlign granularity.
class Arena {
public:
    void reset(size_t size) {
        free_.clear();
        if (size) free_[0] = size;
        size_ = size;
    }
    bool alloc(size_t bytes, size_t* off) {
        bytes = align_up(bytes, kAlign);
        for (auto it = free_.begin(); it != free_.end(); ++it) {
            if (it->second >= bytes) {
                *off = it->first;
                const size_t rest = it->second - bytes, start = it->first + bytes;
                free_.erase(it);
                if (rest) free_[start] = rest;
                return true;
            }
        }
        return false;
    }
    void release(size_t off, size_t bytes) {
        bytes = align_up(bytes, kAlign);
        auto it = free_.emplace(off, bytes).first;
        auto next = std::next(it);
        if (next != free_.end() && it->first + it->second == next->first) {
            it->second += next->second;
            free_.erase(next);
        }
        if (it != free_.begin()) {
            auto prev = std::prev(it);
            if (prev->first + prev->second == it->first) {
                prev->second += it->second;
                free_.erase(it);
            }
        }
    }

private:
    std::map<size_t, size_t> free_;
    size_t size_ = 0;
};

struct Member {
    bool used = false;
    Lattice lat;
    size_t off = 0, bytes = 0;
    long long target = 0, done = 0;
};

}  // namespace

// A launch configuration the tuner chooses: work partition and tile shape.
struct Choice {
    int seg;                 // > 0 segments of seg tiles; -1 contiguous runs; 0 the model's
    int spt;                 // sites per thread (tiles of 8 spt rows)
};

struct lb_pool {
    lb_params shared;
    int forced_seg;          // 0: autotune; else the partition to use (-1: contiguous runs)
    int forced_spt;          // 0: autotune; else the sites per thread to use
    cudaStream_t stream;
    bool own_stream;
    int device, sms;
    char* arena_mem;
    size_t budget;
    Arena arena;
    std::vector<Member> members;
    // launch area: descriptors, arrival counter, item tables
    char* desc_mem;
    unsigned int* ticket;
    double* slots;
    size_t slot_cap;         // doubles
    void* host_desc;         // staging of the descriptors (128-byte aligned)
    // current active set and its launch
    std::vector<int> active;
    bool built;
    Launch launch;
    cudaGraphExec_t graph;
    std::map<std::string, Choice> tuned;   // member-set signature -> tuned choice
};

namespace {

bool same_shared(const lb_params& a, const lb_params& b) {
    return a.precision == b.precision && a.psi_form == b.psi_form &&
           a.force_scheme == b.force_scheme && a.tau_A == b.tau_A && a.tau_B == b.tau_B &&
           a.G_A1 == b.G_A1 && a.G_A2 == b.G_A2 && a.G_B1 == b.G_B1 && a.G_B2 == b.G_B2 &&
           a.G_X == b.G_X && a.g_x == b.g_x && a.kolmo_amp == b.kolmo_amp &&
           a.kolmo_k == b.kolmo_k && a.rounding == b.rounding;
}

std::string signature(lb_pool* P) {
    std::vector<std::string> parts;
    for (int j : P->active) {
        const lb_params& p = P->members[(size_t)j].lat.p;
        parts.push_back(std::to_string(p.nx) + "x" + std::to_string(p.ny) + (p.boundary ? "c" : "p"));
    }
    std::sort(parts.begin(), parts.end());
    std::string s;
    for (auto& x : parts) s += x + ",";
    return s;
}

void drop_graph(lb_pool* P) {
    if (P->graph) {
        cudaGraphExecDestroy(P->graph);
        P->graph = nullptr;
    }
}

lb_status build(lb_pool* P, Choice c) {
    drop_graph(P);
    std::vector<Lattice*> lats;
    for (int j : P->active) lats.push_back(&P->members[(size_t)j].lat);
    const int nlat = (int)lats.size();
    // item tables: items are most numerous for seg = 1 (one per tile)
    size_t tiles = 0, strips = 0;
    for (Lattice* L : lats) {
        tiles += (size_t)L->nstrips * (size_t)L->ntiles_y;
        strips += (size_t)L->nstrips;
    }
    const size_t need = launch_area_doubles(tiles, strips, P->sms);
    if (need > P->slot_cap) {
        cudaError_t e = cudaStreamSynchronize(P->stream);
        if (P->slots) cudaFree(P->slots);
        P->slots = nullptr;
        P->slot_cap = 0;
        if (e == cudaSuccess) e = cudaMalloc(&P->slots, need * sizeof(double));
        if (e != cudaSuccess) return cuda_status(e);
        P->slot_cap = need;
    }
    cudaError_t ce = kernels_configure(P->shared.precision);   // before any graph capture
    if (ce != cudaSuccess) return cuda_status(ce);
    lb_status s = launch_build(P->launch, lats.data(), nlat, P->desc_mem, P->slots, P->ticket,
                               P->sms, P->stream, P->host_desc, c.seg, c.spt);
    P->built = s == LB_OK;
    return s;
}

// Capture kGraphChunk launches of the built launch into the pool's graph
// (nothing executes during the capture).
lb_status capture_graph(lb_pool* P) {
    if (P->graph) return LB_OK;
    cudaGraph_t g = nullptr;
    cudaError_t e = cudaStreamBeginCapture(P->stream, cudaStreamCaptureModeThreadLocal);
    if (e != cudaSuccess) return cuda_status(e);
    lb_status s = LB_OK;
    for (int i = 0; i < kGraphChunk && s == LB_OK; ++i) s = launch_run(P->launch, P->stream);
    e = cudaStreamEndCapture(P->stream, &g);
    if (s != LB_OK) {
        if (g) cudaGraphDestroy(g);
        return s;
    }
    if (e == cudaSuccess) e = cudaGraphInstantiate(&P->graph, g, 0);
    if (g) cudaGraphDestroy(g);
    if (e != cudaSuccess) {
        P->graph = nullptr;
        return cuda_status(e);
    }
    return LB_OK;
}

// Run k steps of the built launch: captured chunks, then single launches.
lb_status run_steps(lb_pool* P, long long k) {
    while (k >= kGraphChunk) {
        lb_status s = capture_graph(P);
        if (s != LB_OK) return s;
        cudaError_t e = cudaGraphLaunch(P->graph, P->stream);
        if (e != cudaSuccess) return cuda_status(e);
        k -= kGraphChunk;
    }
    for (long long i = 0; i < k; ++i) {
        lb_status s = launch_run(P->launch, P->stream);
        if (s != LB_OK) return s;
    }
    return LB_OK;
}

void advanced(lb_pool* P, long long k) {
    for (int j : P->active) {
        Member& m = P->members[(size_t)j];
        lattice_advanced(m.lat, k);
        m.done += k;
    }
}

// The choices open to the tuner (the fixed dimensions of lb_pool_set_partition
// and lb_pool_set_tile_rows kept), and the untuned default.
std::vector<Choice> candidates(lb_pool* P) {
    const int prec = P->shared.precision;
    std::vector<int> spts;
    if (P->forced_spt != 0) spts.push_back(P->forced_spt);
    else for (int k = 1; k <= max_spt(prec); ++k) spts.push_back(k);
    std::vector<Choice> out;
    for (int spt : spts) {
        std::vector<int> segs;
        if (P->forced_seg != 0) {
            segs.push_back(P->forced_seg);
        } else {
            // contiguous runs per CTA, the load-balance model's segments, then fixed segments
            std::vector<int> ns, nt;
            int tiles = 0;
            for (int j : P->active) {
                const Lattice& L = P->members[(size_t)j].lat;
                ns.push_back(L.nstrips);
                nt.push_back(tiles_y(L, spt));
                tiles = std::max(tiles, nt.back());
            }
            segs = {-1, choose_seg(ns.data(), nt.data(), (int)ns.size(), P->sms)};
            for (int c : {1, 2, 4, 8, 16, 32, 64})
                if (c <= tiles && std::find(segs.begin(), segs.end(), c) == segs.end()) segs.push_back(c);
        }
        for (int seg : segs) out.push_back({seg, spt});
    }
    return out;
}
Choice untuned(lb_pool* P) {
    return {P->forced_seg, P->forced_spt != 0 ? P->forced_spt : default_spt(P->shared.precision)};
}
std::string cache_key(lb_pool* P) {
    return signature(P) + "|" + std::to_string(P->forced_seg) + "|" + std::to_string(P->forced_spt);
}

// Time kTuneSteps real steps for each candidate (tile shape, partition) and
// keep the fastest.  Returns the steps consumed.
long long tune(lb_pool* P, long long budget_steps, lb_status* st) {
    *st = LB_OK;
    const std::vector<Choice> cand = candidates(P);
    if (cand.size() < 2) {   // nothing to choose between
        *st = build(P, cand.empty() ? untuned(P) : cand[0]);
        return 0;
    }
    if ((long long)cand.size() * kTuneSteps * kTuneShare > budget_steps) return 0;
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    Choice best = cand[0];
    float best_ms = 1e30f;
    long long used = 0;
    for (const Choice& c : cand) {
        *st = build(P, c);
        if (*st != LB_OK) break;
        cudaEventRecord(e0, P->stream);
        *st = run_steps(P, kTuneSteps);
        cudaEventRecord(e1, P->stream);
        if (*st != LB_OK) break;
        cudaEventSynchronize(e1);
        float ms = 0.f;
        cudaEventElapsedTime(&ms, e0, e1);
        advanced(P, kTuneSteps);
        used += kTuneSteps;
        if (ms < best_ms) {
            best_ms = ms;
            best = c;
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (*st == LB_OK) {
        P->tuned[cache_key(P)] = best;
        *st = build(P, best);
    }
    return used;
}

// Members with steps left (in slot order), and the largest step count, up to
// `limit`, that all of them can take.
long long active_members(lb_pool* P, long long limit, std::vector<int>& act) {
    act.clear();
    long long k = limit;
    for (size_t j = 0; j < P->members.size(); ++j) {
        const Member& m = P->members[j];
        if (m.used && m.done < m.target) {
            act.push_back((int)j);
            k = std::min(k, m.target - m.done);
        }
    }
    return k;
}

}  // namespace

extern "C" {

lb_status lb_pool_prepare(lb_pool* P) {
    if (!P) return LB_ERR_INVALID;
    std::vector<int> act;
    active_members(P, 1, act);
    if (act.empty()) return LB_OK;
    if (!P->built || act != P->active) {
        P->active = act;
        auto it = P->tuned.find(cache_key(P));
        lb_status s = build(P, it != P->tuned.end() ? it->second : untuned(P));
        if (s != LB_OK) return s;
    }
    return capture_graph(P);
}

lb_status lb_pool_footprint(const lb_params* p, size_t* bytes) {
    lb_status s = validate_params(p);
    if (s != LB_OK) return s;
    if (!bytes) return LB_ERR_INVALID;
    *bytes = align_up(lattice_bytes(p), kAlign);
    return LB_OK;
}

lb_status lb_pool_create(const lb_params* shared, size_t bytes_budget, int32_t max_jobs,
                         void* stream, lb_pool** out) {
    if (!out || max_jobs < 1 || max_jobs > (1 << 20)) return LB_ERR_INVALID;
    *out = nullptr;
    lb_status s = validate_params(shared);
    if (s != LB_OK) return s;
    lb_pool* P = new (std::nothrow) lb_pool();
    if (!P) return LB_ERR_NOMEM;
    P->shared = *shared;
    P->stream = reinterpret_cast<cudaStream_t>(stream);
    P->own_stream = false;
    cudaGetDevice(&P->device);
    P->sms = device_sms(P->device);
    P->budget = bytes_budget;
    P->members.resize((size_t)max_jobs);
    P->built = false;
    P->graph = nullptr;
    P->slots = nullptr;
    P->slot_cap = 0;
    P->arena_mem = nullptr;
    P->desc_mem = nullptr;
    P->host_desc = nullptr;
    cudaError_t e = cudaSuccess;
    if (!P->stream) {   // graphs need a capturable stream
        e = cudaStreamCreateWithFlags(&P->stream, cudaStreamNonBlocking);
        P->own_stream = e == cudaSuccess;
    }
    const size_t dbytes = align_up(sizeof(LatDesc<double>) * (size_t)max_jobs, kAlign);
    if (e == cudaSuccess && bytes_budget) e = cudaMalloc(&P->arena_mem, bytes_budget);
    if (e == cudaSuccess) e = cudaMalloc(&P->desc_mem, dbytes + kAlign);
    if (e == cudaSuccess) {
        P->ticket = reinterpret_cast<unsigned int*>(P->desc_mem + dbytes);
        e = cudaMemsetAsync(P->ticket, 0, sizeof(unsigned int), P->stream);
    }
    if (e == cudaSuccess) {
        P->host_desc = std::aligned_alloc(128, dbytes);
        if (!P->host_desc) e = cudaErrorMemoryAllocation;
    }
    if (e != cudaSuccess) {
        lb_pool_destroy(P);
        return cuda_status(e);
    }
    P->arena.reset(bytes_budget);
    *out = P;
    return LB_OK;
}

lb_status lb_pool_admit(lb_pool* P, const lb_params* p, uint64_t seed, int64_t steps, lb_job* job) {
    if (!P || !p || !job || steps < 0) return LB_ERR_INVALID;
    lb_status s = validate_params(p);
    if (s != LB_OK) return s;
    if (!same_shared(P->shared, *p)) return LB_ERR_INVALID;
    int slot = -1;
    for (size_t j = 0; j < P->members.size(); ++j)
        if (!P->members[j].used) {
            slot = (int)j;
            break;
        }
    if (slot < 0) return LB_ERR_INVALID;
    const size_t bytes = align_up(lattice_bytes(p), kAlign);
    size_t off = 0;
    if (!P->arena.alloc(bytes, &off)) return LB_ERR_NOMEM;
    Member& m = P->members[(size_t)slot];
    s = cuda_status(cudaMemsetAsync(P->arena_mem + off, 0, bytes, P->stream));
    if (s == LB_OK) s = lattice_setup(m.lat, p, P->arena_mem + off);
    if (s == LB_OK) s = lattice_init_seeded(m.lat, seed, P->stream);
    if (s != LB_OK) {
        P->arena.release(off, bytes);
        return s;
    }
    m.used = true;
    m.off = off;
    m.bytes = bytes;
    m.target = steps;
    m.done = 0;
    *job = slot;
    return LB_OK;
}

lb_status lb_pool_run(lb_pool* P, int64_t quantum, int32_t* active_out) {
    if (!P || quantum < 0) return LB_ERR_INVALID;
    struct Range {   // a profiler range around the quantum (free without a tool)
        Range() { nvtxRangePushA("lb_pool_run"); }
        ~Range() { nvtxRangePop(); }
    } range;
    long long remaining = quantum;
    lb_status s = LB_OK;
    while (remaining > 0) {
        std::vector<int> act;
        long long k = active_members(P, remaining, act);
        if (act.empty()) break;
        if (!P->built || act != P->active) {
            P->active = act;
            P->built = false;   // the previous member set's launch no longer applies
            drop_graph(P);
            auto it = P->tuned.find(cache_key(P));
            if (it != P->tuned.end()) {
                s = build(P, it->second);
            } else {
                const long long used = tune(P, k, &s);
                if (s != LB_OK) return s;
                if (!P->built) s = build(P, untuned(P));   // too few steps to tune
                k -= used;
                remaining -= used;
            }
            if (s != LB_OK) return s;
        }
        if (k > 0) {
            s = run_steps(P, k);
            if (s != LB_OK) return s;
            advanced(P, k);
            remaining -= k;
        }
    }
    if (active_out) {
        int32_t n = 0;
        for (const Member& m : P->members)
            if (m.used && m.done < m.target) ++n;
        *active_out = n;
    }
    return s;
}

lb_status lb_pool_poll(lb_pool* P, lb_job job, int64_t* steps_done, int32_t* done) {
    if (!P || job < 0 || (size_t)job >= P->members.size() || !P->members[(size_t)job].used)
        return LB_ERR_INVALID;
    const Member& m = P->members[(size_t)job];
    if (steps_done) *steps_done = m.done;
    if (done) *done = m.done >= m.target ? 1 : 0;
    return LB_OK;
}

lb_status lb_pool_fields(lb_pool* P, lb_job job, double* rho_A, double* rho_B, double* ux,
                         double* uy) {
    if (!P || job < 0 || (size_t)job >= P->members.size() || !P->members[(size_t)job].used)
        return LB_ERR_INVALID;
    return lattice_fields(P->members[(size_t)job].lat, rho_A, rho_B, ux, uy, P->stream);
}

lb_status lb_pool_init_fields(lb_pool* P, lb_job job, const double* rho_A, const double* rho_B,
                              const double* ux, const double* uy) {
    if (!P || !rho_A || !rho_B || job < 0 || (size_t)job >= P->members.size() ||
        !P->members[(size_t)job].used)
        return LB_ERR_INVALID;
    Member& m = P->members[(size_t)job];
    lb_status s = lattice_init_fields(m.lat, rho_A, rho_B, ux, uy, P->stream);
    if (s == LB_OK) m.done = 0;   // the member restarts from these fields
    return s;
}

lb_status lb_pool_stress(lb_pool* P, lb_job job, lb_stress_out* out) {
    if (!P || !out || job < 0 || (size_t)job >= P->members.size() || !P->members[(size_t)job].used)
        return LB_ERR_INVALID;
    return lattice_stress(P->members[(size_t)job].lat, out, P->stream);
}

lb_status lb_pool_release(lb_pool* P, lb_job job) {
    if (!P || job < 0 || (size_t)job >= P->members.size() || !P->members[(size_t)job].used)
        return LB_ERR_INVALID;
    // the member's memory may still be read by enqueued steps
    cudaError_t e = cudaStreamSynchronize(P->stream);
    Member& m = P->members[(size_t)job];
    P->arena.release(m.off, m.bytes);
    m.used = false;
    if (std::find(P->active.begin(), P->active.end(), job) != P->active.end()) {
        P->built = false;
        drop_graph(P);
    }
    return cuda_status(e);
}

int32_t lb_pool_segment(const lb_pool* P) { return P && P->built ? P->launch.seg : 0; }

lb_status lb_pool_set_partition(lb_pool* P, int32_t seg) {
    if (!P || seg < -1) return LB_ERR_INVALID;
    P->forced_seg = seg;
    P->built = false;   // rebuilt with it before the next step
    drop_graph(P);
    return LB_OK;
}

lb_status lb_pool_set_tile_rows(lb_pool* P, int32_t rows) {
    if (!P) return LB_ERR_INVALID;
    const int ty = kernel_tile_y(P->shared.precision);
    if (rows != 0 && rows != ty && rows != 2 * ty) return LB_ERR_INVALID;
    const int spt = rows / ty;
    if (spt > max_spt(P->shared.precision)) return LB_ERR_INVALID;
    P->forced_spt = spt;
    P->built = false;
    drop_graph(P);
    return LB_OK;
}

int32_t lb_pool_tile_rows(const lb_pool* P) {
    return P && P->built ? P->launch.spt * kernel_tile_y(P->shared.precision) : 0;
}

lb_status lb_pool_destroy(lb_pool* P) {
    if (!P) return LB_OK;
    cudaError_t e = P->stream ? cudaStreamSynchronize(P->stream) : cudaSuccess;
    drop_graph(P);
    if (P->slots) cudaFree(P->slots);
    if (P->desc_mem) cudaFree(P->desc_mem);
    if (P->arena_mem) cudaFree(P->arena_mem);
    if (P->host_desc) std::free(P->host_desc);
    if (P->own_stream) cudaStreamDestroy(P->stream);
    delete P;
    return cuda_status(e);
}

}  // extern "C"
