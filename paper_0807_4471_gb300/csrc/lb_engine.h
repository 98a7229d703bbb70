// lb_engine.h -- host-side engine shared by the single-lattice ABI
// (lb_api.cu) and the lattice pool (lb_pool.cu): device regions of lattices,
// their TMA descriptors and coefficients, the work partition and launch of
// the persistent step kernel, and the observe/initialise helpers.
#pragma once

#include <vector>

#include "lb_internal.h"

namespace lbgb {

// Host-side state of one resident lattice.
struct Lattice {
    lb_params p;
    Geom g;
    char* region;            // device region: stats | observe slots | wall columns | wall sums |
                             // buffer 0 | buffer 1
    DevStats* st;
    double* slots;           // observe partial sums, 4 per tile
    char* wallx;             // the step's wall-momentum pairs: [2][nx] (bottom, top), compute type
    double* wsum;            // their per-strip sums: [2][nstrips]
    char* fbuf[2];
    size_t fbytes;
    CUtensorMap tblock[2];   // step kernel: 8-row block loads of buffer b
    CUtensorMap ttile[2];    // step kernel: tile stores into buffer b, clipped at the lattice edge
    CUtensorMap tobs[2];     // observe kernel: tile + halo loads of buffer b
    Coef<double> kd;
    Coef<float> kf;
    int nstrips, ntiles_y, seg;
    int cur, pull;           // host mirror of DevStats::cur / pull
    bool inited;
    long long t;             // host mirror of the step count
    unsigned int err_latched;
    long long next_sample;   // source of the device's DevStats::next_sample (lives with
                             // the lattice, so the asynchronous copy needs no wait)
};

// One launch of the persistent step kernel over a set of lattices.
struct Launch {
    int precision;
    int variant;             // bit 0: all periodic; bit 1: general forcing; bit 2: 1 - omega = 0
    int spt;                 // sites per thread: tiles of 8 spt rows
    dim3 grid;
    int nitems, seg;
    BatchArgs<double> ad;
    BatchArgs<float> af;
};

size_t align_up(size_t v, size_t a);
lb_status validate_params(const lb_params* p);
lb_status cuda_status(cudaError_t e);
int device_sms(int device);

// Bytes of a lattice's device region, and binding a lattice to one.
size_t lattice_bytes(const lb_params* p);
lb_status lattice_setup(Lattice& L, const lb_params* p, char* region);

// Host-only plan of one launch's work items (the lb_plan_partition entry).
lb_status plan_partition(const lb_params* ps, int nlat, int seg, int tile_rows, int sms,
                         int32_t* items, int32_t* nitems, int32_t* cta, int32_t* grid,
                         int32_t* seg_used);

// Segment length (tiles per work item) minimising the most loaded CTA.
int choose_seg(const int* nstrips, const int* ntiles_y, int nlat, int G);

// Sites per thread of the step kernel: the tile shapes a precision has
// (tiles of 8 spt rows), the library's default, and a lattice's tile rows.
int max_spt(int precision);
int default_spt(int precision);
int tiles_y(const Lattice& L, int spt);

// Write the lattices' descriptors to `descs` (device, 128-byte aligned, room
// for nlat LatDesc<double>) through `host_scratch` (as large, host) and fill
// the launch.  Synchronises the stream.  All lattices share the precision
// and the coefficients of lats[0] (couplings, tau, forcing).  seg > 0 forces
// the segment length; seg = 0 takes choose_seg's; seg < 0 cuts the tiles
// into one contiguous run per CTA.  `slots` holds launch_area_doubles(tiles,
// strips, sms) doubles for the lattices' total tiles and strips: the item
// tables.
// spt: sites per thread of the launch's kernel (1 or 2, see max_spt).
lb_status launch_build(Launch& Ln, Lattice* const* lats, int nlat, void* descs, double* slots,
                       unsigned int* ticket, int sms, cudaStream_t stream, void* host_scratch,
                       int seg = 0, int spt = 1);
size_t launch_area_doubles(size_t tiles, size_t strips, int sms);
lb_status launch_run(const Launch& Ln, cudaStream_t s);

lb_status lattice_init_seeded(Lattice& L, uint64_t seed, cudaStream_t s);
lb_status lattice_init_fields(Lattice& L, const double* rho_A, const double* rho_B,
                              const double* ux, const double* uy, cudaStream_t s);
// Resume from populations [2][9][ny][nx] (host FP64, as lattice_populations
// writes them) at step t; stress averages restart.
// pulled = 1: f holds the stored post-collision state f*(t-1) (a raw
// checkpoint); 0: the populations f(t) before collision.
lb_status lattice_load_populations(Lattice& L, const double* f, long long t, int pulled,
                                   cudaStream_t s);
void lattice_advanced(Lattice& L, long long n);
lb_status lattice_observe(Lattice& L, int obs, double* out, int q0, int q1, cudaStream_t s);
lb_status lattice_fields(Lattice& L, double* rho_A, double* rho_B, double* ux, double* uy,
                         cudaStream_t s);
// raw = 0: f(t) after streaming; raw = 1: the stored state as it is (f*(t-1)
// when L.pull, else f(t)), for an exact checkpoint.
lb_status lattice_populations(Lattice& L, double* f, cudaStream_t s, int raw = 0);
lb_status lattice_stress(Lattice& L, lb_stress_out* out, cudaStream_t s);
lb_status lattice_read_stats(Lattice& L, DevStats* out, cudaStream_t s);

}  // namespace lbgb
