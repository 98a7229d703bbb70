// lb_internal.h -- structures shared by the host side of the C ABI
// (lb_api.cu) and the kernels (lb_kernels.cu).  Not part of the public ABI.
#pragma once

#include <cstddef>
#include <cstdint>

#include <cuda.h>           // CUtensorMap (type only; the driver is reached via
#include <cuda_runtime.h>   // cudaGetDriverEntryPointByVersion)

#include "../../include/lb.h"

namespace lbgb {

// Device-resident counters and accumulators of one lattice.
struct DevStats {
    unsigned int err;       // bit 0: non-finite density, bit 1: TMA wait timeout
    unsigned int ticket;    // CTA arrival counter of the observe reductions
    long long t;            // completed time steps
    double sum_bot;         // sum of per-step bottom-wall samples
    double sum_top;         // sum of per-step top-wall samples
    long long samples;      // number of samples in the sums
    double totals[4];       // last observe pass: mass_A, mass_B, mom_x, mom_y
    int cur;                // buffer holding the current state (0 or 1)
    int pull;               // 1: it holds post-collision f*(t-1); 0: f(t) in place
    long long next_sample;  // the next step whose wall momentum is sampled
                            // (stress_t0 + k stress_every >= t; set by the host
                            // with t, advanced by the kernel)
    double pad_[5];
};
static_assert(sizeof(DevStats) == 128, "DevStats is one 128-byte line");

enum : unsigned int { ERR_NONFINITE = 1u, ERR_TIMEOUT = 2u };

// The bounded-wait self-test kernel (lb_selftest_wait).
cudaError_t launch_wait_selftest(unsigned int* err, int limit, cudaStream_t s);
// The FP32 exp(x) - 1 / reciprocal probe (lb_selftest_math).
cudaError_t launch_math_probe(const float* x, float* out, long long n, cudaStream_t s);

// Geometry of the ghost-padded population planes.  Plane i (i = 0..8, the
// D2Q9 direction) holds (ny + 2*kGY) rows of `pitch` interleaved (A, B)
// pairs; lattice site (x, y) sits at row y + kGY, pair column x + gx.  The
// kGY = 3 rows and gx >= 3 columns on each side hold periodic copies so that
// the tile loads never wrap.
constexpr int kGY = 3;

struct Geom {
    int nx, ny;
    int pitch;          // (A, B) pairs per padded row (row bytes a multiple of 16)
    int rows;           // ny + 2*kGY
    long long plane;    // pairs per direction plane = rows * pitch
    int gx;             // ghost columns on each side
    int periodic;       // 1: periodic in y; 0: Couette walls in y
    // Lattice columns x >= x_tail (at most 3) are written by plain stores,
    // not by the tile's bulk tensor store: a clipped bulk store ends on a
    // 16-byte boundary, so its descriptor stops at the last 16-byte
    // boundary of the lattice row and leaves the ghost column beside it alone.
    int x_tail;
};

// The (A, B) pair type of a compute precision.
template <typename C> struct PairOf;
template <> struct PairOf<float> { typedef float2 T; };
template <> struct PairOf<double> { typedef double2 T; };

// Per-launch model coefficients, in the compute precision C.  The stencil
// sums of Eq. (2) are taken row by row (see the step kernel): with
// K(|d|^2) = G^a w(|d|^2) + G^r p(|d|^2) per species, the like-species
// weights are the (A, B) pairs KC = {K(1), K(2), K(5), 2 K(4), 2 K(5),
// 2 K(8)} (the factors 2 are the stencil components |d_x| or |d_y| = 2,
// exact), and the cross-species ones WC = {w(1), w(2)} for both species.
template <typename C>
struct Coef {
    typedef typename PairOf<C>::T C2;
    C2 KC[6];          // like-species row weights, (A, B) pairs
    C2 WC[2];          // cross-species row weights, equal in both lanes
    C gx_rho0;         // G_X / rho0
    C psi_ref;         // Psi(rho_ref)
    C psi_scale;       // P exp(-rho_ref / rho0)
    C inv_rho0;        // 1 / rho0
    C rho_ref;         // reference density of the stored offsets
    C tau3[2];         // 3 tau_s (the velocity shift is taken for v = 3u)
    C omega[2];        // 1 / tau
    C2 omw[3];         // omega_s S w for the D2Q9 classes |c|^2 = 0, 1, 2 (S the storage scale)
    C2 omm;            // 1 - omega_s
    C u_wall;          // Couette wall speed (top +, bottom -)
    C g_x;             // uniform body acceleration
    C kolmo_amp;       // Kolmogorov acceleration amplitude
    C kolmo_w;         // 2 pi kolmo_k / ny
    int sr;            // 1: half formats stored with stochastic rounding
    int source;        // 1: additive source term; 0: velocity shift
    int has_accel;     // 1 if g_x or kolmo_amp is nonzero
};

// Values that vary between the lattices of one step launch.
template <typename C>
struct LatVals {
    C rho_ref, psi_ref, psi_scale, inv_rho0, gx_rho0, u_wall;
    C kolmo_w;         // 2 pi kolmo_k / ny (ny is per lattice)
};

// One lattice of a step launch, in device memory (128-byte aligned for the
// tensor maps).  Both buffers are described; the device-side DevStats::cur
// says which one holds the current state.
template <typename C>
struct alignas(128) LatDesc {
    CUtensorMap tin[2];    // 8-row block loads of buffer b: box {2 BX, 8, 9}
    CUtensorMap tout[2];   // tile stores into buffer b: box {2 TX, 8, 9}, clipped at x = x_tail, y = ny
    Geom g;
    LatVals<C> v;
    void* fbuf[2];
    DevStats* st;
    void* wallx;           // [2][nx] compute-type pairs: x-momentum handed to the bottom
                           // (then top) wall by the links leaving site x, this step
    double* wsum;          // [2][nstrips]: those summed per strip (bottom, then top)
    int nstrips;           // ceil(nx / TX)
    int ntiles_y;          // tile rows of the launch's tile shape
    int stress_every;
    long long stress_t0;
    double inv_nx;         // 1 / nx: the wall samples are momentum per unit length
};

// Arguments of the (multi-lattice) step kernel.
template <typename C>
struct BatchArgs {
    Coef<C> k;                  // coefficients shared by all lattices of the launch
    const LatDesc<C>* lat;      // nlat descriptors
    int nlat;
    int nitems;                 // total work items
    // Work items (lattice, strip, first tile row, end tile row), grouped by
    // CTA: CTA b takes items cta_items[b] .. cta_items[b + 1] - 1 in order.
    const int4* items;
    const int* cta_items;
    unsigned int* ticket;       // CTA arrival counter of the launch (zero between launches)
    int l2_resident;            // one buffer of all lattices fits in L2: cache-policy hints
    int early_release;          // kernel variant bit 2 only: a tile's ring slots are refilled
                                // after its density phase (else after its site phase)
};

// Observe-mode outputs (the kernel writes FP64 planes of nx*ny values).
enum ObsKind : int { OBS_NONE = 0, OBS_FIELDS = 1, OBS_POPS = 2, OBS_TOTALS = 3 };

template <typename C>
struct StepArgs {
    Geom g;
    Coef<C> k;
    void* fout;            // output population buffer (padded planes)
    DevStats* st;
    double* slots;         // per-CTA partial sums
    int pull;              // 1: input holds post-collision f*(t-1); 0: f(t) in place
    int obs;               // ObsKind; OBS_NONE = a time step
    double* obs_out;       // observe output base
    int q0, q1;            // OBS_POPS: planes [q0, q1) written
    long long stress_t0;
    int stress_every;
};

// Host-side launch helpers (lb_dispatch.cu).
int kernel_smem_bytes(int precision);
int kernel_tile_x(int precision);
int kernel_tile_y(int precision);
int kernel_ghost_x(int precision);
int kernel_elem_bytes(int precision);
int kernel_smem_obs_bytes(int precision);
int kernel_block_rows(int precision);
int kernel_scale_log2(int precision);
// 1 if the step kernel with spt sites per thread leaves through a staging
// tile (its periodic ghost copies are then separate stores after the tile)
int kernel_staged(int precision, int spt);

// Step: the persistent multi-lattice kernel (args: BatchArgs<C>), variant
// bit 0 = every lattice periodic, bit 1 = general forcing, bit 2 = 1 - omega
// rounds to zero for both species (the collision reads no populations), spt sites per
// thread (tiles of 8 spt rows).  Observe: one lattice, one CTA per 8-row
// tile (args: StepArgs<C>, tin: tile-box load map).
cudaError_t launch_step(int precision, const void* args, int variant, int spt, dim3 grid,
                        cudaStream_t s);
// Opt the kernels of a precision into their shared memory (once per device;
// call before capturing launches into a graph).
cudaError_t kernels_configure(int precision);
cudaError_t launch_observe(int precision, const CUtensorMap* tin, const void* args, dim3 grid,
                           cudaStream_t s);
cudaError_t launch_init_seeded(int precision, const Geom& g, const void* coef, void* fout,
                               double rho0, double amp, double u_wall, int init_shear,
                               unsigned long long seed, cudaStream_t s);
cudaError_t launch_init_fields(int precision, const Geom& g, const void* coef, void* fout,
                               const double* fields, cudaStream_t s);

// Restore directions [i0, i1) from FP64 populations [i1 - i0][2][ny][nx].
cudaError_t launch_load_pops(int precision, const Geom& g, const void* coef, void* fout,
                             const double* pops, int i0, int i1, cudaStream_t s);

// Per-precision launchers, one explicit instantiation per compilation of
// lb_kernels.cu (-DLB_PREC=P).
template <int P>
cudaError_t configure_prec();
template <int P>
cudaError_t launch_step_prec(const void* args, int variant, int spt, dim3 grid, cudaStream_t s);
template <int P>
cudaError_t launch_observe_prec(const CUtensorMap* tin, const void* args, dim3 grid,
                                cudaStream_t s);
template <int P>
cudaError_t launch_load_pops_prec(const Geom& g, const void* coef, void* fout, const double* pops,
                                  int i0, int i1, cudaStream_t s);
template <int P>
cudaError_t launch_init_prec(const Geom& g, const void* coef, void* fout, int mode,
                             const double* fields, double rho0, double amp, double u_wall,
                             int init_shear, unsigned long long seed, cudaStream_t s);

}  // namespace lbgb
