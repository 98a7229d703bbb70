/*
 * lb.h -- C ABI of the GB300 two-species multi-range pseudo-potential
 * lattice Boltzmann library (liblbgb.so).
 *
 * The model is the one of Benzi, Chibbaro & Succi, "Mesoscopic lattice
 * Boltzmann modeling of flowing soft systems" (arXiv:0807.4471):
 *  - Eq. (1): per species s in {A, B}, D2Q9 BGK relaxation with time tau_s
 *    toward the local equilibrium, a body force F_s, and free streaming;
 *  - Eq. (2): F_s = F^a_s + F^r_s + F^X_s, a like-species attraction G^a_s on
 *    the first belt (D2Q9 weights w), a like-species repulsion G^r_s on both
 *    belts (24 neighbours, 8th-order isotropic weights p) acting on the
 *    pseudo-potential Psi_s(rho) = P (1 - exp(-rho/rho0)), and a cross-species
 *    repulsion (G_AB/rho0) rho_s sum w_i rho_s'(r + c_i) c_i on the first belt;
 *  - the Fig. 2 caption gives the couplings G_A1, G_A2, G_B1, G_B2, G^X.
 * Every force term carries an overall minus sign, so that positive G is
 * repulsive as the text after Eq. (2) states.  The paper has no walls;
 * plane-Couette moving-wall bounce-back is an addition of this library.
 *
 * Conventions for every entry point:
 *  - The status is returned; nothing crosses the ABI as an exception.
 *  - A handle owns its device memory (unless created with lb_create_in, in
 *    which case the caller owns the workspace and must keep it alive until
 *    lb_destroy).  The caller owns every host buffer.
 *  - Work is enqueued on the CUDA stream given at creation (NULL = legacy
 *    default stream).  lb_step returns once its kernels are enqueued; device
 *    errors (non-finite density, a TMA wait that timed out) are latched on the
 *    device and returned by the next synchronising call (lb_fields,
 *    lb_populations, lb_stress, lb_sync).
 *  - Calls on one handle are not thread-safe; different handles are
 *    independent.
 *  - Host field arrays are FP64, row-major [ny][nx] (x fastest), whatever the
 *    storage precision.
 */
#ifndef LB_H
#define LB_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct lb_handle lb_handle;

typedef enum {
    LB_OK = 0,
    LB_ERR_INVALID = -1,     /* bad argument or parameter                      */
    LB_ERR_NOMEM = -2,       /* device allocation failed / workspace too small */
    LB_ERR_CUDA = -3,        /* a CUDA runtime call failed                      */
    LB_ERR_NONFINITE = -4,   /* a density became NaN or Inf                     */
    LB_ERR_TIMEOUT = -5,     /* a bounded device-side wait gave up             */
    LB_ERR_STATE = -6,       /* call out of order (e.g. step before init)      */
    LB_ERR_UNSUPPORTED = -7  /* no kernel for this configuration               */
} lb_status;

/* Storage precision of the populations.  Arithmetic is FP64 for LB_FP64 and
 * FP32 otherwise; every format stores the offsets f_i - w_i rho_ref, and the
 * half formats decode them to FP32.  LB_FP16_OFFSET stores the offsets times
 * 2^10 (exact), so that offsets down to 2^-24 keep binary16's full 11-bit
 * precision; offsets must stay below 64 in magnitude. */
typedef enum { LB_FP64 = 0, LB_FP32 = 1, LB_FP16_OFFSET = 2, LB_BF16_OFFSET = 3 } lb_precision;

/* Rounding of the half formats when a step stores its populations (FP32 and
 * FP64 always round to nearest).  LB_ROUND_STOCHASTIC rounds to one of the
 * two neighbours with probability given by the distance to them (the
 * hardware's stochastic-rounding conversion), with random bits from a
 * counter-based hash of (site, step), so results stay reproducible and
 * independent of how lattices share a launch; round-to-nearest biases slow
 * shear flows (the stored non-equilibrium part is below one FP16 ulp near
 * the walls), stochastic rounding does not on average. */
typedef enum { LB_ROUND_NEAREST = 0, LB_ROUND_STOCHASTIC = 1 } lb_rounding;

/* LB_COUETTE: x periodic, halfway bounce-back walls at y = -1/2 (velocity
 * -u_wall) and y = ny - 1/2 (velocity +u_wall). */
typedef enum { LB_PERIODIC = 0, LB_COUETTE = 1 } lb_boundary;

/* Prefactor P of Psi = P (1 - exp(-rho/rho0)): sqrt(rho0) as printed after
 * Eq. (2), or rho0. */
typedef enum { LB_PSI_SQRT_RHO0 = 0, LB_PSI_RHO0 = 1 } lb_psi_form;

/* How F_s enters Eq. (1): Shan-Chen equilibrium-velocity shift
 * u_s^eq = u' + tau_s F_s / rho_s with the common velocity
 * u' = sum_s (j_s/tau_s) / sum_s (rho_s/tau_s), or the additive term
 * F_is = w_i (c_i . F_s) / c_s^2 with f^eq at u'. */
typedef enum { LB_FORCE_SHIFT = 0, LB_FORCE_SOURCE = 1 } lb_force_scheme;

typedef struct {
    int32_t nx, ny;            /* lattice size, each >= 8; x is fastest        */
    int32_t boundary;          /* lb_boundary                                  */
    int32_t precision;         /* lb_precision                                 */
    int32_t psi_form;          /* lb_psi_form                                  */
    int32_t force_scheme;      /* lb_force_scheme                              */
    int32_t init_shear;        /* lb_init_seeded velocity: 0 rest, 1 the linear
                                  Couette profile u_x = u_wall (2y+1-ny)/ny     */
    int32_t stress_every;      /* wall-stress sample period in steps (>= 1)    */
    int64_t stress_t0;         /* first step index that is sampled            */
    double tau_A, tau_B;       /* relaxation times, > 1/2                      */
    double G_A1, G_A2;         /* species A: attraction (belt 1), repulsion (belts 1+2) */
    double G_B1, G_B2;         /* species B: attraction, repulsion             */
    double G_X;                /* cross-species coupling G_AB                  */
    double rho0;               /* reference density (> 0)                      */
    double u_wall;             /* Couette wall speed                           */
    double init_amp;           /* lb_init_seeded: rho = rho0 (1 + amp (2u-1))  */
    double rho_ref;            /* offset base of the half formats (0 => rho0)  */
    double g_x;                /* uniform body acceleration along x            */
    double kolmo_amp;          /* Kolmogorov acceleration amplitude            */
    double kolmo_k;            /* a_x += kolmo_amp sin(2 pi kolmo_k y / ny)    */
    int32_t rounding;          /* lb_rounding of the half formats              */
    int32_t tile_rows;         /* step-kernel tile height of an lb_create handle:
                                  0 = library default, 8 (one site per thread)
                                  or 16 (two per thread; not LB_FP64); results
                                  are bitwise the same; pools choose their own */
} lb_params;

typedef struct {
    double mass_A, mass_B;     /* sum of rho_A, rho_B at the current time      */
    double mom_x, mom_y;       /* sum_r sum_s (j_s + F_s/2)                    */
    double sigma_bot, sigma_top; /* time-averaged x-momentum given to the bottom
                                  / top wall per unit length and step          */
    double sigma_mean;         /* (sigma_bot - sigma_top)/2                    */
    double nu_eff;             /* sigma_mean / (shear rate * mean density)     */
    double response_R;         /* nu0 / nu_eff, nu0 = c_s^2 (tau - 1/2)        */
    int64_t samples;           /* number of wall-stress samples averaged       */
    int64_t step;              /* current time step                            */
} lb_stress_out;

/* Fill *p with the Fig. 2 caption couplings, tau = 1, rho0 = 0.70, a periodic
 * 128 x 128 FP32 lattice, init_amp = 0.03, stress_every = 1, stochastic
 * rounding of the half formats. */
void lb_params_default(lb_params* p);

/* Device bytes a handle needs for *p (both population buffers and the
 * reduction area).  LB_ERR_INVALID if *p is not valid. */
lb_status lb_workspace_size(const lb_params* p, size_t* bytes);

/* Validate *p, allocate device memory with cudaMalloc, build the TMA
 * descriptors.  stream is a cudaStream_t (NULL = default stream).  On error
 * *out is NULL and nothing is leaked. */
lb_status lb_create(const lb_params* p, void* stream, lb_handle** out);

/* As lb_create, but the device memory is the caller's: `workspace` must be a
 * device pointer aligned to 256 bytes holding at least lb_workspace_size
 * bytes.  LB_ERR_NOMEM if `bytes` is too small. */
lb_status lb_create_in(const lb_params* p, void* stream, void* workspace, size_t bytes,
                       lb_handle** out);

/* Random initial densities ("random initial conditions for the two
 * densities", text after Eq. (5)): rho_s(x,y) = rho0 (1 + init_amp (2u - 1))
 * with u = (z >> 11) 2^-53, z = mix64(seed ^ mix64(idx + 0x9E3779B97F4A7C15)),
 * idx = (s ny + y) nx + x, mix64 the SplitMix64 finaliser; velocity zero (or
 * the Couette profile if init_shear); populations at equilibrium.  Resets the
 * step counter and the stress averages. */
lb_status lb_init_seeded(lb_handle* h, uint64_t seed);

/* Initial state from host FP64 fields [ny][nx]: f = f^eq(rho_s, u).  ux and
 * uy may be NULL (zero).  Resets the step counter and the stress averages.
 * Synchronises the stream. */
lb_status lb_init_fields(lb_handle* h, const double* rho_A, const double* rho_B,
                         const double* ux, const double* uy);

/* Start from given populations f_is(r, t) [2][9][ny][nx] (host FP64, after
 * streaming and before collision, as lb_populations writes them) at step
 * t >= 0; the wall-stress averages restart.  Synchronises. */
lb_status lb_init_populations(lb_handle* h, const double* f, int64_t t);

/* Checkpoint / restart for long runs (the paper's runs reach 5e6 steps,
 * text before Fig. 4).  lb_checkpoint writes the stored state as it is --
 * [2][9][ny][nx] FP64 values f = stored offset + w_i rho_ref, the step count
 * and `pulled` (1: the state is the post-collision f*(t-1); 0: f(t)) -- and
 * lb_restore loads it into a handle with the same parameters.  The run then
 * continues bitwise as the original for FP32/FP16/BF16 storage (FP64 offsets
 * round-trip to within one ulp); wall-stress averages restart.  Both
 * synchronise. */
lb_status lb_checkpoint(lb_handle* h, double* state, int64_t* t, int32_t* pulled);
lb_status lb_restore(lb_handle* h, const double* state, int64_t t, int32_t pulled);

/* Advance n >= 0 time steps of Eq. (1) (asynchronous on the stream). */
lb_status lb_step(lb_handle* h, int64_t n);

/* Copy the fields at the current time to host FP64 arrays [ny][nx]: the
 * densities and the barycentric velocity u = sum_s (j_s + F_s/2) / sum_s rho_s.
 * Any pointer may be NULL.  Synchronises. */
lb_status lb_fields(lb_handle* h, double* rho_A, double* rho_B, double* ux, double* uy);

/* Copy the populations f_is(r, t) at the current time (after streaming,
 * before collision), decoded to FP64, to a host array [2][9][ny][nx]
 * (species, D2Q9 direction in the order rest, +x, +y, -x, -y, (+1,+1),
 * (-1,+1), (-1,-1), (+1,-1)).  Synchronises. */
lb_status lb_populations(lb_handle* h, double* f);

/* Totals at the current time and the time-averaged wall stress of the
 * Couette walls (response R = nu0/nu_eff as defined after Fig. 3).
 * Synchronises. */
lb_status lb_stress(lb_handle* h, lb_stress_out* out);

/* Wait for the handle's stream and return any latched device error. */
lb_status lb_sync(lb_handle* h);

/* Number of completed time steps. */
int64_t lb_time(const lb_handle* h);

/* Release the handle (NULL is accepted).  Synchronises. */
lb_status lb_destroy(lb_handle* h);

/* ------------------------------------------------------------------------
 * Lattice pool: many resident lattices stepped together, one persistent
 * launch per time step over all active members (builder addition; the paper
 * runs one lattice at a time, and its ensemble averages -- the overlap of
 * Eq. (6) -- need many independent realisations).
 *
 * All members share the pool's precision, couplings (G_A1..G_X), tau_A,
 * tau_B, psi_form, force_scheme and body forces; nx, ny, boundary, rho0,
 * u_wall, init_amp, init_shear, rho_ref and the stress sampling vary per
 * member.  Device memory is one arena of `bytes_budget` bytes allocated at
 * creation; members are placed in it first-fit and admission fails with
 * LB_ERR_NOMEM when a member's footprint does not fit.  Steps run on the
 * pool's stream (a private stream is created when `stream` is NULL); runs of
 * consecutive steps over an unchanged member set are captured once into a
 * CUDA graph and replayed.  The work partition (segment length of the
 * column strips) is tuned by timing candidate partitions on the first steps
 * of each new member set (those steps are real steps) and cached; a member
 * set that runs fewer than 8 times the steps the timing takes (about 400 to
 * 500 steps) keeps the load-balance model's partition instead.
 * ------------------------------------------------------------------------ */
typedef struct lb_pool lb_pool;
typedef int32_t lb_job;

/* Device bytes one member with parameters *p occupies in a pool arena. */
lb_status lb_pool_footprint(const lb_params* p, size_t* bytes);

lb_status lb_pool_create(const lb_params* shared, size_t bytes_budget, int32_t max_jobs,
                         void* stream, lb_pool** out);

/* Admit a member: place it in the arena, initialise it with lb_init_seeded's
 * rule and `seed`, and schedule `steps` time steps.  *job receives its id.
 * LB_ERR_NOMEM if it does not fit; LB_ERR_INVALID if the shared fields of *p
 * differ from the pool's or the pool is full (max_jobs). */
lb_status lb_pool_admit(lb_pool* pool, const lb_params* p, uint64_t seed, int64_t steps,
                        lb_job* job);

/* Advance every active member by min(quantum, its remaining steps); members
 * that reach their step count drop out of the launches.  *active (may be
 * NULL) receives the number of members with steps left afterwards.
 * Asynchronous except for re-partitioning and tuning. */
lb_status lb_pool_run(lb_pool* pool, int64_t quantum, int32_t* active);

/* Set up the step launch of the current member set without taking a step:
 * build its work partition (the cached tuned one, the fixed one of
 * lb_pool_set_partition, or else the load-balance model's -- no tuning) and
 * capture its CUDA graph, so that the next lb_pool_run replays the graph
 * with no capture or instantiation in its way.  A later lb_pool_run on the
 * same member set keeps this partition.  Synchronises the pool stream when
 * it builds; LB_OK with nothing to do when no member has steps left. */
lb_status lb_pool_prepare(lb_pool* pool);

/* Steps done and whether the member has finished (all its steps). */
lb_status lb_pool_poll(lb_pool* pool, lb_job job, int64_t* steps_done, int32_t* done);

/* As lb_init_fields for one member: restart it from caller FP64 host fields
 * (rho_A, rho_B required; ux, uy may be NULL for rest) at step 0, with its
 * scheduled step count unchanged and none of it done. */
lb_status lb_pool_init_fields(lb_pool* pool, lb_job job, const double* rho_A, const double* rho_B,
                              const double* ux, const double* uy);

/* As lb_fields / lb_stress for one member (synchronise the pool stream). */
lb_status lb_pool_fields(lb_pool* pool, lb_job job, double* rho_A, double* rho_B, double* ux,
                         double* uy);
lb_status lb_pool_stress(lb_pool* pool, lb_job job, lb_stress_out* out);

/* Free a member's arena space (finished or not). */
lb_status lb_pool_release(lb_pool* pool, lb_job job);

/* Work partition the current member set runs with: > 0, segments of that
 * many tiles dealt to the CTAs in turn; -1, one contiguous run of tiles per
 * CTA; 0 if none is built. */
int32_t lb_pool_segment(const lb_pool* pool);

/* Fix the work partition instead of measuring candidates: seg > 0 segments
 * of seg tiles dealt to the CTAs in turn, -1 one contiguous run of tiles per
 * CTA, 0 back to autotuning.  Applies from the next lb_pool_run. */
lb_status lb_pool_set_partition(lb_pool* pool, int32_t seg);

/* Tile height of the step kernel: the autotuner times both tile shapes (8
 * rows, one site per thread; 16 rows, two vertically adjacent sites per
 * thread sharing their stencil rows -- not for FP64) together with the
 * partitions.  lb_pool_set_tile_rows fixes it (8 or 16; 0 back to
 * autotuning; LB_ERR_INVALID for a shape the pool's precision lacks), from
 * the next lb_pool_run; lb_pool_tile_rows returns the current launch's, or
 * 0 if none is built.  Every shape gives bitwise the same results. */
lb_status lb_pool_set_tile_rows(lb_pool* pool, int32_t rows);
int32_t lb_pool_tile_rows(const lb_pool* pool);

lb_status lb_pool_destroy(lb_pool* pool);

/* Host only, no device work (usable without a GPU): the work items that one
 * step launch over `nlat` lattices with parameters ps[0 .. nlat-1] would use
 * on a device with `sms` SMs.  seg > 0: segments of seg tiles, each given in
 * band order to the CTA with the least estimated work; -1: one cost-balanced
 * contiguous run of tiles per CTA; 0: the library's default for these sizes.
 * A tile is TX x tile_rows sites (TX = 60; 28 for FP64), a strip a TX-wide
 * column of tiles; tile_rows is 8 (or 0, meaning 8) or 16 (not for FP64).  On entry *nitems is the capacity of `items` (in items of
 * 4 int32: lattice index, strip, first tile row, end tile row) and *grid the
 * capacity of `cta` (in entries); on return they hold the item count and the
 * number of CTAs, items lists the items CTA by CTA, the items of CTA b are
 * items[cta[b] .. cta[b + 1]) (grid + 1 entries), and *seg_used the
 * partition applied.  LB_ERR_INVALID for an invalid lattice, mixed
 * precisions, nlat or sms < 1, or a capacity too small (the sizes needed
 * are still returned).  No pointer is retained. */
lb_status lb_plan_partition(const lb_params* ps, int32_t nlat, int32_t seg, int32_t tile_rows,
                            int32_t sms, int32_t* items, int32_t* nitems, int32_t* cta,
                            int32_t* grid, int32_t* seg_used);

/* Largest lattice, nx * ny, that lb_totals_noalloc accepts (4096 x 4096). */
#define LB_NOALLOC_MAX_SITES 16777216

/* Totals of caller-owned FP64 device fields, without allocating anything.
 * The paper has no counterpart; this entry point exists for callers that may
 * not call cudaMalloc -- for instance code that runs inside a fixed device
 * arena it cannot grow, or inside a framework that forbids allocation on its
 * hot path.  It is the mass/momentum reduction of lb_stress (FP64 warp sums,
 * one slot per CTA, the last CTA adds the slots in a fixed order) run on
 * fields the caller passes in.
 *
 * Inputs: device arrays rho_A, rho_B, ux, uy of nx * ny FP64 values each
 * (any layout, e.g. [ny][nx] as lb_fields writes them).  Output: `totals`, a
 * device array of 4 doubles, receives {sum rho_A, sum rho_B,
 * sum (rho_A + rho_B) ux, sum (rho_A + rho_B) uy}, asynchronously on `stream`
 * (a cudaStream_t, NULL = default stream).  Returns LB_ERR_INVALID for a NULL
 * pointer, nx or ny < 1, or nx * ny > LB_NOALLOC_MAX_SITES.
 *
 * Scratch: the per-CTA slots and the arrival counter live in one static
 * device array of 128 KB + 256 B that every GPU which loads the library keeps
 * until the process exits.  The first call on a device looks up that array's
 * device address (cudaGetSymbolAddress); make that first call before any
 * stream capture.  The address is kept per device and context: after a
 * cudaDeviceReset the next call on the new context looks it up again (and is
 * then again a first call).  Each call clears the counter with cudaMemsetAsync on
 * `stream` and overwrites the slots it uses.  All calls on a device share the
 * array, so calls whose kernels may overlap on the GPU (different streams with
 * no ordering between them) race: order them on one stream or with events. */
lb_status lb_totals_noalloc(int32_t nx, int32_t ny, const double* rho_A, const double* rho_B,
                            const double* ux, const double* uy, double* totals, void* stream);

/* Diagnostic, no counterpart in the paper: runs the step kernel's bounded
 * mbarrier wait on a barrier that nothing will complete, with a bound of
 * `limit` polls (>= 1), on `stream`.  The wait gives up and the kernel
 * latches its timeout flag, which comes back as LB_ERR_TIMEOUT; the context
 * stays usable.  Any other status means the wait or the error path is
 * broken.  Allocates (and frees) one word of device memory. */
lb_status lb_selftest_wait(void* stream, int32_t limit);

/* Diagnostic, no counterpart in the paper: evaluates the FP32 functions the
 * step kernel uses for the pseudo-potential and the velocities -- its
 * exp(x) - 1 (Cody-Waite reduction x = k ln 2 + r, degree-7 Taylor series of
 * expm1(r), about 2 ulp) and its reciprocal (rcp.approx.ftz, within 1 ulp)
 * -- on n caller values, next to the CUDA library's expm1f, so that their
 * error can be measured over the arguments the kernel sees.  x: device
 * array of n floats; out: device array of 3 n floats, receiving
 * {pexpm1(x[k]), expm1f(x[k]), recip(x[k])} at out[3k .. 3k + 2] (reciprocal
 * flushes subnormal results to zero).  Asynchronous on `stream`;
 * LB_ERR_INVALID for n < 0 or a NULL pointer with n > 0. */
lb_status lb_selftest_math(const float* x, float* out, int64_t n, void* stream);

/* Static description of a status code. */
const char* lb_status_string(lb_status s);

#ifdef __cplusplus
}
#endif

#endif /* LB_H */
