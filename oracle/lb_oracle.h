/*
 * lb_oracle.h -- FP64 CPU oracle for the two-species multi-range
 * pseudo-potential lattice Boltzmann model of Benzi, Chibbaro & Succi,
 * "Mesoscopic lattice Boltzmann modeling of flowing soft systems"
 * (arXiv:0807.4471).
 *
 * TEST INFRASTRUCTURE ONLY.  This code is the slow, plain, obviously-correct
 * statement of what one time step computes.  Only the test-suite, the smoke
 * check and the timed CPU baseline of bench.py may load it.  The GPU library
 * (paper_0807_4471_gb300) shares no code, header, table or constant with it.
 *
 * Storage: array of sites, f[((y*nx + x)*2 + s)*9 + i], s = 0 (A), 1 (B),
 * i the D2Q9 direction index of or_velocities().  All arrays are caller-owned.
 */
#ifndef LB_ORACLE_H
#define LB_ORACLE_H
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* Model parameters (the paper's couplings, plus the readings the paper
 * leaves open).  Doubles first so the layout is the same under ctypes. */
typedef struct {
    double tau[2];      /* relaxation times tau_A, tau_B (Eq. 1)            */
    double Ga[2];       /* G^a_s: like-species attraction, belt 1, weights w */
    double Gr[2];       /* G^r_s: like-species repulsion, belts 1+2, weights p */
    double GX;          /* G_AB: cross-species repulsion, belt 1, weights w  */
    double rho0;        /* reference density of Psi and of F^X               */
    double u_wall;      /* Couette: top wall +u_wall, bottom wall -u_wall    */
    double init_amp;    /* seeded init: rho = rho0 (1 + amp (2u - 1))       */
    double g_x;         /* uniform body acceleration along x (0: none)      */
    double kolmo_amp;   /* Kolmogorov acceleration amplitude (0: none)      */
    double kolmo_k;     /* Kolmogorov wave number: a_x += amp sin(2 pi k y / ny) */
    int32_t nx, ny;
    int32_t boundary;      /* 0 periodic; 1 Couette (x periodic, walls in y) */
    int32_t psi_form;      /* 0: sqrt(rho0)(1-e^{-rho/rho0}); 1: rho0(1-e^{-rho/rho0}) */
    int32_t force_scheme;  /* 0: Shan-Chen velocity shift; 1: additive source term */
    int32_t init_shear;    /* seeded init velocity: 0 rest; 1 linear Couette profile */
    int32_t stress_every;  /* wall-stress sample period (>= 1)                */
    int32_t pad_;
    int64_t stress_t0;     /* first sampled step                             */
} or_params;

/* Time-averaged wall momentum exchange (Couette). */
typedef struct {
    double sum_bot, sum_top;   /* sums of per-step samples              */
    int64_t samples;
} or_accum;

/* 25-vector stencil: index 0 rest, 1..8 first belt (D2Q9 order), 9..24
 * second belt.  w[0..8] are the D2Q9 weights, p[0..24] the multi-range
 * weights (p[0] the rest weight fixed by sum p = 1). */
void or_velocities(int32_t cx[25], int32_t cy[25]);
void or_weights(double w[9], double p[25]);
int32_t or_opposite(int32_t i);

double or_psi(const or_params* P, double rho);
void or_feq(double rho, double ux, double uy, double feq[9]);

uint64_t or_mix64(uint64_t z);
double or_uniform(uint64_t seed, uint64_t idx);

void or_init_seeded(const or_params* P, uint64_t seed, double* f);
void or_init_fields(const or_params* P, const double* rhoA, const double* rhoB,
                    const double* ux, const double* uy, double* f);

void or_moments(const or_params* P, const double* f, double* rho, double* jx, double* jy);
void or_forces(const or_params* P, const double* rho, double* Fx, double* Fy);
void or_forces_interaction(const or_params* P, const double* rho, double* Fx, double* Fy);

int or_step(const or_params* P, double* f, double* scratch, int64_t t, or_accum* acc);
int or_run(const or_params* P, double* f, int64_t t0, int64_t nsteps, or_accum* acc);
void or_stream_only(const or_params* P, double* f, int64_t nsteps);

void or_fields(const or_params* P, const double* f, double* rhoA, double* rhoB,
               double* ux, double* uy);
void or_totals(const or_params* P, const double* f, double out[4]);

#ifdef __cplusplus
}
#endif
#endif
