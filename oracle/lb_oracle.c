/*
 * lb_oracle.c -- FP64 CPU oracle of the two-species multi-range
 * pseudo-potential lattice Boltzmann model (Benzi, Chibbaro & Succi,
 * arXiv:0807.4471).
 *
 * TEST INFRASTRUCTURE ONLY: the plain, slow, obviously-correct statement of
 * one time step, used by the tests, the smoke check and the CPU baseline of
 * the benchmark.  The GPU path shares no code with this file.
 *
 * One step follows the order of the paper's kinetic equation, Eq. (1):
 *   1. moments        rho_s = sum_i f_is, j_s = sum_i f_is c_i
 *   2. pseudo-potential Psi_s(rho_s)             (definition after Eq. (2))
 *   3. forces F^a_s + F^r_s + F^X_s              (Eq. (2))
 *   4. BGK relaxation toward the local equilibrium with the force  (Eq. (1))
 *   5. free streaming along c_i (push)           (left-hand side of Eq. (1))
 * Plain loops, array-of-sites storage, no tiling, no fusion.
 *
 * Readings of points the paper leaves open (each is also listed in the
 * design notes of the repository):
 *  - Force sign: the paper states that positive G codes for repulsion, so
 *    every term of Eq. (2) carries an overall minus sign (Shan-Chen form).
 *  - Weights w (D2Q9) and p (25-vector multi-range stencil) are not printed;
 *    they are the unique solution of the paper's normalisation constraints
 *    (sum = 1, second moment = c_s^2 = 1/3) plus isotropy to 8th order, which
 *    the paper requires of the 24-speed lattice.  The tests re-derive them.
 *  - The force enters Eq. (1) either by the Shan-Chen velocity shift (the
 *    scheme of the paper's ref. for Psi; default) or as the additive term
 *    F_is = w_i (c_i . F_s) / c_s^2 (force_scheme = 1).
 *  - Equilibrium: the second-order D2Q9 polynomial ("local Maxwellian").
 *  - Psi prefactor sqrt(rho0) (paper) or rho0 (psi_form = 1).
 *  - Couette walls: halfway bounce-back with moving-wall term, walls at
 *    y = -1/2 (velocity -U) and y = ny - 1/2 (velocity +U); the wall density
 *    is the pre-streaming density of the boundary node, i.e. the sum of its
 *    post-collision populations; Psi and rho beyond a wall are mirrored about
 *    the wall (neutral wetting).
 */
#include "lb_oracle.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>

/* ---------------------------------------------------------------- lattice */

/* First belt: the D2Q9 speeds (rest, 4 axis, 4 diagonal), b1 = 8.
 * Second belt: the 16 speeds with |c|^2 in {4, 5, 8}, b2 = 16, b = 24.
 * (Paragraph after Eq. (2): "the first belt is discretized with 9 speeds,
 * the second with 16".) */
static const int32_t CX[25] = {0, 1, 0, -1, 0, 1, -1, -1, 1,
                               2, 0, -2, 0,
                               2, 1, -1, -2, -2, -1, 1, 2,
                               2, -2, -2, 2};
static const int32_t CY[25] = {0, 0, 1, 0, -1, 1, 1, -1, -1,
                               0, 2, 0, -2,
                               1, 2, 2, 1, -1, -2, -2, -1,
                               2, 2, -2, -2};
static const int32_t OPP[9] = {0, 3, 4, 1, 2, 7, 8, 5, 6};

static const double CS2 = 1.0 / 3.0; /* lattice sound speed squared */

/* D2Q9 weights by |c|^2: 0 -> 4/9, 1 -> 1/9, 2 -> 1/36. */
static double w_of(int c2) {
    if (c2 == 0) return 4.0 / 9.0;
    if (c2 == 1) return 1.0 / 9.0;
    return 1.0 / 36.0;
}

/* Multi-range weights by |c|^2 (8th-order isotropic, second moment 1/3):
 * 1 -> 4/63, 2 -> 4/135, 4 -> 1/180, 5 -> 2/945, 8 -> 1/15120;
 * the rest weight closes sum p = 1. */
static double p_of(int c2) {
    switch (c2) {
        case 1: return 4.0 / 63.0;
        case 2: return 4.0 / 135.0;
        case 4: return 1.0 / 180.0;
        case 5: return 2.0 / 945.0;
        case 8: return 1.0 / 15120.0;
        default: break;
    }
    /* rest: 1 - sum over the 24 moving speeds */
    double s = 0.0;
    for (int i = 1; i < 25; ++i) s += p_of(CX[i] * CX[i] + CY[i] * CY[i]);
    return 1.0 - s;
}

void or_velocities(int32_t cx[25], int32_t cy[25]) {
    for (int i = 0; i < 25; ++i) { cx[i] = CX[i]; cy[i] = CY[i]; }
}

void or_weights(double w[9], double p[25]) {
    for (int i = 0; i < 9; ++i) w[i] = w_of(CX[i] * CX[i] + CY[i] * CY[i]);
    for (int i = 0; i < 25; ++i) p[i] = p_of(CX[i] * CX[i] + CY[i] * CY[i]);
}

int32_t or_opposite(int32_t i) { return OPP[i]; }

/* -------------------------------------------------------- local functions */

/* Pseudo-potential (definition after Eq. (2)): P (1 - exp(-rho/rho0)),
 * P = sqrt(rho0) as printed, or P = rho0 (psi_form = 1). */
double or_psi(const or_params* P, double rho) {
    double pref = (P->psi_form == 1) ? P->rho0 : sqrt(P->rho0);
    return pref * (1.0 - exp(-rho / P->rho0));
}

/* Local equilibrium, second order in u (D2Q9, c_s^2 = 1/3). */
void or_feq(double rho, double ux, double uy, double feq[9]) {
    double usq = ux * ux + uy * uy;
    for (int i = 0; i < 9; ++i) {
        double cu = CX[i] * ux + CY[i] * uy;
        feq[i] = w_of(CX[i] * CX[i] + CY[i] * CY[i]) * rho *
                 (1.0 + cu / CS2 + cu * cu / (2.0 * CS2 * CS2) - usq / (2.0 * CS2));
    }
}

/* SplitMix64 finaliser (Steele, Lea & Flood, OOPSLA 2014). */
uint64_t or_mix64(uint64_t z) {
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
    return z ^ (z >> 31);
}

/* Counter-based uniform in [0,1): z = mix64(seed ^ mix64(idx + golden)),
 * u = (z >> 11) 2^-53. */
double or_uniform(uint64_t seed, uint64_t idx) {
    uint64_t z = or_mix64(seed ^ or_mix64(idx + 0x9E3779B97F4A7C15ULL));
    return (double)(z >> 11) * (1.0 / 9007199254740992.0);
}

static int64_t site(const or_params* P, int x, int y) { return (int64_t)y * P->nx + x; }

static int wrap(int a, int n) { a %= n; return a < 0 ? a + n : a; }

/* Neighbour row for the force stencils: periodic wrap, or the mirror image
 * about the halfway wall for Couette. */
static int nb_row(const or_params* P, int y) {
    if (P->boundary == 1) {
        if (y < 0) return -1 - y;
        if (y >= P->ny) return 2 * P->ny - 1 - y;
        return y;
    }
    return wrap(y, P->ny);
}

/* External acceleration along x at row y (uniform part + Kolmogorov). */
static double accel_x(const or_params* P, int y) {
    double a = P->g_x;
    if (P->kolmo_amp != 0.0)
        a += P->kolmo_amp * sin(2.0 * M_PI * P->kolmo_k * (double)y / (double)P->ny);
    return a;
}

/* ------------------------------------------------------------- initialise */

void or_init_fields(const or_params* P, const double* rhoA, const double* rhoB,
                    const double* ux, const double* uy, double* f) {
    int64_t n = (int64_t)P->nx * P->ny;
    for (int64_t r = 0; r < n; ++r) {
        double u = ux ? ux[r] : 0.0, v = uy ? uy[r] : 0.0;
        or_feq(rhoA[r], u, v, f + (r * 2 + 0) * 9);
        or_feq(rhoB[r], u, v, f + (r * 2 + 1) * 9);
    }
}

/* Random initial densities ("random initial conditions for the two
 * densities", after Fig. 2): rho_s = rho0 (1 + amp (2u - 1)), u from the
 * counter generator at index (s ny + y) nx + x; f = f^eq(rho_s, u0(y)). */
void or_init_seeded(const or_params* P, uint64_t seed, double* f) {
    int nx = P->nx, ny = P->ny;
    for (int y = 0; y < ny; ++y) {
        double u0 = 0.0;
        if (P->init_shear)
            u0 = P->u_wall * (2.0 * y + 1.0 - ny) / (double)ny;
        for (int x = 0; x < nx; ++x) {
            for (int s = 0; s < 2; ++s) {
                uint64_t idx = ((uint64_t)s * ny + y) * nx + x;
                double rho = P->rho0 * (1.0 + P->init_amp * (2.0 * or_uniform(seed, idx) - 1.0));
                or_feq(rho, u0, 0.0, f + (site(P, x, y) * 2 + s) * 9);
            }
        }
    }
}

/* ---------------------------------------------------------------- moments */

/* rho[s*N + r], jx[s*N + r], jy[s*N + r]. */
void or_moments(const or_params* P, const double* f, double* rho, double* jx, double* jy) {
    int64_t n = (int64_t)P->nx * P->ny;
    for (int64_t r = 0; r < n; ++r)
        for (int s = 0; s < 2; ++s) {
            const double* fi = f + (r * 2 + s) * 9;
            double d = 0, mx = 0, my = 0;
            for (int i = 0; i < 9; ++i) { d += fi[i]; mx += fi[i] * CX[i]; my += fi[i] * CY[i]; }
            rho[s * n + r] = d;
            if (jx) jx[s * n + r] = mx;
            if (jy) jy[s * n + r] = my;
        }
}

/* ----------------------------------------------------------------- forces */

/* Interaction force of Eq. (2), with the overall minus sign:
 *   F^a_s = -G^a_s Psi_s(r) sum_{belt1} w_i Psi_s(r + c_i) c_i
 *   F^r_s = -G^r_s Psi_s(r) [sum_{belt1} p_i Psi_s(r + c_i) c_i
 *                            + sum_{belt2} p_i Psi_s(r + c_i) c_i]
 *   F^X_s = -(G_AB / rho0) rho_s(r) sum_{belt1} w_i rho_s'(r + c_i) c_i
 * (the rest speed contributes nothing).  rho[s*N + r] in, F[s*N + r] out. */
void or_forces_interaction(const or_params* P, const double* rho, double* Fx, double* Fy) {
    int nx = P->nx, ny = P->ny;
    int64_t n = (int64_t)nx * ny;
    double w[9], p[25];
    or_weights(w, p);
    double* psi = (double*)malloc(sizeof(double) * 2 * n);
    for (int64_t k = 0; k < 2 * n; ++k) psi[k] = or_psi(P, rho[k]);

    for (int y = 0; y < ny; ++y)
        for (int x = 0; x < nx; ++x) {
            int64_t r = site(P, x, y);
            for (int s = 0; s < 2; ++s) {
                int so = 1 - s;
                const double* ps = psi + s * n;
                const double* ro = rho + so * n;
                double ax = 0, ay = 0;   /* attraction sum (belt 1, w)     */
                double rx = 0, ry = 0;   /* repulsion sum (belts 1+2, p)   */
                double xx = 0, xy = 0;   /* cross sum (belt 1, w, rho_s')  */
                for (int i = 1; i <= 8; ++i) {
                    int64_t q = site(P, wrap(x + CX[i], nx), nb_row(P, y + CY[i]));
                    ax += w[i] * ps[q] * CX[i];
                    ay += w[i] * ps[q] * CY[i];
                    xx += w[i] * ro[q] * CX[i];
                    xy += w[i] * ro[q] * CY[i];
                }
                for (int i = 1; i <= 8; ++i) {
                    int64_t q = site(P, wrap(x + CX[i], nx), nb_row(P, y + CY[i]));
                    rx += p[i] * ps[q] * CX[i];
                    ry += p[i] * ps[q] * CY[i];
                }
                for (int i = 9; i <= 24; ++i) {
                    int64_t q = site(P, wrap(x + CX[i], nx), nb_row(P, y + CY[i]));
                    rx += p[i] * ps[q] * CX[i];
                    ry += p[i] * ps[q] * CY[i];
                }
                double Fax = -P->Ga[s] * ps[r] * ax, Fay = -P->Ga[s] * ps[r] * ay;
                double Frx = -P->Gr[s] * ps[r] * rx, Fry = -P->Gr[s] * ps[r] * ry;
                double FXx = -(P->GX / P->rho0) * rho[s * n + r] * xx;
                double FXy = -(P->GX / P->rho0) * rho[s * n + r] * xy;
                Fx[s * n + r] = Fax + Frx + FXx;
                Fy[s * n + r] = Fay + Fry + FXy;
            }
        }
    free(psi);
}

/* Total force on species s: the interaction force plus rho_s a(y). */
void or_forces(const or_params* P, const double* rho, double* Fx, double* Fy) {
    int nx = P->nx, ny = P->ny;
    int64_t n = (int64_t)nx * ny;
    or_forces_interaction(P, rho, Fx, Fy);
    for (int y = 0; y < ny; ++y) {
        double a = accel_x(P, y);
        if (a == 0.0) continue;
        for (int x = 0; x < nx; ++x)
            for (int s = 0; s < 2; ++s) Fx[s * n + site(P, x, y)] += rho[s * n + site(P, x, y)] * a;
    }
}

/* ------------------------------------------------------------------- step */

static int sampled(const or_params* P, int64_t t) {
    int64_t every = P->stress_every > 0 ? P->stress_every : 1;
    return t >= P->stress_t0 && ((t - P->stress_t0) % every) == 0;
}

/* One time step t -> t+1 of Eq. (1).  f holds f(t) on entry and f(t+1) on
 * exit; scratch must hold 18 N doubles.  Returns 0, or 1 if a density is
 * not finite. */
int or_step(const or_params* P, double* f, double* scratch, int64_t t, or_accum* acc) {
    int nx = P->nx, ny = P->ny;
    int64_t n = (int64_t)nx * ny;
    double* rho = (double*)malloc(sizeof(double) * 2 * n);
    double* jx = (double*)malloc(sizeof(double) * 2 * n);
    double* jy = (double*)malloc(sizeof(double) * 2 * n);
    double* Fx = (double*)malloc(sizeof(double) * 2 * n);
    double* Fy = (double*)malloc(sizeof(double) * 2 * n);
    double* fs = scratch;   /* post-collision populations */
    int bad = 0;

    /* 1-3: moments, pseudo-potential, forces */
    or_moments(P, f, rho, jx, jy);
    for (int64_t k = 0; k < 2 * n; ++k)
        if (!isfinite(rho[k])) bad = 1;
    or_forces(P, rho, Fx, Fy);

    /* 4: collision.  Common velocity u' = sum_s (j_s/tau_s) / sum_s (rho_s/tau_s). */
    double w[9], p[25];
    or_weights(w, p);
    for (int64_t r = 0; r < n; ++r) {
        double den = rho[r] / P->tau[0] + rho[n + r] / P->tau[1];
        double upx = 0.0, upy = 0.0;
        if (den != 0.0) {
            upx = (jx[r] / P->tau[0] + jx[n + r] / P->tau[1]) / den;
            upy = (jy[r] / P->tau[0] + jy[n + r] / P->tau[1]) / den;
        }
        for (int s = 0; s < 2; ++s) {
            const double* fi = f + (r * 2 + s) * 9;
            double* fo = fs + (r * 2 + s) * 9;
            double d = rho[s * n + r], F_x = Fx[s * n + r], F_y = Fy[s * n + r];
            double tau = P->tau[s], feq[9];
            if (P->force_scheme == 0) {
                /* velocity shift: u_s^eq = u' + tau_s F_s / rho_s */
                double ueqx = upx, ueqy = upy;
                if (d != 0.0) { ueqx += tau * F_x / d; ueqy += tau * F_y / d; }
                or_feq(d, ueqx, ueqy, feq);
                for (int i = 0; i < 9; ++i) fo[i] = fi[i] - (fi[i] - feq[i]) / tau;
            } else {
                /* additive source F_is = w_i (c_i . F_s) / c_s^2 */
                or_feq(d, upx, upy, feq);
                for (int i = 0; i < 9; ++i)
                    fo[i] = fi[i] - (fi[i] - feq[i]) / tau + w[i] * (CX[i] * F_x + CY[i] * F_y) / CS2;
            }
        }
    }

    /* 5: streaming (push), with halfway bounce-back at the Couette walls. */
    double sb = 0.0, st = 0.0;
    for (int y = 0; y < ny; ++y)
        for (int x = 0; x < nx; ++x) {
            int64_t r = site(P, x, y);
            for (int s = 0; s < 2; ++s) {
                const double* fo = fs + (r * 2 + s) * 9;
                double rho_w = 0.0;
                for (int i = 0; i < 9; ++i) rho_w += fo[i];
                for (int i = 0; i < 9; ++i) {
                    int yd = y + CY[i];
                    if (P->boundary == 1 && (yd < 0 || yd >= ny)) {
                        double uw = (yd < 0) ? -P->u_wall : P->u_wall;
                        int ib = OPP[i];
                        double back = fo[i] - 2.0 * w[i] * rho_w * (CX[i] * uw) / CS2;
                        f[(r * 2 + s) * 9 + ib] = back;
                        double dp = CX[i] * (fo[i] + back);  /* momentum to the wall */
                        if (yd < 0) sb += dp; else st += dp;
                    } else {
                        int xd = wrap(x + CX[i], nx);
                        int yw = (P->boundary == 1) ? yd : wrap(yd, ny);
                        f[(site(P, xd, yw) * 2 + s) * 9 + i] = fo[i];
                    }
                }
            }
        }
    if (acc && P->boundary == 1 && sampled(P, t)) {
        acc->sum_bot += sb / nx;
        acc->sum_top += st / nx;
        acc->samples += 1;
    }
    free(rho); free(jx); free(jy); free(Fx); free(Fy);
    return bad;
}

int or_run(const or_params* P, double* f, int64_t t0, int64_t nsteps, or_accum* acc) {
    int64_t n = (int64_t)P->nx * P->ny;
    double* scratch = (double*)malloc(sizeof(double) * 18 * n);
    int bad = 0;
    for (int64_t k = 0; k < nsteps; ++k) bad |= or_step(P, f, scratch, t0 + k, acc);
    free(scratch);
    return bad;
}

/* Free streaming alone (no collision, no force): a permutation of f. */
void or_stream_only(const or_params* P, double* f, int64_t nsteps) {
    int nx = P->nx, ny = P->ny;
    int64_t n = (int64_t)nx * ny;
    double* g = (double*)malloc(sizeof(double) * 18 * n);
    for (int64_t k = 0; k < nsteps; ++k) {
        memcpy(g, f, sizeof(double) * 18 * n);
        for (int y = 0; y < ny; ++y)
            for (int x = 0; x < nx; ++x)
                for (int s = 0; s < 2; ++s)
                    for (int i = 0; i < 9; ++i) {
                        double v = g[(site(P, x, y) * 2 + s) * 9 + i];
                        int yd = y + CY[i];
                        if (P->boundary == 1 && (yd < 0 || yd >= ny))
                            f[(site(P, x, y) * 2 + s) * 9 + OPP[i]] = v;
                        else
                            f[(site(P, wrap(x + CX[i], nx), wrap(yd, ny)) * 2 + s) * 9 + i] = v;
                    }
    }
    free(g);
}

/* ------------------------------------------------------------ observables */

/* Densities and the barycentric velocity u = sum_s (j_s + F_s/2) / sum_s rho_s
 * at the current time.  Any output may be NULL. */
void or_fields(const or_params* P, const double* f, double* rhoA, double* rhoB,
               double* ux, double* uy) {
    int64_t n = (int64_t)P->nx * P->ny;
    double* rho = (double*)malloc(sizeof(double) * 2 * n);
    double* jx = (double*)malloc(sizeof(double) * 2 * n);
    double* jy = (double*)malloc(sizeof(double) * 2 * n);
    double* Fx = (double*)malloc(sizeof(double) * 2 * n);
    double* Fy = (double*)malloc(sizeof(double) * 2 * n);
    or_moments(P, f, rho, jx, jy);
    or_forces(P, rho, Fx, Fy);
    for (int64_t r = 0; r < n; ++r) {
        double tot = rho[r] + rho[n + r];
        if (rhoA) rhoA[r] = rho[r];
        if (rhoB) rhoB[r] = rho[n + r];
        double mx = jx[r] + jx[n + r] + 0.5 * (Fx[r] + Fx[n + r]);
        double my = jy[r] + jy[n + r] + 0.5 * (Fy[r] + Fy[n + r]);
        if (ux) ux[r] = tot != 0.0 ? mx / tot : 0.0;
        if (uy) uy[r] = tot != 0.0 ? my / tot : 0.0;
    }
    free(rho); free(jx); free(jy); free(Fx); free(Fy);
}

/* out = {mass_A, mass_B, momentum_x, momentum_y}, momentum of the
 * barycentric velocity, sum_r sum_s (j_s + F_s/2). */
void or_totals(const or_params* P, const double* f, double out[4]) {
    int64_t n = (int64_t)P->nx * P->ny;
    double* rho = (double*)malloc(sizeof(double) * 2 * n);
    double* jx = (double*)malloc(sizeof(double) * 2 * n);
    double* jy = (double*)malloc(sizeof(double) * 2 * n);
    double* Fx = (double*)malloc(sizeof(double) * 2 * n);
    double* Fy = (double*)malloc(sizeof(double) * 2 * n);
    or_moments(P, f, rho, jx, jy);
    or_forces(P, rho, Fx, Fy);
    double mA = 0, mB = 0, px = 0, py = 0;
    for (int64_t r = 0; r < n; ++r) {
        mA += rho[r];
        mB += rho[n + r];
        px += jx[r] + jx[n + r] + 0.5 * (Fx[r] + Fx[n + r]);
        py += jy[r] + jy[n + r] + 0.5 * (Fy[r] + Fy[n + r]);
    }
    out[0] = mA; out[1] = mB; out[2] = px; out[3] = py;
    free(rho); free(jx); free(jy); free(Fx); free(Fy);
}
