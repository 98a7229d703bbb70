"""Seeded synthetic workloads shared by the tests, the smoke check and the bench.

This module holds only input data and seeded generators: the coupling
constants printed in the paper (Fig. 2 caption), the lattice sizes, seeds and
sweeps of the benchmark workloads, and numpy-driven samplers for the batched
and served job mixes.  It contains none of the model's arithmetic, so both the
FP64 CPU oracle and the GPU library can be fed from it.
"""
from __future__ import annotations

import math

import numpy as np

# Couplings of the Fig. 2 caption: G_A1 = -12.55 (A attraction, belt 1),
# G_A2 = 11.70 (A repulsion, belts 1+2), G_B1 = -11.80, G_B2 = 10.95,
# G^X = 0.58, rho0 = 0.70.  tau is not given in the paper; 1.0 is used.
CAPTION = dict(Ga=(-12.55, -11.80), Gr=(11.70, 10.95), GX=0.58, rho0=0.70)
TAU = (1.0, 1.0)
INIT_AMP = 0.03

# Plain method, FP64: 128^2 periodic, seed 0, 500 steps.
CFG_PLAIN = dict(nx=128, ny=128, seed=0, steps=500, boundary=0)
# FP32 at the paper's resolution: 512^2 periodic, seed 1, rho0 sweep.
CFG_SWEEP = dict(nx=512, ny=512, seed=1, rho0s=(0.55, 0.65, 0.70, 0.75, 0.83),
                 steps=100_000, snapshot_every=10_000)
# Plane Couette shear: 512 x 512, walls in y, seed 2, 8 log-spaced shear rates.
CFG_COUETTE = dict(nx=512, ny=512, seed=2, rho0=0.70, steps=200_000)
# Peak-bandwidth lattice.
CFG_PEAK = dict(nx=4096, ny=4096, seed=5)
# Batched: steps of every lattice of the 64-lattice mix.
CFG_BATCH_STEPS = 20_000


def couette_shear_rates(n: int = 8, lo: float = 1e-6, hi: float = 1e-4):
    """The 8 log-spaced shear rates 1e-6 .. 1e-4."""
    return [float(v) for v in np.logspace(math.log10(lo), math.log10(hi), n)]


def wall_speed(shear_rate: float, ny: int) -> float:
    """Wall speed U for shear rate 2U/H with H = ny (walls at y=-1/2, ny-1/2)."""
    return shear_rate * ny / 2.0


def uniforms(seed: int, shape):
    """Plain U[0,1) draws (numpy PCG64) for explicitly supplied fields."""
    return np.random.default_rng(seed).random(shape)


def sample_batch(seed: int = 3, count: int = 64,
                 sizes=(128, 256, 512, 1024)):
    """Batched workload: lattices with sizes drawn uniformly from `sizes`,
    rho0 ~ U[0.55, 0.83], half periodic and half Couette (shear rate
    log-uniform in [1e-6, 1e-4])."""
    rng = np.random.default_rng(seed)
    jobs = []
    for k in range(count):
        L = int(rng.choice(sizes))
        rho0 = float(rng.uniform(0.55, 0.83))
        couette = k >= count // 2
        rate = float(10 ** rng.uniform(-6, -4)) if couette else 0.0
        jobs.append(dict(nx=L, ny=L, rho0=rho0, boundary=1 if couette else 0,
                         shear_rate=rate, seed=int(rng.integers(0, 2**31))))
    return jobs


def sample_serving(seed: int = 4, count: int = 2000, lmin: int = 64,
                   lmax: int = 2048, steps_lo: float = 1e3, steps_hi: float = 1e5):
    """Served workload: jobs with square lattices of side log-uniform in
    [lmin, lmax] (rounded up to a multiple of 8), rho0 ~ U[0.55, 0.83],
    shear rate from {0} and the 8 Couette rates, step counts log-uniform.
    Arrival times are returned in units of the mean inter-arrival gap
    (multiply by the chosen gap in seconds)."""
    rng = np.random.default_rng(seed)
    rates = [0.0] + couette_shear_rates()
    jobs = []
    t = 0.0
    for _ in range(count):
        t += float(rng.exponential(1.0))
        L = float(math.exp(rng.uniform(math.log(lmin), math.log(lmax))))
        L = int(math.ceil(L / 8.0) * 8)
        rate = float(rates[int(rng.integers(0, len(rates)))])
        steps = int(round(math.exp(rng.uniform(math.log(steps_lo), math.log(steps_hi)))))
        jobs.append(dict(arrival=t, nx=L, ny=L, rho0=float(rng.uniform(0.55, 0.83)),
                         boundary=1 if rate > 0 else 0, shear_rate=rate, steps=steps,
                         seed=int(rng.integers(0, 2**31))))
    return jobs
