"""Observables of the experiments module against closed forms, and the
oracle against two physical facts they rely on: the steady Kolmogorov
amplitude of a passive fluid, and mechanical equilibrium (equal bulk
pressure of Eq. (3)) across a flat A/B interface."""
import math

import numpy as np
import pytest

from paper_0807_4471_gb300 import experiments as E
from _oracle_lb import OracleLb as _OracleLb


def test_structure_factor_parseval_and_peak():
    n = 64
    y, x = np.mgrid[0:n, 0:n]
    phi = 0.3 * np.cos(2 * np.pi * 5 * x / n) + 0.1 * np.sin(2 * np.pi * 3 * y / n) + 0.7
    k, s, c = E.structure_factor(phi)
    assert abs((s * c).sum() - ((phi - phi.mean()) ** 2).sum()) < 1e-9
    top = np.argsort(s * c)[-2:]
    assert set(top) == {3, 5}
    assert abs(k[5] - 2 * np.pi * 5 / n) < 1e-12
    assert (s * c)[5] == pytest.approx(2 * n * n * 0.3 ** 2 / 4, rel=1e-12)


def test_interface_indicator_closed_form():
    n, m = 48, 3
    q = 2 * np.pi * m / n
    x = np.arange(n)
    a = np.tile(np.cos(q * x), (n, 1))
    b = np.tile(-2 * np.cos(q * x), (n, 1))
    # central differences: d/dx cos(q x) -> -sin(q) sin(q x)
    want = -2 * n * n * math.sin(q) ** 2 / 2
    assert E.interface_indicator(a, b) == pytest.approx(want, rel=1e-12)


def test_sine_projection_and_overlap():
    ny = 40
    ux = 0.07 * np.sin(2 * np.pi * np.arange(ny) / ny)[:, None] * np.ones((1, 12)) + 0.01
    assert E.sine_projection(ux) == pytest.approx(0.07, rel=1e-12)
    phi = np.random.default_rng(1).standard_normal((16, 16))
    num, den = E.overlap(phi, phi)
    assert num == den
    num, den = E.overlap(phi, -phi)
    assert num == -den


def test_kolmogorov_steady_amplitude_oracle(O):
    """Passive two-species fluid (all G = 0) forced by a_x = nu0 k^2 U0 sin(ky):
    the steady amplitude is U0 (R = 1) up to the lattice error O(k^2)."""
    n, U0, tau = 32, 0.01, 1.0
    nu0 = (tau - 0.5) / 3
    k = 2 * np.pi / n
    P = O.make_params(4, n, Ga=(0.0, 0.0), Gr=(0.0, 0.0), GX=0.0, rho0=0.5, init_amp=0.0,
                      kolmo_amp=nu0 * k * k * U0, kolmo_k=1.0)
    f = O.init_seeded(P, 0)
    O.run(P, f, 12000)
    _, _, ux, _ = O.fields(P, f)
    R = E.sine_projection(ux) / U0
    assert abs(R - 1.0) < 0.01


def test_flat_interface_pressure_balance_oracle(O, caption):
    """A flat A/B interface relaxes to mechanical equilibrium: the bulk
    pressure of Eq. (3) is the same in the A-rich and the B-rich phase."""
    nx, ny = 4, 64
    y = np.arange(ny)[:, None].repeat(nx, 1)
    s = 0.5 * (1 + np.tanh((np.minimum(y - 16, 48 - y)) / 2.0))
    r0 = caption["rho0"]
    ra = 0.1 * r0 + 1.5 * r0 * s
    rb = 1.6 * r0 - 1.5 * r0 * s
    P = O.make_params(nx, ny, **caption, psi_form=1)
    f = O.init_fields(P, ra, rb)
    O.run(P, f, 6000)
    fa, fb, ux, uy = O.fields(P, f)
    p = E.bulk_pressure(fa, fb, caption["Ga"], caption["Gr"], caption["GX"], r0, r0)
    p_a, p_b = p[32, 0], p[0, 0]
    assert fa[32, 0] > fb[32, 0] and fb[0, 0] > fa[0, 0]      # two bulk phases
    assert abs(p_a - p_b) < 2e-3 * abs(p_a)
    # spurious currents at the interface stay small (1e-6 here)
    assert np.abs(ux).max() < 1e-5 and np.abs(uy).max() < 1e-5


def test_ageing_driver_on_oracle(O, caption):
    """C(t_w, tau) from the pooled driver equals Eq. (6) evaluated on
    separately run oracle realisations; C(t_w, 0) = 1."""
    lb = _OracleLb(O, caption)
    seeds, n = (0, 1, 2), 16
    t_ws, taus = (20, 40), (0, 10, 30)
    _, C = E.ageing_overlap(lb, n, seeds, t_ws, taus, precision="fp64", psi_form=1)
    assert C.shape == (2, 3) and np.allclose(C[:, 0], 1.0, rtol=0, atol=1e-15)
    P = lb.make_params(n, n, psi_form=1).P
    phi = {}
    for sd in seeds:
        f = O.init_seeded(P, sd)
        t = 0
        for when in sorted({w + u for w in t_ws for u in taus}):
            O.run(P, f, when - t, t0=t)
            t = when
            ra, rb, _, _ = O.fields(P, f)
            phi[sd, when] = ra - rb
    for a, w in enumerate(t_ws):
        den = sum((phi[sd, w] ** 2).sum() for sd in seeds)
        for b, u in enumerate(taus):
            num = sum((phi[sd, w] * phi[sd, w + u]).sum() for sd in seeds)
            assert abs(C[a, b] - num / den) < 1e-13
    _, c1 = E.ageing_overlap(lb, n, seeds, 40, taus, precision="fp64", psi_form=1)
    assert np.array_equal(c1, C[1])


def test_laplace_driver_on_oracle(O, caption):
    """The Laplace driver on oracle drops (psi_form = 1, rho0 = 0.55): the
    pressure jump is positive, falls as 1/R within 20 %, and the dense
    interior stays one uniform phase."""
    out = E.laplace_test(_OracleLb(O, caption), 0.55, radii=(8, 12), n=48, steps=3000,
                         avg_from=2000, every=500, precision="fp64", psi_form=1)
    (r1, r2) = out["rows"]
    assert out["uniform"] and out["sigma"] > 0
    assert r1["dp"] > r2["dp"] > 0
    assert abs(r1["dp"] * r1["R"] / (r2["dp"] * r2["R"]) - 1) < 0.2


def test_sweep_driver_on_oracle(O, caption):
    """The rho0-sweep driver on oracle lattices: one S(k) and domain length
    per lattice and sample time, S(k) summing to the variance of phi."""
    lb = _OracleLb(O, caption)
    out = E.sweep_structure_factor(lb, rho0s=(0.55, 0.83), precision="fp64", n=24, steps=60,
                                   every=30, seed=1)
    assert out["t"] == [30, 60] and set(out["rho0"]) == {0.55, 0.83}
    for rec in out["rho0"].values():
        assert len(rec["S"]) == 2 and len(rec["L"]) == 2
        assert all(np.isfinite(rec["L"])) and all(v > 0 for v in rec["L"])
    P = lb.make_params(24, 24, rho0=0.83, psi_form=1).P
    f = O.init_seeded(P, 1)
    O.run(P, f, 60)
    ra, rb, _, _ = O.fields(P, f)
    k, S, c = E.structure_factor(ra - rb)
    assert np.allclose(out["rho0"][0.83]["S"][1], S, rtol=1e-12, atol=0)
