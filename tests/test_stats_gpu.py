"""Long-run statistics of the reduced-precision storage paths against the
FP64 GPU path (itself held to the oracle element by element by the parity
tests).  Beyond ~10^2 steps the demixing dynamics is chaotic, so runs of
different precisions are compared through ensemble statistics of the order
parameter phi = rho_A - rho_B: its variance (the integral of the structure
factor S(k)) and the domain length 2 pi sum S / sum k S, over 32 seeded
realisations stepped together in one lattice pool.  The experiment drivers
themselves (Kolmogorov forcing, Couette stress) are checked against closed
forms on a passive fluid."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def lb():
    import torch
    if not torch.cuda.is_available():
        pytest.fail("a CUDA GPU is required for -m gpu tests")
    import paper_0807_4471_gb300 as lb
    from paper_0807_4471_gb300 import build
    build.build()
    lb.load()
    return lb


def _ensemble(lb, prec, seeds=range(32), n=128, steps=2000):
    from paper_0807_4471_gb300 import experiments as E
    p = lb.make_params(n, n, prec, psi_form=1)
    budget = lb.Pool.footprint(p) * len(seeds) + (64 << 20)
    L, var = [], []
    with lb.Pool(p, budget, max_jobs=len(seeds)) as pool:
        jobs = [pool.admit(p, s, steps) for s in seeds]
        pool.run(steps)
        for j in jobs:
            ra, rb, _, _ = pool.fields(j)
            phi = ra - rb
            L.append(E.domain_length(phi))
            k, s, c = E.structure_factor(phi)
            var.append(float((s * c).sum()))
    return np.array(L), np.array(var)


@pytest.fixture(scope="module")
def ensembles(lb):
    return {p: _ensemble(lb, p) for p in ("fp64", "fp32", "fp16", "bf16")}


def test_ensemble_statistics_fp32(ensembles):
    L0, v0 = ensembles["fp64"]
    L, v = ensembles["fp32"]
    assert abs(L.mean() / L0.mean() - 1) < 1e-3
    assert abs(v.mean() / v0.mean() - 1) < 1e-3


def test_ensemble_statistics_fp16_within_one_percent(ensembles):
    """FP16 offsets: ensemble domain length and phi variance within 1 % of
    FP64 after 2000 steps (measured 0.2 % and 0.06 %)."""
    L0, v0 = ensembles["fp64"]
    L, v = ensembles["fp16"]
    assert abs(L.mean() / L0.mean() - 1) < 0.01
    assert abs(v.mean() / v0.mean() - 1) < 0.01


def test_ensemble_statistics_bf16_bounded(ensembles):
    """BF16 offsets (8-bit significand) shift the statistics measurably
    (domain length +3.7 % after 2000 steps); they stay bounded here, and the
    1 % target is not claimed for BF16."""
    L0, v0 = ensembles["fp64"]
    L, v = ensembles["bf16"]
    assert np.isfinite(L).all() and np.isfinite(v).all()
    assert abs(L.mean() / L0.mean() - 1) < 0.1
    assert abs(v.mean() / v0.mean() - 1) < 0.05


def test_kolmogorov_passive_response(lb):
    """The Kolmogorov body force a_x = nu0 k^2 U0 sin(k y) on a passive fluid
    (all couplings zero) sustains u_x = U0 sin(k y): R -> 1 up to the
    lattice error O(k^2)."""
    from paper_0807_4471_gb300 import experiments as E
    rows = E.kolmogorov_run(lb, n=64, U0=0.01, steps=8000, every=4000, G_A1=0.0, G_A2=0.0,
                            G_B1=0.0, G_B2=0.0, G_X=0.0, init_amp=0.0)
    assert abs(rows[-1][1] - 1.0) < 0.01
    assert abs(rows[-1][2]) < 1e-12        # no interfaces: I_AB = 0


@pytest.mark.parametrize("prec", ["fp64", "fp32", "fp16"])
def test_couette_passive_wall_stress(lb, prec):
    """Passive fluid between walls at -U and +U (shear rate 2U/ny), started
    on the steady linear profile: the time-averaged wall stress is
    rho nu0 gamma with nu0 = c_s^2 (tau - 1/2) (both species, rho = 2 rho0).
    FP16 runs with the default stochastic rounding."""
    from paper_0807_4471_gb300 import experiments as E
    rate = 1e-4
    out = E.couette_study(lb, [rate], precisions=(prec,), n=128, steps=2000, avg_from=1000,
                          psi_form=1, G_A1=0.0, G_A2=0.0, G_B1=0.0, G_B2=0.0, G_X=0.0,
                          init_amp=0.0)[prec][0]
    want = 2 * 0.70 * (1.0 / 6.0) * rate
    # storage rounding biases the steady state: FP32 by 4e-4 here; FP16 with
    # stochastic rounding stays inside the 1 % target (nearest: 3 %)
    tol = 1e-9 if prec == "fp64" else (2e-3 if prec == "fp32" else 0.01)
    assert abs(out["sigma"] / want - 1) < tol
    assert out["samples"] == 1000
