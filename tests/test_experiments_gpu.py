"""The experiment drivers of the paper's Fig. 4 (the overlap C(t_w, tau) of
Eq. (6)) and Fig. 2, left (the Laplace test), run on the GPU library with
FP64 storage, against the same drivers run on the FP64 CPU oracle with the
same seeds and initial fields.  Both runs stay far below the length at which
the demixing dynamics amplifies rounding differences, so the drivers'
outputs agree to 1e-10."""
import numpy as np
import pytest

from _oracle_lb import OracleLb

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


def test_ageing_overlap_gpu_equals_oracle(lb, O, caption):
    """C(t_w, tau), Eq. (6), over three seeded 16^2 realisations stepped in
    one lattice pool on the GPU, against the driver on oracle realisations."""
    from paper_0807_4471_gb300 import experiments as E
    seeds, n = (0, 1, 2), 16
    t_ws, taus = (20, 40), (0, 10, 30)
    _, C_gpu = E.ageing_overlap(lb, n, seeds, t_ws, taus, precision="fp64", psi_form=1)
    _, C_or = E.ageing_overlap(OracleLb(O, caption), n, seeds, t_ws, taus, precision="fp64",
                               psi_form=1)
    print("C(t_w, tau) gpu", C_gpu.tolist(), "max |diff|", float(np.abs(C_gpu - C_or).max()))
    assert C_gpu.shape == C_or.shape == (2, 3)
    assert np.allclose(C_gpu[:, 0], 1.0, rtol=0, atol=1e-15)
    assert float(np.abs(C_gpu - C_or).max()) < 1e-10


def test_laplace_test_gpu_equals_oracle(lb, O, caption):
    """Pressure jumps of two drops (R = 8, 12) on 48^2 lattices, rho0 = 0.55,
    Psi prefactor rho0: per radius the measured radius and Delta p agree
    with the oracle's within 1e-10 relative, and so does sigma."""
    from paper_0807_4471_gb300 import experiments as E
    kw = dict(radii=(8, 12), n=48, steps=3000, avg_from=2000, every=500, precision="fp64",
              psi_form=1)
    g = E.laplace_test(lb, 0.55, **kw)
    o = E.laplace_test(OracleLb(O, caption), 0.55, **kw)
    print("laplace gpu", g, "oracle", o)
    assert g["uniform"] and o["uniform"]
    for rg, ro in zip(g["rows"], o["rows"]):
        assert abs(rg["R"] - ro["R"]) <= 1e-10 * abs(ro["R"])
        assert abs(rg["dp"] - ro["dp"]) <= 1e-10 * abs(ro["dp"])
    assert abs(g["sigma"] - o["sigma"]) <= 1e-10 * abs(o["sigma"])
