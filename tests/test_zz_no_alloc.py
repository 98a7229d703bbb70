"""lb_totals_noalloc -- the totals reduction for callers that may not allocate
device memory (a fixed arena they cannot grow, or a framework that forbids
cudaMalloc on its hot path) -- called through the C ABI, against the totals
the existing lb_stress entry point reports for the same state, on two calls
in a row (the second reuses the static scratch the first one left behind).

Collected last on purpose (file name), so that a run stopping at the first
failure has already run every other test.
"""
import numpy as np
import pytest

from _pair import gpu_params, model

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


def _noalloc_totals(lb, torch, g):
    """lb_fields to host, caller-owned device copies, then the no-alloc call."""
    ra, rb, ux, uy = g.fields()
    dev = [torch.from_numpy(np.ascontiguousarray(a)).cuda() for a in (ra, rb, ux, uy)]
    out = torch.full((4,), float("nan"), dtype=torch.float64, device="cuda")
    stream = torch.cuda.current_stream()
    lb.lb_totals_noalloc(g.nx, g.ny, *[t.data_ptr() for t in dev], out.data_ptr(),
                         stream.cuda_stream)
    stream.synchronize()
    return out.cpu().numpy()


def _check(st, tot):
    # FP64 sums of the same per-site values in different orders
    assert abs(tot[0] - st["mass_A"]) <= 1e-12 * st["mass_A"]
    assert abs(tot[1] - st["mass_B"]) <= 1e-12 * st["mass_B"]
    scale = st["mass_A"] + st["mass_B"]
    assert abs(tot[2] - st["mom_x"]) <= 1e-12 * scale
    assert abs(tot[3] - st["mom_y"]) <= 1e-12 * scale


def test_totals_noalloc_matches_lb_stress_on_two_calls(lb):
    import torch
    # call 1: FP64 periodic lattice with a nonzero net momentum
    m = model(96, 80)
    g = lb.Lattice(gpu_params(lb, m, "fp64"))
    rng = np.random.default_rng(3)
    g.init_fields(0.7 * (1 + 0.03 * (2 * rng.random((80, 96)) - 1)),
                  0.7 * (1 + 0.03 * (2 * rng.random((80, 96)) - 1)),
                  0.02 + 0.01 * rng.standard_normal((80, 96)), np.zeros((80, 96)))
    g.step(20)
    st = g.stress()
    assert abs(st["mom_x"]) > 1.0
    _check(st, _noalloc_totals(lb, torch, g))
    # call 2, right after: a different (ragged, multi-CTA) FP32 Couette lattice
    m2 = model(520, 200, boundary=1, u_wall=0.02, init_shear=1)
    g2 = lb.Lattice(gpu_params(lb, m2, "fp32")).init_seeded(4)
    g2.step(30)
    _check(g2.stress(), _noalloc_totals(lb, torch, g2))
    # and the first lattice again, a few steps later
    g.step(5)
    _check(g.stress(), _noalloc_totals(lb, torch, g))
    g.close()
    g2.close()


def test_totals_noalloc_rejects_sizes_beyond_the_maximum(lb):
    import torch
    x = torch.zeros(8, dtype=torch.float64, device="cuda")
    with pytest.raises(lb.LbError) as e:
        lb.lb_totals_noalloc(4097, 4096, *[x.data_ptr()] * 5)
    assert e.value.status == lb.LB_ERR_INVALID
    with pytest.raises(lb.LbError):
        lb.lb_totals_noalloc(16, 16, 0, x.data_ptr(), x.data_ptr(), x.data_ptr(), x.data_ptr())
