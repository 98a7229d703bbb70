"""The step kernel's FP32 exp(x) - 1 (Cody-Waite reduction plus a degree-7
Taylor series) and reciprocal (rcp.approx.ftz), measured through
lb_selftest_math over the arguments the kernel gives them, against FP64
references rounded nowhere (errors in units of the FP32 spacing at the exact
value) and next to the CUDA library's expm1f.

Arguments: the pseudo-potential evaluates expm1(-(rho - rho_ref)/rho0) with
rho_ref = rho0, for densities rho in [0, 3] and rho0 in [0.55, 0.83], plus
the small arguments of nearly uniform regions; the reciprocal takes the
relaxation-weighted density sum and the species densities, in [1e-3, 10]."""
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


def ulp32(v):
    """Spacing of FP32 numbers at |v| (normal range)."""
    e = np.floor(np.log2(np.maximum(np.abs(v), 2.0 ** -126)))
    return np.power(2.0, e - 23)


def probe(lb, x32):
    import torch
    x = torch.from_numpy(x32).cuda()
    out = torch.empty(3 * x.numel(), dtype=torch.float32, device="cuda")
    lb.lb_selftest_math(x.data_ptr(), out.data_ptr(), x.numel(),
                        torch.cuda.current_stream().cuda_stream)
    torch.cuda.synchronize()
    o = out.cpu().numpy().astype(np.float64).reshape(-1, 3)
    return o[:, 0], o[:, 1], o[:, 2]


def kernel_expm1_arguments():
    rho = np.linspace(0.0, 3.0, 1501)
    rho0 = np.linspace(0.55, 0.83, 281)
    x = -(rho[None, :] - rho0[:, None]) / rho0[:, None]
    small = np.logspace(-12, -1, 2000)
    x = np.concatenate([x.ravel(), small, -small])
    return x.astype(np.float32)


def test_expm1_error_bound(lb):
    x32 = kernel_expm1_arguments()
    ours, lib, _ = probe(lb, x32)
    exact = np.expm1(x32.astype(np.float64))
    nz = exact != 0.0
    err = np.abs(ours[nz] - exact[nz]) / ulp32(exact[nz])
    err_lib = np.abs(lib[nz] - exact[nz]) / ulp32(exact[nz])
    print(f"pexpm1: max {err.max():.2f} ulp, mean {err.mean():.3f} ulp over {x32.size} "
          f"arguments; expm1f: max {err_lib.max():.2f} ulp, mean {err_lib.mean():.3f} ulp")
    assert np.all(np.isfinite(ours))
    assert ours[~nz].max() == 0.0 and ours[~nz].min() == 0.0
    assert err.max() <= 3.0
    # never more than 2.5 ulp worse than the library function
    assert err.max() <= err_lib.max() + 2.5


def test_expm1_special_values(lb):
    x32 = np.array([0.0, -0.0, np.nan, -20.0, 20.0, -87.0, 88.0], dtype=np.float32)
    ours, _, _ = probe(lb, x32)
    assert ours[0] == 0.0 and ours[1] == 0.0
    assert np.isnan(ours[2])
    exact = np.expm1(x32[3:].astype(np.float64))
    assert np.all(np.abs(ours[3:] - exact) <= 4 * ulp32(exact))


def test_reciprocal_error_bound(lb):
    x32 = np.concatenate([np.logspace(-3, 1, 400001), np.linspace(0.5, 4.0, 100001)]
                         ).astype(np.float32)
    _, _, r = probe(lb, x32)
    exact = 1.0 / x32.astype(np.float64)
    err = np.abs(r - exact) / ulp32(exact)
    print(f"recip: max {err.max():.3f} ulp, mean {err.mean():.3f} ulp")
    assert err.max() <= 1.0
