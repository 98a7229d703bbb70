"""Failure detection without faulting the GPU: the step kernel's bounded
waits give up with a status the host reads (a barrier that nothing
completes), the context stays usable afterwards, and a pool member
cancelled in the middle of a run leaves the others' results untouched."""
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


def test_bounded_wait_times_out_and_context_survives(lb):
    assert lb.lb_selftest_wait(1024) == lb.LB_ERR_TIMEOUT
    assert lb.lb_selftest_wait(4) == lb.LB_ERR_TIMEOUT
    assert lb.lb_selftest_wait(0) == lb.LB_ERR_INVALID
    # the same process keeps stepping lattices normally
    g = lb.Lattice(gpu_params(lb, model(64, 40), "fp32")).init_seeded(1)
    g.step(10)
    ra, rb, _, _ = g.fields()
    assert np.isfinite(ra).all() and np.isfinite(rb).all()
    g.close()


def test_pool_member_cancelled_mid_run(lb):
    """Releasing a running member frees its memory for the next admission;
    the member stepped alongside it is bitwise what it is alone."""
    m = model(96, 64)
    p = gpu_params(lb, m, "fp32")
    fp = lb.Pool.footprint(p)
    with lb.Pool(p, 2 * fp, max_jobs=4) as pool:
        keep = pool.admit(p, 3, 40)
        drop = pool.admit(p, 4, 1000)
        with pytest.raises(lb.LbError):
            pool.admit(p, 5, 10)          # arena full
        pool.run(15)
        pool.release(drop)                # cancelled mid-run
        late = pool.admit(p, 5, 25)       # its memory is reused
        pool.run(25)
        assert pool.poll(keep) == (40, True) and pool.poll(late) == (25, True)
        got = pool.fields(keep)
    g = lb.Lattice(p).init_seeded(3)
    g.step(40)
    for a, b in zip(got, g.fields()):
        assert np.array_equal(a, b)
    g.close()
