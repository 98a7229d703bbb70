"""The server on the GPU: a job's result is the same alone and in a mix of
other jobs arriving while it runs (bitwise: the per-site arithmetic does not
depend on which lattices share a launch), and jobs queue until memory frees."""
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


def _server(lb, budget, keep_fields=True):
    from paper_0807_4471_gb300.serve import Server, job_params
    shared = dict(psi_form=lb.LB_PSI_RHO0)
    make = job_params(lb, shared, "fp16")
    pool = lb.Pool(make(dict(nx=64, ny=64, steps=1)), budget, max_jobs=64)
    return Server(pool, make, quantum=20, keep_fields=keep_fields), pool


TARGET = dict(nx=128, ny=96, rho0=0.7, shear_rate=2e-4, steps=90, seed=11)


def test_result_same_alone_and_in_mix(lb):
    srv, pool = _server(lb, 1 << 28)
    alone = srv.submit(TARGET)
    srv.run_until_idle()
    pool.close()
    srv, pool = _server(lb, 1 << 28)
    early = srv.submit(dict(nx=256, ny=256, rho0=0.6, shear_rate=0.0, steps=70, seed=1))
    srv.step()
    mixed = srv.submit(TARGET)           # arrives while another job runs
    srv.step()
    late = [srv.submit(dict(nx=64 + 32 * k, ny=64, rho0=0.75, shear_rate=1e-4 * (k % 2),
                            steps=30 + 10 * k, seed=20 + k)) for k in range(4)]
    srv.run_until_idle()
    pool.close()
    assert all(j.done and j.error is None for j in [early, mixed] + late)
    for a, b in zip(alone.result["fields"], mixed.result["fields"]):
        assert np.array_equal(a, b)
    for key in ("sigma_bot", "sigma_top", "samples", "mass_A", "mass_B", "step"):
        assert alone.result[key] == mixed.result[key]
    assert mixed.result["step"] == 90 and mixed.result["samples"] == 90


def test_queueing_under_a_small_arena(lb):
    import paper_0807_4471_gb300 as L
    from paper_0807_4471_gb300.serve import job_params
    make = job_params(lb, dict(psi_form=lb.LB_PSI_RHO0), "fp16")
    one = L.Pool.footprint(make(dict(nx=256, ny=256)))
    srv, pool = _server(lb, int(2.5 * one), keep_fields=False)
    jobs = [srv.submit(dict(nx=256, ny=256, rho0=0.7, shear_rate=0.0, steps=40, seed=k))
            for k in range(6)]
    srv.step()
    assert sum(1 for j in jobs if j.admitted is not None) == 2
    srv.run_until_idle()
    pool.close()
    assert all(j.done and j.error is None for j in jobs)
    assert srv.stats.refused_nomem > 0
