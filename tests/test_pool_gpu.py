"""Lattice pool (lb_pool_*): members stepped together by one persistent
launch per step give bitwise the same result as each lattice stepped alone
(the per-site arithmetic does not depend on the work partition), admission
is by arena footprint, and members stop at their own step counts."""
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


MEMBERS = [dict(nx=64, ny=40), dict(nx=128, ny=128, rho0=0.55), dict(nx=200, ny=72, rho0=0.83),
           dict(nx=96, ny=64, boundary=1, u_wall=0.02, init_shear=1),
           dict(nx=256, ny=48, boundary=1, u_wall=0.01, rho0=0.65), dict(nx=60, ny=8)]


def _single(lb, m, prec, seed, steps):
    g = lb.Lattice(gpu_params(lb, m, prec)).init_seeded(seed)
    g.step(steps)
    f = g.fields()
    st = g.stress()
    g.close()
    return f, st


@pytest.mark.parametrize("prec", ["fp32", "fp16", "fp64"])
def test_pool_members_match_single_lattices(lb, prec):
    shared = gpu_params(lb, model(64, 64), prec)
    with lb.Pool(shared, budget=1 << 30, max_jobs=16) as pool:
        jobs = []
        for k, kw in enumerate(MEMBERS):
            steps = 30 if k == 2 else 60     # one member finishes early
            m = model(**kw)
            jobs.append((pool.admit(gpu_params(lb, m, prec), 100 + k, steps), m, steps, 100 + k))
        left = pool.run(25)
        assert left == len(MEMBERS)
        left = pool.run(25)
        assert left == len(MEMBERS) - 1       # the 30-step member is done
        assert pool.poll(jobs[2][0]) == (30, True)
        assert pool.run(25) == 0
        assert pool.segment != 0              # a partition was built (-1: contiguous runs)
        for j, m, steps, seed in jobs:
            assert pool.poll(j) == (steps, True)
            got = pool.fields(j)
            want, st_single = _single(lb, m, prec, seed, steps)
            for a, b in zip(got, want):
                assert np.array_equal(a, b)
            st = pool.stress(j)
            for key in ("mass_A", "mass_B", "sigma_bot", "sigma_top", "samples", "step"):
                assert st[key] == st_single[key], key


def test_pool_admission_by_footprint(lb):
    shared = gpu_params(lb, model(64, 64), "fp32")
    p = gpu_params(lb, model(256, 256), "fp32")
    fp = lb.Pool.footprint(p)
    with lb.Pool(shared, budget=2 * fp + fp // 2, max_jobs=8) as pool:
        a = pool.admit(p, 1, 10)
        b = pool.admit(p, 2, 10)
        with pytest.raises(lb.LbError) as e:
            pool.admit(p, 3, 10)
        assert e.value.status == lb.LB_ERR_NOMEM
        small = gpu_params(lb, model(64, 64), "fp32")
        c = pool.admit(small, 4, 10)           # fits in the remaining space
        pool.release(a)
        d = pool.admit(p, 5, 10)               # the freed space is reused
        assert pool.run(10) == 0
        for j in (b, c, d):
            assert pool.poll(j) == (10, True)
        bad = gpu_params(lb, model(64, 64, GX=0.3), "fp32")
        with pytest.raises(lb.LbError) as e:
            pool.admit(bad, 6, 10)             # couplings differ from the pool's
        assert e.value.status == lb.LB_ERR_INVALID


def test_pool_init_fields_matches_handle(lb):
    """lb_pool_init_fields restarts a member from host fields: the member then
    steps bitwise like a handle initialised with lb_init_fields."""
    m = model(120, 48, boundary=1, u_wall=0.01)
    p = gpu_params(lb, m, "fp32")
    rng = np.random.default_rng(21)
    ra = np.ascontiguousarray(0.7 * (1 + 0.03 * (2 * rng.random((48, 120)) - 1)))
    rb = np.ascontiguousarray(0.7 * (1 + 0.03 * (2 * rng.random((48, 120)) - 1)))
    g = lb.Lattice(p).init_fields(ra, rb)
    g.step(17)
    want = g.fields()
    g.close()
    with lb.Pool(p, 4 * lb.Pool.footprint(p), max_jobs=2) as pool:
        j = pool.admit(p, 5, 17)
        other = pool.admit(p, 6, 40)
        pool.run(3)                     # the member's seeded start is discarded
        pool.init_fields(j, ra, rb)
        assert pool.poll(j) == (0, False)
        pool.run(17)
        assert pool.poll(j) == (17, True)
        got = pool.fields(j)
        for a, b in zip(got, want):
            assert np.array_equal(a, b)
        assert pool.poll(other)[0] == 20


@pytest.mark.parametrize("prec", ["fp32", "fp16"])
def test_pool_tuned_partitions_match_single_lattices(lb, prec):
    """A run long enough for the autotuner to time every candidate partition
    (dealt segments, contiguous runs) on the real steps, then a forced
    contiguous partition, still gives bitwise the single-lattice result: the
    per-site arithmetic and the wall-sum order do not depend on the
    partition."""
    members = [dict(nx=200, ny=136), dict(nx=96, ny=64, boundary=1, u_wall=0.02, init_shear=1),
               dict(nx=128, ny=128, rho0=0.55)]
    steps = 400                         # the member set runs long enough to be tuned
    shared = gpu_params(lb, model(64, 64), prec)
    ps = [gpu_params(lb, model(**m), prec) for m in members]
    budget = sum(lb.Pool.footprint(p) for p in ps) + (1 << 20)
    with lb.Pool(shared, budget, max_jobs=len(members)) as pool:
        jobs = [pool.admit(p, 11 + k, steps) for k, p in enumerate(ps)]
        assert pool.run(steps - 20) == len(members)
        assert pool.segment != 0
        pool.set_partition(-1)
        assert pool.run(20) == 0
        assert pool.segment == -1
        for k, (j, m) in enumerate(zip(jobs, members)):
            want, st_single = _single(lb, model(**m), prec, 11 + k, steps)
            for a, b in zip(pool.fields(j), want):
                assert np.array_equal(a, b)
            st = pool.stress(j)
            for key in ("sigma_bot", "sigma_top", "samples", "step"):
                assert st[key] == st_single[key], key
