"""The step kernel's two tile shapes -- 8-row tiles with one site per thread
(leaving through a staging tile and a TMA bulk store) and 16-row tiles with
two vertically adjacent sites per thread that share their stencil rows
(stored to global memory directly) -- compute every site with the same
operations in the same order, so they give bitwise the same populations
and wall-stress sums: for single lattices (lb_params.tile_rows) and for
pool members (lb_pool_set_tile_rows, and the autotuner's choice), on
ragged sizes, periodic and Couette, with and without body forces."""
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


STRESS_KEYS = ("mass_A", "mass_B", "mom_x", "mom_y", "sigma_bot", "sigma_top", "samples", "step")


def run_single(lb, m, prec, rows, seed, steps, fields=False):
    p = gpu_params(lb, m, prec)
    p.tile_rows = rows
    g = lb.Lattice(p).init_seeded(seed)
    g.step(steps)
    out = (g.fields() if fields else g.populations()), g.stress()
    g.close()
    return out


DIMS = [(72, 40, 0), (100, 27, 1), (8, 8, 0), (60, 16, 1), (130, 9, 0), (1020, 136, 1),
        (512, 512, 0), (33, 17, 1), (131, 21, 0)]


@pytest.mark.parametrize("prec", ["fp32", "fp16", "bf16"])
@pytest.mark.parametrize("dims", DIMS)
def test_single_lattice_tile_shapes_bitwise(lb, prec, dims):
    nx, ny, b = dims
    m = model(nx, ny, boundary=b, u_wall=0.02 if b else 0.0, init_shear=b)
    f8, s8 = run_single(lb, m, prec, 8, 12, 37)
    f16, s16 = run_single(lb, m, prec, 16, 12, 37)
    assert np.array_equal(f8, f16)
    for key in STRESS_KEYS:
        assert s8[key] == s16[key], key


@pytest.mark.parametrize("variant", ["accel", "source", "tau", "tau_fp16_couette"])
def test_tile_shapes_bitwise_with_forcing(lb, variant):
    if variant == "accel":
        m = model(96, 40, boundary=1, u_wall=0.01, g_x=1e-4, kolmo_amp=2e-4, kolmo_k=1.0)
    elif variant == "source":
        c = model(96, 40)
        m = model(96, 40, force_scheme=1, Ga=tuple(0.5 * v for v in c["Ga"]),
                  Gr=tuple(0.5 * v for v in c["Gr"]))
    elif variant == "tau":
        m = model(96, 40, tau=(1.0, 0.8))
    else:
        m = model(130, 40, boundary=1, u_wall=0.01, init_shear=1, tau=(0.9, 0.8))
    prec = "fp16" if variant == "tau_fp16_couette" else "fp32"
    f8, s8 = run_single(lb, m, prec, 8, 3, 41)
    f16, s16 = run_single(lb, m, prec, 16, 3, 41)
    assert np.array_equal(f8, f16)
    for key in STRESS_KEYS:
        assert s8[key] == s16[key], key


MEMBERS = [dict(nx=64, ny=40), dict(nx=128, ny=128, rho0=0.55), dict(nx=200, ny=72, rho0=0.83),
           dict(nx=96, ny=64, boundary=1, u_wall=0.02, init_shear=1),
           dict(nx=256, ny=48, boundary=1, u_wall=0.01, rho0=0.65), dict(nx=60, ny=8)]


@pytest.mark.parametrize("prec", ["fp32", "fp16"])
@pytest.mark.parametrize("rows,steps", [(8, 40), (16, 40), (0, 1200)])
def test_pool_tile_shapes_match_single_lattices(lb, prec, rows, steps):
    """Members of a pool run with 8-row tiles, 16-row tiles, or the
    autotuner's choice over shapes and partitions (1200 steps: enough for the
    tuner to run) equal the lattices run alone with the 8-row tile."""
    shared = gpu_params(lb, model(64, 64), prec)
    with lb.Pool(shared, budget=1 << 30, max_jobs=16) as pool:
        if rows:
            pool.set_tile_rows(rows)
        jobs = []
        for k, kw in enumerate(MEMBERS):
            m = model(**kw)
            jobs.append((pool.admit(gpu_params(lb, m, prec), 200 + k, steps), m, 200 + k))
        assert pool.run(steps) == 0
        assert pool.tile_rows in (8, 16) and (rows == 0 or pool.tile_rows == rows)
        for j, m, seed in jobs:
            want, st_single = run_single(lb, m, prec, 8, seed, steps, fields=True)
            got = pool.fields(j)
            for a, b in zip(got, want):
                assert np.array_equal(a, b)
            st = pool.stress(j)
            for key in ("mass_A", "mass_B", "sigma_bot", "sigma_top", "samples", "step"):
                assert st[key] == st_single[key], key


def test_pool_tile_rows_validation(lb):
    with lb.Pool(gpu_params(lb, model(64, 64), "fp64"), budget=1 << 26, max_jobs=2) as pool:
        with pytest.raises(lb.LbError):
            pool.set_tile_rows(16)          # FP64 has only the 8-row tile
        pool.set_tile_rows(8)
    with lb.Pool(gpu_params(lb, model(64, 64), "fp32"), budget=1 << 26, max_jobs=2) as pool:
        with pytest.raises(lb.LbError):
            pool.set_tile_rows(24)
        assert pool.tile_rows == 0          # nothing built yet
