"""Work partition of the step launch (host logic, no GPU): every tile of
every lattice is updated exactly once per launch, work items are well
formed, the dealt segments are balanced by the cost model and the
contiguous runs follow the tile order.  The plan comes from the library's
own host code through lb_plan_partition."""
import numpy as np
import pytest

TX = {"fp64": 28, "fp32": 60, "fp16": 60, "bf16": 60}
TY = 8


@pytest.fixture(scope="module")
def lb():
    import paper_0807_4471_gb300 as lb
    from paper_0807_4471_gb300 import build
    build.build()
    lb.load()
    return lb


def lattices(lb, dims, prec="fp32"):
    return [lb.make_params(nx, ny, prec, psi_form=1, boundary=b, u_wall=0.01 if b else 0.0)
            for nx, ny, b in dims]


ITEM = 0.8   # an item's start, in tiles


def tile_cost(nx, ny, periodic, tx, sx, ty, rows=TY, staged=True):
    """The cost model the library documents: an interior tile 1; a ragged
    tile 1.07; a Couette tile holding a wall row 1.38; +0.21 for writing
    periodic ghost columns and +0.25 for ghost rows (+0.02 where the kernel
    stores them directly, FP32 with 16-row tiles)."""
    x0, y0 = sx * tx, ty * rows
    if not (x0 + tx <= nx and y0 + rows <= ny):
        return 1.07
    if not periodic and (y0 == 0 or y0 + rows >= ny):
        return 1.38
    c = 1.0
    if x0 < 3 or x0 + tx > nx - 3:
        c += 0.21
    if periodic and (y0 < 3 or y0 + rows > ny - 3):
        c += 0.25 if staged else 0.02
    return c


def check_cover(items, cta, dims, tx, sms, ty_rows=TY):
    G = len(cta) - 1
    assert 1 <= G <= sms
    assert cta[0] == 0 and cta[-1] == len(items) and np.all(np.diff(cta) >= 1)
    seen = {}
    for l, sx, a, b in items:
        nx, ny, _ = dims[l]
        nt = -(-ny // ty_rows)
        assert 0 <= sx < -(-nx // tx) and 0 <= a < b <= nt
        for ty in range(a, b):
            key = (l, sx, ty)
            assert key not in seen, key
            seen[key] = True
    want = sum(-(-nx // tx) * -(-ny // ty_rows) for nx, ny, _ in dims)
    assert len(seen) == want


CASES = [
    [(512, 512, 0)] * 5,                                   # the rho0 sweep
    [(4096, 4096, 0)],
    [(128, 128, 0), (256, 256, 1), (512, 512, 0), (1024, 1024, 1), (200, 72, 0), (60, 8, 1)],
    [(1020, 136, 1), (96, 64, 0), (8, 8, 0)],
]


@pytest.mark.parametrize("dims", CASES)
@pytest.mark.parametrize("seg", [0, -1, 1, 5, 47])
@pytest.mark.parametrize("sms", [152, 7])
def test_every_tile_once(lb, dims, seg, sms):
    items, cta, used = lb.lb_plan_partition(lattices(lb, dims), seg, sms)
    check_cover(items, cta, dims, TX["fp32"], sms)
    if seg != 0:
        assert used == seg


@pytest.mark.parametrize("prec", ["fp64", "fp16"])
def test_tile_width_follows_precision(lb, prec):
    dims = [(200, 72, 0), (96, 64, 1)]
    items, cta, _ = lb.lb_plan_partition(lattices(lb, dims, prec), -1, 152)
    check_cover(items, cta, dims, TX[prec], 152)


@pytest.mark.parametrize("dims", CASES)
@pytest.mark.parametrize("seg", [1, 5, 47])
def test_segments_balanced_by_cost(lb, dims, seg):
    """Each item is one segment [a, min(a + seg, nt)); every segment is
    placed once, the CTAs' estimated work differs by at most one item's
    (the bound of giving each item to the least loaded CTA), and each CTA
    takes its items in band order."""
    items, cta, _ = lb.lb_plan_partition(lattices(lb, dims), seg, 152)
    tx = TX["fp32"]
    for l, sx, a, b in items:
        nt = -(-dims[l][1] // TY)
        assert a % seg == 0 and b == min(a + seg, nt)

    def cost(it):
        l, sx, a, b = it
        nx, ny, bnd = dims[l]
        return ITEM + sum(tile_cost(nx, ny, bnd == 0, tx, sx, ty) for ty in range(a, b))

    loads = [sum(cost(items[k]) for k in range(cta[c], cta[c + 1])) for c in range(len(cta) - 1)]
    wmax = max(cost(it) for it in items)
    assert max(loads) - min(loads) <= wmax + 1e-9
    band = {tuple(it): k for k, it in enumerate(
        (l, sx, a, min(a + seg, -(-dims[l][1] // TY)))
        for l in range(len(dims)) for a in range(0, -(-dims[l][1] // TY), seg)
        for sx in range(-(-dims[l][0] // tx)))}
    assert len(band) == len(items)
    for c in range(len(cta) - 1):
        order = [band[tuple(items[k])] for k in range(cta[c], cta[c + 1])]
        assert order == sorted(order)


@pytest.mark.parametrize("dims", CASES)
@pytest.mark.parametrize("rows,sms", [(8, 152), (16, 152), (16, 7)])
def test_contiguous_runs(lb, dims, rows, sms):
    """seg = -1: the CTAs' items, concatenated, walk the tiles in order
    (lattice, strip, tile row), each CTA's run one stretch of it, an item
    per strip it touches; and the largest run cost is the least any split
    into at most sms contiguous runs achieves: packing the runs greedily
    under any smaller bound takes more than sms runs."""
    items, cta, _ = lb.lb_plan_partition(lattices(lb, dims), -1, sms, tile_rows=rows)
    tx = TX["fp32"]
    staged = rows == 8          # FP32 with 16-row tiles stores directly
    order = [(l, sx, ty) for l, (nx, ny, _) in enumerate(dims)
             for sx in range(-(-nx // tx)) for ty in range(-(-ny // rows))]
    walk = [(l, sx, ty) for l, sx, a, b in items for ty in range(a, b)]
    assert walk == order
    G = len(cta) - 1
    assert 1 <= G <= sms
    loads = []
    for c in range(G):
        w = 0.0
        for l, sx, a, b in items[cta[c]:cta[c + 1]]:
            nx, ny, bnd = dims[l]
            w += ITEM + sum(tile_cost(nx, ny, bnd == 0, tx, sx, ty, rows, staged) for ty in range(a, b))
        loads.append(w)
    # tile costs in order, with an item start where a strip begins
    seq = [(tile_cost(dims[l][0], dims[l][1], dims[l][2] == 0, tx, sx, ty, rows, staged), ty == 0)
           for l, sx, ty in order]

    def greedy_runs(bound):
        n, acc = 0, 0.0
        for c, first in seq:
            add = c + (ITEM if first else 0.0)
            if n and acc + add <= bound:
                acc += add
            else:
                n, acc = n + 1, c + ITEM
        return n

    B = max(loads)
    assert greedy_runs(B * (1 + 1e-9)) <= sms
    if B > max(c for c, _ in seq) + ITEM + 1e-9:   # not a single tile's bound
        assert greedy_runs(B * (1 - 1e-5)) > sms
    mean = sum(loads) / G
    assert B <= mean + max(c for c, _ in seq) + ITEM + 1e-9


def test_default_rule(lb):
    """Cost-balanced contiguous runs while each CTA has up to 40 tiles, the
    model's dealt segments beyond."""
    _, _, used = lb.lb_plan_partition(lattices(lb, [(512, 512, 0)] * 5), 0, 152)
    assert used == -1
    _, _, used = lb.lb_plan_partition(lattices(lb, [(4096, 4096, 0)]), 0, 152)
    assert used > 0


def test_invalid_plans(lb):
    from paper_0807_4471_gb300 import LbError
    mixed = lattices(lb, [(64, 64, 0)], "fp32") + lattices(lb, [(64, 64, 0)], "fp16")
    with pytest.raises(LbError):
        lb.lb_plan_partition(mixed, 0, 152)
    with pytest.raises(LbError):
        lb.lb_plan_partition(lattices(lb, [(64, 64, 0)]), 0, 0)


@pytest.mark.parametrize("dims", CASES)
@pytest.mark.parametrize("seg", [0, -1, 1, 3])
def test_every_tile_once_16_row_tiles(lb, dims, seg):
    """The two-sites-per-thread kernel's 16-row tiles: every tile once."""
    items, cta, _ = lb.lb_plan_partition(lattices(lb, dims), seg, 152, tile_rows=16)
    check_cover(items, cta, dims, TX["fp32"], 152, ty_rows=16)


def test_tile_rows_validation(lb):
    with pytest.raises(lb.LbError):
        lb.lb_plan_partition(lattices(lb, [(64, 64, 0)]), 0, 152, tile_rows=12)
    with pytest.raises(lb.LbError):        # FP64 has only the 8-row tile
        lb.lb_plan_partition(lattices(lb, [(64, 64, 0)], "fp64"), 0, 152, tile_rows=16)
    p = lb.make_params(64, 64, "fp64", tile_rows=16)
    with pytest.raises(lb.LbError):
        lb.lb_workspace_size(p)
    for rows in (0, 8, 16):
        assert lb.lb_workspace_size(lb.make_params(64, 64, "fp32", tile_rows=rows)) > 0
