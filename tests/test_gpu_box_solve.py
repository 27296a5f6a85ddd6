"""GPU vs oracle: the transform exact solve on single boxes (Algorithm 1,
exact_solve) and the restricted additive Schwarz preconditioner (Sec. II-B),
float64, relative error <= 1e-11."""
import numpy as np
import pytest

from oracle import box, ras, yee
from paper_2508_07193_b300 import workloads as wl
from tests._gpu import FP64_TOL, box_rel2, context, dev, host, rel

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("grid", [(32, 32, 32), (8, 8, 8), (2, 2, 2), (5, 7, 3), (36, 34, 33), (80, 9, 12)])
def test_box_solve_matches_oracle(grid):
    rng = np.random.default_rng(sum(grid))
    eps = rng.uniform(1, 10)
    nx, ny, nz = grid
    w = wl.make_workload("box", grid, seed=sum(grid), uniform_eps=True, overlap=0)
    from paper_2508_07193_b300 import flashmp as F
    ctx = F.Context(grid, np.full((nz, ny, nx), eps), 0.25)
    x = host(ctx.box_solve(0, dev(w.rhs)))
    ref = box.exact_solve(w.rhs, eps, 0.25)
    assert rel(x, ref) <= FP64_TOL
    assert np.all(x[ras.box_wall(grid)] == 0.0)


@pytest.mark.parametrize("axis", [0, 1, 2])
def test_box_solve_every_extent_2_to_40(axis):
    """Single boxes whose extent along one axis runs through 2 .. 40, the other
    two 6 and 5: every folding shape of the float64 transforms (odd extents,
    even ones whose halves are odd or even, and the third level's inner
    transforms of 1 .. 20 points), for the DCT-II axis of one component and
    the DST-I axes of the others."""
    from paper_2508_07193_b300 import flashmp as F
    worst = 0.0
    for m in range(2, 41):
        grid = [6, 5, 6]
        grid[axis] = m
        nx, ny, nz = grid
        w = wl.make_workload("box", tuple(grid), seed=m + 100 * axis, uniform_eps=True, overlap=0)
        ctx = F.Context(tuple(grid), np.full((nz, ny, nx), 3.0), 0.25)
        x = host(ctx.box_solve(0, dev(w.rhs)))
        ctx.close()
        ref = box.exact_solve(w.rhs, 3.0, 0.25)
        worst = max(worst, rel(x, ref))
        assert rel(x, ref) <= FP64_TOL, (grid, rel(x, ref))
        assert np.all(x[ras.box_wall(tuple(grid))] == 0.0)
    print("worst", worst)


def test_box32_workload_residual():
    w = wl.box32()
    ctx = context(w)
    x = host(ctx.box_solve(0, dev(w.rhs)))
    A = yee.system_matrix(w.grid, yee.edge_eps(w.grid, None), w.beta)
    r = np.linalg.norm(A @ x.reshape(-1) - w.rhs.reshape(-1)) / np.linalg.norm(w.rhs)
    assert r <= 1e-12
    # the same through the preconditioner entry (one box = whole grid)
    z = host(ctx.precond_apply(dev(w.rhs)))
    assert rel(z, x) <= 1e-15


@pytest.mark.parametrize("w", [
    wl.small(),
    wl.small(grid=(33, 17, 9), cuts=((11, 11, 11), (17,), (4, 5)), overlap=1, seed=21, n_eps_boxes=5),
    wl.small(grid=(24, 24, 24), cuts=((8, 8, 8),) * 3, overlap=3, seed=22, n_eps_boxes=6),
    wl.small(grid=(12, 10, 8), cuts=((3, 3, 3, 3), (2, 8), (8,)), overlap=2, seed=23, n_eps_boxes=3, beta=25.0),
], ids=["small", "ragged", "27boxes", "beta25"])
def test_precond_apply_matches_oracle(w):
    ctx = context(w)
    ee = yee.edge_eps(w.grid, w.eps_cell)
    z = host(ctx.precond_apply(dev(w.rhs)))
    boxes = ras.partition(w.grid, w.cuts, w.overlap)
    ref = ras.precond_apply(w.rhs, boxes, ee, w.beta)
    assert rel(z, ref) <= FP64_TOL
    assert box_rel2(z, ref, boxes) <= FP64_TOL
    # run twice: scratch reuse must not leak state between applies
    z2 = host(ctx.precond_apply(dev(w.rhs)))
    assert np.array_equal(z, z2)


def test_precond_128_sampled_boxes():
    # the 128^3 workload in the launch configuration the benchmark uses;
    # the oracle checks the owned block of a few boxes one by one
    w = wl.grid128()
    ctx = context(w)
    z = host(ctx.precond_apply(dev(w.rhs)))
    ee = yee.edge_eps(w.grid, w.eps_cell)
    boxes = ras.partition(w.grid, w.cuts, w.overlap)
    for i in (0, 21, 42, 63):
        b = boxes[i]
        eb = box.exact_solve(ras.restrict(w.rhs, b), ras.eps_bar(ee, b), w.beta)
        part = np.zeros_like(w.rhs)
        ras.prolong_owned(part, eb, b)
        (x0, y0, z0), (x1, y1, z1) = b.own_lo, b.own_hi
        sl = (slice(None), slice(z0, z1), slice(y0, y1), slice(x0, x1))
        assert rel(z[sl], part[sl]) <= FP64_TOL


def test_precond_uneven_sampled_boxes_per_size_class():
    """The uneven 320 x 256 x 192 workload (extents 28-68) in float64: its
    boxes run in several launches of each pass, grouped by the shared memory
    they need. Owned blocks of the smallest, the largest and two more boxes
    against the oracle one by one."""
    w = wl.grid_uneven()
    ctx = context(w)
    z = host(ctx.precond_apply(dev(w.rhs)))
    ee = yee.edge_eps(w.grid, w.eps_cell)
    boxes = ras.partition(w.grid, w.cuts, w.overlap)
    size = lambda i: np.prod([boxes[i].ext_hi[a] - boxes[i].ext_lo[a] for a in range(3)])
    picks = {min(range(len(boxes)), key=size), max(range(len(boxes)), key=size), 0, len(boxes) // 2}
    for i in sorted(picks):
        b = boxes[i]
        eb = box.exact_solve(ras.restrict(w.rhs, b), ras.eps_bar(ee, b), w.beta)
        part = np.zeros_like(w.rhs)
        ras.prolong_owned(part, eb, b)
        (x0, y0, z0), (x1, y1, z1) = b.own_lo, b.own_hi
        sl = (slice(None), slice(z0, z1), slice(y0, y1), slice(x0, x1))
        assert rel(z[sl], part[sl]) <= FP64_TOL
    ctx.close()
