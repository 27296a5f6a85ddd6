"""The streamed reduced-precision solve (one persistent launch over boxes of
any extent, work items pulled from an atomic counter, per-box dependency
counts between its passes) against the float64 oracle: ragged multi-box
grids with boxes above the fused kernel's 40 cells, extents 2 to 80, the
uneven 320 x 256 x 192 workload's largest and smallest boxes, and the
bounded waits (a test mode whose last-pass items wait for an item that
never comes: NaN in that box, an error status, the context usable after)."""
import numpy as np
import pytest

from oracle import box, ras, yee
from paper_2508_07193_b300 import flashmp as F
from paper_2508_07193_b300 import workloads as wl
from tests._gpu import context, dev, host, owned_slices
from tests.test_gpu_mixed import _oracle_owned, check

pytestmark = pytest.mark.gpu

RAGGED = [
    wl.small(grid=(80, 24, 16), cuts=((20, 60), (12, 12), (16,)), overlap=2, seed=23, n_eps_boxes=5),
    wl.small(grid=(70, 41, 33), cuts=((33, 37), (41,), (15, 18)), overlap=3, seed=41, n_eps_boxes=6),
    wl.small(grid=(33, 17, 9), cuts=((11, 11, 11), (17,), (4, 5)), overlap=1, seed=21, n_eps_boxes=5),
]


@pytest.mark.parametrize("fused", [40, 0], ids=["with_fused", "all_streamed"])
@pytest.mark.parametrize("prec", ["bf16", "fp16"])
@pytest.mark.parametrize("w", RAGGED, ids=lambda w: "x".join(map(str, w.grid)))
def test_streamed_precond_matches_oracle(w, prec, fused):
    ctx = context(w, precision=prec)
    ctx.set_fused(fused)
    mode, nb = ctx.get_streamed()
    assert mode == 1 and nb == ctx.num_boxes() - ctx.get_fused()[1] and (nb > 0 or fused)
    ee = yee.edge_eps(w.grid, w.eps_cell)
    boxes = ras.partition(w.grid, w.cuts, w.overlap)
    ref = ras.precond_apply(w.rhs, boxes, ee, w.beta)
    r = dev(w.rhs)
    z = host(ctx.precond_apply(r))
    check(z, ref, prec, boxes)
    assert np.all(z[wl.edge_wall_mask(w.grid)] == 0.0)
    assert ctx.stream_check() == F.FMP_OK
    # repeated applies are bitwise equal (counters reset, scratch fully rewritten)
    assert np.array_equal(host(ctx.precond_apply(r)), z)
    # the three-pass kernels reach the same oracle bound
    ctx.set_streamed(0)
    assert ctx.get_streamed() == (0, 0)
    check(host(ctx.precond_apply(r)), ref, prec, boxes)
    ctx.close()


@pytest.mark.parametrize("grid", [(2, 3, 64), (80, 9, 12), (41, 80, 5), (67, 45, 71), (17, 40, 3)])
def test_streamed_single_box_extents(grid):
    nx, ny, nz = grid
    w = wl.make_workload("box", grid, seed=sum(grid), uniform_eps=True, overlap=0)
    for prec in ("bf16", "fp16"):
        ctx = F.Context(grid, np.full((nz, ny, nx), 2.5), 0.25, precision=prec)
        ctx.set_fused(0)
        z = host(ctx.precond_apply(dev(w.rhs)))
        ref = box.exact_solve(w.rhs, 2.5, 0.25)
        check(z, ref, prec)
        ctx.close()


def test_uneven_workload_streamed_boxes_match_oracle():
    """The uneven workload in bf16 with the streamed solve (boxes above 40 in
    one persistent launch, the rest fused): its largest and smallest boxes
    against the oracle, and the same with every box streamed."""
    w = wl.grid_uneven()
    ee = yee.edge_eps(w.grid, w.eps_cell)
    boxes = ras.partition(w.grid, w.cuts, w.overlap)
    ext = [max(b.ext_hi[a] - b.ext_lo[a] for a in range(3)) for b in boxes]
    big = max(range(len(boxes)), key=lambda i: ext[i])
    small = min(range(len(boxes)), key=lambda i: ext[i])
    refs = [_oracle_owned(w, ee, boxes[i]) for i in (small, big)]
    ctx = context(w, precision="bf16")
    r = dev(w.rhs)
    for fused in (40, 0):
        ctx.set_fused(fused)
        z = host(ctx.precond_apply(r))
        for sl, ref in refs:
            check(z[sl], ref, "bf16")
    assert ctx.stream_check() == F.FMP_OK
    ctx.close()


@pytest.mark.parametrize("prec", ["bf16", "fp16"])
def test_fgmres_with_streamed_precond(prec):
    w = RAGGED[1]
    ctx = context(w, precision=prec, rtol=1e-10)
    ctx.set_fused(0)
    x, info = ctx.krylov_solve(dev(w.rhs))
    ee = yee.edge_eps(w.grid, w.eps_cell)
    A = yee.system_matrix(w.grid, ee, w.beta)
    b = w.rhs.reshape(-1)
    assert np.linalg.norm(b - A @ host(x).reshape(-1)) / np.linalg.norm(b) <= 1e-10
    ctx.close()


def test_bounded_wait_runs_out_cleanly():
    """Mode 2 makes one box's last-pass items wait for a count that is never
    reached: after about a second each wait gives up, that box's owned cells
    get NaN, the other boxes are exact, the status is FMP_ERR_CUDA once, and
    the next applies in mode 1 are correct again."""
    w = RAGGED[0]
    ctx = context(w, precision="bf16")
    ctx.set_fused(0)
    ee = yee.edge_eps(w.grid, w.eps_cell)
    boxes = ras.partition(w.grid, w.cuts, w.overlap)
    ref = ras.precond_apply(w.rhs, boxes, ee, w.beta)
    r = dev(w.rhs)
    ctx.set_streamed(2)
    z = host(ctx.precond_apply(r))
    assert ctx.stream_check() == F.FMP_ERR_CUDA
    assert ctx.stream_check() == F.FMP_OK
    bad = [i for i, b in enumerate(boxes) if np.isnan(z[owned_slices(b)]).any()]
    assert len(bad) == 1
    assert np.isnan(z[owned_slices(boxes[bad[0]])]).all()
    for i, b in enumerate(boxes):
        if i != bad[0]:
            check(z[owned_slices(b)], ref[owned_slices(b)], "bf16")
    ctx.set_streamed(1)
    check(host(ctx.precond_apply(r)), ref, "bf16", boxes)
    assert ctx.stream_check() == F.FMP_OK
    ctx.close()
