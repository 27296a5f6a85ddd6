"""Compact-layout preconditioner (Algorithm 1 with Step 4's Woodbury boundary
correction) on the GPU against the float64 oracle, and at full size against
the property that a single compact box over the whole grid is the exact
solve."""
import numpy as np
import pytest

from oracle import compact as cp, ras, yee
from paper_2508_07193_b300 import workloads as wl
from tests._gpu import FP64_TOL, context, dev, host, rel

pytestmark = pytest.mark.gpu

CASES = [
    wl.small(grid=(12, 10, 8), cuts=((6, 6), (5, 5), (8,)), overlap=1, seed=41, n_eps_boxes=3),
    wl.small(grid=(11, 9, 7), cuts=((4, 7), (9,), (3, 4)), overlap=2, seed=42, n_eps_boxes=3),
    wl.small(grid=(9, 8, 10), cuts=((9,), (8,), (10,)), overlap=0, seed=43, n_eps_boxes=2),
]


@pytest.mark.parametrize("w", CASES, ids=lambda w: "x".join(map(str, w.grid)))
def test_compact_precond_matches_oracle(w):
    ctx = context(w)
    ctx.set_subdomain_form("compact")
    form, nbytes = ctx.get_subdomain_form()
    assert form == "compact" and nbytes > 0
    ee = yee.edge_eps(w.grid, w.eps_cell)
    ref = cp.precond_apply(w.rhs, ras.partition(w.grid, w.cuts, w.overlap), ee, w.beta)
    z = host(ctx.precond_apply(dev(w.rhs)))
    assert rel(z, ref) <= FP64_TOL
    assert np.all(z[wl.edge_wall_mask(w.grid)] == 0.0)
    # back to the Yee-box form: a different (also exact) local solve
    ctx.set_subdomain_form("yee")
    z2 = host(ctx.precond_apply(dev(w.rhs)))
    assert rel(z2, ras.precond_apply(w.rhs, ras.partition(w.grid, w.cuts, w.overlap), ee, w.beta)) <= FP64_TOL


@pytest.mark.parametrize("n", [16, 32])
def test_single_compact_box_is_the_exact_solve(n):
    """One compact box covering an n^3 grid (eps boxes in [1, 10]): the
    preconditioner is (eps_bar I + beta K)^{-1}; with eps = eps_bar everywhere
    its output solves the global system, checked by the sparse residual."""
    w = wl.small(grid=(n, n, n), cuts=((n,),) * 3, overlap=0, seed=44, n_eps_boxes=0)
    ctx = context(w)
    ctx.set_subdomain_form("compact")
    z = host(ctx.precond_apply(dev(w.rhs))).reshape(-1)
    ee = yee.edge_eps(w.grid, w.eps_cell)
    A = yee.system_matrix(w.grid, ee, w.beta)
    b = w.rhs.reshape(-1)
    assert np.linalg.norm(b - A @ z) <= 1e-11 * np.linalg.norm(b)


def test_fgmres_with_compact_boxes_converges():
    w = CASES[0]
    ctx = context(w, rtol=1e-10)
    ctx.set_subdomain_form("compact")
    x, info = ctx.krylov_solve(dev(w.rhs))
    ee = yee.edge_eps(w.grid, w.eps_cell)
    A = yee.system_matrix(w.grid, ee, w.beta)
    b = w.rhs.reshape(-1)
    assert np.linalg.norm(b - A @ host(x).reshape(-1)) <= 1e-10 * np.linalg.norm(b)
    assert info["status"] == 0


def test_compact_form_needs_float64():
    w = CASES[0]
    ctx = context(w, precision="bf16")
    ctx.set_subdomain_form("compact")
    with pytest.raises(Exception):
        ctx.precond_apply(dev(w.rhs))
