"""Checked mode (fmp_set_checked): the layout contract of the C ABI -- wall
slots of E-shaped fields (PEC edges) and of H (wall-normal faces) must be
zero on input -- is verified on request and a violation is reported as
FMP_ERR_ARG before anything is computed."""
import numpy as np
import pytest

from paper_2508_07193_b300 import workloads as wl
from tests._gpu import context, dev, host

pytestmark = pytest.mark.gpu


def _err(fn):
    from paper_2508_07193_b300 import flashmp as F
    with pytest.raises(F.FlashMPError) as e:
        fn()
    return e.value.status


@pytest.mark.parametrize("c, k, j, i", [(0, 0, 3, 4), (0, 2, 0, 4), (1, 2, 3, 0), (1, 0, 3, 4), (2, 2, 0, 4),
                                        (2, 2, 3, 0)])
def test_nonzero_wall_slot_is_rejected(c, k, j, i):
    from paper_2508_07193_b300 import flashmp as F
    w = wl.small()
    ctx = context(w)
    ctx.set_checked(True)
    r = w.rhs.copy()
    r[c, k, j, i] = 1.0
    z = ctx.empty_field()
    z.fill_(7.0)
    assert _err(lambda: ctx.precond_apply(dev(r), z)) == F.FMP_ERR_ARG
    assert float(z.min()) == 7.0 and float(z.max()) == 7.0   # nothing was computed
    assert _err(lambda: ctx.curlcurl_apply(dev(r))) == F.FMP_ERR_ARG
    assert _err(lambda: ctx.krylov_solve(dev(r))) == F.FMP_ERR_ARG


def test_clean_fields_pass_and_mode_can_be_switched_off():
    w = wl.small()
    ctx = context(w)
    ctx.set_checked(True)
    z = host(ctx.precond_apply(dev(w.rhs)))
    assert np.all(z[wl.edge_wall_mask(w.grid)] == 0.0)
    x, info = ctx.krylov_solve(dev(w.rhs))
    assert info["true_rel_res"] <= 1e-8
    r = w.rhs.copy()
    r[0, 0, 3, 4] = 1.0
    ctx.set_checked(False)
    z2 = host(ctx.precond_apply(dev(r)))   # unchecked: computed, walls still written as zero
    assert np.all(z2[wl.edge_wall_mask(w.grid)] == 0.0)


def test_cn_step_checks_E_H_and_J():
    from paper_2508_07193_b300 import flashmp as F
    w = wl.small()
    ctx = context(w)
    ctx.set_checked(True)
    dt = 2.0 * np.sqrt(w.beta)
    E, H = ctx.empty_field(), ctx.empty_field()
    J = dev(-w.rhs / dt)
    info = ctx.cn_step(E, H, J, dt)
    assert info["true_rel_res"] <= 1e-8
    Hb = H.clone()
    Hb[0, 2, 3, 0] = 1.0           # Hx on the x = 0 wall
    assert _err(lambda: ctx.cn_step(E, Hb, J, dt)) == F.FMP_ERR_ARG
    Jb = J.clone()
    Jb[2, 2, 0, 4] = 1.0           # Ez on the y = 0 wall
    assert _err(lambda: ctx.cn_step(E, H, Jb, dt)) == F.FMP_ERR_ARG
    Hc = H.clone()
    Hc[0, 2, 0, 4] = 1.0           # Hx off the x = 0 wall: allowed
    ctx.cn_step(E, Hc, J, dt)


def test_box_solve_checks_the_box_grid():
    from paper_2508_07193_b300 import flashmp as F
    grid = (8, 8, 8)
    w = wl.make_workload("box", grid, seed=3, uniform_eps=True, overlap=0)
    ctx = F.Context(grid, np.full((8, 8, 8), 2.0), 0.25)
    ctx.set_checked(True)
    ctx.box_solve(0, dev(w.rhs))
    r = w.rhs.copy()
    r[1, 0, 5, 5] = 1.0            # Ey at k = 0
    assert _err(lambda: ctx.box_solve(0, dev(r))) == F.FMP_ERR_ARG


@pytest.mark.parametrize("prec, tol", [("fp64", 1e-11), ("fp64_ozaki", 1e-11), ("bf16", 3e-2), ("tf32", 5e-3)])
def test_nan_canary_in_the_transform_scratch(prec, tol):
    """Checked mode fills the transform scratch with NaN before every apply:
    a pass that read a slot its predecessor did not write would turn the
    output NaN. Ragged boxes, odd extents and a box with one-cell overlap."""
    from oracle import ras, yee
    w = wl.small(grid=(33, 17, 9), cuts=((11, 11, 11), (17,), (4, 5)), overlap=1, seed=21, n_eps_boxes=5)
    ctx = context(w, precision=prec)
    if prec == "bf16":
        ctx.set_fused(0)   # the three-pass kernels are the ones that use the scratch
    ctx.set_checked(True)
    z = host(ctx.precond_apply(dev(w.rhs)))
    assert np.all(np.isfinite(z))
    ee = yee.edge_eps(w.grid, w.eps_cell)
    ref = ras.precond_apply(w.rhs, ras.partition(w.grid, w.cuts, w.overlap), ee, w.beta)
    assert np.linalg.norm(z - ref) / np.linalg.norm(ref) <= tol
