"""GPU vs oracle: edge permittivity, box means, double-curl SpMV, CN rhs and H
update (deterministic float64 maps, relative error <= 1e-11)."""
import numpy as np
import pytest

from oracle import cn, ras, yee
from paper_2508_07193_b300 import workloads as wl
from tests._gpu import FP64_TOL, context, dev, host, rel

pytestmark = pytest.mark.gpu

CASES = [
    wl.small(),
    wl.small(grid=(33, 17, 9), cuts=((11, 11, 11), (17,), (4, 5)), overlap=1, seed=21, n_eps_boxes=5),
    wl.small(grid=(2, 3, 2), cuts=((2,), (3,), (2,)), overlap=0, seed=5, n_eps_boxes=1),
]


@pytest.mark.parametrize("w", CASES, ids=lambda w: "x".join(map(str, w.grid)))
def test_eps_edge_and_box_means(w):
    ctx = context(w)
    ee = yee.edge_eps(w.grid, w.eps_cell)
    assert rel(host(ctx.eps_edge()), ee) <= 1e-15
    boxes = ras.partition(w.grid, w.cuts, w.overlap)
    assert ctx.num_boxes() == len(boxes)
    for i, b in enumerate(boxes):
        g = ctx.box(i)
        assert g["ext_lo"] == b.ext_lo and g["m"] == b.m and g["own_lo"] == b.own_lo
        assert g["eps_bar"] == pytest.approx(ras.eps_bar(ee, b), rel=1e-14)


@pytest.mark.parametrize("w", CASES, ids=lambda w: "x".join(map(str, w.grid)))
@pytest.mark.parametrize("c_eps,c_k", [(1.0, 0.25), (1.0, -0.25), (0.0, 1.0), (2.5, 7.0)])
def test_curlcurl_apply(w, c_eps, c_k):
    ctx = context(w)
    ee = yee.edge_eps(w.grid, w.eps_cell)
    y = host(ctx.curlcurl_apply(dev(w.rhs), c_eps=c_eps, c_k=c_k))
    ref = yee.operator_apply(w.grid, ee, w.rhs, c_eps, c_k)
    assert rel(y, ref) <= FP64_TOL
    assert np.all(y[wl.edge_wall_mask(w.grid)] == 0.0)


@pytest.mark.parametrize("w", CASES[:2], ids=lambda w: "x".join(map(str, w.grid)))
def test_cn_rhs_and_h_update(w):
    ctx = context(w)
    g = w.grid
    ee = yee.edge_eps(g, w.eps_cell)
    rng = np.random.default_rng(4)
    E = w.rhs
    H = rng.uniform(-1, 1, E.shape); H[wl.face_wall_mask(g)] = 0
    J = rng.uniform(-1, 1, E.shape); J[wl.edge_wall_mask(g)] = 0
    dt = 2.0 * np.sqrt(w.beta)
    R = host(ctx.cn_rhs(dev(E), dev(H), dev(J), dt))
    assert rel(R, cn.rhs(g, ee, E, H, J, dt)) <= FP64_TOL
    R0 = host(ctx.cn_rhs(dev(E), dev(H), None, dt))
    assert rel(R0, cn.rhs(g, ee, E, H, None, dt)) <= FP64_TOL
    En = rng.uniform(-1, 1, E.shape); En[wl.edge_wall_mask(g)] = 0
    Hd = dev(H)
    ctx.h_update(Hd, dev(En), dev(E), dt)
    assert rel(host(Hd), cn.h_update(g, H, En, E, dt)) <= FP64_TOL


def test_cn_rhs_rejects_mismatched_dt():
    from paper_2508_07193_b300 import flashmp as F
    w = CASES[0]
    ctx = context(w)
    z = ctx.empty_field()
    with pytest.raises(F.FlashMPError):
        ctx.cn_rhs(z, z.clone(), None, 0.9)


def test_curlcurl_is_exact_on_integer_fields():
    """K has integer coefficients and the apply evaluates K x exactly in
    fixed point: on small integer fields (c_eps = 0, c_k = 1) the result is
    the oracle's sparse product bit for bit."""
    w = CASES[1]
    ctx = context(w)
    rng = np.random.default_rng(9)
    x = rng.integers(-1000, 1001, size=w.rhs.shape).astype(np.float64)
    x[wl.edge_wall_mask(w.grid)] = 0.0
    y = host(ctx.curlcurl_apply(dev(x), c_eps=0.0, c_k=1.0))
    ref = (yee.double_curl(w.grid) @ x.reshape(-1)).reshape(x.shape)
    ref[wl.edge_wall_mask(w.grid)] = 0.0
    assert np.array_equal(y, ref)


@pytest.mark.parametrize("grid", [(20, 18, 14), (33, 17, 37), (40, 9, 3), (9, 40, 70)])
def test_curlcurl_exact_with_plane_scales(grid):
    """Each z-plane of an integer field scaled by its own power of two (up and
    down along z, so the running exponent maximum of a column grows in steps
    and older planes shift into it): K x stays exact, bit for bit against the
    oracle's sparse product. Grids whose nz leaves ragged and single-plane
    columns."""
    w = wl.make_workload("planes", grid, seed=sum(grid), n_eps_boxes=2, cuts=tuple((n,) for n in grid),
                         overlap=0)
    ctx = context(w)
    rng = np.random.default_rng(11)
    x = rng.integers(-100, 101, size=w.rhs.shape).astype(np.float64)
    s = (np.arange(grid[2]) * 37) % 31           # per-plane exponent, 0 .. 30
    x *= np.ldexp(1.0, s)[None, :, None, None]
    x[wl.edge_wall_mask(w.grid)] = 0.0
    y = host(ctx.curlcurl_apply(dev(x), c_eps=0.0, c_k=1.0))
    ref = (yee.double_curl(w.grid) @ x.reshape(-1)).reshape(x.shape)
    ref[wl.edge_wall_mask(w.grid)] = 0.0
    assert np.array_equal(y, ref)


def test_curlcurl_wide_dynamic_range_and_tiny_tiles():
    """Values 2^-300 .. 2^300 across and inside the 32 x 8 tiles and along
    their columns: the error stays below the float64 bar relative to the
    field; a field of values near 2^-1000 (exponents below the split scale)
    too."""
    w = CASES[0]
    ctx = context(w)
    ee = yee.edge_eps(w.grid, w.eps_cell)
    rng = np.random.default_rng(10)
    for lo, hi in ((-300, 301), (-1010, -990)):
        x = w.rhs * np.ldexp(1.0, rng.integers(lo, hi, size=w.rhs.shape))
        x[wl.edge_wall_mask(w.grid)] = 0.0
        y = host(ctx.curlcurl_apply(dev(x), c_eps=1.0, c_k=0.25))
        ref = yee.operator_apply(w.grid, ee, x, 1.0, 0.25)
        assert rel(y, ref) <= FP64_TOL


def test_curlcurl_nonfinite_and_zero_tiles():
    w = CASES[0]
    ctx = context(w)
    x = np.zeros_like(w.rhs)
    y = host(ctx.curlcurl_apply(dev(x)))
    assert not np.any(y)
    x = w.rhs.copy()
    x[0, 5, 6, 7] = np.inf
    y = host(ctx.curlcurl_apply(dev(x)))
    assert not np.all(np.isfinite(y))
