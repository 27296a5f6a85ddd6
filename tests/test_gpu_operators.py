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
