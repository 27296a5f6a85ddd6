"""GPU vs oracle: the digit-split float64 transforms (FMP_PREC_FP64_OZAKI,
bf16 tensor-core digit planes with exact fp32 accumulation). The bar is the
float64 one: relative error <= 1e-11 against the oracle's exact solve
(Algorithm 1, exact_solve) and RAS apply (Sec. II-B); plus properties the
splitting guarantees exactly (power-of-two scaling, zero in -> zero out)."""
import numpy as np
import pytest

from oracle import box, ras, yee
from paper_2508_07193_b300 import workloads as wl
from tests._gpu import FP64_TOL, context, dev, host, maxrel, rel, rel2

pytestmark = pytest.mark.gpu


def _box_ctx(grid, eps, **kw):
    from paper_2508_07193_b300 import flashmp as F
    nx, ny, nz = grid
    return F.Context(grid, np.full((nz, ny, nx), eps), 0.25, precision="fp64_ozaki", **kw)


@pytest.mark.parametrize("grid", [(32, 32, 32), (8, 8, 8), (2, 2, 2), (5, 7, 3), (36, 34, 33), (40, 40, 40),
                                  (17, 40, 3)])
def test_box_solve_matches_oracle(grid):
    rng = np.random.default_rng(sum(grid))
    eps = rng.uniform(1, 10)
    w = wl.make_workload("box", grid, seed=sum(grid), uniform_eps=True, overlap=0)
    ctx = _box_ctx(grid, eps)
    x = host(ctx.box_solve(0, dev(w.rhs)))
    ref = box.exact_solve(w.rhs, eps, 0.25)
    assert rel(x, ref) <= FP64_TOL
    assert np.all(x[ras.box_wall(grid)] == 0.0)


def test_box32_error_against_native_float64():
    """The configuration-1 box: the split path agrees with the float64 path
    far inside the float64 bar (each axis transform keeps ~46 bits)."""
    w = wl.box32()
    nat = context(w)
    oz = context(w, precision="fp64_ozaki")
    a = host(nat.box_solve(0, dev(w.rhs)))
    b = host(oz.box_solve(0, dev(w.rhs)))
    assert rel2(b, a) <= 1e-13 and maxrel(b, a) <= 3e-13
    A = yee.system_matrix(w.grid, yee.edge_eps(w.grid, None), w.beta)
    r = np.linalg.norm(A @ b.reshape(-1) - w.rhs.reshape(-1)) / np.linalg.norm(w.rhs)
    assert r <= 1e-12


@pytest.mark.parametrize("grid", [(48, 48, 48), (80, 9, 12), (64, 33, 41), (41, 5, 70)])
def test_box_solve_long_lines_match_oracle(grid):
    """Extents 41-80: the contraction is accumulated in two-k-step fp32
    partials moved into 64-bit sums (each partial exact)."""
    rng = np.random.default_rng(sum(grid))
    eps = rng.uniform(1, 10)
    w = wl.make_workload("box", grid, seed=sum(grid), uniform_eps=True, overlap=0)
    x = host(_box_ctx(grid, eps).box_solve(0, dev(w.rhs)))
    ref = box.exact_solve(w.rhs, eps, 0.25)
    assert rel(x, ref) <= FP64_TOL
    assert np.all(x[ras.box_wall(grid)] == 0.0)


def test_uneven_workload_sampled_boxes_and_native_agreement():
    """The 320 x 256 x 192 uneven workload (extents 28-68): owned blocks of
    three boxes against the oracle, the whole field against the float64 kernels."""
    w = wl.grid_uneven()
    ctx = context(w, precision="fp64_ozaki")
    z = host(ctx.precond_apply(dev(w.rhs)))
    ee = yee.edge_eps(w.grid, w.eps_cell)
    boxes = ras.partition(w.grid, w.cuts, w.overlap)
    big = max(range(len(boxes)), key=lambda i: max(boxes[i].ext_hi[a] - boxes[i].ext_lo[a] for a in range(3)))
    for i in (0, big, len(boxes) - 1):
        b = boxes[i]
        eb = box.exact_solve(ras.restrict(w.rhs, b), ras.eps_bar(ee, b), w.beta)
        part = np.zeros_like(w.rhs)
        ras.prolong_owned(part, eb, b)
        (x0, y0, z0), (x1, y1, z1) = b.own_lo, b.own_hi
        sl = (slice(None), slice(z0, z1), slice(y0, y1), slice(x0, x1))
        assert rel(z[sl], part[sl]) <= FP64_TOL
    zn = host(context(w).precond_apply(dev(w.rhs)))
    assert rel2(z, zn) <= 1e-13 and maxrel(z, zn) <= 3e-13


@pytest.mark.parametrize("w", [
    wl.small(),
    wl.small(grid=(33, 17, 9), cuts=((11, 11, 11), (17,), (4, 5)), overlap=1, seed=21, n_eps_boxes=5),
    wl.small(grid=(24, 24, 24), cuts=((8, 8, 8),) * 3, overlap=3, seed=22, n_eps_boxes=6),
    wl.small(grid=(12, 10, 8), cuts=((3, 3, 3, 3), (2, 8), (8,)), overlap=2, seed=23, n_eps_boxes=3, beta=25.0),
], ids=["small", "ragged", "27boxes", "beta25"])
def test_precond_apply_matches_oracle(w):
    ctx = context(w, precision="fp64_ozaki")
    ee = yee.edge_eps(w.grid, w.eps_cell)
    z = host(ctx.precond_apply(dev(w.rhs)))
    ref = ras.precond_apply(w.rhs, ras.partition(w.grid, w.cuts, w.overlap), ee, w.beta)
    assert rel(z, ref) <= FP64_TOL
    z2 = host(ctx.precond_apply(dev(w.rhs)))
    assert np.array_equal(z, z2)


def test_precond_128_sampled_boxes_and_native_agreement():
    """The 128^3 workload in the benchmark's launch configuration: owned
    blocks of four boxes against the oracle one by one, the whole field
    against the float64 kernels."""
    w = wl.grid128()
    ctx = context(w, precision="fp64_ozaki")
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
    zn = host(context(w).precond_apply(dev(w.rhs)))
    assert rel2(z, zn) <= 1e-13 and maxrel(z, zn) <= 3e-13


def test_power_of_two_scaling_is_exact_and_zero_stays_zero():
    """Digits are taken relative to each line's exponent, so scaling the input
    by 2^k scales every output by exactly 2^k (no over/underflow)."""
    w = wl.small()
    ctx = context(w, precision="fp64_ozaki")
    z = host(ctx.precond_apply(dev(w.rhs)))
    for k in (-600, -37, 1, 500):
        zk = host(ctx.precond_apply(dev(np.ldexp(w.rhs, k))))
        assert np.array_equal(zk, np.ldexp(z, k))
    z0 = host(ctx.precond_apply(dev(np.zeros_like(w.rhs))))
    assert not np.any(z0)


def test_wide_dynamic_range_input():
    """Values spanning 2^-80 .. 2^80 inside the lines: the error stays within
    the bar relative to the whole field."""
    w = wl.small(grid=(24, 24, 24), cuts=((8, 8, 8),) * 3, overlap=3, seed=22, n_eps_boxes=6)
    rng = np.random.default_rng(5)
    r = w.rhs * np.ldexp(1.0, rng.integers(-80, 81, size=w.rhs.shape))
    r[wl.edge_wall_mask(w.grid)] = 0.0
    ctx = context(w, precision="fp64_ozaki")
    ee = yee.edge_eps(w.grid, w.eps_cell)
    z = host(ctx.precond_apply(dev(r)))
    ref = ras.precond_apply(r, ras.partition(w.grid, w.cuts, w.overlap), ee, w.beta)
    assert rel(z, ref) <= FP64_TOL


def test_nonfinite_input_stays_nonfinite():
    w = wl.small()
    ctx = context(w, precision="fp64_ozaki")
    r = w.rhs.copy()
    r[0, 3, 4, 5] = np.nan
    z = host(ctx.precond_apply(dev(r)))
    assert np.isnan(z).any()


def test_fgmres_converges_like_float64():
    w = wl.small(grid=(24, 24, 24), cuts=((8, 8, 8),) * 3, overlap=2, seed=22, n_eps_boxes=6)
    xn, inf_n = context(w, rtol=1e-10).krylov_solve(dev(w.rhs))
    xo, inf_o = context(w, rtol=1e-10, precision="fp64_ozaki").krylov_solve(dev(w.rhs))
    assert inf_o["true_rel_res"] <= 1e-10
    assert inf_o["iters"] == inf_n["iters"]
    assert rel(host(xo), host(xn)) <= 1e-9


def test_bicgstab_and_graph_replay():
    """BiCGSTAB reaches rtol with the split transforms; the graph-replayed
    FGMRES cycle equals the host loop bit for bit."""
    w = wl.small()
    x, inf = context(w, rtol=1e-10, precision="fp64_ozaki", krylov="bicgstab").krylov_solve(dev(w.rhs))
    assert inf["true_rel_res"] <= 1e-10
    a, ia = context(w, rtol=1e-10, precision="fp64_ozaki", use_graph=False).krylov_solve(dev(w.rhs))
    g, ig = context(w, rtol=1e-10, precision="fp64_ozaki", use_graph=True).krylov_solve(dev(w.rhs))
    assert ia["iters"] == ig["iters"] and np.array_equal(host(a), host(g))


def test_cn_steps_match_float64_kernels():
    """Three CN steps with the split transforms stay within the solve
    tolerance of the same steps with the float64 kernels."""
    w = wl.small(grid=(24, 24, 24), cuts=((8, 8, 8),) * 3, overlap=2, seed=22, n_eps_boxes=6)
    dt = 2.0 * np.sqrt(w.beta)
    out = []
    for prec in ("fp64", "fp64_ozaki"):
        ctx = context(w, rtol=1e-11, precision=prec)
        E, H = ctx.empty_field(), ctx.empty_field()
        J = dev(-w.rhs / dt)
        for _ in range(3):
            info = ctx.cn_step(E, H, J, dt)
            assert info["true_rel_res"] <= 1e-11
        out.append((host(E), host(H)))
    assert rel(out[1][0], out[0][0]) <= 1e-9 and rel(out[1][1], out[0][1]) <= 1e-9
