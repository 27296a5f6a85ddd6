"""Learned component: GPU convolution forward / backward against the float64
oracle CNN, training reduces the loss, and the learned solver paths still
solve to the requested true residual (with the fallback rule)."""
import numpy as np
import pytest

from oracle import cn, cnn, yee
from paper_2508_07193_b300 import workloads as wl
from tests._gpu import context, dev, host, rel

pytestmark = pytest.mark.gpu


def bf16(x):
    """Round float64 -> bfloat16 (nearest even), returned as float64."""
    u = np.ascontiguousarray(x, dtype=np.float32).view(np.uint32).astype(np.uint64)
    u = ((u + 0x7FFF + ((u >> 16) & 1)) & 0xFFFF0000).astype(np.uint32)
    return u.view(np.float32).astype(np.float64)


def flat(params):
    return np.concatenate([np.concatenate([w.reshape(-1), b]) for w, b in params]).astype(np.float32)


def unflat(v):
    out, o = [], 0
    for ci, co in cnn.LAYERS:
        nw = co * ci * 27
        out.append((v[o:o + nw].reshape(co, ci, 3, 3, 3), v[o + nw:o + nw + co]))
        o += nw + co
    return out


def seeded_params(seed=3):
    rng = np.random.default_rng(seed)
    p = cnn.init_params(seed)
    p = [(w, rng.uniform(-0.05, 0.05, b.shape)) for w, b in p]
    f = flat(p)
    return f, unflat(f.astype(np.float64))


def net_input(w, r):
    s = np.sqrt(np.mean(r ** 2))
    eps = np.ones(w.grid[::-1]) if w.eps_cell is None else w.eps_cell
    return s, np.concatenate([r / s, eps[None] * 0.1])


def test_cnn_apply_matches_oracle():
    w = wl.small()
    ctx = context(w)
    f, params = seeded_params()
    ctx.cnn_set_params(f)
    assert np.array_equal(ctx.cnn_get_params(), f)
    out = host(ctx.cnn_apply(dev(w.rhs)))
    s, x = net_input(w, w.rhs)
    y, _ = cnn.forward(params, x)
    ref = y * s
    ref[wl.edge_wall_mask(w.grid)] = 0.0
    assert rel(out, ref) <= 3e-2
    assert np.all(out[wl.edge_wall_mask(w.grid)] == 0.0)


def test_cnn_gradients_match_oracle():
    w = wl.small(grid=(24, 20, 16), cuts=((24,), (20,), (16,)), overlap=0, seed=9)
    ctx = context(w)
    f, params = seeded_params(5)
    ctx.cnn_set_params(f)
    rng = np.random.default_rng(6)
    e = rng.uniform(-1, 1, w.rhs.shape)
    ctx.cnn_add_sample(dev(w.rhs), dev(e))
    assert ctx.cnn_num_samples() == 1
    lo, crop = (3, 2, 1), 12
    loss, g = ctx.cnn_grad(0, lo, crop)
    s, x = net_input(w, w.rhs)
    sl = (slice(None), slice(lo[2], lo[2] + crop), slice(lo[1], lo[1] + crop), slice(lo[0], lo[0] + crop))
    xc = bf16(x)[sl]
    tc = (e / s).astype(np.float32).astype(np.float64)[sl]
    out, acts = cnn.forward(params, xc)
    L, grads = cnn.backward(params, acts, tc)
    assert loss == pytest.approx(L, rel=2e-2)
    gg = unflat(g.astype(np.float64))
    for li in range(4):
        for q in range(2):
            assert rel(gg[li][q], grads[li][q]) <= 6e-2, (li, q, rel(gg[li][q], grads[li][q]))


def test_cnn_training_reduces_loss():
    w = wl.small(grid=(24, 20, 16), cuts=((12, 12), (20,), (16,)), overlap=2, seed=11)
    ctx = context(w, rtol=1e-10)
    rng = np.random.default_rng(12)
    for _ in range(3):
        b = rng.uniform(-1, 1, w.rhs.shape); b[wl.edge_wall_mask(w.grid)] = 0
        bd = dev(b)
        x, _ = ctx.krylov_solve(bd)
        ctx.cnn_add_sample(bd, x)
    l0, _ = ctx.cnn_grad(0, (4, 4, 2), 12)
    ctx.cnn_train(300, 12, lr=2e-3, seed=1)
    l1, _ = ctx.cnn_grad(0, (4, 4, 2), 12)
    assert l1 < 0.5 * l0, (l0, l1)


@pytest.mark.parametrize("mode", [1, 2])
def test_learned_cn_steps_solve_to_tolerance(mode):
    w = wl.small(grid=(16, 14, 12), cuts=((8, 8), (7, 7), (12,)), overlap=2, seed=31, n_eps_boxes=3)
    g = w.grid
    ee = yee.edge_eps(g, w.eps_cell)
    dt = 2.0 * np.sqrt(w.beta)
    ctx = context(w, rtol=1e-11, use_learned=mode, experimental=mode >= 2)
    E = np.zeros_like(w.rhs); H = np.zeros_like(E)
    Ed, Hd = dev(E), dev(H)
    for n in range(3):
        J = wl.dipole_current(g, n + 20, dt) * 10 + (w.rhs if n == 0 else 0)
        info = ctx.cn_step(Ed, Hd, dev(J), dt)
        E, H = cn.step(g, ee, E, H, J, dt)
        assert info["used_fallback"] in (0, 1)
    assert rel(host(Ed), E) <= 1e-8 and rel(host(Hd), H) <= 1e-8


def _oracle_out(params, w, r, s):
    """The oracle network on the whole volume, rescaled, walls zeroed."""
    eps = np.ones(w.grid[::-1]) if w.eps_cell is None else w.eps_cell
    y, _ = cnn.forward(params, np.concatenate([r / s, eps[None] * 0.1]))
    y = y * s
    y[wl.edge_wall_mask(w.grid)] = 0.0
    return y


@pytest.mark.parametrize("grid,xcuts", [((20, 18, 14), (20,)), ((131, 19, 7), (44, 44, 43)),
                                        ((129, 9, 3), (43, 43, 43)), ((5, 3, 2), (5,))],
                         ids=["small", "two-x-tiles-ragged", "x-tail-one", "tiny"])
def test_cnn_apply_tcgen05_matches_oracle(grid, xcuts):
    """The full-volume apply (16-channel layers on tcgen05, TMA zero fill as
    the convolution's padding) on volumes with ragged x tiles (128 voxels),
    ragged y tiles (8 rows) and short z-columns."""
    w = wl.make_workload("cnn", grid, seed=sum(grid), n_eps_boxes=3, cuts=(xcuts, (grid[1],), (grid[2],)),
                         overlap=1 if len(xcuts) > 1 else 0)
    ctx = context(w)
    f, params = seeded_params()
    ctx.cnn_set_params(f)
    out = host(ctx.cnn_apply(dev(w.rhs)))
    s = np.sqrt(np.mean(w.rhs ** 2))
    ref = _oracle_out(params, w, w.rhs, s)
    assert rel(out, ref) <= 3e-2
    assert np.all(out[wl.edge_wall_mask(w.grid)] == 0.0)


def test_cnn_apply_scales_exactly_with_the_residual():
    """The input is r / rms(r) and the output is rescaled by rms(r), so a
    residual scaled by 2^400 or 2^-400 gives the same bf16 input and an
    output scaled by exactly that power of two (the input conversion's
    exponent arithmetic over a wide range)."""
    w = wl.small(grid=(40, 12, 6), cuts=((40,), (12,), (6,)), overlap=0, seed=33, n_eps_boxes=2)
    ctx = context(w)
    f, _ = seeded_params()
    ctx.cnn_set_params(f)
    a = host(ctx.cnn_apply(dev(w.rhs)))
    assert np.any(a)
    for p in (400, -400):
        b = host(ctx.cnn_apply(dev(np.ldexp(w.rhs, p))))
        assert np.array_equal(b, np.ldexp(a, p)), p


def test_cnn_apply_tcgen05_agrees_with_mma_sync():
    """tcgen05 and mma.sync evaluate the same bf16 network; they differ only in
    the fp32 summation order (and the bf16 roundings that flips)."""
    w = wl.small(grid=(140, 21, 9), cuts=((70, 70), (21,), (9,)), overlap=1, seed=31, n_eps_boxes=4)
    ctx = context(w)
    f, _ = seeded_params()
    ctx.cnn_set_params(f)
    a = host(ctx.cnn_apply(dev(w.rhs)))
    ctx.cnn_set_tc(False)
    b = host(ctx.cnn_apply(dev(w.rhs)))
    ctx.cnn_set_tc(True)
    c = host(ctx.cnn_apply(dev(w.rhs)))
    assert np.array_equal(a, c)   # deterministic
    assert rel(a, b) <= 1e-2


def test_cnn_apply_128_sampled_voxels_match_oracle():
    """The 128^3 workload: sampled output voxels, each against the oracle
    network on the 9^3 neighbourhood that determines it (clipped at the
    volume, where the padding is the volume's own)."""
    w = wl.grid128()
    ctx = context(w)
    f, params = seeded_params()
    ctx.cnn_set_params(f)
    out = host(ctx.cnn_apply(dev(w.rhs)))
    s = np.sqrt(np.mean(w.rhs ** 2))
    eps = w.eps_cell
    nx, ny, nz = w.grid
    rng = np.random.default_rng(11)
    pts = [(0, 0, 0), (nz - 1, ny - 1, nx - 1), (0, 64, 127), (127, 7, 8), (64, 8, 0), (3, 127, 126)]
    pts += [tuple(int(v) for v in rng.integers(0, 128, 3)) for _ in range(10)]
    got, want = [], []
    for k, j, i in pts:
        lo = [max(0, k - 4), max(0, j - 4), max(0, i - 4)]
        hi = [min(nz, k + 5), min(ny, j + 5), min(nx, i + 5)]
        sl = tuple(slice(a, b) for a, b in zip(lo, hi))
        x = np.concatenate([w.rhs[(slice(None),) + sl] / s, eps[sl][None] * 0.1])
        y, _ = cnn.forward(params, x)
        want.append(y[:, k - lo[0], j - lo[1], i - lo[2]] * s)
        got.append(out[:, k, j, i])
    want = np.array(want)
    mask = wl.edge_wall_mask(w.grid)
    for q, (k, j, i) in enumerate(pts):
        want[q][mask[:, k, j, i]] = 0.0
    assert rel(np.array(got), want) <= 3e-2


def test_cnn_tcgen05_wait_runs_out_cleanly():
    """The tcgen05 kernels' bounded waits: with every input-plane wait of the
    first layer expecting bytes that never arrive, the waits run out, the
    kernel returns, the apply reports FMP_ERR_CUDA, and the context still
    works (the next applies are exact again)."""
    from paper_2508_07193_b300 import flashmp as F
    w = wl.small()
    ctx = context(w)
    f, _ = seeded_params()
    ctx.cnn_set_params(f)
    good = host(ctx.cnn_apply(dev(w.rhs)))
    ctx.cnn_set_tc(2)
    with pytest.raises(F.FlashMPError) as ei:
        ctx.cnn_apply(dev(w.rhs))
    assert "FMP_ERR_CUDA" in str(ei.value)
    ctx.cnn_set_tc(True)
    assert np.array_equal(host(ctx.cnn_apply(dev(w.rhs))), good)
    z = host(ctx.precond_apply(dev(w.rhs)))
    assert np.isfinite(z).all()
    for bad in (3, -1):
        with pytest.raises(F.FlashMPError) as ei:
            ctx.cnn_set_tc(bad)
        assert "FMP_ERR_ARG" in str(ei.value)


def test_in_fgmres_correction_needs_the_experimental_flag():
    w = wl.small(grid=(16, 14, 12), cuts=((8, 8), (7, 7), (12,)), overlap=2, seed=31, n_eps_boxes=3)
    with pytest.raises(ValueError):
        context(w, use_learned=2)
    ctx = context(w, use_learned=1)
    with pytest.raises(ValueError):
        ctx.set_options(use_learned=2)
    ctx.set_options(use_learned=2, experimental=True)
    ctx.close()
