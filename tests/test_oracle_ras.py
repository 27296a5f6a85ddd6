"""Pins of the oracle's restricted additive Schwarz preconditioner (Sec. II-B)."""
import numpy as np
import pytest

from oracle import ras, yee
from paper_2508_07193_b300 import workloads as wl


def test_single_box_constant_eps_is_exact_inverse():
    g = (7, 6, 5)
    rng = np.random.default_rng(2)
    r = rng.uniform(-1, 1, (3, 5, 6, 7)); r[wl.edge_wall_mask(g)] = 0
    ee = yee.edge_eps(g, np.full((5, 6, 7), 2.5))
    boxes = ras.partition(g, ((7,), (6,), (5,)), overlap=2)
    z = ras.precond_apply(r, boxes, ee, 0.25)
    A = yee.system_matrix(g, ee, 0.25)
    assert np.linalg.norm(A @ z.reshape(-1) - r.reshape(-1)) <= 1e-13 * np.linalg.norm(r)


def test_partition_owns_every_cell_once_and_clips():
    g = (20, 18, 14)
    boxes = ras.partition(g, ((7, 6, 7), (9, 9), (5, 9)), overlap=2)
    owner = np.zeros((14, 18, 20), int)
    for b in boxes:
        (x0, y0, z0), (x1, y1, z1) = b.own_lo, b.own_hi
        owner[z0:z1, y0:y1, x0:x1] += 1
        for a in range(3):
            assert b.ext_lo[a] == max(0, b.own_lo[a] - 2)
            assert b.ext_hi[a] == min(g[a], b.own_hi[a] + 2)
    assert np.all(owner == 1)
    assert len(boxes) == 12


def test_ras_equals_explicit_matrix_sum():
    # M^{-1} = sum_i S0_i^T A_i^{-1} S_i with A_i^{-1} the dense inverse of the
    # assembled box operator: compare column by column on a tiny problem.
    g = (6, 5, 4)
    rng = np.random.default_rng(4)
    eps = rng.uniform(1, 10, (4, 5, 6))
    ee = yee.edge_eps(g, eps)
    beta = 0.25
    boxes = ras.partition(g, ((3, 3), (2, 3), (4,)), overlap=1)
    r = rng.uniform(-1, 1, (3, 4, 5, 6)); r[wl.edge_wall_mask(g)] = 0
    z = ras.precond_apply(r, boxes, ee, beta)
    z_ref = np.zeros_like(r)
    for b in boxes:
        m = b.m
        rb = ras.restrict(r, b)
        Ab = yee.system_matrix(m, np.full(rb.shape, ras.eps_bar(ee, b)), beta)
        u = yee.unknowns(m)
        xb = np.zeros(rb.size)
        xb[u] = np.linalg.solve(Ab[u][:, u].toarray(), rb.reshape(-1)[u])
        ras.prolong_owned(z_ref, xb.reshape(rb.shape), b)
    assert np.abs(z - z_ref).max() <= 1e-13 * np.abs(z_ref).max()


def test_eps_bar_is_mean_over_interior_edges():
    g = (6, 5, 4)
    eps = np.full((4, 5, 6), 3.0)
    ee = yee.edge_eps(g, eps)
    b = ras.partition(g, ((6,), (5,), (4,)), overlap=0)[0]
    assert ras.eps_bar(ee, b) == pytest.approx(3.0, abs=1e-15)


def test_eps_bar_brute_force_over_box_edges():
    # mean over the extended box's interior edges, enumerated edge by edge
    g = (7, 6, 5)
    rng = np.random.default_rng(9)
    ee = yee.edge_eps(g, rng.uniform(1, 10, (5, 6, 7)))
    b = ras.partition(g, ((3, 4), (6,), (2, 3)), overlap=1)[3]
    (x0, y0, z0), (x1, y1, z1) = b.ext_lo, b.ext_hi
    vals = []
    for c in range(3):
        for k in range(z0, z1):
            for j in range(y0, y1):
                for i in range(x0, x1):
                    on_wall = [(j == y0) or (k == z0), (i == x0) or (k == z0), (i == x0) or (j == y0)][c]
                    if not on_wall:
                        vals.append(ee[c, k, j, i])
    assert ras.eps_bar(ee, b) == pytest.approx(np.mean(vals), rel=1e-14)


def _cut_edges(sizes):
    """Owned cell intervals [a, a + n) of one axis, from its cut sizes."""
    out, a = [], 0
    for n in sizes:
        out.append((a, a + n))
        a += n
    return out


RAGGED = ((11, 9, 7), ((4, 3, 4), (5, 4), (2, 5)), 2)


def test_restrict_slot_by_slot_on_clipped_ragged_boxes():
    """S_i^gamma enumerated slot by slot with plain index loops, using neither
    restrict nor the partition's boxes: every slot of a box's extended array
    holds the global slot at (extended low corner + local index), the
    extended corner being the owned corner minus gamma clipped at 0, and the
    box's own wall slots (local j = 0 or k = 0 for Ex, i = 0 or k = 0 for Ey,
    i = 0 or j = 0 for Ez) are 0. Global values are distinct, so a shifted
    or transposed copy fails."""
    g, cuts, ov = RAGGED
    nx, ny, nz = g
    r = np.arange(1, 3 * nz * ny * nx + 1, dtype=np.float64).reshape(3, nz, ny, nx)
    boxes = ras.partition(g, cuts, ov)
    t = 0
    for (az, bz) in _cut_edges(cuts[2]):
        for (ay, by) in _cut_edges(cuts[1]):
            for (ax, bx) in _cut_edges(cuts[0]):
                lo = (max(0, ax - ov), max(0, ay - ov), max(0, az - ov))
                hi = (min(nx, bx + ov), min(ny, by + ov), min(nz, bz + ov))
                rb = ras.restrict(r, boxes[t])
                assert rb.shape == (3, hi[2] - lo[2], hi[1] - lo[1], hi[0] - lo[0])
                for c in range(3):
                    for kl in range(hi[2] - lo[2]):
                        for jl in range(hi[1] - lo[1]):
                            for il in range(hi[0] - lo[0]):
                                wall = ((jl == 0 or kl == 0), (il == 0 or kl == 0), (il == 0 or jl == 0))[c]
                                want = 0.0 if wall else r[c, lo[2] + kl, lo[1] + jl, lo[0] + il]
                                assert rb[c, kl, jl, il] == want, (t, c, kl, jl, il)
                t += 1
    assert t == len(boxes)


def test_prolong_owned_slot_by_slot_on_clipped_ragged_boxes():
    """S_i^0T enumerated slot by slot: each global slot (c, k, j, i) receives
    the value that its owning box (the one whose owned cell intervals contain
    (i, j, k), found by walking the cut sizes) holds at local index
    (i, j, k) - that box's extended low corner. Box-local values encode
    (box, local slot), so taking the owned corner for the extended one, or
    writing overlap cells, fails."""
    g, cuts, ov = RAGGED
    nx, ny, nz = g
    boxes = ras.partition(g, cuts, ov)
    sols = []
    z = np.zeros((3, nz, ny, nx))
    for t, b in enumerate(boxes):
        m = b.m
        eb = (1000.0 * (t + 1) + np.arange(3 * m[2] * m[1] * m[0], dtype=np.float64)).reshape(3, m[2], m[1], m[0])
        sols.append(eb)
        ras.prolong_owned(z, eb, b)
    ex, ey, ez = (_cut_edges(c) for c in cuts)

    def owner(v, edges):
        for q, (a, b) in enumerate(edges):
            if a <= v < b:
                return q, a
        raise AssertionError(v)
    for c in range(3):
        for k in range(nz):
            qz, az = owner(k, ez)
            for j in range(ny):
                qy, ay = owner(j, ey)
                for i in range(nx):
                    qx, ax = owner(i, ex)
                    t = (qz * len(ey) + qy) * len(ex) + qx
                    lo = (max(0, ax - ov), max(0, ay - ov), max(0, az - ov))
                    assert z[c, k, j, i] == sols[t][c, k - lo[2], j - lo[1], i - lo[0]], (c, k, j, i)
