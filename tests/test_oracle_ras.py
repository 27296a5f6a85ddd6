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
