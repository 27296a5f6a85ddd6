"""Pins of the oracle's Yee operators against exact discrete identities.

Sec. III-A, Eq. (6) (curl) and the double-curl M; Sec. II-A Eq. (7).
"""
import numpy as np
import pytest

from oracle import yee
from paper_2508_07193_b300 import workloads as wl

GRIDS = [(3, 3, 3), (4, 3, 5), (6, 5, 4)]


@pytest.mark.parametrize("g", GRIDS)
def test_div_curl_and_curl_grad_vanish_exactly(g):
    C, G, Dv = yee.curl_matrix(g), yee.gradient_matrix(g), yee.divergence_matrix(g)
    assert abs(C @ G).max() == 0.0
    assert abs(Dv @ C).max() == 0.0
    K = yee.double_curl(g)
    assert abs(K @ G).max() == 0.0


@pytest.mark.parametrize("g", GRIDS)
def test_curl_has_four_unit_entries_per_interior_face(g):
    C = yee.curl_matrix(g).toarray()
    assert set(np.unique(C)) <= {-1.0, 0.0, 1.0}
    # a face fully inside the box touches four non-wall edges
    nx, ny, nz = g
    r = yee.slot(g, 2, 1, 1, 1)   # Hz at (1.5, 1.5, 1)
    assert np.count_nonzero(C[r]) == 4


@pytest.mark.parametrize("g", GRIDS)
def test_double_curl_symmetric_and_diagonal(g):
    K = yee.double_curl(g)
    assert abs(K - K.T).max() == 0.0
    # interior edge: 4 faces touch it -> diagonal 4
    assert K[yee.slot(g, 0, 1, 1, 1), yee.slot(g, 0, 1, 1, 1)] == 4.0


def test_double_curl_is_grad_div_minus_laplacian_on_interior_edge():
    # (curl curl E)_x = d_x(div E) - lap E_x : at an interior Ex edge the
    # stencil is 4 on itself, -1 on its four y/z neighbours, and the mixed
    # second differences +-1 on the Ey and Ez edges around it.
    g = (5, 5, 5)
    K = yee.double_curl(g).toarray()
    S = lambda c, k, j, i: yee.slot(g, c, k, j, i)
    row = K[S(0, 2, 2, 2)]
    expect = {S(0, 2, 2, 2): 4, S(0, 2, 3, 2): -1, S(0, 2, 1, 2): -1, S(0, 3, 2, 2): -1, S(0, 1, 2, 2): -1,
              S(1, 2, 2, 3): 1, S(1, 2, 2, 2): -1, S(1, 2, 1, 3): -1, S(1, 2, 1, 2): 1,
              S(2, 2, 2, 3): 1, S(2, 2, 2, 2): -1, S(2, 1, 2, 3): -1, S(2, 1, 2, 2): 1}
    got = {int(c): row[c] for c in np.flatnonzero(row)}
    assert got == expect


def test_system_matrix_spd_with_gershgorin_bounds():
    g = (5, 4, 4)
    rng = np.random.default_rng(3)
    eps_cell = rng.uniform(1, 10, (4, 4, 5))
    ee = yee.edge_eps(g, eps_cell)
    beta = 0.25
    A = yee.system_matrix(g, ee, beta)
    u = yee.unknowns(g)
    ev = np.linalg.eigvalsh(A[u][:, u].toarray())
    e = ee.reshape(-1)[u]
    assert ev.min() >= e.min() - 1e-12
    assert ev.max() <= e.max() + 12 * beta + 1e-12   # ||K|| <= 12 (Gershgorin: 4 + 8)


def test_edge_eps_mean_of_four_cells():
    g = (3, 3, 3)
    eps = np.arange(27, dtype=float).reshape(3, 3, 3) + 1
    ee = yee.edge_eps(g, eps)
    # Ex at (i+1/2, j=1, k=1), i=0: cells (0, 0|1, 0|1)
    assert ee[0, 1, 1, 0] == np.mean([eps[0, 0, 0], eps[0, 1, 0], eps[1, 0, 0], eps[1, 1, 0]])
    assert ee[0, 0, 1, 0] == 0.0 and ee[1, 1, 1, 0] == 0.0 and ee[2, 1, 0, 1] == 0.0


def test_operator_apply_matches_matrix_and_zeroes_walls():
    w = wl.small(grid=(6, 5, 4), cuts=((6,), (5,), (4,)))
    ee = yee.edge_eps(w.grid, w.eps_cell)
    y = yee.operator_apply(w.grid, ee, w.rhs, 1.0, 0.25)
    A = yee.system_matrix(w.grid, ee, 0.25)
    assert np.allclose(y.reshape(-1), A @ w.rhs.reshape(-1))
    assert np.all(y[wl.edge_wall_mask(w.grid)] == 0)


def test_curl_transpose_pair():
    g = (4, 5, 3)
    rng = np.random.default_rng(5)
    E = rng.standard_normal((3, 3, 5, 4)); E[wl.edge_wall_mask(g)] = 0
    H = rng.standard_normal((3, 3, 5, 4)); H[wl.face_wall_mask(g)] = 0
    assert np.isclose(np.sum(yee.curl_apply(g, E) * H), np.sum(E * yee.curl_t_apply(g, H)))
