"""Pins of the oracle's subdomain exact solve (Algorithm 1, exact_solve).

* Sec. III-A Step 1 / Eq. (12): G K G^T is block diagonal with the per-mode
  blocks |sigma|^2 I - sigma sigma^T (brute force on small boxes).
* The transform solve equals a dense LU solve of the assembled PEC-box system
  (8^3 box) and has a tiny residual at 32^3.
"""
import numpy as np
import pytest
import scipy.sparse.linalg as spla

from oracle import box, ras, transforms as tf, yee


@pytest.mark.parametrize("m", [(3, 3, 3), (4, 3, 5), (5, 6, 4)])
def test_transformed_double_curl_is_block_diagonal(m):
    mx, my, mz = m
    G = tf.forward_matrix(mx, my, mz)
    K = yee.double_curl(m).toarray()
    T = G @ K @ G.T
    sx, sy, sz = tf.sigma(mx), tf.sigma(my), tf.sigma(mz)
    n = mx * my * mz
    expect = np.zeros_like(T)
    for kz in range(mz):
        for ky in range(my):
            for kx in range(mx):
                s = np.array([sx[kx], sy[ky], sz[kz]])
                blk = (s @ s) * np.eye(3) - np.outer(s, s)
                idx = [c * n + (kz * my + ky) * mx + kx for c in range(3)]
                expect[np.ix_(idx, idx)] = blk
    live = np.abs(G).sum(axis=1) > 0      # padded DST modes are empty rows of G
    expect *= live[:, None] * live[None, :]
    assert np.abs(T - expect).max() < 1e-13


def _dense_box_solve(m, eps_bar, beta, R):
    A = yee.system_matrix(m, np.full(R.shape, eps_bar), beta)
    u = yee.unknowns(m)
    x = np.zeros(R.size)
    x[u] = np.linalg.solve(A[u][:, u].toarray(), R.reshape(-1)[u])
    return x.reshape(R.shape)


@pytest.mark.parametrize("m,eps_bar,beta", [((8, 8, 8), 1.0, 0.25), ((7, 5, 6), 3.3, 0.25),
                                            ((4, 6, 5), 1.0, 25.0)])
def test_exact_solve_matches_dense_lu(m, eps_bar, beta):
    rng = np.random.default_rng(11)
    R = rng.uniform(-1, 1, (3, m[2], m[1], m[0]))
    R[ras.box_wall(m)] = 0.0
    E = box.exact_solve(R, eps_bar, beta)
    E_ref = _dense_box_solve(m, eps_bar, beta, R)
    assert np.abs(E - E_ref).max() <= 1e-13 * np.abs(E_ref).max()
    assert np.all(E[ras.box_wall(m)] == 0.0)


def test_exact_solve_32_residual():
    # the 32^3 PEC box workload (eps = 1, beta = 0.25, rhs from seed 0)
    from paper_2508_07193_b300 import workloads as wl
    w = wl.box32()
    g = w.grid
    E = box.exact_solve(w.rhs, 1.0, w.beta)
    A = yee.system_matrix(g, yee.edge_eps(g, None), w.beta)
    res = np.linalg.norm(A @ E.reshape(-1) - w.rhs.reshape(-1)) / np.linalg.norm(w.rhs)
    assert res <= 1e-13


def test_exact_solve_matches_spsolve_12():
    g = (12, 12, 12)
    rng = np.random.default_rng(12)
    R = rng.uniform(-1, 1, (3, 12, 12, 12)); R[ras.box_wall(g)] = 0
    E = box.exact_solve(R, 1.0, 0.25)
    A = yee.system_matrix(g, yee.edge_eps(g, None), 0.25)
    u = yee.unknowns(g)
    x = spla.spsolve(A[u][:, u].tocsc(), R.reshape(-1)[u])
    assert np.abs(E.reshape(-1)[u] - x).max() <= 1e-12


def test_block_matrices_are_the_printed_B():
    # B_ijk of Sec. III-A at one mode, written out entry by entry.
    B = box.block_matrices(4, 5, 6, 2.0, 0.5)
    sx, sy, sz = tf.sigma(4)[3], tf.sigma(5)[2], tf.sigma(6)[1]
    a = 0.5
    ref = 2.0 * np.eye(3) + a * np.array([[sy**2 + sz**2, -sx * sy, -sx * sz],
                                          [-sx * sy, sx**2 + sz**2, -sy * sz],
                                          [-sx * sz, -sy * sz, sx**2 + sy**2]])
    assert np.allclose(B[1, 2, 3], ref)
