"""Pins of the oracle's 1-D tables and axis transforms against closed forms.

Sec. III-A, Eq. (8): D^f = U S V^T; Eq. (9): TrX/TrY/TrZ.
"""
import numpy as np
import pytest

from oracle import transforms as tf


@pytest.mark.parametrize("m", [2, 3, 4, 7, 8, 17, 34, 36])
def test_sigma_matches_svd_of_rectangular_difference(m):
    # D: m cells x (m-1) interior nodes, (D v)_c = v_{c+1} - v_c, v_0 = v_m = 0.
    D = np.zeros((m, m - 1))
    for c in range(m):
        if c - 1 >= 0:
            D[c, c - 1] = -1.0      # node c   (interior index c-1)
        if c < m - 1:
            D[c, c] = 1.0           # node c+1 (interior index c)
    s = np.sort(np.linalg.svd(D, compute_uv=False))
    assert np.allclose(s, np.sort(tf.sigma(m)[1:]), atol=1e-13)


@pytest.mark.parametrize("n", [1, 2, 5, 8, 31])
def test_sigma_squared_are_dirichlet_laplacian_eigenvalues(n):
    # 1-D Dirichlet Laplacian on n interior nodes: eigenvalues 2 - 2 cos(pi k/(n+1)).
    L = 2 * np.eye(n) - np.eye(n, k=1) - np.eye(n, k=-1)
    ev = np.sort(np.linalg.eigvalsh(L))
    k = np.arange(1, n + 1)
    assert np.allclose(ev, 2 - 2 * np.cos(np.pi * k / (n + 1)), atol=1e-13)
    assert np.allclose(np.sort(tf.sigma(n + 1)[1:] ** 2), ev, atol=1e-13)


@pytest.mark.parametrize("m", [2, 3, 5, 8, 34, 36])
def test_tables_orthonormal(m):
    C = tf.dct2(m)
    S = tf.dst1(m)
    assert np.allclose(C @ C.T, np.eye(m), atol=1e-13)
    assert np.allclose(S[0], 0) and np.allclose(S[:, 0], 0)
    Si = S[1:, 1:]
    assert np.allclose(Si @ Si.T, np.eye(m - 1), atol=1e-13)


@pytest.mark.parametrize("m", [2, 3, 6, 9, 34])
def test_difference_factorises_with_positive_sigma(m):
    # D = U diag(sigma) V^T with U^T = C, V^T = S (padded): D = C^T diag(sigma) S.
    D = tf.difference(m)
    assert np.allclose(tf.dct2(m).T @ np.diag(tf.sigma(m)) @ tf.dst1(m), D, atol=1e-13)


def test_axis_transforms_match_explicit_loops():
    rng = np.random.default_rng(0)
    mz, my, mx = 3, 4, 5
    F = rng.standard_normal((mz, my, mx))
    Tx, Ty, Tz = (rng.standard_normal((m, m)) for m in (mx, my, mz))
    ox = np.zeros_like(F); oy = np.zeros_like(F); oz = np.zeros_like(F)
    for k in range(mz):
        for j in range(my):
            for i in range(mx):
                ox[k, j, i] = sum(Tx[i, q] * F[k, j, q] for q in range(mx))
                oy[k, j, i] = sum(Ty[j, q] * F[k, q, i] for q in range(my))
                oz[k, j, i] = sum(Tz[k, q] * F[q, j, i] for q in range(mz))
    assert np.allclose(tf.tr_x(Tx, F), ox)
    assert np.allclose(tf.tr_y(Ty, F), oy)
    assert np.allclose(tf.tr_z(Tz, F), oz)


def test_forward_inverse_roundtrip_on_non_wall_slots():
    rng = np.random.default_rng(1)
    from oracle.ras import box_wall
    m = (6, 5, 7)
    R = rng.standard_normal((3, m[2], m[1], m[0]))
    R[box_wall(m)] = 0.0
    tabs = tf.component_tables(*m)
    assert np.allclose(tf.inverse(tf.forward(R, tabs), tabs), R, atol=1e-13)
