"""1-D transform tables and the tensor-product axis transforms (oracle, test-only).

Sec. III-A "Key Idea", Eq. (8): the forward difference operator is factored by
its SVD, D = U S V^T, and the backward difference reuses it (D^b = -V S U^T).

Reading for a Yee box of m cells per axis with PEC walls: along an axis, a
component that sits at nodes has m-1 interior nodes (node 0 and node m are
walls); its difference lands on the m cell centres. D is therefore the m x (m-1)
matrix (D v)_c = v_{c+1} - v_c (v_0 = v_m = 0). Its SVD has
  U = DCT-II vectors  C[k, i] = sqrt((2 - delta_k0)/m) cos(pi k (i + 1/2) / m),
  V = DST-I vectors   S[k, j] = sqrt(2/m) sin(pi k j / m),  j = 1..m-1,
  sigma_k = 2 sin(pi k / (2m)),   k = 0..m-1 (sigma_0 = 0 pairs with no V).
Both tables are stored m x m: S keeps the wall slot j = 0 and the empty mode
k = 0 as a zero column and row, so every component of a box has m^3 slots.

Eq. (9): TrX/TrY/TrZ contract one axis of an m_x x m_y x m_z tensor with a
square matrix. Arrays here are indexed [z][y][x].
"""
from __future__ import annotations

import numpy as np


def dct2(m):
    """Orthonormal DCT-II table C[k, i] (rows are the left singular vectors U^T)."""
    k = np.arange(m)[:, None]
    i = np.arange(m)[None, :]
    scale = np.where(k == 0, np.sqrt(1.0 / m), np.sqrt(2.0 / m))
    return scale * np.cos(np.pi * k * (i + 0.5) / m)


def dst1(m):
    """Zero-padded orthonormal DST-I table S[k, j] (rows are V^T), j, k in 0..m-1."""
    k = np.arange(m)[:, None]
    j = np.arange(m)[None, :]
    return np.sqrt(2.0 / m) * np.sin(np.pi * k * j / m)


def sigma(m):
    """Singular values sigma_k = 2 sin(pi k / 2m), k = 0..m-1 (sigma_0 = 0)."""
    return 2.0 * np.sin(np.pi * np.arange(m) / (2.0 * m))


def difference(m):
    """Padded forward difference D (m x m): cells <- nodes, column 0 is the wall node."""
    D = np.zeros((m, m))
    for c in range(m):
        if c >= 1:
            D[c, c] = -1.0
        if c + 1 < m:
            D[c, c + 1] = 1.0
    return D


def tr_x(T, F):
    """Eq. (9) TrX: out[k, j, a] = sum_i T[a, i] F[k, j, i]."""
    return np.einsum("ai,kji->kja", T, F)


def tr_y(T, F):
    """Eq. (9) TrY: out[k, b, i] = sum_j T[b, j] F[k, j, i]."""
    return np.einsum("bj,kji->kbi", T, F)


def tr_z(T, F):
    """Eq. (9) TrZ: out[c, j, i] = sum_k T[c, k] F[k, j, i]."""
    return np.einsum("ck,kji->cji", T, F)


def component_tables(mx, my, mz):
    """Per component (x, y, z) tables along (x, y, z), following the definition
    of G in Sec. III-A: Ex takes U^T along x and V^T along y, z; Ey takes U^T
    along y; Ez takes U^T along z."""
    Cx, Cy, Cz = dct2(mx), dct2(my), dct2(mz)
    Sx, Sy, Sz = dst1(mx), dst1(my), dst1(mz)
    return ((Cx, Sy, Sz), (Sx, Cy, Sz), (Sx, Sy, Cz))


def forward(R, tables):
    """G R for a [3][mz][my][mx] field (Sec. III-A Step 1): TrZ(TrY(TrX(.)))."""
    out = np.empty_like(R, dtype=np.float64)
    for c in range(3):
        Tx, Ty, Tz = tables[c]
        out[c] = tr_z(Tz, tr_y(Ty, tr_x(Tx, R[c])))
    return out


def inverse(Rh, tables):
    """G^{-1} = G^T applied to a transformed field (Sec. III-A Step 3)."""
    out = np.empty_like(Rh, dtype=np.float64)
    for c in range(3):
        Tx, Ty, Tz = tables[c]
        out[c] = tr_x(Tx.T, tr_y(Ty.T, tr_z(Tz.T, Rh[c])))
    return out


def forward_matrix(mx, my, mz):
    """Dense G (3 m^3 x 3 m^3) as Kronecker products, for brute-force checks."""
    blocks = []
    for Tx, Ty, Tz in component_tables(mx, my, mz):
        blocks.append(np.kron(Tz, np.kron(Ty, Tx)))
    n = mx * my * mz
    G = np.zeros((3 * n, 3 * n))
    for c in range(3):
        G[c * n:(c + 1) * n, c * n:(c + 1) * n] = blocks[c]
    return G
