"""Yee-grid incidence matrices and the double-curl system (oracle, test-only).

Sec. II-A, Eqs. (1)-(5): the Crank-Nicolson update leads to
(I + (dt^2/4) curl curl) E = R. Sec. III-A, Eq. (6) writes the curl with
forward/backward differences and Eq. (7) the system (I + alpha M) E = R.

Discretisation (reading of the paper, which normalises eps = mu = 1 and fixes
no boundary): a Yee grid of nx*ny*nz unit cells inside a perfectly conducting
box. E lives on edges, H on faces; tangential E and normal H vanish on the
walls. The system solved is A = diag(eps_edge) + beta * K with K = C^T C, where
C is the edge-to-face incidence (discrete curl), beta = (dt/2)^2; with eps = 1
this is exactly Eq. (7) with alpha = beta.

All matrices act on full slot vectors of length 3*nx*ny*nz (layout of
``paper_2508_07193_b300.workloads``); columns and rows of wall slots are
dropped, so wall slots map to zero.
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp


def _ijk(grid):
    nx, ny, nz = grid
    k, j, i = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    return i.ravel(), j.ravel(), k.ravel()


def slot(grid, c, k, j, i):
    """Flat index of slot (c, k, j, i) in a [3][nz][ny][nx] array."""
    nx, ny, nz = grid
    return ((c * nz + k) * ny + j) * nx + i


def edge_is_wall(grid):
    """Flat boolean mask of PEC edge slots (tangential E = 0 on the walls)."""
    nx, ny, nz = grid
    i, j, k = _ijk(grid)
    return np.concatenate([(j == 0) | (k == 0), (i == 0) | (k == 0), (i == 0) | (j == 0)])


def face_is_wall(grid):
    """Flat boolean mask of wall faces (normal H = 0 on the walls)."""
    i, j, k = _ijk(grid)
    return np.concatenate([i == 0, j == 0, k == 0])


def node_is_wall(grid):
    """Flat boolean mask of wall nodes for a [nz][ny][nx] node array."""
    i, j, k = _ijk(grid)
    return (i == 0) | (j == 0) | (k == 0)


def _coo(grid, entries, n_rows, n_cols, col_wall, row_wall=None):
    """Assemble a CSR matrix from (row, col, val, valid) lists, dropping wall
    columns (and rows) and out-of-range neighbours."""
    rows, cols, vals = [], [], []
    for r, c, v, ok in entries:
        rows.append(r[ok]); cols.append(c[ok]); vals.append(np.full(int(ok.sum()), v, dtype=np.float64))
    rows = np.concatenate(rows); cols = np.concatenate(cols); vals = np.concatenate(vals)
    keep = ~col_wall[cols]
    if row_wall is not None:
        keep &= ~row_wall[rows]
    return sp.csr_matrix((vals[keep], (rows[keep], cols[keep])), shape=(n_rows, n_cols))


def curl_matrix(grid):
    """Discrete curl C: edges -> faces (Eq. 6, with the row-2 typo read as dz Ex - dx Ez).

    (CE)_x at face (i, j+1/2, k+1/2) = [Ez(j+1) - Ez(j)] - [Ey(k+1) - Ey(k)]
    (CE)_y at face (i+1/2, j, k+1/2) = [Ex(k+1) - Ex(k)] - [Ez(i+1) - Ez(i)]
    (CE)_z at face (i+1/2, j+1/2, k) = [Ey(i+1) - Ey(i)] - [Ex(j+1) - Ex(j)]
    Edges beyond the high walls are wall edges (zero) and are dropped.
    """
    nx, ny, nz = grid
    n = nx * ny * nz
    i, j, k = _ijk(grid)
    S = lambda c, kk, jj, ii: slot(grid, c, kk, jj, ii)
    true = np.ones_like(i, dtype=bool)
    e = []
    # face x rows: c = 0
    r = S(0, k, j, i)
    e += [(r, S(2, k, np.minimum(j + 1, ny - 1), i), +1.0, j + 1 < ny),
          (r, S(2, k, j, i), -1.0, true),
          (r, S(1, np.minimum(k + 1, nz - 1), j, i), -1.0, k + 1 < nz),
          (r, S(1, k, j, i), +1.0, true)]
    r = S(1, k, j, i)
    e += [(r, S(0, np.minimum(k + 1, nz - 1), j, i), +1.0, k + 1 < nz),
          (r, S(0, k, j, i), -1.0, true),
          (r, S(2, k, j, np.minimum(i + 1, nx - 1)), -1.0, i + 1 < nx),
          (r, S(2, k, j, i), +1.0, true)]
    r = S(2, k, j, i)
    e += [(r, S(1, k, j, np.minimum(i + 1, nx - 1)), +1.0, i + 1 < nx),
          (r, S(1, k, j, i), -1.0, true),
          (r, S(0, k, np.minimum(j + 1, ny - 1), i), -1.0, j + 1 < ny),
          (r, S(0, k, j, i), +1.0, true)]
    return _coo(grid, e, 3 * n, 3 * n, edge_is_wall(grid))


def gradient_matrix(grid):
    """Discrete gradient G: nodes -> edges (phi = 0 on the wall nodes)."""
    nx, ny, nz = grid
    n = nx * ny * nz
    i, j, k = _ijk(grid)
    node = lambda kk, jj, ii: (kk * ny + jj) * nx + ii
    S = lambda c: slot(grid, c, k, j, i)
    true = np.ones_like(i, dtype=bool)
    e = [(S(0), node(k, j, np.minimum(i + 1, nx - 1)), +1.0, i + 1 < nx),
         (S(0), node(k, j, i), -1.0, true),
         (S(1), node(k, np.minimum(j + 1, ny - 1), i), +1.0, j + 1 < ny),
         (S(1), node(k, j, i), -1.0, true),
         (S(2), node(np.minimum(k + 1, nz - 1), j, i), +1.0, k + 1 < nz),
         (S(2), node(k, j, i), -1.0, true)]
    return _coo(grid, e, 3 * n, n, node_is_wall(grid), row_wall=edge_is_wall(grid))


def divergence_matrix(grid):
    """Discrete divergence Dv: faces -> cells."""
    nx, ny, nz = grid
    n = nx * ny * nz
    i, j, k = _ijk(grid)
    cell = (k * ny + j) * nx + i
    S = lambda c, kk, jj, ii: slot(grid, c, kk, jj, ii)
    true = np.ones_like(i, dtype=bool)
    e = [(cell, S(0, k, j, np.minimum(i + 1, nx - 1)), +1.0, i + 1 < nx),
         (cell, S(0, k, j, i), -1.0, true),
         (cell, S(1, k, np.minimum(j + 1, ny - 1), i), +1.0, j + 1 < ny),
         (cell, S(1, k, j, i), -1.0, true),
         (cell, S(2, np.minimum(k + 1, nz - 1), j, i), +1.0, k + 1 < nz),
         (cell, S(2, k, j, i), -1.0, true)]
    return _coo(grid, e, n, 3 * n, face_is_wall(grid))


def double_curl(grid):
    """K = C^T C on edge slots (the matrix M of Sec. III-A, symmetric)."""
    C = curl_matrix(grid)
    return (C.T @ C).tocsr()


def edge_eps(grid, eps_cell):
    """Permittivity per edge: the mean of the four cells sharing the edge.

    The paper normalises eps = 1 (Sec. II-A); with a cell-wise eps the edge
    value is the arithmetic mean of its four neighbour cells. Wall slots get 0.
    """
    nx, ny, nz = grid
    out = np.zeros((3, nz, ny, nx))
    if eps_cell is None:
        out[:] = 1.0
        out.reshape(-1)[edge_is_wall(grid)] = 0.0
        return out
    e = np.asarray(eps_cell, dtype=np.float64)
    # Ex(i+1/2, j, k): cells (i, j-1|j, k-1|k)
    out[0, 1:, 1:, :] = 0.25 * (e[:-1, :-1, :] + e[:-1, 1:, :] + e[1:, :-1, :] + e[1:, 1:, :])
    # Ey(i, j+1/2, k): cells (i-1|i, j, k-1|k)
    out[1, 1:, :, 1:] = 0.25 * (e[:-1, :, :-1] + e[:-1, :, 1:] + e[1:, :, :-1] + e[1:, :, 1:])
    # Ez(i, j, k+1/2): cells (i-1|i, j-1|j, k)
    out[2, :, 1:, 1:] = 0.25 * (e[:, :-1, :-1] + e[:, :-1, 1:] + e[:, 1:, :-1] + e[:, 1:, 1:])
    return out


def system_matrix(grid, eps_edge, beta):
    """A = diag(eps_edge) + beta * K on all slots (wall rows/cols zero)."""
    K = double_curl(grid)
    wall = edge_is_wall(grid)
    d = np.where(wall, 0.0, np.asarray(eps_edge, dtype=np.float64).reshape(-1))
    return (sp.diags(d) + beta * K).tocsr()


def unknowns(grid):
    """Flat indices of the non-wall edge slots (the unknowns)."""
    return np.flatnonzero(~edge_is_wall(grid))


def operator_apply(grid, eps_edge, x, c_eps, c_k):
    """y = c_eps * eps o x + c_k * K x on a [3][nz][ny][nx] field; walls -> 0."""
    K = double_curl(grid)
    wall = edge_is_wall(grid)
    xf = np.asarray(x, dtype=np.float64).reshape(-1).copy()
    xf[wall] = 0.0
    y = c_eps * np.asarray(eps_edge).reshape(-1) * xf + c_k * (K @ xf)
    y[wall] = 0.0
    return y.reshape(x.shape)


def curl_apply(grid, E):
    """H-shaped C E for an edge field E."""
    return (curl_matrix(grid) @ np.asarray(E).reshape(-1)).reshape(E.shape)


def curl_t_apply(grid, H):
    """Edge-shaped C^T H for a face field H (wall edges come out zero)."""
    C = curl_matrix(grid)
    y = C.T @ np.asarray(H).reshape(-1)
    y[edge_is_wall(grid)] = 0.0
    return y.reshape(H.shape)
