"""Compact-layout subdomain solve with the low-rank boundary correction
(oracle, test-only): Algorithm 1 in full, Sec. III-A Steps 1-4.

A compact box keeps every field component on the same n_x x n_y x n_z slots
of the global Yee grid; all of them are unknowns. Differences use the square
forward difference of Sec. III-A,
    D^f = -I + (superdiagonal of ones)     (n x n),
whose last row has no +1: the slot beyond the box reads as zero. With D_l^f
acting along axis l, the compact curl is
    (C E)_x = D_y^f Ez - D_z^f Ey,  (C E)_y = D_z^f Ex - D_x^f Ez,
    (C E)_z = D_x^f Ey - D_y^f Ex,
and the compact double curl is M = C^T C (D^b = -(D^f)^T), the matrix M of
Sec. III-A with its garbled entries read as the curl-curl they come from.

M misses, on each component's two low transverse faces, the face that lies
outside the box; Step 4's diagonal Lambda (delta in {0, 1, 2}: the number of
low transverse faces a slot sits on) restores it, so M + Lambda is the global
double curl restricted to the box. The box operator is
    A_box = eps_bar I + beta (M + Lambda)
and Algorithm 1 inverts it by the Woodbury formula around the transform solve
of A_M = eps_bar I + beta M:
    E = A_M^{-1} R;  E <- E - A_M^{-1} Q C^{-1} Q^T E,
    C = W^{-1} + Q^T A_M^{-1} Q,  beta Lambda = Q W Q^T.
Q selects the slots with delta > 0 (6n^2 - 3n of them in a cube).

Slots of a box that are PEC walls of the global grid (tangential E on a low
global wall) lie on those same low faces. They are kept at zero by giving them
W^{-1} = 0 in C: the Woodbury step is then the exact solve with those slots
constrained to zero (a Lagrange multiplier per wall slot).

The transform tables come from numpy's SVD of D^f (D^f V = U S); the 3x3 per
mode is solved by dense LU.
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp

from . import yee


def difference(n):
    """Square forward difference D^f (Sec. III-A)."""
    return -np.eye(n) + np.eye(n, k=1)


def tables(n):
    """(U, sigma, V) with D^f V = U diag(sigma), from numpy's SVD."""
    U, s, Vt = np.linalg.svd(difference(n))
    return U, s, Vt.T


def _kron_axis(D, shape, axis):
    """Matrix of applying D along `axis` (0 = x, 1 = y, 2 = z) of a [nz][ny][nx] array."""
    nx, ny, nz = shape
    Ix, Iy, Iz = sp.identity(nx), sp.identity(ny), sp.identity(nz)
    Ds = sp.csr_matrix(D)
    if axis == 0:
        return sp.kron(Iz, sp.kron(Iy, Ds))
    if axis == 1:
        return sp.kron(Iz, sp.kron(Ds, Ix))
    return sp.kron(Ds, sp.kron(Iy, Ix))


def curl(shape):
    """Compact curl on a box of shape (nx, ny, nz): [3][nz][ny][nx] edges -> faces."""
    nx, ny, nz = shape
    Dx = _kron_axis(difference(nx), shape, 0)
    Dy = _kron_axis(difference(ny), shape, 1)
    Dz = _kron_axis(difference(nz), shape, 2)
    Z = sp.csr_matrix(Dx.shape)
    return sp.bmat([[Z, -Dz, Dy], [Dz, Z, -Dx], [-Dy, Dx, Z]]).tocsr()


def double_curl(shape):
    """M = C^T C for the compact box."""
    C = curl(shape)
    return (C.T @ C).tocsr()


def delta(shape):
    """Lambda's diagonal, [3][nz][ny][nx]: for component c, the number of its
    two transverse indices that are 0 (Step 4, 0-based)."""
    nx, ny, nz = shape
    k, j, i = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    return np.stack([(j == 0).astype(int) + (k == 0),
                     (i == 0).astype(int) + (k == 0),
                     (i == 0).astype(int) + (j == 0)]).astype(np.float64)


def box_slots(grid, lo, shape):
    """Global flat slot indices of a box [lo, lo + shape) in [3][nz][ny][nx] order."""
    nx, ny, nz = shape
    k, j, i = np.meshgrid(np.arange(nz) + lo[2], np.arange(ny) + lo[1], np.arange(nx) + lo[0], indexing="ij")
    return np.concatenate([yee.slot(grid, c, k, j, i).ravel() for c in range(3)])


def restricted_double_curl(grid, lo, shape):
    """The global double curl K restricted to the box's slots (wall rows and
    columns are zero in K)."""
    s = box_slots(grid, lo, shape)
    return yee.double_curl(grid)[s][:, s].tocsr()


def box_walls(grid, lo, shape):
    """[3][nz][ny][nx] boolean mask of the box slots that are global PEC walls."""
    return yee.edge_is_wall(grid)[box_slots(grid, lo, shape)].reshape((3, shape[2], shape[1], shape[0]))


# ---- transform solve of A_M = eps_bar I + beta M (Steps 1-3) ----------------

def _tr(T, F, axis):
    """Apply T (n_out x n_in) along axis (0 = x, 1 = y, 2 = z) of F[nz][ny][nx]."""
    ax = {0: 2, 1: 1, 2: 0}[axis]
    return np.moveaxis(np.tensordot(T, np.moveaxis(F, ax, 0), axes=(1, 0)), 0, ax)


def forward(R):
    """G R: component c takes U^T along its own axis and V^T along the others."""
    _, nz, ny, nx = R.shape
    tab = [tables(nx), tables(ny), tables(nz)]
    out = np.empty_like(R)
    for c in range(3):
        F = R[c]
        for a in range(3):
            U, _, V = tab[a]
            F = _tr((U if a == c else V).T, F, a)
        out[c] = F
    return out


def inverse(Rh):
    """G^{-1} = G^T."""
    _, nz, ny, nx = Rh.shape
    tab = [tables(nx), tables(ny), tables(nz)]
    out = np.empty_like(Rh)
    for c in range(3):
        F = Rh[c]
        for a in range(3):
            U, _, V = tab[a]
            F = _tr(U if a == c else V, F, a)
        out[c] = F
    return out


def block_matrices(shape, eps_bar, beta):
    """Per mode: eps_bar I + beta (|s|^2 I - s s^T), s = (sx, sy, sz), [mz][my][mx][3][3]."""
    nx, ny, nz = shape
    sx = tables(nx)[1][None, None, :]
    sy = tables(ny)[1][None, :, None]
    sz = tables(nz)[1][:, None, None]
    s = np.stack(np.broadcast_arrays(sx, sy, sz), axis=-1)
    B = beta * ((s * s).sum(-1)[..., None, None] * np.eye(3) - s[..., :, None] * s[..., None, :])
    return B + eps_bar * np.eye(3)


def transform_solve(R, eps_bar, beta):
    """A_M^{-1} R by Steps 1-3 (per-mode 3x3 by dense LU)."""
    _, nz, ny, nx = R.shape
    Rh = forward(R)
    B = block_matrices((nx, ny, nz), eps_bar, beta)
    rhs = np.moveaxis(Rh, 0, -1)[..., None]
    Eh = np.moveaxis(np.linalg.solve(B, rhs)[..., 0], -1, 0)
    return inverse(Eh)


# ---- Step 4: Woodbury correction ---------------------------------------------

def boundary(shape, walls=None):
    """Q's slots (flat indices into [3][nz][ny][nx]) and the diagonal of W^{-1}
    for them: 1 / (beta delta) is applied by the caller; wall slots get 0."""
    d = delta(shape).reshape(-1)
    q = np.flatnonzero(d > 0)
    wall = np.zeros(d.size, dtype=bool) if walls is None else np.asarray(walls).reshape(-1)
    return q, d[q], wall[q]


def correction_matrix(shape, eps_bar, beta, walls=None):
    """C = W^{-1} + Q^T A_M^{-1} Q, built from one transform solve per column."""
    nx, ny, nz = shape
    q, dq, wq = boundary(shape, walls)
    C = np.zeros((q.size, q.size))
    for a, s in enumerate(q):
        e = np.zeros(3 * nx * ny * nz)
        e[s] = 1.0
        C[:, a] = transform_solve(e.reshape(3, nz, ny, nx), eps_bar, beta).reshape(-1)[q]
    winv = np.where(wq, 0.0, 1.0 / (beta * dq))
    return C + np.diag(winv), q


def woodbury_solve(R, eps_bar, beta, walls=None):
    """Algorithm 1: E = exact_solve(R); E <- E - exact_solve(Q C^{-1} Q^T E).
    Slots flagged in `walls` must have R = 0; they come out zero."""
    _, nz, ny, nx = R.shape
    C, q = correction_matrix((nx, ny, nz), eps_bar, beta, walls)
    E = transform_solve(R, eps_bar, beta)
    cor = np.zeros(R.size)
    cor[q] = np.linalg.solve(C, E.reshape(-1)[q])
    return E - transform_solve(cor.reshape(R.shape), eps_bar, beta)


# ---- restricted additive Schwarz with compact boxes ---------------------------

def eps_bar(eps_edge, grid, lo, shape):
    """Mean edge permittivity over the box's non-wall slots."""
    s = box_slots(grid, lo, shape)
    keep = ~yee.edge_is_wall(grid)[s]
    return float(np.asarray(eps_edge).reshape(-1)[s][keep].mean())


def precond_apply(r, boxes, eps_edge, beta):
    """z = sum_i S_i^{0T} A_box_i^{-1} S_i r with compact boxes (Sec. II-B):
    each extended box is solved by Algorithm 1 and writes its owned slots."""
    grid = (r.shape[3], r.shape[2], r.shape[1])
    z = np.zeros_like(r)
    for b in boxes:
        lo = b.ext_lo
        shape = tuple(b.ext_hi[a] - b.ext_lo[a] for a in range(3))
        sl = (slice(None), slice(lo[2], lo[2] + shape[2]), slice(lo[1], lo[1] + shape[1]),
              slice(lo[0], lo[0] + shape[0]))
        walls = box_walls(grid, lo, shape)
        Rb = np.where(walls, 0.0, r[sl])
        Eb = woodbury_solve(Rb, eps_bar(eps_edge, grid, lo, shape), beta, walls)
        (x0, y0, z0), (x1, y1, z1) = b.own_lo, b.own_hi
        osl = (slice(None), slice(z0 - lo[2], z1 - lo[2]), slice(y0 - lo[1], y1 - lo[1]),
               slice(x0 - lo[0], x1 - lo[0]))
        z[:, z0:z1, y0:y1, x0:x1] = Eb[osl]
    z.reshape(-1)[yee.edge_is_wall(grid)] = 0.0
    return z
