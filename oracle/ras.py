"""Restricted additive Schwarz preconditioner (oracle, test-only).

Sec. II-B, "Domain Decomposition": M_RAS^{-1} = sum_i S_i^{0T} A_i^{-1} S_i^gamma,
with S_i^gamma the restriction to subdomain i extended by the overlap gamma and
S_i^0 the restriction to its non-overlapping (owned) part.

Readings taken here:
* Owned cells of box i are a tensor product of per-axis intervals [a, a+n);
  the extended box is [a - gamma, a + n + gamma) clipped to the grid.
* A_i is replaced by the exact inverse of eps_bar_i I + beta K_i, K_i the
  double-curl of the extended box with PEC walls, eps_bar_i the mean of
  eps_edge over the box's interior edge slots. (With constant eps this equals
  S_i A S_i^T exactly.)
* Slot (c, k, j, i) is owned by the box whose owned cell range contains cell
  (i, j, k); the prolongation overwrites, no averaging.
"""
from __future__ import annotations

import dataclasses

import numpy as np

from . import box as box_mod


@dataclasses.dataclass
class Box:
    own_lo: tuple   # (x, y, z) global cell index
    own_hi: tuple
    ext_lo: tuple
    ext_hi: tuple

    @property
    def m(self):
        return tuple(h - l for l, h in zip(self.ext_lo, self.ext_hi))


def partition(grid, cuts, overlap):
    """Boxes from per-axis owned sizes; ordered z-major, then y, then x."""
    bounds = []
    for n_cells, sizes in zip(grid, cuts):
        edges = np.concatenate([[0], np.cumsum(sizes)]).astype(int)
        assert edges[-1] == n_cells
        bounds.append([(int(edges[t]), int(edges[t + 1])) for t in range(len(sizes))])
    boxes = []
    for bz in bounds[2]:
        for by in bounds[1]:
            for bx in bounds[0]:
                lo = (bx[0], by[0], bz[0])
                hi = (bx[1], by[1], bz[1])
                elo = tuple(max(0, l - overlap) for l in lo)
                ehi = tuple(min(n, h + overlap) for h, n in zip(hi, grid))
                boxes.append(Box(lo, hi, elo, ehi))
    return boxes


def box_wall(m):
    """Boolean [3][mz][my][mx] mask of the extended box's own PEC wall slots."""
    mx, my, mz = m
    k = np.arange(mz)[:, None, None]
    j = np.arange(my)[None, :, None]
    i = np.arange(mx)[None, None, :]
    w = np.zeros((3, mz, my, mx), dtype=bool)
    w[0] = (j == 0) | (k == 0)
    w[1] = (i == 0) | (k == 0)
    w[2] = (i == 0) | (j == 0)
    return w


def restrict(r, b):
    """S_i^gamma: copy the extended box out of a global field, wall slots zeroed."""
    (x0, y0, z0), (x1, y1, z1) = b.ext_lo, b.ext_hi
    rb = np.array(r[:, z0:z1, y0:y1, x0:x1], dtype=np.float64)
    rb[box_wall(b.m)] = 0.0
    return rb


def prolong_owned(z, eb, b):
    """S_i^{0T}: write the owned cells of a box solution into the global field."""
    (x0, y0, z0) = b.ext_lo
    (ox0, oy0, oz0), (ox1, oy1, oz1) = b.own_lo, b.own_hi
    z[:, oz0:oz1, oy0:oy1, ox0:ox1] = eb[:, oz0 - z0:oz1 - z0, oy0 - y0:oy1 - y0, ox0 - x0:ox1 - x0]


def eps_bar(eps_edge, b):
    """Mean of eps_edge over the box's interior (non-wall) edge slots."""
    e = restrict(eps_edge, b)
    return float(e[~box_wall(b.m)].mean())


def precond_apply(r, boxes, eps_edge, beta):
    """z = M_RAS^{-1} r with per-box exact transform solves (Sec. II-B)."""
    z = np.zeros_like(r, dtype=np.float64)
    for b in boxes:
        eb = box_mod.exact_solve(restrict(r, b), eps_bar(eps_edge, b), beta)
        prolong_owned(z, eb, b)
    return z
