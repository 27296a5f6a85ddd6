"""Seeded synthetic inputs for the Crank-Nicolson Yee-grid workloads.

This module only draws random numbers and lays them out; it holds none of the
method's arithmetic (no operator, no transform, no averaging, no partition
geometry). Both the CUDA path and the CPU oracle take their inputs from here.

Layout conventions (shared contract of every field array):

* A grid has ``nx, ny, nz`` cells with unit spacing.
* Cell arrays are ``[nz][ny][nx]`` float64, x fastest.
* Edge fields (E, b, J) are ``[3][nz][ny][nx]`` float64. Slot ``(c, k, j, i)``
  is Ex(i+1/2, j, k), Ey(i, j+1/2, k) or Ez(i, j, k+1/2). Slots lying on the
  perfectly conducting walls (Ex: j == 0 or k == 0; Ey: i == 0 or k == 0;
  Ez: i == 0 or j == 0) hold zero; the walls at j == ny etc. are not stored.
* Face fields (H) are ``[3][nz][ny][nx]``: Hx(i, j+1/2, k+1/2) etc., with the
  wall faces Hx at i == 0, Hy at j == 0, Hz at k == 0 held at zero.

Draw order for a workload (one ``numpy.random.default_rng(seed)``): partition
cuts (uneven workloads only, axes x, y, z), then the permittivity boxes, then
the right-hand side.
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np

EPS_LO, EPS_HI = 1.0, 10.0
CUT_CHOICES = (24, 32, 40, 48, 64)


def edge_wall_mask(grid):
    """Boolean ``[3][nz][ny][nx]`` mask of the PEC wall slots (layout rule)."""
    nx, ny, nz = grid
    k = np.arange(nz)[:, None, None]
    j = np.arange(ny)[None, :, None]
    i = np.arange(nx)[None, None, :]
    m = np.zeros((3, nz, ny, nx), dtype=bool)
    m[0] = (j == 0) | (k == 0)
    m[1] = (i == 0) | (k == 0)
    m[2] = (i == 0) | (j == 0)
    return m


def face_wall_mask(grid):
    """Boolean ``[3][nz][ny][nx]`` mask of the wall faces (layout rule)."""
    nx, ny, nz = grid
    k = np.arange(nz)[:, None, None]
    j = np.arange(ny)[None, :, None]
    i = np.arange(nx)[None, None, :]
    m = np.zeros((3, nz, ny, nx), dtype=bool)
    m[0] = np.broadcast_to(i == 0, (nz, ny, nx))
    m[1] = np.broadcast_to(j == 0, (nz, ny, nx))
    m[2] = np.broadcast_to(k == 0, (nz, ny, nx))
    return m


def draw_eps_boxes(rng, grid, n_boxes):
    """Piecewise-constant relative permittivity per cell.

    Background 1; each box has a low corner uniform in [0, N) per axis, a size
    uniform in [N/8, N/2] per axis (clipped at the grid), a value uniform in
    [1, 10]; later boxes overwrite earlier ones.
    """
    nx, ny, nz = grid
    eps = np.ones((nz, ny, nx), dtype=np.float64)
    dims = (nx, ny, nz)
    for _ in range(n_boxes):
        lo = [int(rng.integers(0, n)) for n in dims]
        size = [int(rng.integers(max(1, n // 8), n // 2 + 1)) for n in dims]
        val = float(rng.uniform(EPS_LO, EPS_HI))
        eps[lo[2]:lo[2] + size[2], lo[1]:lo[1] + size[1], lo[0]:lo[0] + size[0]] = val
    return eps


def draw_rhs(rng, grid):
    """Right-hand side uniform in [-1, 1] per slot, wall slots zeroed."""
    nx, ny, nz = grid
    b = rng.uniform(-1.0, 1.0, size=(3, nz, ny, nx))
    b[edge_wall_mask(grid)] = 0.0
    return b


def draw_cuts(rng, n_cells, choices=CUT_CHOICES, max_tries=100000):
    """Owned subdomain sizes along one axis, drawn from ``choices``.

    Sizes are drawn until their sum reaches ``n_cells``; the draw is kept only
    if the sum is exactly ``n_cells``, otherwise the axis is drawn again.
    """
    for _ in range(max_tries):
        sizes = []
        while sum(sizes) < n_cells:
            sizes.append(int(choices[int(rng.integers(0, len(choices)))]))
        if sum(sizes) == n_cells:
            return sizes
    raise RuntimeError(f"could not partition {n_cells} cells from {choices}")


def even_cuts(n_cells, n_parts):
    """Equal owned sizes (the last part takes the remainder)."""
    base = n_cells // n_parts
    cuts = [base] * n_parts
    cuts[-1] += n_cells - base * n_parts
    return cuts


@dataclasses.dataclass
class Workload:
    """One seeded problem instance: grid, materials, partition and rhs."""
    name: str
    grid: tuple            # (nx, ny, nz) cells
    beta: float            # (c dt / 2h)^2 in grid units
    eps_cell: np.ndarray | None   # [nz][ny][nx] or None for eps == 1
    cuts: tuple            # per-axis owned sizes, (cx, cy, cz)
    overlap: int
    rhs: np.ndarray        # [3][nz][ny][nx]
    seed: int

    @property
    def n_slots(self):
        nx, ny, nz = self.grid
        return 3 * nx * ny * nz

    @property
    def n_boxes(self):
        return len(self.cuts[0]) * len(self.cuts[1]) * len(self.cuts[2])


def make_workload(name, grid, *, seed, n_eps_boxes=16, cuts=None, overlap=2,
                  beta=0.25, uneven=False, uniform_eps=False):
    """Build a workload with the draw order stated in the module docstring."""
    rng = np.random.default_rng(seed)
    nx, ny, nz = grid
    if uneven:
        cuts = tuple(tuple(draw_cuts(rng, n)) for n in (nx, ny, nz))
    elif cuts is None:
        cuts = ((nx,), (ny,), (nz,))
    else:
        cuts = tuple(tuple(int(v) for v in c) for c in cuts)
    for c, n in zip(cuts, grid):
        if sum(c) != n:
            raise ValueError(f"cuts {c} do not sum to {n}")
    eps = None if uniform_eps else draw_eps_boxes(rng, grid, n_eps_boxes)
    rhs = draw_rhs(rng, grid)
    return Workload(name, tuple(grid), float(beta), eps, cuts, int(overlap), rhs, seed)


# The five named workloads. Sizes, seeds and structure follow the problem
# statement: one PEC box; 128^3 with 4^3 subdomains; 256^3 with 8^3
# subdomains; an uneven 320x256x192 partition; the 256^3 dipole run.

def box32(seed=0):
    """32^3 PEC box, eps == 1, beta = 0.25, rhs uniform[-1,1] from seed 0."""
    return make_workload("box32_pec_eps1", (32, 32, 32), seed=seed,
                         uniform_eps=True, overlap=0)


def grid128(seed=1):
    """128^3, 16 eps boxes in [1,10], 4x4x4 subdomains of 32^3, overlap 2."""
    return make_workload("yee128_ras4x4x4_ol2", (128, 128, 128), seed=seed,
                         n_eps_boxes=16, cuts=[even_cuts(128, 4)] * 3, overlap=2)


def grid256(seed=2):
    """256^3, 16 eps boxes, 8x8x8 subdomains of 32^3, overlap 2."""
    return make_workload("yee256_ras8x8x8_ol2", (256, 256, 256), seed=seed,
                         n_eps_boxes=16, cuts=[even_cuts(256, 8)] * 3, overlap=2)


def grid_uneven(seed=3):
    """320x256x192, uneven cuts from {24,32,40,48,64}, 32 eps boxes, overlap 2."""
    return make_workload("yee320x256x192_uneven_ol2", (320, 256, 192), seed=seed,
                         n_eps_boxes=32, uneven=True, overlap=2)


def small(grid=(20, 18, 14), cuts=((7, 6, 7), (9, 9), (5, 9)), overlap=2, seed=7,
          n_eps_boxes=4, beta=0.25):
    """A small ragged workload for parity tests (several boxes, odd extents)."""
    return make_workload("small", grid, seed=seed, n_eps_boxes=n_eps_boxes,
                         cuts=cuts, overlap=overlap, beta=beta)


# Dipole source: a z-directed current on the single Ez edge nearest the grid
# centre, a Gaussian-modulated sine at 20 cells per wavelength (c = h = 1).

DIPOLE_CELLS_PER_WAVELENGTH = 20.0


def dipole_waveform(t, cells_per_wavelength=DIPOLE_CELLS_PER_WAVELENGTH):
    """J(t) = sin(2 pi f0 (t - t0)) exp(-((t - t0)/tau)^2), f0 = 1/20, tau = 1/f0, t0 = 3 tau."""
    f0 = 1.0 / cells_per_wavelength
    tau = 1.0 / f0
    t0 = 3.0 * tau
    return math.sin(2.0 * math.pi * f0 * (t - t0)) * math.exp(-((t - t0) / tau) ** 2)


def dipole_slot(grid):
    """Slot (c, k, j, i) of the Ez edge carrying the dipole current."""
    nx, ny, nz = grid
    return (2, nz // 2, ny // 2, nx // 2)


def dipole_current(grid, step, dt):
    """Full ``[3][nz][ny][nx]`` current density at time (step + 1/2) dt."""
    J = np.zeros((3,) + tuple(reversed(grid)), dtype=np.float64)
    J[dipole_slot(grid)] = dipole_waveform((step + 0.5) * dt)
    return J
