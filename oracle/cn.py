"""Crank-Nicolson FDTD step (oracle, test-only).

Sec. II-A, Eqs. (2)-(4), with eps kept per edge (the paper sets eps = mu = 1)
and an impressed current J:
    eps (E^{n+1} - E^n)/dt =  1/2 C^T (H^{n+1} + H^n) - J^{n+1/2}
        (H^{n+1} - H^n)/dt = -1/2 C (E^{n+1} + E^n)
Eliminating H^{n+1} gives Eq. (4)/(5):
    (eps + beta K) E^{n+1} = (eps - beta K) E^n + dt C^T H^n - dt J,  beta = dt^2/4,
after which H^{n+1} = H^n - (dt/2) C (E^{n+1} + E^n).
"""
from __future__ import annotations

import numpy as np
import scipy.sparse.linalg as spla

from . import yee


def rhs(grid, eps_edge, E, H, J, dt):
    """R = (eps - beta K) E + dt C^T H - dt J (walls zero)."""
    beta = dt * dt / 4.0
    R = yee.operator_apply(grid, eps_edge, E, 1.0, -beta) + dt * yee.curl_t_apply(grid, H)
    if J is not None:
        R = R - dt * J
    R.reshape(-1)[yee.edge_is_wall(grid)] = 0.0
    return R


def h_update(grid, H, E_new, E_old, dt):
    """H^{n+1} = H^n - (dt/2) C (E^{n+1} + E^n) (Eq. 3)."""
    return H - 0.5 * dt * yee.curl_apply(grid, E_new + E_old)


def step(grid, eps_edge, E, H, J, dt, solve=None):
    """One CN step; ``solve(A_sparse, R_flat_unknowns)`` defaults to spsolve."""
    beta = dt * dt / 4.0
    R = rhs(grid, eps_edge, E, H, J, dt)
    A = yee.system_matrix(grid, eps_edge, beta)
    u = yee.unknowns(grid)
    Au = A[u][:, u].tocsc()
    E_new = np.zeros_like(E)
    if solve is None:
        E_new.reshape(-1)[u] = spla.spsolve(Au, R.reshape(-1)[u])
    else:
        E_new.reshape(-1)[u] = solve(Au, R.reshape(-1)[u])
    return E_new, h_update(grid, H, E_new, E, dt)


def energy(eps_edge, E, H):
    """Discrete energy sum eps E^2 + sum H^2, conserved by CN when J = 0."""
    return float(np.sum(eps_edge * E * E) + np.sum(H * H))
