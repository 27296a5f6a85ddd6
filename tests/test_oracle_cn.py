"""Pins of the oracle's Crank-Nicolson step (Sec. II-A, Eqs. 2-4).

* With J = 0 the scheme is a Cayley transform of a skew-adjoint system, so the
  discrete energy sum eps E^2 + sum H^2 is conserved exactly.
* A single cavity eigenmode with eps = 1 advances by the phase
  2 atan(omega dt / 2) per step, omega = |sigma| (closed form).
"""
import numpy as np
import pytest

from oracle import cn, ras, transforms as tf, yee
from paper_2508_07193_b300 import workloads as wl


def test_energy_conserved_without_source():
    g = (6, 5, 4)
    rng = np.random.default_rng(8)
    ee = yee.edge_eps(g, rng.uniform(1, 4, (4, 5, 6)))
    E = rng.standard_normal((3, 4, 5, 6)); E[wl.edge_wall_mask(g)] = 0
    H = rng.standard_normal((3, 4, 5, 6)); H[wl.face_wall_mask(g)] = 0
    w0 = cn.energy(ee, E, H)
    for _ in range(5):
        E, H = cn.step(g, ee, E, H, None, dt=1.0)
    assert abs(cn.energy(ee, E, H) - w0) <= 1e-11 * w0


@pytest.mark.parametrize("dt", [0.5, 1.0, 3.0])
def test_single_mode_phase_advance(dt):
    g = (6, 5, 4)
    mx, my, mz = g
    kx, ky, kz = 2, 3, 1
    s = np.array([tf.sigma(mx)[kx], tf.sigma(my)[ky], tf.sigma(mz)[kz]])
    # a transverse mode amplitude (perpendicular to sigma)
    e_hat = np.cross(s, [0.3, -0.7, 0.2]); e_hat /= np.linalg.norm(e_hat)
    Eh = np.zeros((3, mz, my, mx))
    Eh[:, kz, ky, kx] = e_hat
    E0 = tf.inverse(Eh, tf.component_tables(mx, my, mz))
    ee = yee.edge_eps(g, None)
    E, H = E0.copy(), np.zeros_like(E0)
    phi = 2 * np.arctan(np.linalg.norm(s) * dt / 2)
    for n in range(1, 4):
        E, H = cn.step(g, ee, E, H, None, dt=dt)
        c = np.sum(E * E0) / np.sum(E0 * E0)
        assert c == pytest.approx(np.cos(n * phi), abs=1e-11)


def test_rhs_with_zero_fields_is_minus_dt_j():
    g = (5, 4, 4)
    ee = yee.edge_eps(g, None)
    J = wl.dipole_current(g, 3, 1.0)
    z = np.zeros((3, 4, 4, 5))
    assert np.allclose(cn.rhs(g, ee, z, z, J, 1.0), -J)
