"""Seeded input generators: determinism, layout and the stated recipes."""
import numpy as np

from paper_2508_07193_b300 import workloads as wl


def test_small_is_deterministic_and_walls_zero():
    a, b = wl.small(), wl.small()
    assert np.array_equal(a.rhs, b.rhs) and np.array_equal(a.eps_cell, b.eps_cell)
    assert np.all(a.rhs[wl.edge_wall_mask(a.grid)] == 0)
    assert a.rhs.shape == (3, 14, 18, 20)


def test_box32_recipe():
    w = wl.box32()
    assert w.grid == (32, 32, 32) and w.eps_cell is None and w.beta == 0.25
    assert w.rhs.min() >= -1 and w.rhs.max() <= 1


def test_uneven_cuts_sum_and_choices():
    rng = np.random.default_rng(3)
    for n in (320, 256, 192):
        c = wl.draw_cuts(rng, n)
        assert sum(c) == n and set(c) <= set(wl.CUT_CHOICES)


def test_eps_range():
    rng = np.random.default_rng(1)
    e = wl.draw_eps_boxes(rng, (32, 24, 16), 16)
    assert e.min() >= 1.0 and e.max() <= 10.0


def test_dipole_waveform_peak_near_t0():
    t = np.arange(0, 120, 0.5)
    v = np.array([abs(wl.dipole_waveform(x)) for x in t])
    assert 40 <= t[v.argmax()] <= 80
