"""Planted mistakes in the oracle (on the CPU) must be caught by its pins.

Each case patches one plausible slip into an oracle function (a flipped sign,
a dropped term, a swapped table, a transposed operand) and checks that one of
the pin tests then fails.
"""
import numpy as np
import pytest

from oracle import box, transforms as tf, yee
import tests.test_oracle_box as tbox
import tests.test_oracle_transforms as ttf
import tests.test_oracle_yee as tyee
import tests.test_oracle_cn as tcn


def _fails(fn, *args):
    with pytest.raises(AssertionError):
        fn(*args)


def test_flipped_coupling_sign_in_block_is_caught(monkeypatch):
    orig = box.block_matrices

    def bad(mx, my, mz, eps_bar, beta):
        B = orig(mx, my, mz, eps_bar, beta)
        off = ~np.eye(3, dtype=bool)
        B[..., off] *= -1.0
        return B
    monkeypatch.setattr(box, "block_matrices", bad)
    _fails(tbox.test_exact_solve_matches_dense_lu, (7, 5, 6), 3.3, 0.25)


def test_swapped_tables_are_caught(monkeypatch):
    orig = tf.component_tables

    def bad(mx, my, mz):
        t = orig(mx, my, mz)
        return ((t[0][0], t[0][1], t[0][2]), (t[1][0], tf.dst1(my), t[1][2]), t[2])
    monkeypatch.setattr(tf, "component_tables", bad)
    _fails(tbox.test_exact_solve_matches_dense_lu, (7, 5, 6), 3.3, 0.25)


def test_untransposed_inverse_is_caught(monkeypatch):
    def bad_inverse(Rh, tables):
        out = np.empty_like(Rh)
        for c in range(3):
            Tx, Ty, Tz = tables[c]
            out[c] = tf.tr_x(Tx, tf.tr_y(Ty, tf.tr_z(Tz, Rh[c])))
        return out
    monkeypatch.setattr(tf, "inverse", bad_inverse)
    _fails(ttf.test_forward_inverse_roundtrip_on_non_wall_slots)


def test_dropped_curl_term_is_caught(monkeypatch):
    orig = yee.curl_matrix

    def bad(grid):
        C = orig(grid).tolil()
        r = yee.slot(grid, 2, 1, 1, 1)
        c = yee.slot(grid, 0, 1, 2, 1)       # drop the Ex(j+1) term of one Hz face
        C[r, c] = 0.0
        return C.tocsr()
    monkeypatch.setattr(yee, "curl_matrix", bad)
    _fails(tyee.test_div_curl_and_curl_grad_vanish_exactly, (4, 3, 5))


def test_wrong_sigma_is_caught(monkeypatch):
    monkeypatch.setattr(tf, "sigma", lambda m: 2.0 * np.sin(np.pi * np.arange(m) / (2.0 * m + 1)))
    _fails(ttf.test_difference_factorises_with_positive_sigma, 6)


def test_wrong_cn_half_step_is_caught(monkeypatch):
    from oracle import cn
    orig = cn.h_update
    monkeypatch.setattr(cn, "h_update", lambda g, H, En, Eo, dt: orig(g, H, En, En, dt))
    _fails(tcn.test_energy_conserved_without_source)


def test_dropped_boundary_weight_is_caught(monkeypatch):
    """Step 4 without the Lambda weights (C = Q^T A_M^{-1} Q alone) is caught."""
    from oracle import compact as cp
    import tests.test_oracle_compact as tcp
    orig = cp.correction_matrix

    def bad(shape, eps_bar, beta, walls=None):
        C, q = orig(shape, eps_bar, beta, walls)
        _, dq, wq = cp.boundary(shape, walls)
        return C - np.diag(np.where(wq, 0.0, 1.0 / (beta * dq))), q
    monkeypatch.setattr(cp, "correction_matrix", bad)
    grid, lo, shape = tcp.BOXES[0]
    _fails(tcp.test_woodbury_solve_matches_dense_restricted_solve, grid, lo, shape, 2.3, 0.25)


def test_upper_diagonal_difference_is_caught(monkeypatch):
    """D^f with its +1 on the subdiagonal (a transposed difference) is caught."""
    from oracle import compact as cp
    import tests.test_oracle_compact as tcp
    monkeypatch.setattr(cp, "difference", lambda n: -np.eye(n) + np.eye(n, k=-1))
    grid, lo, shape = tcp.BOXES[0]
    _fails(tcp.test_M_plus_lambda_is_the_restricted_double_curl, grid, lo, shape)
