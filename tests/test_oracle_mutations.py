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


def test_prolong_with_owned_corner_for_extended_corner_is_caught(monkeypatch):
    """S_i^0T reading the box solution at (owned corner) instead of (extended
    corner) offsets: caught by the slot-by-slot prolongation pin."""
    from oracle import ras
    import tests.test_oracle_ras as tras

    def bad(z, eb, b):
        (x0, y0, z0) = b.own_lo
        (ox0, oy0, oz0), (ox1, oy1, oz1) = b.own_lo, b.own_hi
        z[:, oz0:oz1, oy0:oy1, ox0:ox1] = eb[:, oz0 - z0:oz1 - z0, oy0 - y0:oy1 - y0, ox0 - x0:ox1 - x0]
    monkeypatch.setattr(ras, "prolong_owned", bad)
    _fails(tras.test_prolong_owned_slot_by_slot_on_clipped_ragged_boxes)


def test_restrict_with_swapped_wall_masks_is_caught(monkeypatch):
    """S_i^gamma zeroing Ey's walls on Ex and Ex's on Ey: caught by the
    slot-by-slot restriction pin."""
    from oracle import ras
    import tests.test_oracle_ras as tras
    orig = ras.box_wall

    def bad(m):
        w = orig(m)
        return w[[1, 0, 2]]
    monkeypatch.setattr(ras, "box_wall", bad)
    _fails(tras.test_restrict_slot_by_slot_on_clipped_ragged_boxes)


def test_restrict_without_clipping_offset_is_caught(monkeypatch):
    """S_i^gamma copying from the owned corner instead of the extended one
    (the halo dropped on the low side): caught by the restriction pin."""
    from oracle import ras
    import tests.test_oracle_ras as tras

    def bad(r, b):
        (x0, y0, z0) = b.own_lo
        m = b.m
        rb = np.zeros((3, m[2], m[1], m[0]))
        src = r[:, z0:z0 + m[2], y0:y0 + m[1], x0:x0 + m[0]]
        rb[:, :src.shape[1], :src.shape[2], :src.shape[3]] = src
        rb[ras.box_wall(m)] = 0.0
        return rb
    monkeypatch.setattr(ras, "restrict", bad)
    _fails(tras.test_restrict_slot_by_slot_on_clipped_ragged_boxes)
