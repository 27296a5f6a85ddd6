"""Subdomain exact solve by discrete transforms (oracle, test-only).

Algorithm 1, function exact_solve, and Sec. III-A Steps 1-3:
  (1) R_hat = G R (component-wise tensor-product transforms),
  (2) per transform mode (i, j, k) solve the 3x3 system B_ijk e = r (Eq. 12),
  (3) E = G^{-1} E_hat.

The block is the one printed for B_ijk in Sec. III-A (its off-diagonals carry a
minus sign; the scalar x-row printed just before it has a sign typo) with the
identity scaled by the subdomain's mean permittivity eps_bar:
  B = eps_bar I + beta [[sy^2+sz^2, -sx sy, -sx sz],
                         [-sx sy, sx^2+sz^2, -sy sz],
                         [-sx sz, -sy sz, sx^2+sy^2]].
Each mode's 3x3 system is solved with a dense LU solve (np.linalg.solve), not
with a closed form, so the GPU's closed-form inverse is checked independently.

Step 2's permutation P (component-major <-> grid-major) is only a reordering;
here it is the stacking of the three components along the last axis.

The Woodbury boundary correction of Step 4 is not used: on a Yee box with PEC
walls (the reading of the boundary taken here) the transforms diagonalise the
box operator exactly.
"""
from __future__ import annotations

import numpy as np

from . import transforms as tf


def block_matrices(mx, my, mz, eps_bar, beta):
    """B_ijk for every mode, shape [mz][my][mx][3][3] (Eq. 12)."""
    sx = tf.sigma(mx)[None, None, :]
    sy = tf.sigma(my)[None, :, None]
    sz = tf.sigma(mz)[:, None, None]
    shape = (mz, my, mx)
    sx, sy, sz = (np.broadcast_to(s, shape) for s in (sx, sy, sz))
    B = np.zeros(shape + (3, 3))
    B[..., 0, 0] = sy ** 2 + sz ** 2
    B[..., 1, 1] = sx ** 2 + sz ** 2
    B[..., 2, 2] = sx ** 2 + sy ** 2
    B[..., 0, 1] = B[..., 1, 0] = -sx * sy
    B[..., 0, 2] = B[..., 2, 0] = -sx * sz
    B[..., 1, 2] = B[..., 2, 1] = -sy * sz
    B *= beta
    for c in range(3):
        B[..., c, c] += eps_bar
    return B


def exact_solve(R, eps_bar, beta):
    """(eps_bar I + beta K_box)^{-1} R for a [3][mz][my][mx] box field.

    Algorithm 1 exact_solve: transform, permute, per-mode 3x3 solve, permute
    back, inverse transform. Box-wall slots of R must be zero; they come out
    zero.
    """
    _, mz, my, mx = R.shape
    tables = tf.component_tables(mx, my, mz)
    Rh = tf.forward(R, tables)
    Xp = np.moveaxis(Rh, 0, -1)                 # P: grid-major [mz][my][mx][3]
    B = block_matrices(mx, my, mz, eps_bar, beta)
    Yp = np.linalg.solve(B, Xp[..., None])[..., 0]
    Eh = np.moveaxis(Yp, -1, 0)                 # P^T: component-major
    return tf.inverse(Eh, tables)
