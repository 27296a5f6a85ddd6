"""Operation and memory counts of the subdomain solve (oracle, test-only).

Sec. III-B, "Theoretical Computational Complexity" and "Theoretical Space
Complexity", and Table 2 (n = 32):
* one tensor product (one axis of one component) costs 2 n^4 flops; G is 9 of
  them (18 n^4), G^{-1} the same, one exact_solve 36 n^4; Algorithm 1 calls
  exact_solve twice: 72 n^4;
* the point-wise 3x3 solve with precomputed B^{-1}: 18 n^3;
* the Woodbury GEMV with C^{-1} of order 6n^2 - 3n: 2 (6n^2 - 3n)^2;
* memory: C^{-1} is (6n^2 - 3n)^2 doubles; E and R are 3 n^3 doubles each;
* a direct method: GEMV with a dense A^{-1}: 2 (3n^3)^2 flops, (3n^3)^2 doubles.
"""
from __future__ import annotations


def boundary_rank(n):
    """Number of nonzeros of Lambda over three components (Sec. III-A Step 4)."""
    return 3 * (2 * n * n - n)


def flashmp_flops(n):
    """Transforms (two exact_solves) + BSpMV + Woodbury GEMV."""
    return 72 * n ** 4 + 18 * n ** 3 + 2 * boundary_rank(n) ** 2


def flashmp_bytes(n):
    """C^{-1} plus the two field vectors E and R, in bytes."""
    return 8 * boundary_rank(n) ** 2 + 2 * 8 * 3 * n ** 3


def direct_flops(n):
    return 2 * (3 * n ** 3) ** 2


def direct_bytes(n):
    return 8 * (3 * n ** 3) ** 2 + 2 * 8 * 3 * n ** 3


def transform_flops_box(mx, my, mz):
    """Flops of one forward + inverse component-wise transform on an mx*my*mz box
    (2 m_a per output per axis pass, 3 components, 3 axes, two directions)."""
    v = mx * my * mz
    return 2 * 3 * 2 * (mx + my + mz) * v
