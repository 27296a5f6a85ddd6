"""Pins of the compact-layout oracle (Algorithm 1 with Step 4's Woodbury
boundary correction) against what the mathematics fixes: the closed-form
singular values of the square difference, the restricted global double curl,
dense solves, and the explicit sum of local inverses."""
import numpy as np
import pytest
import scipy.sparse as sp

from oracle import compact as cp, ras, yee
from paper_2508_07193_b300 import workloads as wl

# (grid, box low corner, box shape): interior, touching two or three low
# walls, and flush with the high walls
BOXES = [((9, 8, 7), (2, 2, 2), (4, 3, 3)),
         ((9, 8, 7), (0, 0, 0), (4, 3, 3)),
         ((9, 8, 7), (0, 3, 1), (3, 4, 2)),
         ((9, 8, 7), (5, 4, 4), (4, 4, 3))]


@pytest.mark.parametrize("n", [1, 2, 5, 12, 33])
def test_singular_values_closed_form(n):
    """sigma_k = 2 sin((2k - 1) pi / (2 (2n + 1))), k = 1..n, for the square D^f."""
    U, s, V = cp.tables(n)
    k = np.arange(1, n + 1)
    closed = 2.0 * np.sin((2 * k - 1) * np.pi / (2 * (2 * n + 1)))
    assert np.allclose(np.sort(s), np.sort(closed), rtol=0, atol=1e-13)
    D = cp.difference(n)
    assert np.allclose(D @ V, U * s, atol=1e-13)
    assert np.allclose(U.T @ U, np.eye(n), atol=1e-13) and np.allclose(V.T @ V, np.eye(n), atol=1e-13)


@pytest.mark.parametrize("grid, lo, shape", BOXES)
def test_M_plus_lambda_is_the_restricted_double_curl(grid, lo, shape):
    """Step 4: M + Lambda equals the global double curl restricted to the box,
    exactly (integer entries), on every non-wall slot."""
    M = cp.double_curl(shape)
    L = sp.diags(cp.delta(shape).reshape(-1))
    K = cp.restricted_double_curl(grid, lo, shape)
    nw = ~cp.box_walls(grid, lo, shape).reshape(-1)
    D = (M + L - K).toarray()[np.ix_(nw, nw)]
    assert np.array_equal(D, np.zeros_like(D))


def test_lambda_counts_and_rank():
    """delta in {0, 1, 2}; 2n^2 - n slots per component, 6n^2 - 3n in all (Fig. 4)."""
    for n in (3, 4, 7):
        d = cp.delta((n, n, n))
        assert set(np.unique(d)) == {0.0, 1.0, 2.0}
        for c in range(3):
            assert int((d[c] > 0).sum()) == 2 * n * n - n
        assert cp.boundary((n, n, n))[0].size == 6 * n * n - 3 * n


def test_transform_space_block_structure():
    """G M G^T = blockdiag(|s|^2 I - s s^T) over the modes, by brute force."""
    shape = (4, 3, 5)
    nx, ny, nz = shape
    n = 3 * nx * ny * nz
    G = np.zeros((n, n))
    for a in range(n):
        e = np.zeros(n)
        e[a] = 1.0
        G[:, a] = cp.forward(e.reshape(3, nz, ny, nx)).reshape(-1)
    assert np.allclose(G @ G.T, np.eye(n), atol=1e-13)
    H = G @ cp.double_curl(shape).toarray() @ G.T
    B = cp.block_matrices(shape, 0.0, 1.0)
    Hb = np.zeros((n, n))
    for k in range(nz):
        for j in range(ny):
            for i in range(nx):
                for c in range(3):
                    for d in range(3):
                        Hb[((c * nz + k) * ny + j) * nx + i, ((d * nz + k) * ny + j) * nx + i] = B[k, j, i, c, d]
    assert np.abs(H - Hb).max() < 1e-12


def test_transform_solve_matches_dense():
    shape = (5, 4, 3)
    nx, ny, nz = shape
    R = np.random.default_rng(1).standard_normal((3, nz, ny, nx))
    eb, beta = 1.7, 0.25
    A = eb * np.eye(R.size) + beta * cp.double_curl(shape).toarray()
    x = np.linalg.solve(A, R.reshape(-1))
    assert np.abs(cp.transform_solve(R, eb, beta).reshape(-1) - x).max() <= 1e-13 * np.abs(x).max()


@pytest.mark.parametrize("grid, lo, shape", BOXES)
@pytest.mark.parametrize("eb, beta", [(2.3, 0.25), (1.0, 25.0)])
def test_woodbury_solve_matches_dense_restricted_solve(grid, lo, shape, eb, beta):
    """Algorithm 1 with Step 4 inverts eps_bar I + beta K restricted to the
    box's unknowns; wall slots come out zero."""
    nx, ny, nz = shape
    w = cp.box_walls(grid, lo, shape)
    R = np.random.default_rng(2).standard_normal((3, nz, ny, nx))
    R[w] = 0.0
    E = cp.woodbury_solve(R, eb, beta, w)
    K = cp.restricted_double_curl(grid, lo, shape).toarray()
    nw = ~w.reshape(-1)
    A = (eb * np.eye(K.shape[0]) + beta * K)[np.ix_(nw, nw)]
    ref = np.zeros(R.size)
    ref[nw] = np.linalg.solve(A, R.reshape(-1)[nw])
    assert np.abs(E.reshape(-1) - ref).max() <= 1e-12 * np.abs(ref).max()
    assert np.abs(E[w]).max(initial=0.0) <= 1e-14 * np.abs(ref).max()


def test_without_step4_the_solve_is_not_exact():
    """The transform solve alone (no Woodbury) misses the restricted operator."""
    grid, lo, shape = BOXES[0]
    nx, ny, nz = shape
    R = np.random.default_rng(3).standard_normal((3, nz, ny, nx))
    K = cp.restricted_double_curl(grid, lo, shape).toarray()
    ref = np.linalg.solve(2.0 * np.eye(K.shape[0]) + 0.25 * K, R.reshape(-1))
    assert np.abs(cp.transform_solve(R, 2.0, 0.25).reshape(-1) - ref).max() > 1e-3 * np.abs(ref).max()


def test_compact_ras_equals_sum_of_local_inverses():
    """z = sum_i S_i^{0T} (eps_bar_i I + beta K_i)^{-1} S_i r, each K_i the
    global double curl restricted to the extended box's unknowns."""
    w = wl.small(grid=(10, 9, 8), cuts=((5, 5), (4, 5), (8,)), overlap=1, seed=31, n_eps_boxes=3)
    ee = yee.edge_eps(w.grid, w.eps_cell)
    boxes = ras.partition(w.grid, w.cuts, w.overlap)
    z = cp.precond_apply(w.rhs, boxes, ee, w.beta)
    K = yee.double_curl(w.grid)
    wall = yee.edge_is_wall(w.grid)
    ref = np.zeros(w.rhs.size)
    for b in boxes:
        shape = tuple(b.ext_hi[a] - b.ext_lo[a] for a in range(3))
        s = cp.box_slots(w.grid, b.ext_lo, shape)
        keep = ~wall[s]
        s = s[keep]
        eb = ee.reshape(-1)[s].mean()
        A = eb * np.eye(s.size) + w.beta * K[s][:, s].toarray()
        x = np.linalg.solve(A, w.rhs.reshape(-1)[s])
        own = np.zeros(w.rhs.shape, dtype=bool)
        (x0, y0, z0), (x1, y1, z1) = b.own_lo, b.own_hi
        own[:, z0:z1, y0:y1, x0:x1] = True
        o = own.reshape(-1)[s]
        ref[s[o]] = x[o]
    assert np.abs(z.reshape(-1) - ref).max() <= 1e-12 * np.abs(ref).max()
