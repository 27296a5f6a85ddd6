"""Pins of the oracle's Krylov solvers (Sec. IV-A, Table 3)."""
import numpy as np
import scipy.sparse.linalg as spla

from oracle import krylov, ras, yee
from paper_2508_07193_b300 import workloads as wl


def _problem(grid=(10, 9, 8), cuts=((5, 5), (4, 5), (8,)), overlap=2, seed=3):
    w = wl.small(grid=grid, cuts=cuts, overlap=overlap, seed=seed, n_eps_boxes=3)
    ee = yee.edge_eps(w.grid, w.eps_cell)
    A = yee.system_matrix(w.grid, ee, w.beta)
    boxes = ras.partition(w.grid, w.cuts, w.overlap)
    shape = w.rhs.shape
    Aop = lambda x: A @ x
    Mop = lambda r: ras.precond_apply(r.reshape(shape), boxes, ee, w.beta).reshape(-1)
    return w, A, Aop, Mop


def test_fgmres_exact_preconditioner_converges_in_one_iteration():
    g = (6, 6, 5)
    rng = np.random.default_rng(0)
    b = rng.uniform(-1, 1, (3, 5, 6, 6)); b[wl.edge_wall_mask(g)] = 0
    ee = yee.edge_eps(g, None)
    A = yee.system_matrix(g, ee, 0.25)
    boxes = ras.partition(g, ((6,), (6,), (5,)), 2)
    M = lambda r: ras.precond_apply(r.reshape(b.shape), boxes, ee, 0.25).reshape(-1)
    x, info = krylov.fgmres(lambda v: A @ v, M, b.reshape(-1), rtol=1e-10)
    assert info["iters"] == 1 and info["true_rel_res"] <= 1e-10


def test_fgmres_matches_spsolve_and_beats_unpreconditioned():
    w, A, Aop, Mop = _problem()
    b = w.rhs.reshape(-1)
    x, info = krylov.fgmres(Aop, Mop, b, rtol=1e-10)
    u = yee.unknowns(w.grid)
    xs = spla.spsolve(A[u][:, u].tocsc(), b[u])
    assert info["true_rel_res"] <= 1e-10
    assert np.abs(x[u] - xs).max() <= 1e-8 * np.abs(xs).max()
    _, info0 = krylov.fgmres(Aop, lambda r: r.copy(), b, rtol=1e-10)
    assert info["iters"] < info0["iters"]


def test_fgmres_restart_path():
    w, A, Aop, _ = _problem()
    b = w.rhs.reshape(-1)
    x, info = krylov.fgmres(Aop, lambda r: r.copy(), b, restart=3, rtol=1e-9)
    assert info["restarts"] >= 2 and info["true_rel_res"] <= 1e-9


def test_bicgstab_converges_and_needs_fewer_iterations_than_gmres():
    w, A, Aop, Mop = _problem()
    b = w.rhs.reshape(-1)
    x, info = krylov.bicgstab(Aop, Mop, b, rtol=1e-10)
    _, ig = krylov.fgmres(Aop, Mop, b, rtol=1e-10)
    assert info["true_rel_res"] <= 1e-9
    assert info["iters"] <= ig["iters"]


def test_fgmres_on_k_distinct_eigenvalues_takes_k_steps_and_minimises_the_residual():
    """Closed forms of GMRES: on a diagonal matrix with k distinct eigenvalues
    (identity preconditioner) the Krylov space of b holds the solution after k
    steps, and the residual norm after j < k steps is the minimum over degree-j
    polynomials p with p(0) = 1 of ||p(A) b||, a small least-squares problem
    solved here independently of the Arnoldi process."""
    rng = np.random.default_rng(7)
    lam = np.array([1.0, 2.5, 4.0, 7.5])
    d = np.repeat(lam, 40)
    b = rng.uniform(-1, 1, d.size)
    Aop = lambda v: d * v
    x, info = krylov.fgmres(Aop, lambda r: r.copy(), b, rtol=1e-12)
    assert info["iters"] == len(lam) and info["true_rel_res"] <= 1e-12
    assert np.abs(x - b / d).max() <= 1e-12 * np.abs(b / d).max()
    for j in (1, 2, 3):
        _, ij = krylov.fgmres(Aop, lambda r: r.copy(), b, rtol=1e-300, max_iters=j, restart=j)
        # min over c of || b - sum_{i=1..j} c_i A^i b ||
        K = np.stack([d ** i * b for i in range(1, j + 1)], axis=1)
        c, *_ = np.linalg.lstsq(K, b, rcond=None)
        best = np.linalg.norm(b - K @ c) / np.linalg.norm(b)
        assert abs(ij["true_rel_res"] - best) <= 1e-10 * max(best, 1e-30) + 1e-14


def test_bicgstab_on_k_distinct_eigenvalues_ends_within_k_iterations():
    """On a diagonal SPD matrix with k distinct eigenvalues the BiCG polynomial
    (CG's, for a symmetric matrix and r^ = r_0) vanishes on the spectrum after
    k steps, so BiCGSTAB's residual Q_i(A) P_i(A) r_0 does too: at most k
    iterations to the tolerance, and the exact solution."""
    rng = np.random.default_rng(8)
    lam = np.array([1.0, 3.0, 4.5, 9.0, 12.0])
    d = np.repeat(lam, 30)
    b = rng.uniform(-1, 1, d.size)
    x, info = krylov.bicgstab(lambda v: d * v, lambda r: r.copy(), b, rtol=1e-11)
    assert info["iters"] <= len(lam) and info["true_rel_res"] <= 1e-11
    assert np.abs(x - b / d).max() <= 1e-10 * np.abs(b / d).max()
