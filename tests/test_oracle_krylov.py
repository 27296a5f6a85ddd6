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
