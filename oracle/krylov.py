"""Outer Krylov solvers (oracle, test-only).

Sec. IV-A "Workloads": GMRES with restart k = 30 and BiCGSTAB with standard
parameters, both preconditioned by the subdomain solver; Table 3 lists their
work per iteration (GMRES: 1 preconditioner apply, 1 SpMV, k_avg + 1 dots;
BiCGSTAB: 2, 2, 4).

Readings: GMRES is right-preconditioned flexible GMRES (the preconditioner may
be nonlinear once it runs in reduced precision), with modified Gram-Schmidt and
Givens rotations (Saad, Iterative Methods for Sparse Linear Systems, FGMRES).
BiCGSTAB is van der Vorst's right-preconditioned form with r_hat_0 = r_0.
Both stop when the TRUE relative residual ||b - A x|| / ||b|| <= rtol.
Iterations count preconditioner applications for GMRES (Arnoldi steps) and
full BiCGSTAB steps (two applications each).
"""
from __future__ import annotations

import numpy as np


def fgmres(A, M, b, x0=None, restart=30, rtol=1e-8, max_iters=1000):
    """Restarted right-preconditioned flexible GMRES with MGS + Givens.

    Returns (x, info) with info = dict(iters, restarts, true_rel_res, history).
    """
    b = np.asarray(b, dtype=np.float64)
    x = np.zeros_like(b) if x0 is None else np.array(x0, dtype=np.float64)
    bnorm = np.linalg.norm(b)
    if bnorm == 0.0:
        return np.zeros_like(b), dict(iters=0, restarts=0, true_rel_res=0.0, history=[])
    iters, restarts, history = 0, 0, []
    while True:
        r = b - A(x)
        rnorm = np.linalg.norm(r)
        rel = rnorm / bnorm
        history.append(rel)
        if rel <= rtol or iters >= max_iters:
            return x, dict(iters=iters, restarts=restarts, true_rel_res=rel, history=history)
        n = b.size
        V = np.zeros((restart + 1, n))
        Z = np.zeros((restart, n))
        H = np.zeros((restart + 1, restart))
        cs = np.zeros(restart); sn = np.zeros(restart)
        g = np.zeros(restart + 1); g[0] = rnorm
        V[0] = r / rnorm
        j_done = 0
        for j in range(restart):
            Z[j] = M(V[j])
            w = A(Z[j])
            for i in range(j + 1):                  # modified Gram-Schmidt
                H[i, j] = np.dot(w, V[i])
                w = w - H[i, j] * V[i]
            hnext = np.linalg.norm(w)
            H[j + 1, j] = hnext
            for i in range(j):                      # previous rotations
                t = cs[i] * H[i, j] + sn[i] * H[i + 1, j]
                H[i + 1, j] = -sn[i] * H[i, j] + cs[i] * H[i + 1, j]
                H[i, j] = t
            den = np.hypot(H[j, j], H[j + 1, j])
            cs[j], sn[j] = H[j, j] / den, H[j + 1, j] / den
            H[j, j] = den
            H[j + 1, j] = 0.0
            g[j + 1] = -sn[j] * g[j]
            g[j] = cs[j] * g[j]
            iters += 1
            j_done = j + 1
            history.append(abs(g[j + 1]) / bnorm)
            if abs(g[j + 1]) / bnorm <= rtol or iters >= max_iters:
                break
            if hnext == 0.0 or not np.isfinite(g[j + 1]):   # lucky breakdown
                break
            V[j + 1] = w / hnext
        y = np.linalg.solve(np.triu(H[:j_done, :j_done]), g[:j_done])
        x = x + y @ Z[:j_done]
        restarts += 1


def bicgstab(A, M, b, x0=None, rtol=1e-8, max_iters=1000):
    """Right-preconditioned BiCGSTAB (van der Vorst 1992), r_hat_0 = r_0."""
    b = np.asarray(b, dtype=np.float64)
    x = np.zeros_like(b) if x0 is None else np.array(x0, dtype=np.float64)
    bnorm = np.linalg.norm(b)
    if bnorm == 0.0:
        return np.zeros_like(b), dict(iters=0, true_rel_res=0.0, history=[])
    r = b - A(x)
    rhat = r.copy()
    rho_old = alpha = omega = 1.0
    v = np.zeros_like(b); p = np.zeros_like(b)
    history = [np.linalg.norm(r) / bnorm]
    it = 0
    while history[-1] > rtol and it < max_iters:
        rho = np.dot(rhat, r)
        if it == 0:
            p = r.copy()
        else:
            beta = (rho / rho_old) * (alpha / omega)
            p = r + beta * (p - omega * v)
        phat = M(p)
        v = A(phat)
        alpha = rho / np.dot(rhat, v)
        s = r - alpha * v
        shat = M(s)
        t = A(shat)
        omega = np.dot(t, s) / np.dot(t, t)
        x = x + alpha * phat + omega * shat
        r = s - omega * t
        rho_old = rho
        it += 1
        history.append(np.linalg.norm(r) / bnorm)
    true_rel = np.linalg.norm(b - A(x)) / bnorm
    return x, dict(iters=it, true_rel_res=true_rel, history=history)
