"""Oracle: restarted GMRES(m) with right preconditioning.

TEST INFRASTRUCTURE ONLY (see oracle/tree.py).

The paper solves its BEM systems with GMRES(m) from x = 0 and stops when the
relative residual ||Ax - b||_2 / ||b||_2 falls below tol (Algorithm 4, Sec. 5.1);
the preconditioner M ~ A^{-1} is applied as v = M r (Algorithm 5).  Readings:
right preconditioning (so the stopping test is on the true residual), classical
Gram-Schmidt applied twice, Givens rotations, and a restart whenever the true
residual is still above tol at the end of a cycle.
"""

from __future__ import annotations

import numpy as np


def gmres(matvec, b, precond=None, restart=30, tol=1e-8, maxit=500):
    """Returns (x, iterations, true relative residual)."""
    M = precond if precond is not None else (lambda v: v)
    b = np.asarray(b, dtype=np.float64)
    n = len(b)
    bnorm = np.linalg.norm(b)
    x = np.zeros(n)
    r = b.copy()
    its = 0
    relres = np.linalg.norm(r) / bnorm
    while its < maxit and relres > tol:
        beta = np.linalg.norm(r)
        m = restart
        V = np.zeros((m + 1, n))
        H = np.zeros((m + 1, m))
        cs, sn = np.zeros(m), np.zeros(m)
        g = np.zeros(m + 1)
        g[0] = beta
        V[0] = r / beta
        k = 0
        for j in range(m):
            w = matvec(M(V[j]))
            its += 1
            h = V[: j + 1] @ w
            w = w - V[: j + 1].T @ h
            h2 = V[: j + 1] @ w
            w = w - V[: j + 1].T @ h2
            h = h + h2
            hn = np.linalg.norm(w)
            H[: j + 1, j] = h
            H[j + 1, j] = hn
            if hn > 0:
                V[j + 1] = w / hn
            for i in range(j):
                t = cs[i] * H[i, j] + sn[i] * H[i + 1, j]
                H[i + 1, j] = -sn[i] * H[i, j] + cs[i] * H[i + 1, j]
                H[i, j] = t
            den = np.hypot(H[j, j], H[j + 1, j])
            cs[j], sn[j] = H[j, j] / den, H[j + 1, j] / den
            H[j, j] = den
            H[j + 1, j] = 0.0
            g[j + 1] = -sn[j] * g[j]
            g[j] = cs[j] * g[j]
            k = j + 1
            if abs(g[j + 1]) / bnorm <= tol or its >= maxit or hn == 0:
                break
        y = np.linalg.solve(np.triu(H[:k, :k]), g[:k])
        x = x + M(V[:k].T @ y)
        r = b - matvec(x)
        relres = np.linalg.norm(r) / bnorm
    return x, its, relres
