"""Oracle: the dense FMM-represented matrix A~ and the direct-summation matvec.

TEST INFRASTRUCTURE ONLY (see oracle/tree.py).

Eliminating y and z from the extended system of Eq. (1) leaves A~ x = b with
    A~_ij = A_ij                                   leaves of i and j equal or adjacent,
    A~_ij = sum_{m,k} S_P(x_i, m) K(m, k) S_Q(x_j, k)   otherwise,
where (P, Q) is the unique pair of ancestors of i's and j's leaves that are in
each other's interaction list (Sec. 2.1), K is evaluated between their Chebyshev
nodes, and S_P is the interpolation of cell P evaluated directly at x_i (the
L2P/L2L chain of Chebyshev interpolants reproduces the ancestor's interpolant
exactly, because an order-p interpolant reproduces polynomials of degree < p).
The IFMM computes an approximate factorization of exactly this matrix; at
eps -> 0 its solve equals A~^{-1}.
"""

from __future__ import annotations

import numpy as np

from .operators import interp_matrix, kernel_block


def fmm_matrix(tree, ops) -> np.ndarray:
    """Assemble A~ densely (user point order).  Meant for N <= a few thousand."""
    N, ell, p = tree.N, tree.depth, ops.p
    At = np.zeros((N, N), dtype=np.complex128 if getattr(ops, "k", 0.0) else np.float64)
    leaf = tree.levels[ell]
    # ancestors of each leaf per level
    anc = {ell: np.arange(leaf.n)}
    for kappa in range(ell, 0, -1):
        anc[kappa - 1] = tree.levels[kappa].parent[anc[kappa]]
    idx = [tree.leaf_points(i) for i in range(leaf.n)]
    S_cache = {}

    def S(i, kappa):
        key = (i, kappa)
        if key not in S_cache:
            a = anc[kappa][i]
            S_cache[key] = interp_matrix(tree.pts[idx[i]], tree.cell_center(kappa, a), tree.cell_halfwidth(kappa), p)
        return S_cache[key]

    K_cache = {}
    for P in range(leaf.n):
        for Q in range(leaf.n):
            cP, cQ = leaf.cells[P], leaf.cells[Q]
            if np.max(np.abs(cP - cQ)) <= 1:
                At[np.ix_(idx[P], idx[Q])] = kernel_block(N, tree.pts[idx[P]], tree.pts[idx[Q]], same=(P == Q),
                                                          k=getattr(ops, "k", 0.0))
                continue
            kappa = ell
            while True:
                a, b = anc[kappa][P], anc[kappa][Q]
                pa, pb = anc[kappa - 1][P], anc[kappa - 1][Q]
                Lk, Lp = tree.levels[kappa], tree.levels[kappa - 1]
                if np.max(np.abs(Lk.cells[a] - Lk.cells[b])) >= 2 and np.max(np.abs(Lp.cells[pa] - Lp.cells[pb])) <= 1:
                    break
                kappa -= 1
            key = (kappa, a, b)
            if key not in K_cache:
                K_cache[key] = ops.m2l(kappa, a, b)
            At[np.ix_(idx[P], idx[Q])] = S(P, kappa).T @ K_cache[key] @ S(Q, kappa)
    return At


def direct_matvec(pts: np.ndarray, x: np.ndarray, rows: np.ndarray | None = None, chunk: int = 512) -> np.ndarray:
    """(A x)_i = (0.5 + 1/sqrt(N)) x_i + sum_{j != i} x_j / (N |x_i - x_j|), for the
    requested rows (all rows by default), in row chunks."""
    N = len(pts)
    rows = np.arange(N) if rows is None else np.asarray(rows)
    out = np.empty(len(rows))
    diag = 0.5 + 1.0 / np.sqrt(N)
    for s in range(0, len(rows), chunk):
        rr = rows[s:s + chunk]
        d = np.sqrt(((pts[rr, None, :] - pts[None, :, :]) ** 2).sum(axis=2))
        self_mask = rr[:, None] == np.arange(N)[None, :]
        d[self_mask] = np.inf
        out[s:s + chunk] = (x[None, :] / (N * d)).sum(axis=1) + diag * x[rr]
    return out
