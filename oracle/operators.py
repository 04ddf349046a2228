"""Oracle: the BEM matrix and the black-box FMM (Chebyshev) operators.

TEST INFRASTRUCTURE ONLY (see oracle/tree.py).

The matrix: a collocation single-layer Laplace system on N surface points with
equal area weights 4pi/N,
    A_ij = (4pi/N) * 1/(4pi |x_i - x_j|) = 1/(N |x_i - x_j|)   (i != j),
    A_ii = 0.5 + 1/sqrt(N),
the electrostatic example of Sec. 2 (Coulomb interaction, Eq. (1) system Ax=b),
with a second-kind 0.5 on the diagonal and 1/sqrt(N) for the self panel.

The Helmholtz variant (the paper's acoustic BEM, Sec. 4.1): with wavenumber k
the kernel is e^{ik|x-y|}/(4pi|x-y|), so
    A_ij = e^{ik r_ij} / (N r_ij)   (i != j),
    A_ii = 0.5 + sin(k rho)/(2k) + i (1 - cos(k rho))/(2k),   rho = 2/sqrt(N),
the self term being the kernel integrated over a disk of area 4pi/N (radius
rho); k -> 0 gives the Laplace entries above.

The FMM operators (Sec. 2.2 lists P2P, P2M, L2P, M2M, M2L, L2L) come from
Chebyshev interpolation, the black-box FMM the paper names as an admissible
choice (Sec. 4.2):
  * order p: p first-kind Chebyshev roots per axis, t_m = cos((2m-1)pi/(2p)),
    r = p^3 nodes per cell, node (a, b, c) at flat index (c*p + b)*p + a;
  * S(x, node (a,b,c)) = l_a(u_x) l_b(u_y) l_c(u_z), Lagrange polynomials on the
    roots, u = (x - centre)/halfwidth;
  * P2M of a leaf = [S(x_j, node_m)] (r x n); L2P = P2M^T;
  * M2M of child c = [S_parent(child node k, parent node m)] (r x r); L2L = M2M^T;
  * M2L between cells = [K(target node m, source node k)] (r x r).
"""

from __future__ import annotations

import math

import numpy as np


def bem_diag(N: int, k: float = 0.0):
    """The diagonal entry: 0.5 plus the kernel integrated over the point's panel (a
    disk of area 4pi/N, radius rho = 2/sqrt(N)): rho/2 for Laplace, and
    (e^{ik rho} - 1)/(2ik) for Helmholtz."""
    rho = 2.0 / math.sqrt(N)
    if k == 0.0:
        return 0.5 + 0.5 * rho
    return 0.5 + math.sin(k * rho) / (2.0 * k) + 1j * (1.0 - math.cos(k * rho)) / (2.0 * k)


def kernel_block(N: int, X: np.ndarray, Y: np.ndarray, same: bool = False, k: float = 0.0) -> np.ndarray:
    """[e^{ik|x_i - y_j|}/(N|x_i - y_j|)] (k = 0: 1/(N|x_i - y_j|)); with same=True the
    diagonal gets bem_diag(N, k)."""
    d = np.sqrt(((X[:, None, :] - Y[None, :, :]) ** 2).sum(axis=2))
    if same:
        np.fill_diagonal(d, 1.0)
    K = 1.0 / (N * d) if k == 0.0 else np.exp(1j * k * d) / (N * d)
    if same:
        np.fill_diagonal(K, bem_diag(N, k))
    return K


def dense_matrix(pts: np.ndarray, k: float = 0.0) -> np.ndarray:
    """The full N x N BEM matrix A (user point order); complex for k != 0."""
    return kernel_block(len(pts), pts, pts, same=True, k=k)


def cheb_roots(p: int) -> np.ndarray:
    m = np.arange(1, p + 1, dtype=np.float64)
    return np.cos((2.0 * m - 1.0) * math.pi / (2.0 * p))


def lagrange_1d(u: np.ndarray, t: np.ndarray) -> np.ndarray:
    """L[j, a] = l_a(u_j) = prod_{b != a} (u_j - t_b)/(t_a - t_b)."""
    p = len(t)
    L = np.ones((len(u), p))
    for a in range(p):
        for b in range(p):
            if b != a:
                L[:, a] *= (u - t[b]) / (t[a] - t[b])
    return L


def interp_matrix(X: np.ndarray, center: np.ndarray, halfwidth: float, p: int) -> np.ndarray:
    """[S(x_j, node_m)] with shape (p^3, len(X)): row m = node (a,b,c), m=(c*p+b)*p+a."""
    t = cheb_roots(p)
    U = (X - center[None, :]) / halfwidth
    Lx, Ly, Lz = lagrange_1d(U[:, 0], t), lagrange_1d(U[:, 1], t), lagrange_1d(U[:, 2], t)
    # S[c, b, a, j] = Lz[j, c] * Ly[j, b] * Lx[j, a]
    S = Lz.T[:, None, None, :] * Ly.T[None, :, None, :] * Lx.T[None, None, :, :]
    return S.reshape(p ** 3, len(X))


def cheb_nodes(center: np.ndarray, halfwidth: float, p: int) -> np.ndarray:
    """Chebyshev nodes of a cell, (p^3, 3), in the flat order of interp_matrix."""
    t = cheb_roots(p)
    c, b, a = np.meshgrid(np.arange(p), np.arange(p), np.arange(p), indexing="ij")
    u = np.stack([t[a.ravel()], t[b.ravel()], t[c.ravel()]], axis=1)
    return center[None, :] + halfwidth * u


class Operators:
    """FMM operators of a tree for the BEM matrix, Chebyshev order p."""

    def __init__(self, tree, p: int, k: float = 0.0):
        self.tree = tree
        self.p = p
        self.r = p ** 3
        self.N = tree.N
        self.k = k  # Helmholtz wavenumber (0: Laplace)

    def leaf_points(self, i: int) -> np.ndarray:
        return self.tree.pts[self.tree.leaf_points(i)]

    def p2p(self, i: int, j: int) -> np.ndarray:
        """Near-field block between leaves i (rows) and j (columns)."""
        X, Y = self.leaf_points(i), self.leaf_points(j)
        return kernel_block(self.N, X, Y, same=(i == j), k=self.k)

    def p2m_leaf(self, i: int) -> np.ndarray:
        d = self.tree.depth
        return interp_matrix(self.leaf_points(i), self.tree.cell_center(d, i), self.tree.cell_halfwidth(d), self.p)

    def m2l(self, kappa: int, a: int, b: int) -> np.ndarray:
        """K between the Chebyshev nodes of target cell a and source cell b at level kappa."""
        h = self.tree.cell_halfwidth(kappa)
        Xa = cheb_nodes(self.tree.cell_center(kappa, a), h, self.p)
        Xb = cheb_nodes(self.tree.cell_center(kappa, b), h, self.p)
        return kernel_block(self.N, Xa, Xb, k=self.k)

    def m2m(self, kappa: int, c: int) -> np.ndarray:
        """Child c (level kappa) -> its parent: [S_parent(child node k, parent node m)]."""
        parent = self.tree.levels[kappa].parent[c]
        Xc = cheb_nodes(self.tree.cell_center(kappa, c), self.tree.cell_halfwidth(kappa), self.p)
        return interp_matrix(Xc, self.tree.cell_center(kappa - 1, parent), self.tree.cell_halfwidth(kappa - 1), self.p)
