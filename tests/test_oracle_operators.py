"""Pins for the oracle's Chebyshev operators and the FMM-represented matrix."""

import numpy as np
import pytest

from oracle.dense import direct_matvec, fmm_matrix
from oracle.operators import Operators, cheb_nodes, cheb_roots, dense_matrix, interp_matrix, kernel_block
from oracle.tree import Tree
from paper_1905_10602_gb300.workloads import fibonacci_sphere


@pytest.mark.parametrize("p", [2, 3, 4, 5])
def test_interpolation_reproduces_polynomials(p):
    """An order-p interpolant reproduces every polynomial of degree < p per axis exactly."""
    rng = np.random.default_rng(p)
    c, h = np.array([0.3, -0.2, 0.1]), 0.7
    X = c + h * rng.uniform(-1, 1, (50, 3))
    nodes = cheb_nodes(c, h, p)
    coef = rng.standard_normal((p, p, p))

    def f(Y):
        u = Y - 0.11
        return sum(coef[a, b, cc] * u[:, 0] ** a * u[:, 1] ** b * u[:, 2] ** cc
                   for a in range(p) for b in range(p) for cc in range(p))

    S = interp_matrix(X, c, h, p)
    assert np.allclose(S.T @ f(nodes), f(X), rtol=0, atol=1e-11 * np.abs(f(X)).max())
    # the interpolation matrix at the nodes themselves is the identity
    assert np.allclose(interp_matrix(nodes, c, h, p), np.eye(p ** 3), atol=1e-13)


def test_cheb_roots_are_roots():
    for p in (3, 4):
        t = cheb_roots(p)
        Tp = np.cos(p * np.arccos(t))
        assert np.abs(Tp).max() < 1e-14


def test_m2m_composes_with_leaf_interpolation():
    """Interpolating through the child cell and then M2M equals interpolating at the
    parent directly (polynomial reproduction), so L2P/L2L chains are exact."""
    T = Tree(fibonacci_sphere(1500, 3), 3)
    ops = Operators(T, 4)
    L = T.levels[3]
    for c in (0, 5, L.n - 1):
        X = ops.leaf_points(c)
        parent = L.parent[c]
        direct = interp_matrix(X, T.cell_center(2, parent), T.cell_halfwidth(2), 4)
        via = ops.m2m(3, c) @ ops.p2m_leaf(c)
        assert np.allclose(via, direct, atol=1e-12)


def test_kernel_matrix_entries():
    pts = fibonacci_sphere(300, 4)
    A = dense_matrix(pts)
    N = len(pts)
    i, j = 17, 251
    assert A[i, j] == pytest.approx(1.0 / (N * np.linalg.norm(pts[i] - pts[j])), rel=1e-15)
    assert A[5, 5] == pytest.approx(0.5 + 1 / np.sqrt(N), rel=1e-15)
    assert np.allclose(A, A.T)
    x = np.random.default_rng(0).standard_normal(N)
    assert np.allclose(direct_matvec(pts, x), A @ x, rtol=1e-13, atol=0)


def test_fmm_matrix_near_blocks_exact_and_converges():
    """A~ equals A on near-field blocks; ||A~ - A|| falls with the Chebyshev order."""
    pts = fibonacci_sphere(1024, 5)
    A = dense_matrix(pts)
    errs = []
    for p in (2, 3, 4, 5):
        T = Tree(pts, 3)
        At = fmm_matrix(T, Operators(T, p))
        leaf = T.levels[3]
        for P in (0, 7):
            for Q in [P] + list(leaf.nbrs[P]):
                ip, iq = T.leaf_points(P), T.leaf_points(int(Q))
                assert np.array_equal(At[np.ix_(ip, iq)], A[np.ix_(ip, iq)])
        errs.append(np.linalg.norm(At - A) / np.linalg.norm(A))
    assert all(b < 0.5 * a for a, b in zip(errs, errs[1:])), errs
    assert errs[-1] < 1e-5
