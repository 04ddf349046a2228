"""Pins for the oracle IFMM (Eq. (1), Algorithms 1-3) and GMRES (Algorithm 4/5)."""

import numpy as np
import pytest

from oracle.dense import fmm_matrix
from oracle.gmres import gmres
from oracle.ifmm import IFMMOracle
from oracle.operators import dense_matrix
from oracle.tree import greedy_coloring
from paper_1905_10602_gb300.workloads import bumpy_sphere, fibonacci_sphere, point_source_rhs, torus


@pytest.mark.parametrize("N,depth,p,sigma", [(400, 2, 3, 6), (1024, 3, 3, 6), (1024, 3, 3, 3), (900, 3, 2, 3)])
def test_exact_at_eps0_equals_dense_elimination(N, depth, p, sigma):
    """At eps -> 0 nothing is truncated and the IFMM is Gaussian elimination on the
    extended system: its solve equals A~^{-1} b, with A~ assembled from its closed form."""
    pts = fibonacci_sphere(N, 1)
    b = point_source_rhs(pts)
    o = IFMMOracle(pts, depth, p, 0.0, sigma).factor()
    At = fmm_matrix(o.tree, o.ops)
    x_ref = np.linalg.solve(At, b)
    x = o.solve(b)
    assert np.linalg.norm(x - x_ref) / np.linalg.norm(x_ref) < 1e-11
    # and it is a different matrix from A (the check is against A~, not A)
    A = dense_matrix(pts)
    assert np.linalg.norm(A - At) / np.linalg.norm(A) > 1e-8


def test_exact_other_surfaces():
    for pts in (torus(800, 2), bumpy_sphere(800, 3)):
        o = IFMMOracle(pts, 3, 3, 0.0, 3).factor()
        At = fmm_matrix(o.tree, o.ops)
        b = np.random.default_rng(1).standard_normal(len(pts))
        x = o.solve(b)
        assert np.linalg.norm(At @ x - b) / np.linalg.norm(b) < 1e-12


def test_error_scales_with_eps():
    """Sec. 5.1: the compression error is controlled by eps; ||M A~ x - x|| falls
    roughly in proportion to eps."""
    pts = fibonacci_sphere(2048, 1)
    x = np.random.default_rng(0).standard_normal(len(pts))
    errs = {}
    At = None
    for eps in (1e-2, 1e-4, 1e-6, 1e-8):
        o = IFMMOracle(pts, 3, 3, eps, 6).factor()
        if At is None:
            At = fmm_matrix(o.tree, o.ops)
        errs[eps] = np.linalg.norm(o.solve(At @ x) - x) / np.linalg.norm(x)
    for eps, e in errs.items():
        assert 1e-3 * eps < e < 10 * eps, errs
    es = [errs[e] for e in (1e-2, 1e-4, 1e-6, 1e-8)]
    assert all(b < 0.05 * a for a, b in zip(es, es[1:])), errs


def test_sigma6_color_permutation_bit_identical():
    """Sec. 3.2: at sigma=6 the nodes of a color are independent, so any order inside
    each color gives bit-identical factors and solves."""
    pts = fibonacci_sphere(2048, 1)
    b = point_source_rhs(pts)
    base = IFMMOracle(pts, 3, 3, 1e-6, 6).factor()
    rng = np.random.default_rng(3)
    perm_groups = {}
    for kappa in (2, 3):
        groups = [list(g) for g in base.colors[kappa]]
        for g in groups:
            rng.shuffle(g)
        perm_groups[kappa] = groups
    other = IFMMOracle(pts, 3, 3, 1e-6, 6, color_groups=perm_groups).factor()
    assert np.array_equal(base.solve(b), other.solve(b))
    assert base.ranks() == other.ranks()


def test_rank_replay_reproduces():
    pts = fibonacci_sphere(1024, 2)
    b = point_source_rhs(pts)
    a = IFMMOracle(pts, 3, 3, 1e-5, 3).factor()
    c = IFMMOracle(pts, 3, 3, 1e-5, 3, rank_replay=a.ranks()).factor()
    assert np.array_equal(a.solve(b), c.solve(b))


def test_gmres_plain_matches_dense_solve():
    pts = fibonacci_sphere(1200, 4)
    A = dense_matrix(pts)
    b = point_source_rhs(pts)
    x, its, rel = gmres(lambda v: A @ v, b, restart=30, tol=1e-10)
    assert rel <= 1e-10
    assert np.linalg.norm(x - np.linalg.solve(A, b)) / np.linalg.norm(x) < 1e-8
    assert 5 < its < 60


def test_gmres_restart_path():
    pts = fibonacci_sphere(600, 4)
    A = dense_matrix(pts)
    b = point_source_rhs(pts)
    x, its, rel = gmres(lambda v: A @ v, b, restart=3, tol=1e-10)
    assert rel <= 1e-10 and its > 3


def test_ifmm_preconditioned_gmres():
    """Algorithm 4/5: GMRES on A with the IFMM solve as right preconditioner reaches
    1e-8 in far fewer iterations than without."""
    pts = fibonacci_sphere(2048, 1)
    A = dense_matrix(pts)
    b = point_source_rhs(pts)
    o = IFMMOracle(pts, 3, 3, 1e-6, 6).factor()
    _, its0, _ = gmres(lambda v: A @ v, b, tol=1e-8)
    x, its, rel = gmres(lambda v: A @ v, b, precond=o.solve, tol=1e-8)
    assert rel <= 1e-8
    assert its < its0 and its <= 6
