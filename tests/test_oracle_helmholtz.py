"""Pins of the complex (Helmholtz) oracle, the paper's acoustic kernel
e^{ik r}/(4 pi r) (Sec. 4.1), against what the mathematics fixes: the self term
equals the kernel integrated over the point's disk panel; k -> 0 reduces every
entry to the Laplace one; at eps -> 0 the complex IFMM is Gaussian elimination
of the complex A~; A~ approaches A with the Chebyshev order; and the error
falls with eps."""

import math

import numpy as np
import pytest
from scipy.integrate import quad

from oracle.dense import fmm_matrix
from oracle.ifmm import IFMMOracle
from oracle.operators import Operators, bem_diag, dense_matrix
from oracle.tree import Tree
from paper_1905_10602_gb300.workloads import fibonacci_sphere, helmholtz_source_rhs, torus


@pytest.mark.parametrize("N,k", [(1000, 3.0), (4000, 16.0), (64, 0.5)])
def test_self_term_is_the_disk_integral(N, k):
    rho = 2.0 / math.sqrt(N)  # disk of area 4 pi / N
    re = quad(lambda r: math.cos(k * r) * 2 * math.pi * r / (4 * math.pi * r), 0.0, rho)[0]
    im = quad(lambda r: math.sin(k * r) * 2 * math.pi * r / (4 * math.pi * r), 0.0, rho)[0]
    d = bem_diag(N, k)
    assert abs(d - (0.5 + re + 1j * im)) < 1e-14


def test_small_wavenumber_reduces_to_laplace():
    pts = fibonacci_sphere(300, 1)
    A0, Ak = dense_matrix(pts), dense_matrix(pts, 1e-7)
    assert np.abs(Ak - A0).max() < 1e-7 * np.abs(A0).max()
    assert np.abs(Ak.imag).max() > 0


@pytest.mark.parametrize("k,p", [(2.0, 3), (8.0, 3)])
def test_exact_at_eps0_equals_dense_elimination(k, p):
    pts = fibonacci_sphere(900, 2)
    b = helmholtz_source_rhs(pts, k)
    o = IFMMOracle(pts, 3, p, 0.0, 3, wavenumber=k).factor()
    At = fmm_matrix(o.tree, o.ops)
    assert np.iscomplexobj(At) and np.abs(At.imag).max() > 0
    x = o.solve(b)
    assert np.linalg.norm(x - np.linalg.solve(At, b)) / np.linalg.norm(x) < 1e-11


def test_fmm_matrix_approaches_A_with_order():
    pts = torus(800, 3)
    tree = Tree(pts, 3)
    A = dense_matrix(pts, 4.0)
    errs = [np.linalg.norm(fmm_matrix(tree, Operators(tree, p, 4.0)) - A) / np.linalg.norm(A) for p in (2, 3, 4, 5)]
    assert all(b < a for a, b in zip(errs, errs[1:])), errs


def test_error_scales_with_eps():
    pts = fibonacci_sphere(1500, 1)
    k = 4.0
    x = np.random.default_rng(0).standard_normal(len(pts)) * (1 + 1j)
    errs = []
    At = None
    for eps in (1e-2, 1e-4, 1e-6):
        o = IFMMOracle(pts, 3, 3, eps, 6, wavenumber=k).factor()
        if At is None:
            At = fmm_matrix(o.tree, o.ops)
        errs.append(np.linalg.norm(o.solve(At @ x) - x) / np.linalg.norm(x))
    assert all(b < 0.05 * a for a, b in zip(errs, errs[1:])), errs
    assert errs[-1] < 1e-4
