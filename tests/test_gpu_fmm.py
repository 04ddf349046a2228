"""The FMM matvec (IFMM_ARITH_FMM: the FMM representation A~ of Sec. 2.2,
Eq. (1), applied by P2M, M2M, M2L, L2L, L2P and the near field) against the
oracle's dense A~ (assembled from its closed form), and as the matvec of GMRES
with the IFMM preconditioner built from the same operators (the paper's FMBEM
structure, Algorithms 4 and 5)."""

import numpy as np
import pytest

from oracle.dense import fmm_matrix
from oracle.operators import Operators, dense_matrix
from oracle.tree import Tree
from paper_1905_10602_gb300 import build as _build
from paper_1905_10602_gb300.workloads import bumpy_sphere, fibonacci_sphere, point_source_rhs, torus

pytestmark = pytest.mark.gpu

_build.build()
from paper_1905_10602_gb300 import ifmm  # noqa: E402


def _rel(a, b):
    return np.linalg.norm(a - b) / np.linalg.norm(b)


@pytest.mark.parametrize("shape,N,depth,p", [("sphere", 1500, 3, 3), ("bumpy", 2000, 4, 4), ("torus", 1200, 3, 2),
                                             ("sphere", 600, 2, 4)])
def test_fmm_matvec_equals_dense_At(shape, N, depth, p):
    """A~ x to FP64 rounding (1e-12 relative): the same operators, summed in a
    different order."""
    pts = {"sphere": fibonacci_sphere, "bumpy": bumpy_sphere, "torus": torus}[shape](N, 3)
    tree = Tree(pts, depth)
    At = fmm_matrix(tree, Operators(tree, p))
    t = ifmm.ifmm_build_tree(pts, depth)
    rng = np.random.default_rng(p)
    for _ in range(2):
        x = rng.standard_normal(N)
        y = ifmm.bem_matvec(t, x, kernel=ifmm.default_kernel(N, "fmm", p))
        assert _rel(y, At @ x) < 1e-12


def test_fmm_matvec_converges_to_A_with_order():
    pts = fibonacci_sphere(3000, 2)
    t = ifmm.ifmm_build_tree(pts, 4)
    x = np.random.default_rng(1).standard_normal(len(pts))
    Ax = dense_matrix(pts) @ x
    errs = [_rel(ifmm.bem_matvec(t, x, kernel=ifmm.default_kernel(len(pts), "fmm", p)), Ax) for p in (2, 3, 4, 5)]
    assert all(b < a for a, b in zip(errs, errs[1:])), errs
    assert errs[-1] < 1e-4, errs


def test_gmres_with_fmm_matvec_and_ifmm_preconditioner():
    """GMRES on A~ x = b with the IFMM of the same operators as preconditioner:
    the preconditioned operator is the identity up to eps, so it converges at
    once; the solution is A~'s."""
    pts = bumpy_sphere(2048, 4)
    b = point_source_rhs(pts)
    t = ifmm.ifmm_build_tree(pts, 3)
    ifmm.ifmm_color(t, 3)
    k = ifmm.default_kernel(len(pts), "fmm", 3)
    f = ifmm.ifmm_factor(t, 3, 1e-10)
    x, its, rel = ifmm.bem_gmres(t, b, precond=f, tol=1e-8, kernel=k)
    assert rel <= 1e-8 and its <= 2
    tree = Tree(pts, 3)
    At = fmm_matrix(tree, Operators(tree, 3))
    assert _rel(x, np.linalg.solve(At, b)) < 1e-7
    _, its0, _ = ifmm.bem_gmres(t, b, tol=1e-8, kernel=k)
    assert its < its0
