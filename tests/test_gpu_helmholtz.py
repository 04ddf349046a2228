"""The Helmholtz kernel e^{ik r}/(4 pi r) (the paper's acoustic BEM, Sec. 4.1)
through the library's real 2 x 2 form of the complex entries, against the
complex NumPy oracle: matvec against the dense complex A, eps = 0 exactness
against the complex A~, the applied inverse with the oracle's ranks replayed
(a complex rank k is 2k real directions) within 1e-9, GMRES, and the reduced
precision modes."""

import numpy as np
import pytest

from oracle.dense import fmm_matrix
from oracle.ifmm import IFMMOracle
from oracle.operators import dense_matrix
from paper_1905_10602_gb300 import build as _build
from paper_1905_10602_gb300.workloads import bumpy_sphere, fibonacci_sphere, helmholtz_source_rhs, torus

pytestmark = pytest.mark.gpu

_build.build()
from paper_1905_10602_gb300 import ifmm  # noqa: E402


def _rel(a, b):
    return np.linalg.norm(a - b) / np.linalg.norm(b)


def _tree(pts, depth, sigma):
    t = ifmm.ifmm_build_tree(pts, depth)
    ifmm.ifmm_color(t, sigma)
    return t


@pytest.mark.parametrize("k", [0.5, 4.0, 16.0])
def test_helmholtz_matvec_matches_dense(k):
    pts = torus(1700, 2)
    t = ifmm.ifmm_build_tree(pts, 3)
    x = np.random.default_rng(1).standard_normal(len(pts)) + 1j * np.random.default_rng(2).standard_normal(len(pts))
    y = ifmm.bem_matvec(t, x, kernel=ifmm.helmholtz_kernel(len(pts), k))
    assert y.dtype == np.complex128
    assert _rel(y, dense_matrix(pts, k) @ x) < 1e-13


@pytest.mark.parametrize("N,depth,p,sigma,k", [(900, 3, 3, 3, 2.0), (1200, 3, 3, 6, 8.0), (600, 2, 2, 3, 4.0),
                                               (200, 2, 2, 3, 2.0), (60, 2, 2, 3, 2.0)])
def test_helmholtz_exact_at_eps0(N, depth, p, sigma, k):
    pts = fibonacci_sphere(N, 2)
    b = helmholtz_source_rhs(pts, k)
    o = IFMMOracle(pts, depth, p, 0.0, sigma, wavenumber=k).factor()
    t = _tree(pts, depth, sigma)
    f = ifmm.ifmm_factor(t, p, 0.0, kernel=ifmm.helmholtz_kernel(N, k))
    x = ifmm.ifmm_solve(f, b)
    At = fmm_matrix(o.tree, o.ops)
    assert _rel(x, np.linalg.solve(At, b)) < 1e-10
    assert _rel(x, o.solve(b)) < 1e-10


@pytest.mark.parametrize("shape,N,depth,p,eps,sigma,k", [("sphere", 2048, 3, 3, 1e-6, 3, 4.0),
                                                          ("bumpy", 2500, 4, 3, 1e-6, 3, 8.0),
                                                          ("torus", 1500, 3, 3, 1e-4, 6, 2.0)])
def test_helmholtz_replay_parity(shape, N, depth, p, eps, sigma, k):
    pts = {"sphere": fibonacci_sphere, "bumpy": bumpy_sphere, "torus": torus}[shape](N, 3)
    o = IFMMOracle(pts, depth, p, eps, sigma, wavenumber=k).factor()
    t = _tree(pts, depth, sigma)
    rep = [list(key) + [2 * r] for key, r in o.ranks().items()]
    f = ifmm.ifmm_factor(t, p, eps, kernel=ifmm.helmholtz_kernel(N, k), rank_mode="replay", replay=rep)
    rng = np.random.default_rng(5)
    R = rng.standard_normal((2, N)) + 1j * rng.standard_normal((2, N))
    V = ifmm.ifmm_solve(f, R)
    for j in range(2):
        assert _rel(V[j], o.solve(R[j])) < 1e-9


def test_helmholtz_free_ranks_are_twice_the_complex_ranks():
    """Without replay the real form keeps the singular-value pairs together: its
    ranks are twice the complex oracle's except where a pair straddles the
    threshold within rounding; the solve is within eps of the oracle's."""
    pts = fibonacci_sphere(2048, 1)
    k = 4.0
    o = IFMMOracle(pts, 3, 3, 1e-6, 6, wavenumber=k).factor()
    t = _tree(pts, 3, 6)
    f = ifmm.ifmm_factor(t, 3, 1e-6, kernel=ifmm.helmholtz_kernel(len(pts), k))
    rg, ro = ifmm.ifmm_fact_ranks(f), o.ranks()
    assert rg.keys() == ro.keys()
    assert sum(abs(rg[q] - 2 * ro[q]) > 1 for q in ro) <= 0.01 * len(ro)
    b = helmholtz_source_rhs(pts, k)
    assert _rel(ifmm.ifmm_solve(f, b), o.solve(b)) < 1e-5


@pytest.mark.parametrize("prec,bound", [("fp64", 1e-9), ("fp32", 1e-4)])
def test_helmholtz_gmres(prec, bound):
    pts = bumpy_sphere(4096, 3)
    k = 8.0
    b = helmholtz_source_rhs(pts, k)
    t = _tree(pts, 4, 3)
    kern = ifmm.helmholtz_kernel(len(pts), k)
    f = ifmm.ifmm_factor(t, 3, 1e-6, kernel=kern, precision=prec)
    x, its, rel = ifmm.bem_gmres(t, b, precond=f, tol=1e-8, kernel=kern)
    _, its0, _ = ifmm.bem_gmres(t, b, tol=1e-8, kernel=kern)
    print(f"Helmholtz k={k} {prec}: GMRES {its} iterations with the IFMM, {its0} without")
    assert rel <= 1e-8 and its < its0
    A = dense_matrix(pts, k)
    assert np.linalg.norm(A @ x - b) / np.linalg.norm(b) <= 1.01e-8
    o64 = ifmm.ifmm_factor(t, 3, 1e-6, kernel=kern)
    assert _rel(ifmm.ifmm_solve(f, b), ifmm.ifmm_solve(o64, b)) < bound


def test_helmholtz_refusals():
    pts = fibonacci_sphere(500, 1)
    t = _tree(pts, 3, 3)
    k = ifmm.helmholtz_kernel(500, 2.0)
    k.arith = 1  # float-pair matvec: Laplace only
    with pytest.raises(ifmm.IFMMError):
        ifmm.bem_matvec(t, np.zeros(500, dtype=np.complex128), kernel=k)
    with pytest.raises(ifmm.IFMMError):
        ifmm.ifmm_bd_factor(t, 3, kernel=ifmm.helmholtz_kernel(500, 2.0))


def test_factor_is_repeatable():
    """The same factorization twice gives bit-identical solves (the pivot blocks
    of the 2 x 2 form need row interchanges, which once raced with the reads of
    the pivot row)."""
    pts = fibonacci_sphere(200, 2)
    k = 2.0
    t = _tree(pts, 2, 3)
    b = helmholtz_source_rhs(pts, k)
    xs = [ifmm.ifmm_solve(ifmm.ifmm_factor(t, 2, 0.0, kernel=ifmm.helmholtz_kernel(200, k)), b) for _ in range(4)]
    for x in xs[1:]:
        assert np.array_equal(x, xs[0])
