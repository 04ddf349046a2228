"""The block-diagonal preconditioner (BD / BDbot, Sec. 4.3) on the GPU against
the oracle, and as a GMRES preconditioner beside the IFMM (the paper's
comparison, Algorithms 4 and 5)."""

import numpy as np
import pytest

from oracle.bd import bd_apply
from oracle.tree import Tree
from paper_1905_10602_gb300 import build as _build
from paper_1905_10602_gb300.workloads import bumpy_sphere, fibonacci_sphere, point_source_rhs

pytestmark = pytest.mark.gpu

_build.build()
from paper_1905_10602_gb300 import ifmm  # noqa: E402


@pytest.mark.parametrize("N,depth,level", [(1500, 3, 3), (1500, 3, 2), (3001, 4, 2), (800, 3, 0), (2500, 4, 4)])
def test_bd_matches_oracle(N, depth, level):
    """Applied preconditioner within 1e-12 of the oracle's block solves (FP64
    Gauss-Jordan against LAPACK on blocks of up to a few hundred points)."""
    pts = bumpy_sphere(N, 7)
    t = ifmm.ifmm_build_tree(pts, depth)
    f = ifmm.ifmm_bd_factor(t, level)
    R = np.random.default_rng(level).standard_normal((2, N))
    V = ifmm.ifmm_solve(f, R)
    tree = Tree(pts, depth)
    for k in range(2):
        ref = bd_apply(tree, level, R[k])
        assert np.linalg.norm(V[k] - ref) / np.linalg.norm(ref) < 1e-12
    st = ifmm.ifmm_fact_stats(f)
    assert st["bd_level"] == level and st["bd_blocks"] == len(tree.levels[level].cells)


def test_bd_in_gmres_and_ifmm_needs_fewer_iterations():
    pts = fibonacci_sphere(4096, 3)
    b = point_source_rhs(pts)
    t = ifmm.ifmm_build_tree(pts, 4)
    ifmm.ifmm_color(t, 3)
    _, its0, _ = ifmm.bem_gmres(t, b, tol=1e-8)
    bd = ifmm.ifmm_bd_factor(t, 4)
    _, its_bd, rel_bd = ifmm.bem_gmres(t, b, precond=bd, tol=1e-8)
    bd2 = ifmm.ifmm_bd_factor(t, 2)
    _, its_bd2, rel_bd2 = ifmm.bem_gmres(t, b, precond=bd2, tol=1e-8)
    f = ifmm.ifmm_factor(t, 3, 1e-6)
    _, its_if, rel_if = ifmm.bem_gmres(t, b, precond=f, tol=1e-8)
    print(f"GMRES iterations: none {its0}, BDb4 {its_bd}, BDb2 {its_bd2}, IFMM {its_if}")
    assert max(rel_bd, rel_bd2, rel_if) <= 1e-8
    # the IFMM preconditioner needs far fewer iterations than BD; on this
    # well-conditioned second-kind system BD itself gains little or nothing
    # over no preconditioner
    assert its_if < min(its_bd, its_bd2) and its_if < its0
