"""Failure paths of the C ABI, all made on the host side (inputs and limits the
caller chooses), none by faulting the GPU: an exactly singular pivot block, a
GMRES run stopped by its iteration limit, a rank above max_rank, and device
points given to ifmm_build_tree."""

import numpy as np
import pytest

from paper_1905_10602_gb300 import build as _build
from paper_1905_10602_gb300.workloads import fibonacci_sphere, point_source_rhs

pytestmark = pytest.mark.gpu

_build.build()
from paper_1905_10602_gb300 import ifmm  # noqa: E402


def _tree(n=600, depth=3, sigma=3):
    t = ifmm.ifmm_build_tree(fibonacci_sphere(n, 1), depth)
    ifmm.ifmm_color(t, sigma)
    return t


def test_exactly_singular_pivot_is_esingular():
    """The zero matrix (scale 0, diagonal 0): every P2P_ii is zero and the far
    field has rank 0, so the first pivot block Pi_i = P2P_ii is exactly singular
    (Algorithm 1's 'factorize P2P_ii' cannot proceed)."""
    t = _tree()
    with pytest.raises(ifmm.IFMMError) as e:
        ifmm.ifmm_factor(t, 3, 1e-6, kernel=ifmm.Kernel(0.0, 0.0, 0, 0, 0.0, 0.0))
    assert e.value.code == 4 and "singular" in str(e.value)
    # the library stays usable afterwards
    f = ifmm.ifmm_factor(t, 3, 1e-6)
    assert np.isfinite(ifmm.ifmm_solve(f, point_source_rhs(fibonacci_sphere(600, 1)))).all()


def test_gmres_iteration_limit_is_enoconv_with_outputs_written():
    n = 600
    t = _tree(n)
    b = point_source_rhs(fibonacci_sphere(n, 1))
    with pytest.raises(ifmm.IFMMError) as e:
        ifmm.bem_gmres(t, b, tol=1e-14, maxit=1)
    assert e.value.code == 5
    x, its, rel = ifmm.bem_gmres(t, b, tol=1e-14, maxit=1, raise_on_noconv=False)
    assert its == 1 and np.isfinite(x).all() and 1e-14 < rel < 1.0
    # the written x is GMRES's one-step iterate: it reduces the residual
    A_x = ifmm.bem_matvec(t, x)
    assert np.linalg.norm(A_x - b) / np.linalg.norm(b) == pytest.approx(rel, rel=1e-10)


def test_rank_above_max_rank_is_erank():
    t = _tree(1024)
    with pytest.raises(ifmm.IFMMError) as e:
        ifmm.ifmm_factor(t, 3, 1e-6, max_rank=2)
    assert e.value.code == 7 and "max_rank" in str(e.value)
    # with room enough the same problem factors
    ifmm.ifmm_factor(t, 3, 1e-6, max_rank=64)


def test_build_tree_from_device_points():
    import torch

    pts = fibonacci_sphere(2000, 3)
    th = ifmm.ifmm_build_tree(pts, 4)
    td = ifmm.ifmm_build_tree(torch.from_numpy(pts).cuda(), 4)
    for what in ("perm", "leaf_ptr"):
        assert np.array_equal(ifmm.ifmm_tree_query(th, 0, what), ifmm.ifmm_tree_query(td, 0, what))
    for lvl in range(2, 5):
        for what in ("cells", "nbr", "il"):
            assert np.array_equal(ifmm.ifmm_tree_query(th, lvl, what), ifmm.ifmm_tree_query(td, lvl, what))
