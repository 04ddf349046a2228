"""The benchmarked workloads at full size, as the bench runs them (FP32 mixed
factor, float-pair direct-sum matvec, GMRES(30) to 1e-8), checked by properties
that hold at any size and that the oracle can verify on samples:

  * the solution's residual, recomputed on sampled rows by the oracle's own
    direct sum (Sec. 4.1's matrix, independent of the GPU's matvec), is at the
    GMRES tolerance;
  * at N = 131,072 the FP64 path (FP64 factor and matvec) reaches a solution
    that agrees with the mixed one to the accuracy both satisfy: with A's
    condition number of a few (a second-kind equation), two solutions at
    relative residual 1e-8 differ by at most a small multiple of 1e-8.
"""

import numpy as np
import pytest

from oracle.dense import direct_matvec
from paper_1905_10602_gb300 import build as _build
from paper_1905_10602_gb300.workloads import WORKLOADS

pytestmark = pytest.mark.gpu

_build.build()
from paper_1905_10602_gb300 import ifmm  # noqa: E402


def _solve(w, precision, arith):
    pts = w.points()
    b = w.rhs(pts)
    t = ifmm.ifmm_build_tree(pts, w.depth)
    ifmm.ifmm_color_levels(t, w.sigma, 2)
    k = ifmm.default_kernel(w.n, arith)
    f = ifmm.ifmm_factor(t, w.cheb_order, w.eps, kernel=k, precision=precision)
    x, its, rel = ifmm.bem_gmres(t, b, precond=f, tol=1e-8, kernel=k)
    return pts, b, x, its, rel


@pytest.mark.parametrize("name", ["bumpy131k", "torus262k"])
def test_mixed_solution_residual_on_sampled_rows(name):
    w = WORKLOADS[name]
    pts, b, x, its, rel = _solve(w, "fp32", "df")
    assert rel <= 1e-8 and its <= 6
    rows = np.random.default_rng(7).choice(w.n, 96, replace=False)
    r = direct_matvec(pts, x, rows) - b[rows]
    assert np.linalg.norm(r) / np.linalg.norm(b[rows]) < 1e-7


def test_mixed_and_fp64_solutions_agree_at_full_size():
    w = WORKLOADS["bumpy131k"]
    _, _, x32, _, rel32 = _solve(w, "fp32", "df")
    _, _, x64, _, rel64 = _solve(w, "fp64", "fp64")
    assert rel32 <= 1e-8 and rel64 <= 1e-8
    assert np.linalg.norm(x32 - x64) / np.linalg.norm(x64) < 1e-7
