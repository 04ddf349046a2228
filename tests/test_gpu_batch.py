"""Independent problems factored and solved together (worker threads and
streams) give exactly what one-at-a-time calls give; the float-pair matvec's
autotuned source tile is one of its candidates and keeps the result exact."""

import numpy as np
import pytest

from oracle.operators import dense_matrix
from paper_1905_10602_gb300 import build as _build
from paper_1905_10602_gb300.workloads import Workload, batch_workloads, fibonacci_sphere, point_source_rhs

pytestmark = pytest.mark.gpu

_build.build()
from paper_1905_10602_gb300 import ifmm  # noqa: E402


def test_batched_factor_and_gmres_equal_individual():
    ws = [Workload("a", "sphere", 3000, 31, 3, 4, 1e-6), Workload("b", "torus", 5000, 32, 4, 4, 1e-6),
          Workload("c", "bumpy", 7000, 33, 4, 4, 1e-6), Workload("d", "sphere", 2500, 34, 3, 3, 1e-6),
          Workload("e", "torus", 9000, 35, 4, 4, 1e-6)]
    trees, bs = [], []
    for w in ws:
        pts = w.points()
        t = ifmm.ifmm_build_tree(pts, w.depth)
        ifmm.ifmm_color(t, w.sigma)
        trees.append(t)
        bs.append(point_source_rhs(pts))
    # the fourth problem has Chebyshev order 3: batch the order-4 ones
    idx = [0, 1, 2, 4]
    fb = ifmm.ifmm_factor_batched([trees[i] for i in idx], 4, 1e-6, precision="fp32", nworkers=3)
    for j, i in enumerate(idx):
        fi = ifmm.ifmm_factor(trees[i], 4, 1e-6, precision="fp32")
        assert np.array_equal(ifmm.ifmm_solve(fb[j], bs[i]), ifmm.ifmm_solve(fi, bs[i]))
    ks = [ifmm.default_kernel(trees[i].n, "df") for i in idx]
    xs, its, rel = ifmm.bem_gmres_batched([trees[i] for i in idx], [bs[i] for i in idx], fb, kernels=ks, nworkers=3)
    assert all(r <= 1e-8 for r in rel) and all(0 < k <= 6 for k in its)
    x1, it1, _ = ifmm.bem_gmres(trees[idx[1]], bs[idx[1]], precond=fb[1], kernel=ks[1])
    assert it1 == its[1] and np.array_equal(x1, xs[1])


def test_batch_workload_recipe():
    ws = batch_workloads(64, 5)
    assert len(ws) == 64 and {w.shape for w in ws} == {"sphere", "torus", "bumpy"}
    assert all(4096 <= w.n <= 65536 and 2 <= w.depth <= 6 and w.cheb_order == 4 for w in ws)


def test_autotuned_matvec_tile():
    pts = fibonacci_sphere(6000, 2)
    t = ifmm.ifmm_build_tree(pts, 4)
    assert list(ifmm.ifmm_tree_query(t, 0, "matvec_block")) == [0, 0]
    x = np.random.default_rng(5).standard_normal(len(pts))
    y = ifmm.bem_matvec(t, x, kernel=ifmm.default_kernel(len(pts), "df"))
    tile = ifmm.ifmm_tree_query(t, 0, "matvec_block")
    assert tile[0] in (128, 256, 512) and tile[1] in (1, 2, 3) and (tile[1] == 1 or tile[0] <= 256)
    ref = dense_matrix(pts) @ x
    assert np.linalg.norm(y - ref) / np.linalg.norm(ref) < 1e-12
