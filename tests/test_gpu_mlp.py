"""Rank-predictor kernels (forward, backward, Adam training) against the NumPy
network, and the learned rank mode of the factorization."""

import numpy as np
import pytest

from oracle import mlp as ref
from paper_1905_10602_gb300 import build as _build
from paper_1905_10602_gb300.workloads import bumpy_sphere, point_source_rhs, torus

pytestmark = pytest.mark.gpu

_build.build()
from paper_1905_10602_gb300 import ifmm  # noqa: E402
from paper_1905_10602_gb300.learned import train_rank_model  # noqa: E402


def _rand(seed, n):
    rng = np.random.default_rng(seed)
    w = (rng.standard_normal(ref.nweights()) * 0.15).astype(np.float32)
    X = rng.uniform(-1, 1, (n, 9)).astype(np.float32)
    t = rng.uniform(0, 1, n).astype(np.float32)
    return w, X, t


def test_forward_matches_numpy():
    w, X, _ = _rand(1, 300)
    y = ifmm.ifmm_mlp_forward(w, X)
    yr, _ = ref.forward(w, X)
    assert np.abs(y - yr).max() <= 1e-5 * max(1.0, np.abs(yr).max())


def test_backward_matches_numpy_backprop():
    w, X, t = _rand(2, 257)
    loss, g = ifmm.ifmm_mlp_grad(w, X, t)
    lr, gr = ref.loss_and_grad(w, X, t)
    assert abs(loss - lr) <= 1e-5 * max(1.0, lr)
    assert np.linalg.norm(g - gr) <= 1e-4 * np.linalg.norm(gr)


def test_training_fits_a_smooth_target():
    rng = np.random.default_rng(3)
    X = rng.uniform(-1, 1, (6000, 9)).astype(np.float32)
    t = (0.3 + 0.2 * np.sin(2 * X[:, 0]) * X[:, 4] + 0.1 * X[:, 8]).astype(np.float32)
    w, loss = ifmm.ifmm_mlp_train(X, t, epochs=150, batch=1000, lr=2e-3, seed=4)
    base = 0.5 * np.var(t)
    assert loss < 0.1 * base, (loss, base)
    y = ifmm.ifmm_mlp_forward(w, X)
    assert abs(0.5 * np.mean((y - t) ** 2) - loss) <= 1e-3 * base + 1e-6


def test_learned_rank_mode_end_to_end():
    """Trained on SVD-mode ranks of smaller problems of the same families, applied
    to a larger torus: the network predicts ranks to about one unit, wide
    recompressions run as a randomized range finder at the predicted rank, few
    fail the residual check, the chosen ranks equal the SVD mode's and GMRES still
    reaches 1e-8.  The time of both modes is printed: what the network gains (or
    costs) over the exact path on this GPU."""
    from paper_1905_10602_gb300.workloads import Workload

    train = (Workload("sph8k", "sphere", 8192, 21, 4, 4, 1e-6), Workload("tor8k", "torus", 8192, 22, 4, 4, 1e-6),
             Workload("tor16k", "torus", 16384, 23, 5, 4, 1e-6))
    w, loss, nev = train_rank_model(train=train, eps_list=(1e-5, 1e-6, 1e-7), epochs=200, precision="fp64")
    assert nev > 5000 and np.isfinite(loss)
    pts = torus(32768, 4)
    b = point_source_rhs(pts)
    t = ifmm.ifmm_build_tree(pts, 5)
    ifmm.ifmm_color(t, 3)
    f_svd = ifmm.ifmm_factor(t, 4, 1e-6, precision="fp64")
    X, r = ifmm.ifmm_fact_events(f_svd)
    pred = ifmm.ifmm_mlp_forward(w, X) * 64
    err_mlp = float(np.abs(pred - r).mean())
    assert err_mlp < 3.0
    # without the network the best one can guess from the level alone is the
    # level's mean rank (taken here from the test events themselves); the
    # network's inputs (block size, current rank, fill rows, geometry) must
    # predict better than that
    lev = np.rint(X[:, 4] * 10).astype(int)
    base = np.zeros_like(pred)
    for L in np.unique(lev):
        base[lev == L] = r[lev == L].mean()
    err_base = float(np.abs(base - r).mean())
    print("mean |rank error|: network", err_mlp, "per-level mean", err_base)
    assert err_mlp < err_base
    f_lrn = ifmm.ifmm_factor(t, 4, 1e-6, precision="fp64", rank_mode="learned", mlp=w)
    s_svd, s_lrn = ifmm.ifmm_fact_stats(f_svd), ifmm.ifmm_fact_stats(f_lrn)
    print("mean |pred - rank|", float(np.abs(pred - r).mean()), "| factor s: svd", s_svd["time_factor"], "learned",
          s_lrn["time_factor"], {k: s_lrn[k] for k in ("learned_events", "learned_sketched", "learned_fallbacks")})
    assert s_lrn["learned_sketched"] > 0.05 * s_lrn["learned_events"]
    assert s_lrn["learned_fallbacks"] < 0.25 * s_lrn["learned_sketched"]
    r_svd, r_lrn = ifmm.ifmm_fact_ranks(f_svd), ifmm.ifmm_fact_ranks(f_lrn)
    same = sum(r_svd[k] == r_lrn.get(k) for k in r_svd) / len(r_svd)
    assert same > 0.95, same
    x, its, rel = ifmm.bem_gmres(t, b, precond=f_lrn, tol=1e-8)
    _, its0, _ = ifmm.bem_gmres(t, b, precond=f_svd, tol=1e-8)
    assert rel <= 1e-8 and its <= its0 + 1
