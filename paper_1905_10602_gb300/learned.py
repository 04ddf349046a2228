"""Training the rank predictor from SVD-mode factorizations (on the GPU).

train_rank_model factors each training problem with exact SVD truncation,
collects every recompression event's inputs and chosen rank (ifmm_fact_events),
and fits the MLP with the library's training kernels (ifmm_mlp_train).  The
targets are rank / 64.
"""

from __future__ import annotations

import numpy as np

from . import ifmm
from .workloads import WORKLOADS, Workload


def collect_events(w: Workload, eps: float, precision: str = "fp32"):
    pts = w.points()
    t = ifmm.ifmm_build_tree(pts, w.depth)
    ifmm.ifmm_color(t, w.sigma)
    f = ifmm.ifmm_factor(t, w.cheb_order, eps, precision=precision)
    X, r = ifmm.ifmm_fact_events(f)
    return X, r


def train_rank_model(train=("sphere2k", "sphere32k", "torus65k"), eps_list=(1e-4, 1e-6, 1e-8), epochs=300,
                     seed=1, precision="fp32"):
    """Returns (weights, final loss, number of training events)."""
    Xs, ys = [], []
    for name in train:
        for eps in eps_list:
            X, r = collect_events(WORKLOADS[name] if isinstance(name, str) else name, eps, precision)
            Xs.append(X)
            ys.append(r.astype(np.float32) / 64.0)
    X = np.concatenate(Xs)
    y = np.concatenate(ys)
    perm = np.random.default_rng(seed).permutation(len(y))
    w, loss = ifmm.ifmm_mlp_train(X[perm], y[perm], epochs=epochs, batch=4096, lr=1e-3, seed=seed)
    return w, loss, len(y)
