"""One IFMM factorization + preconditioned GMRES through the C ABI, without
PyTorch, for profilers: `python -m paper_1905_10602_gb300.profile_case
--shape bumpy --n 16384 --depth 5 --order 4 --eps 1e-6 --sigma 3 --precision fp32`."""

from __future__ import annotations

import argparse
import json
import time

from . import build as _build


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--shape", default="bumpy")
    ap.add_argument("--n", type=int, default=16384)
    ap.add_argument("--depth", type=int, default=5)
    ap.add_argument("--order", type=int, default=4)
    ap.add_argument("--eps", type=float, default=1e-6)
    ap.add_argument("--sigma", type=int, default=3)
    ap.add_argument("--seed", type=int, default=3)
    ap.add_argument("--precision", default="fp32")
    a = ap.parse_args()
    _build.build()
    from . import ifmm
    from .workloads import point_source_rhs, surface

    pts = surface(a.shape, a.n, a.seed)
    b = point_source_rhs(pts)
    t = ifmm.ifmm_build_tree(pts, a.depth)
    ifmm.ifmm_color(t, a.sigma)
    arith = "fp64" if a.precision == "fp64" else "df"
    k = ifmm.default_kernel(a.n, arith)
    t0 = time.perf_counter()
    f = ifmm.ifmm_factor(t, a.order, a.eps, kernel=k, precision=a.precision)
    x, its, rel = ifmm.bem_gmres(t, b, precond=f, tol=1e-8, kernel=k)
    st = ifmm.ifmm_fact_stats(f)
    print(json.dumps({"seconds": time.perf_counter() - t0, "gmres_iterations": its, "relres": rel,
                      "factor_s": st["time_factor"], "flops_qr": st["flops_qr"], "flops_svd": st["flops_svd"]}))


if __name__ == "__main__":
    main()
