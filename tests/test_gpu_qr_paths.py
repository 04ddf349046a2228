"""The size paths of the recompression QR: one warp per block, one CTA per block,
the in-place tall reduction, a thread-block cluster per block (rows split over
2-8 CTAs, exchanging through distributed shared memory), and the global-memory
kernel.  On the small parity cases nearly every block takes the first two paths,
so these tests lower the per-CTA shared-memory limit (IFMM_QR_CTA_LIMIT_KB, read
once per process) in a child process (and, for the pivot inverses, send large
blocks to the batched multi-CTA Gauss-Jordan with IFMM_INV_FALLBACK_N); the factor must still reproduce the
oracle's applied inverse to 1e-9 with its ranks replayed (FP64) and keep GMRES
convergence in FP32.
"""

import json
import os
import subprocess
import sys

import pytest

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

CHILD = r"""
import json, sys
import numpy as np
sys.path.insert(0, %(root)r)
from oracle.ifmm import IFMMOracle
from paper_1905_10602_gb300 import build as _build
from paper_1905_10602_gb300.workloads import bumpy_sphere, point_source_rhs
_build.build()
from paper_1905_10602_gb300 import ifmm
pts = bumpy_sphere(3000, 3)
b = point_source_rhs(pts)
o = IFMMOracle(pts, 4, 4, 1e-6, 3).factor()
t = ifmm.ifmm_build_tree(pts, 4)
ifmm.ifmm_color(t, 3)
rep = [list(k) + [v] for k, v in o.ranks().items()]
ifmm.ifmm_profile(False)
f = ifmm.ifmm_factor(t, 4, 1e-6, rank_mode="replay", replay=rep)
R = np.random.default_rng(7).standard_normal((2, len(pts)))
V = ifmm.ifmm_solve(f, R)
err = max(np.linalg.norm(V[k] - o.solve(R[k])) / np.linalg.norm(o.solve(R[k])) for k in range(2))
prof = ifmm.ifmm_profile_query()
f32 = ifmm.ifmm_factor(t, 4, 1e-6, precision="fp32")
x, its, rel = ifmm.bem_gmres(t, b, precond=f32, tol=1e-8, kernel=ifmm.default_kernel(len(pts), "df"))
print(json.dumps({"err": err, "its": its, "rel": rel,
                  "cluster": prof.get("qr_cluster_fp64", (0, 0.0))[0],
                  "global": prof.get("qr_global_fp64", (0, 0.0))[0],
                  "gj_batched": prof.get("gauss_jordan_big", (0, 0.0))[0]}))
"""


def _run(limit_kb, env_extra=None):
    env = dict(os.environ, IFMM_QR_CTA_LIMIT_KB=str(limit_kb), **(env_extra or {}))
    out = subprocess.run([sys.executable, "-c", CHILD % {"root": ROOT}], capture_output=True, text=True, env=env,
                         timeout=900)
    assert out.returncode == 0, out.stderr[-3000:]
    return json.loads(out.stdout.strip().splitlines()[-1])


@pytest.mark.parametrize("limit_kb", [8, 24])
def test_qr_paths_replay_parity(limit_kb):
    r = _run(limit_kb)
    assert r["err"] < 1e-9, r
    assert r["rel"] <= 1e-8, r
    # the lowered limit sends blocks to the cluster kernel
    assert r["cluster"] > 0, r


def test_qr_global_memory_path_replay_parity():
    """At a 4 KB per-CTA limit even an 8-CTA cluster holds only 32 KB: the larger
    blocks take the global-memory pivoted QR (k_qrcp)."""
    r = _run(4)
    assert r["err"] < 1e-9 and r["rel"] <= 1e-8, r
    assert r["global"] > 0, r


def test_gauss_jordan_multi_cta_path_replay_parity():
    """IFMM_INV_FALLBACK_N sends every pivot block of >= 40 rows to the batched
    multi-CTA Gauss-Jordan (k_gjb_*); the factor still matches the oracle."""
    base = _run(220)
    r = _run(220, {"IFMM_INV_FALLBACK_N": "40"})
    assert r["err"] < 1e-9 and r["rel"] <= 1e-8, r
    # beyond the level-1 inverse's own launches (the same in both runs)
    assert r["gj_batched"] > base["gj_batched"], (base, r)
