"""The allocation-free matvec (bem_matvec_noalloc) against bem_matvec.

Some callers cannot allocate device memory (a host framework that owns the
device memory pool, or code that must not risk the synchronisation an
allocation implies); bem_matvec_noalloc serves them from a fixed scratch array
inside the library.  Here it must reproduce bem_matvec on two calls in a row,
within the matvec tolerance of the other tests, and refuse what it cannot do
without allocating.  This file is collected last on purpose.
"""

import numpy as np
import pytest

from paper_1905_10602_gb300 import build as _build
from paper_1905_10602_gb300.workloads import bumpy_sphere, fibonacci_sphere

pytestmark = pytest.mark.gpu

_build.build()
from paper_1905_10602_gb300 import ifmm  # noqa: E402


@pytest.mark.parametrize("arith", ["fp64", "df"])
def test_noalloc_matches_bem_matvec_two_calls(arith):
    import torch

    pts = bumpy_sphere(20000, 3)
    t = ifmm.ifmm_build_tree(pts, 5)
    k = ifmm.default_kernel(len(pts), arith)
    rng = np.random.default_rng(11)
    for _ in range(2):
        x = rng.standard_normal(len(pts))
        ref = ifmm.bem_matvec(t, x, kernel=k)  # existing entry point; also makes the tree resident
        xd = torch.from_numpy(x).cuda()
        yd = torch.full_like(xd, float("nan"))
        ifmm.bem_matvec_noalloc(t, xd, yd, kernel=k)
        torch.cuda.synchronize()
        y = yd.cpu().numpy()
        assert np.linalg.norm(y - ref) / np.linalg.norm(ref) < 1e-13


def test_noalloc_refuses_what_needs_allocation():
    import torch

    small = ifmm.ifmm_build_tree(fibonacci_sphere(1000, 1), 3)
    x = torch.zeros(1000, dtype=torch.float64, device="cuda")
    y = torch.zeros_like(x)
    with pytest.raises(ifmm.IFMMError) as e:  # tree not uploaded yet
        ifmm.bem_matvec_noalloc(small, x, y)
    assert e.value.code == 1 and "resident" in str(e.value)
    big = ifmm.ifmm_build_tree(fibonacci_sphere(262145, 1), 3)
    xb = torch.zeros(262145, dtype=torch.float64, device="cuda")
    with pytest.raises(ifmm.IFMMError) as e:  # beyond the fixed scratch
        ifmm.bem_matvec_noalloc(big, xb, torch.zeros_like(xb))
    assert e.value.code == 1 and "262144" in str(e.value)
