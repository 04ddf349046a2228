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
from paper_1905_10602_gb300.workloads import bumpy_sphere, fibonacci_sphere, torus

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
    for call in range(2):
        x = rng.standard_normal(len(pts))
        ref = ifmm.bem_matvec(t, x, kernel=k)  # existing entry point; also makes the tree resident
        xd = torch.from_numpy(x).cuda()
        yd = torch.full_like(xd, float("nan"))
        torch.cuda.synchronize()
        free0 = torch.cuda.mem_get_info()[0]
        ifmm.bem_matvec_noalloc(t, xd, yd, kernel=k)
        torch.cuda.synchronize()
        # the call itself takes no device memory (its module was loaded when the
        # tree was made resident)
        assert torch.cuda.mem_get_info()[0] == free0, call
        y = yd.cpu().numpy()
        assert np.linalg.norm(y - ref) / np.linalg.norm(ref) < 1e-13


def test_noalloc_float_pairs_against_fp64_second_surface():
    """The float-pair sums of the allocation-free path against its own FP64 sums
    on another surface and size (a randomly sampled torus, odd N), two calls in a
    row, row by row within the bound of the pair representation: each
    coordinate is a float pair within 2^-49 |p| of its double (so a distance
    moves by at most 2^-46 R, R the largest coordinate, and the term x_j / r_ij
    by 2^-46 R |x_j| / r_ij^2: close pairs dominate), and the pair arithmetic
    adds at most 2^-40 |x_j| / r_ij per term."""
    import torch

    pts = torus(9001, 6)
    n = len(pts)
    t = ifmm.ifmm_build_tree(pts, 5)
    ifmm.bem_matvec(t, np.zeros(n))  # makes the tree resident
    rng = np.random.default_rng(12)
    R = np.abs(pts).max()
    for _ in range(2):
        x = rng.standard_normal(n)
        xd = torch.from_numpy(x).cuda()
        y64, ydf = torch.empty_like(xd), torch.empty_like(xd)
        ifmm.bem_matvec_noalloc(t, xd, y64, kernel=ifmm.default_kernel(n, "fp64"))
        ifmm.bem_matvec_noalloc(t, xd, ydf, kernel=ifmm.default_kernel(n, "df"))
        torch.cuda.synchronize()
        diff = np.abs(ydf.cpu().numpy() - y64.cpu().numpy())
        s1, s2 = np.empty(n), np.empty(n)
        for a in range(0, n, 512):
            d = np.sqrt(((pts[a:a + 512, None, :] - pts[None, :, :]) ** 2).sum(axis=2))
            d[np.arange(d.shape[0]), np.arange(a, a + d.shape[0])] = np.inf
            s1[a:a + 512] = (np.abs(x)[None, :] / d).sum(axis=1)
            s2[a:a + 512] = (np.abs(x)[None, :] / d ** 2).sum(axis=1)
        bound = (2.0 ** -40 * s1 + 2.0 ** -46 * R * s2) / n
        assert np.all(diff <= bound), (diff / bound).max()


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
