"""The binary64 -> binary32 conversion the FP32 kernels apply to their FP64
storage with integer operations (GB300's FP64 pipe is narrow), checked against
IEEE round-to-nearest as NumPy computes it: identical except at exact ties
(rounded away from zero here, to even by IEEE), flushing below the binary32
normal range to signed zero, and exact widening back."""

import numpy as np
import pytest

from paper_1905_10602_gb300 import build as _build

pytestmark = pytest.mark.gpu

_build.build()
from paper_1905_10602_gb300 import ifmm  # noqa: E402


@pytest.mark.parametrize("shift", [0, -37, 21])
def test_conversion_matches_ieee_rounding(shift):
    rng = np.random.default_rng(11)
    x = rng.standard_normal(200000) * 10.0 ** rng.uniform(-30, 30, 200000)
    x[:8] = [0.0, -0.0, 1.0, -1.5, 2.0 ** -126, 2.0 ** -127, 3.4e38, np.nextafter(1.0, 2.0)]
    # exact ties: 24 significant bits then a single 1
    x[8:16] = (1.0 + np.arange(8) * 2.0 ** -20 + 2.0 ** -24) * 2.0 ** (-shift)
    f, back = ifmm.ifmm_convert_check(x, shift)
    xs = x * 2.0 ** shift
    ref = xs.astype(np.float32)
    normal = (np.abs(xs) >= np.finfo(np.float32).tiny) & (np.abs(xs) < 3.0e38)
    bits = xs.view(np.uint64) & np.uint64((1 << 29) - 1)
    tie = bits == np.uint64(1 << 28)
    same = (f == ref) | (np.isinf(f) & np.isinf(ref))
    assert np.all(same[normal & ~tie])
    # ties: rounded away from zero
    assert np.all(np.abs(f[normal & tie].astype(np.float64)) >= np.abs(xs[normal & tie]))
    # below the normal range: signed zero
    small = (np.abs(xs) < np.finfo(np.float32).tiny)
    assert np.all(f[small] == 0.0) and np.all(np.signbit(f[small]) == np.signbit(xs[small]))
    # widening is exact
    fin = np.isfinite(f) & (f != 0)
    assert np.array_equal(back[fin], f[fin].astype(np.float64) * 2.0 ** (-shift))
