"""The recompression QR kernels (Algorithm 1 truncates each fill-in block by a
pivoted QR; the weight stacks take a plain QR), through the diagnostic C-ABI
entry ifmm_qr_check, on Gaussian matrices whose shapes select each size class:
a warp per problem, a CTA per problem in each shared-memory size class,
row-chunked reduction for blocks taller than a CTA's shared memory, wide
blocks (m < n), ragged widths.

Checks, against the plain definitions (NumPy):
  * R^T R = A^T A (A P for the pivoted QR) to (m + n) u ||A||_F^2, the
    backward-error bound of Householder QR (u = 2^-24 in FP32, 2^-53 in FP64);
  * R equals NumPy's R up to the sign of each row (R is unique up to those
    signs for a full-rank A), to cond(A) (m + n) u relative;
  * pivoted: a permutation, min(m, n) steps, and |R_kk| non-increasing (each
    step takes the column of largest remaining norm; up to rounding);
  * two calls give bit-identical results."""

import numpy as np
import pytest

from paper_1905_10602_gb300 import build as _build

pytestmark = pytest.mark.gpu

_build.build()
from paper_1905_10602_gb300 import ifmm  # noqa: E402

U = {"fp32": 2.0 ** -24, "fp64": 2.0 ** -53}
SHAPES = [(20, 8), (1, 5), (5, 1), (100, 60), (300, 60), (700, 60), (500, 33), (260, 130), (3000, 60), (64, 100),
          (900, 17), (150, 47)]


def _matrix(m, n, seed):
    rng = np.random.default_rng(seed)
    A = rng.standard_normal((m, n))
    return A * np.exp2(rng.integers(-3, 4, size=(1, n)))  # column scales over a few binades


@pytest.mark.parametrize("prec", ["fp32", "fp64"])
@pytest.mark.parametrize("shape", SHAPES)
def test_plain_qr(prec, shape):
    m, n = shape
    A = _matrix(m, n, m * 1000 + n)
    if prec == "fp32":
        A = A.astype(np.float32).astype(np.float64)  # the kernels see FP32 data
    R = ifmm.ifmm_qr_check(A, prec)
    u, k = U[prec], min(m, n)
    nA2 = np.linalg.norm(A) ** 2
    assert R.shape == (k, n)
    assert np.linalg.norm(A.T @ A - R.T @ R) <= (m + n) * u * nA2
    Rn = np.linalg.qr(A, mode="r")
    if k == n and m >= n:
        s = np.sign(np.diag(R)) * np.sign(np.diag(Rn))
        cond = np.linalg.cond(A)
        assert np.linalg.norm(s[:, None] * R - Rn) <= cond * (m + n) * u * np.linalg.norm(Rn)
    assert np.array_equal(R, ifmm.ifmm_qr_check(A, prec))


@pytest.mark.parametrize("prec", ["fp32", "fp64"])
@pytest.mark.parametrize("shape", [(20, 8), (100, 60), (300, 60), (64, 100), (500, 33), (150, 47)])
def test_pivoted_qr(prec, shape):
    m, n = shape
    A = _matrix(m, n, 7 * m + n)
    if prec == "fp32":
        A = A.astype(np.float32).astype(np.float64)
    R, jp, k = ifmm.ifmm_qr_check(A, prec, pivoted=True)
    u, kk = U[prec], min(m, n)
    assert k == kk
    assert sorted(jp.tolist()) == list(range(n))
    Ap = A[:, jp]
    assert np.linalg.norm(Ap.T @ Ap - R.T @ R) <= (m + n) * u * np.linalg.norm(A) ** 2
    d = np.abs(np.diag(R))
    assert np.all(d[1:] <= d[:-1] * (1 + 64 * u) + 1e-300)
    R2, jp2, _ = ifmm.ifmm_qr_check(A, prec, pivoted=True)
    assert np.array_equal(R, R2) and np.array_equal(jp, jp2)
