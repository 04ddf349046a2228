"""The FP64 Gauss-Jordan inverse of the pivot blocks (Algorithm 1 inverts every
Pi_i), through the diagnostic C-ABI entry ifmm_inv_check, on matrices that need
row interchanges at almost every step (Gaussian entries): orders spanning the
one-CTA shared-memory class, the cluster class (alone and in a batch, so with 8
and with fewer CTAs per block) and ragged orders; bit-identical results over
repeated calls (a missing barrier after the pivot-row swap once made them vary);
an exactly singular block reported through info.

Bound: Gauss-Jordan with partial pivoting has a residual ||A X - I|| of order
n u ||A|| ||X|| (u = 2^-53); the test allows 8 n u, normwise (Frobenius)."""

import numpy as np
import pytest

from paper_1905_10602_gb300 import build as _build

pytestmark = pytest.mark.gpu

_build.build()
from paper_1905_10602_gb300 import ifmm  # noqa: E402

U = 2.0 ** -53


def _residual(A, X):
    n = A.shape[0]
    return np.linalg.norm(A @ X - np.eye(n)) / (np.linalg.norm(A) * np.linalg.norm(X))


@pytest.mark.parametrize("orders", [[1, 2, 5, 31, 32, 33], [100, 160, 161], [300], [517], [200] * 12, [64] * 40])
def test_inverse_residual_and_repeatability(orders):
    rng = np.random.default_rng(sum(orders))
    mats = [rng.standard_normal((n, n)) for n in orders]
    X, info = ifmm.ifmm_inv_check(mats)
    assert not info.any()
    for A, Xi in zip(mats, X):
        n = A.shape[0]
        assert _residual(A, Xi) <= 8 * n * U, (n, _residual(A, Xi))
    for _ in range(3):
        X2, _ = ifmm.ifmm_inv_check(mats)
        for a, b in zip(X, X2):
            assert np.array_equal(a, b)


def test_complex_two_by_two_form():
    """The real 2 x 2 form of a complex matrix (the Helmholtz pivot blocks): its
    inverse is the real form of the complex inverse."""
    rng = np.random.default_rng(7)
    n = 90
    Z = rng.standard_normal((n, n)) + 1j * rng.standard_normal((n, n))
    R = np.zeros((2 * n, 2 * n))
    R[0::2, 0::2] = Z.real
    R[1::2, 0::2] = Z.imag
    R[0::2, 1::2] = -Z.imag
    R[1::2, 1::2] = Z.real
    (X,), info = ifmm.ifmm_inv_check([R])
    assert info[0] == 0
    Zi = np.linalg.inv(Z)
    assert np.abs(X[0::2, 0::2] - Zi.real).max() <= 1e-10 * np.abs(Zi).max()
    assert np.abs(X[1::2, 0::2] - Zi.imag).max() <= 1e-10 * np.abs(Zi).max()


def test_singular_block_reports_step():
    rng = np.random.default_rng(3)
    A = rng.standard_normal((40, 40))
    A[:, 7] = 0.0  # column 7 is zero: no pivot at step 7 (0-based) whatever the row order
    B = rng.standard_normal((20, 20))
    X, info = ifmm.ifmm_inv_check([A, B])
    assert info[0] == 8 and info[1] == 0
    assert _residual(B, X[1]) <= 8 * 20 * U
