"""The batched GEMM of the Schur updates, element by element against the FP64
product (NumPy), through the diagnostic C-ABI entry ifmm_gemm_check.

Bounds follow from each arithmetic, relative to (|alpha| |op(A)| |op(B)| +
|beta| |C|) element by element, with u = 2^-24:
  fp32 (3xTF32 tensor-core MMAs): every operand is split into two TF32 parts
    whose sum is within 2^-22 of it, the dropped tail*tail term is below 2^-22,
    and the FP32 accumulation over k terms adds at most about k * 2u: bound
    (k + 8) * 2^-22.  A single TF32 pass would sit near 2^-11 normwise; the
    normwise error here must stay below 2e-6.
  bf16: operands rounded to bfloat16 (8 significant bits: relative error up
    to 2^-8 each, 2^-7 per product), FP32 accumulation:
    2^-7 + (k + 8) * 2^-22; and the result must differ from the fp32 mode's.
  fp64: (k + 2) * 2^-52.
Shapes span one and several tiles of both tile classes (64 and 128), ragged
tails in every dimension, k = 1 and k beyond one 32-deep slice, all four
transpose combinations and alpha, beta in {1, -1, 0.3, 0}.
"""

import numpy as np
import pytest

from paper_1905_10602_gb300 import build as _build

pytestmark = pytest.mark.gpu

_build.build()
from paper_1905_10602_gb300 import ifmm  # noqa: E402

SHAPES = [(33, 40, 7), (64, 64, 64), (65, 130, 31), (200, 129, 300), (1, 70, 5), (70, 1, 9), (128, 128, 1),
          (129, 257, 33), (512, 96, 513), (40, 33, 0)]


def _case(m, n, k, ta, tb, seed):
    rng = np.random.default_rng(seed)
    A = rng.standard_normal((k, m) if ta else (m, k))
    B = rng.standard_normal((n, k) if tb else (k, n))
    # magnitudes spread over many binades (exercises the FP64 -> FP32 conversion)
    A *= np.exp2(rng.integers(-12, 13, size=A.shape))
    C = rng.standard_normal((m, n))
    return A, B, C


def _ref(A, B, C, alpha, beta, ta, tb):
    oA = A.T if ta else A
    oB = B.T if tb else B
    exact = alpha * (oA @ oB) + beta * C
    scale = abs(alpha) * (np.abs(oA) @ np.abs(oB)) + abs(beta) * np.abs(C)
    return exact, scale


@pytest.mark.parametrize("prec", ["fp32", "bf16", "fp64"])
@pytest.mark.parametrize("shape", SHAPES)
def test_gemm_against_fp64_product(prec, shape):
    m, n, k = shape
    for ta in (False, True):
        for tb in (False, True):
            for alpha, beta in ((1.0, 0.0), (-1.0, 1.0), (0.3, 0.3)):
                A, B, C = _case(m, n, k, ta, tb, hash((m, n, k, ta, tb)) % 2 ** 31)
                out = ifmm.ifmm_gemm_check(prec, A, B, C, alpha, beta, ta, tb)
                exact, scale = _ref(A, B, C, alpha, beta, ta, tb)
                if prec == "fp32":
                    bound = (k + 8) * 2.0 ** -22
                elif prec == "bf16":
                    bound = 2.0 ** -7 + (k + 8) * 2.0 ** -22
                else:
                    bound = (k + 2) * 2.0 ** -52
                err = np.abs(out - exact)
                assert np.all(err <= bound * scale + 1e-300), (prec, shape, ta, tb, alpha, beta, (err / scale).max())
                if prec == "fp32" and k:
                    assert np.linalg.norm(err) <= 2e-6 * np.linalg.norm(scale), np.linalg.norm(err) / np.linalg.norm(scale)


def test_bf16_rounds_operands():
    """The BF16 mode really rounds its operands: it differs from the fp32 mode by
    about the bfloat16 unit, far more than FP32 rounding."""
    A, B, C = _case(200, 129, 300, False, False, 3)
    o32 = ifmm.ifmm_gemm_check("fp32", A, B)
    o16 = ifmm.ifmm_gemm_check("bf16", A, B)
    d = np.linalg.norm(o16 - o32) / np.linalg.norm(o32)
    assert 1e-5 < d < 1e-2, d
