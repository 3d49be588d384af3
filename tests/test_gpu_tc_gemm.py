"""The tcgen05 BF16 GEMM tile (tensor memory accumulator) against float64
products of the same BF16-rounded operands."""

import numpy as np
import pytest

from paper_2005_02498_gb300 import ptadd

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("M,N,K", [(128, 16, 16), (200, 256, 256), (64, 32, 96), (1000, 48, 512), (37, 16, 32),
                                   (300, 112, 80), (128, 80, 64), (513, 256, 272)])
def test_tc_gemm_matches_float64(M, N, K):
    rng = np.random.default_rng(M * 7 + N * 3 + K)
    A = ptadd.to_bf16_bits(rng.normal(size=(M, K)).astype(np.float32))
    B = ptadd.to_bf16_bits(rng.normal(size=(N, K)).astype(np.float32))
    C = ptadd.gemm_bf16(A, B)
    ref = ptadd.from_bf16_bits(A).astype(np.float64) @ ptadd.from_bf16_bits(B).astype(np.float64).T
    assert C.shape == (M, N)
    err = np.max(np.abs(C - ref)) / np.max(np.abs(ref))
    assert err <= 1e-5, err


def test_bf16_rounding_helper():
    x = np.array([1.0, 1.00390625, 1.005859375, -3.3e-5, 65504.0], np.float32)
    b = ptadd.to_bf16_bits(x)
    y = ptadd.from_bf16_bits(b)
    assert y[0] == 1.0 and y[1] == 1.0  # tie rounds to even
    assert y[2] == np.float32(1.0078125)
    assert abs(y[3] / x[3] - 1) < 2 ** -8
