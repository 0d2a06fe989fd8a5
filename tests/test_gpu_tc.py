"""The tensor-core complex GEMM (tcgen05, 3xTF32) against the FP64 product.

Shapes cover the contractions of the one-site, two-site and bond effective
Hamiltonians and environment updates at chi in {16, 32, 64} (e.g. 320 x 128 x
64 and 128 x 64 x 320 at chi = 64), ragged sizes that leave partial M, N and K
tiles, both operand layouts and conjugation.  3xTF32 keeps FP32 accuracy: the
error is bounded by a few FP32 units of sum_k |A_ik| |B_kj|.
"""
import numpy as np
import pytest

from paper_2501_17913_gb300 import tjm

from gpu_common import lib_ready

pytestmark = pytest.mark.gpu


def _rand(rng, m, n):
    return (rng.standard_normal((m, n)) + 1j * rng.standard_normal((m, n))) / np.sqrt(2)


SHAPES = [(128, 16, 8), (320, 128, 64), (128, 64, 320), (64, 64, 320), (160, 64, 32), (80, 32, 16),
          (640, 256, 64), (256, 64, 640), (1, 1, 1), (37, 13, 29), (129, 130, 17), (200, 8, 3)]


@pytest.mark.parametrize("M,N,K", SHAPES)
def test_tc_cgemm_matches_fp64_product(M, N, K):
    lib_ready()
    rng = np.random.default_rng(M * 1000003 + N * 1009 + K)
    A = _rand(rng, M, K)
    B = _rand(rng, K, N)
    ref = A @ B
    bound = np.abs(A) @ np.abs(B)
    for ca, cb, acm, bkc in [(0, 0, 0, 0), (1, 0, 1, 0), (0, 1, 0, 1), (1, 1, 1, 1)]:
        Ao = A.conj() if ca else A
        Bo = B.conj() if cb else B
        C = tjm.selftest_tc_cgemm(A, B, ca, cb, acm, bkc)
        err = np.abs(C - Ao @ Bo)
        # inputs are rounded to FP32 (2^-24 each) and 3xTF32 drops terms near 2^-22 relative
        assert (err <= 4e-6 * bound + 1e-30).all(), (M, N, K, ca, cb, acm, bkc, float((err / bound).max()))
    assert np.abs(ref).max() > 0
