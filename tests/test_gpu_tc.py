"""The tensor-core engine of the mixed form (QLB_PREC_TC): the 3xTF32 complex GEMM
on tcgen05 that applies the Kraus MPO (Sec. V.A), through the C-ABI, against the
FP64 product on ragged shapes (tails in every dimension, several 128 x 64 tiles,
K from 0 to several stages).  The bound per entry is the 3xTF32 one: each operand
keeps ~21 bits (2^-21 relative per product, the lo*lo term dropped) and the sum is
accumulated in FP32, so |C - AB|_ij <= (2^-19 + K 2^-23) sum_k |A_ik| |B_kj|.  The
error must also sit far below what a single TF32 pass (10-bit mantissa) gives."""
import numpy as np
import pytest

from paper_2605_27515_gb300 import qlb as Q

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("m,n,k", [(1, 1, 1), (5, 3, 0), (17, 63, 15), (128, 64, 16), (130, 65, 17),
                                   (300, 129, 100), (257, 200, 64), (64, 256, 333)])
def test_tc_zgemm_matches_fp64(m, n, k):
    rng = np.random.default_rng(m * 1000 + n * 10 + k)
    A = rng.normal(size=(m, k)) + 1j * rng.normal(size=(m, k))
    B = rng.normal(size=(k, n)) + 1j * rng.normal(size=(k, n))
    A *= np.exp(rng.uniform(-3, 3, size=(m, 1)))  # rows of different scales
    C = Q.qlb_tc_zgemm(0, A, B)
    ref = A @ B
    bound = (2.0 ** -19 + k * 2.0 ** -23) * (np.abs(A) @ np.abs(B)) + 1e-300
    assert np.all(np.abs(C - ref) <= bound), np.max(np.abs(C - ref) / bound)
    if k > 0:
        rel = np.linalg.norm(C - ref) / np.linalg.norm(ref)
        assert rel < 2e-5, rel  # one TF32 pass would leave ~1e-3


def test_tc_zgemm_exact_on_small_integers():
    """Integers below 2^10 are exact in TF32 (hi holds them, lo is zero) and their
    products and sums below 2^24 are exact in FP32: the engine returns AB exactly,
    which pins the complex embedding (signs and positions of the re/im parts)."""
    rng = np.random.default_rng(5)
    A = rng.integers(-7, 8, size=(70, 40)) + 1j * rng.integers(-7, 8, size=(70, 40))
    B = rng.integers(-7, 8, size=(40, 90)) + 1j * rng.integers(-7, 8, size=(40, 90))
    C = Q.qlb_tc_zgemm(0, A, B)
    np.testing.assert_array_equal(C, A @ B)
