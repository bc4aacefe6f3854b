"""The step's GEMM engines through qlb_zgemm_check (C-ABI): the FP64 work-distributed
GEMM (run-time K split over a fixed grid, partials added in part order by the last
CTA of each tile), the same GEMM in double-float (the mixed forms) and the
tensor-core 3xTF32 GEMM, against numpy's complex128 product.

Bars (relative Frobenius error of C): FP64 8 eps sqrt(k), double-float 2^-44
sqrt(k) (a ~48-bit significand per operation).  Tensor cores, per entry: 3xTF32
keeps ~21 bits of each operand (2^-19 for the products) and every one of the 2k
real additions into the FP32 accumulator in tensor memory may lose up to 2^-23 of
the running sum (the accumulation is not round-to-nearest, so these losses add up
with K instead of averaging out): |C - AB| <= (2^-19 + 2k 2^-23) |A| |B|.  Shapes cover a single tile, ragged edges, the split path
(few tiles over a long K), many tiles (no split) and K = 0."""
import numpy as np
import pytest

from paper_2605_27515_gb300 import qlb as Q

pytestmark = pytest.mark.gpu

SHAPES = [(1, 1, 1), (7, 5, 3), (32, 32, 16), (33, 65, 17), (60, 60, 2600), (20, 300, 74), (128, 2368, 60),
          (300, 300, 300), (16, 16, 0)]


def _mats(m, n, k, seed):
    rng = np.random.default_rng(seed)
    A = rng.normal(size=(m, k)) + 1j * rng.normal(size=(m, k))
    B = rng.normal(size=(k, n)) + 1j * rng.normal(size=(k, n))
    return A, B


@pytest.mark.parametrize("engine", [Q.GEMM_FP64, Q.GEMM_DF64, Q.GEMM_TC])
@pytest.mark.parametrize("m,n,k", SHAPES)
def test_engine_against_numpy(engine, m, n, k):
    A, B = _mats(m, n, k, seed=m * 1000 + n + k)
    ref = A @ B
    C, ms = Q.qlb_zgemm_check(0, engine, A, B)
    if k == 0:
        assert np.all(C == 0)
        return
    if engine == Q.GEMM_TC:
        bound = (2.0 ** -19 + 2 * k * 2.0 ** -23) * (np.abs(A) @ np.abs(B))
        assert np.all(np.abs(C - ref) <= bound), np.max(np.abs(C - ref) / bound)
    else:
        err = np.linalg.norm(C - ref) / np.linalg.norm(ref)
        bar = {Q.GEMM_FP64: 8 * 2.2e-16 * np.sqrt(k), Q.GEMM_DF64: 2.0 ** -44 * np.sqrt(k)}[engine]
        assert err < bar, (err, bar)
    assert ms > 0


@pytest.mark.parametrize("engine", [Q.GEMM_FP64, Q.GEMM_DF64])
def test_split_sum_is_deterministic(engine):
    """Few tiles over a long K take the split path; two launches give the same bits."""
    A, B = _mats(40, 40, 3000, seed=3)
    C1, _ = Q.qlb_zgemm_check(0, engine, A, B)
    C2, _ = Q.qlb_zgemm_check(0, engine, A, B)
    assert np.array_equal(C1, C2)
