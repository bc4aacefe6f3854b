"""Each truncation solver on its own, through qlb_eig_check (C-ABI): the one-CTA
Jacobi, the cluster Jacobi over 8 and 16 CTAs, Householder + QL, the zip-up range
basis and the step's own dispatch, in FP64 and double-float, on seeded Hermitian
positive semi-definite matrices G = M M^dag.

What pins them (Sec. V.A truncation through the Gram matrix):
  * the eigenvalues against LAPACK's (numpy.linalg.eigvalsh) within the backward
    error of a Hermitian eigen-solve, c n eps ||G||;
  * the kept vectors orthonormal and eigenvectors (residual G v - lambda v);
  * on a matrix of exact rank r the kept count is r (the tail is rounding);
  * the range basis: orthonormal, its discarded weight Tr G - Tr(U^dag G U) below
    the cutoff (or the rounding level when the cutoff is below it), and the cap
    handed to the Jacobi solve (k = -1) when the rank exceeds it.
"""
import numpy as np
import pytest

from paper_2605_27515_gb300 import qlb as Q

pytestmark = pytest.mark.gpu

EPS = {Q.PREC_F64: 2.220446049250313e-16, Q.PREC_MIXED: 1.4210854715202004e-14}
SIZES = [1, 2, 7, 24, 25, 33, 64, 65, 100, 128, 129, 200]


def _gram(n, rank, seed, graded=False):
    rng = np.random.default_rng(seed)
    M = rng.normal(size=(n, rank)) + 1j * rng.normal(size=(n, rank))
    if graded:  # singular values spread over 1e-6: weights over 1e-12
        M = M * np.logspace(0, -6, rank)[None, :]
    G = M @ M.conj().T
    return 0.5 * (G + G.conj().T)


def _valid(solver, prec, n):
    if solver == Q.SOLVER_CLUSTER8:
        return n <= 128
    if solver == Q.SOLVER_CLUSTER16:
        return n <= 256
    if solver == Q.SOLVER_QL:
        return prec == Q.PREC_F64 and n <= 64
    return True


EIG_SOLVERS = [Q.SOLVER_STEP, Q.SOLVER_JACOBI, Q.SOLVER_CLUSTER8, Q.SOLVER_CLUSTER16, Q.SOLVER_QL]


@pytest.mark.parametrize("prec", [Q.PREC_F64, Q.PREC_MIXED])
@pytest.mark.parametrize("solver", EIG_SOLVERS)
@pytest.mark.parametrize("n", SIZES)
def test_eigen_solver_against_lapack(solver, prec, n):
    if not _valid(solver, prec, n):
        pytest.skip("size or precision outside this solver")
    G = _gram(n, n, seed=1000 + n, graded=True)
    ref = np.sort(np.linalg.eigvalsh(G))[::-1]
    lam, V, k, ms = Q.qlb_eig_check(0, prec, solver, G, tol=0.0, cap=n)
    scale = np.linalg.norm(G, 2)
    tol_l = 40 * n * EPS[prec] * scale
    assert np.max(np.abs(lam - np.maximum(ref, 0))) <= tol_l, (np.max(np.abs(lam - np.maximum(ref, 0))), tol_l)
    assert k >= 1 and V is not None
    orth = np.max(np.abs(V.conj().T @ V - np.eye(k)))
    assert orth <= 40 * n * EPS[prec], orth
    res = np.max(np.linalg.norm(G @ V - V * lam[:k][None, :], axis=0))
    assert res <= tol_l, (res, tol_l)
    assert ms > 0


@pytest.mark.parametrize("prec", [Q.PREC_F64, Q.PREC_MIXED])
@pytest.mark.parametrize("solver", EIG_SOLVERS + [Q.SOLVER_RANGE])
@pytest.mark.parametrize("n,rank", [(24, 5), (64, 17), (100, 33), (128, 40), (200, 64)])
def test_kept_count_is_the_rank(solver, prec, n, rank):
    """Exact rank r (tail at the rounding level), cutoff 1e-12: every solver keeps r."""
    if not _valid(solver, prec, n):
        pytest.skip("size or precision outside this solver")
    G = _gram(n, rank, seed=7 * n + rank)
    lam, U, k, _ = Q.qlb_eig_check(0, prec, solver, G, tol=1e-12, cap=n)
    assert k == rank, (k, rank)
    assert np.max(np.abs(U.conj().T @ U - np.eye(k))) <= 40 * n * EPS[prec]
    kept = np.trace(U.conj().T @ G @ U).real
    assert np.trace(G).real - kept <= 1e-12 * np.trace(G).real + 40 * n * EPS[prec] * np.linalg.norm(G)


@pytest.mark.parametrize("prec", [Q.PREC_F64, Q.PREC_MIXED])
@pytest.mark.parametrize("n", [7, 33, 64, 100, 128, 200])
def test_range_basis_at_the_zip_up_cutoff(prec, n):
    """A graded full-rank G at the zip-up cutoff 1e-18 (below the rounding level of
    G): the basis is orthonormal and leaves only rounding-level weight outside."""
    G = _gram(n, n, seed=31 + n, graded=True)
    _, U, k, _ = Q.qlb_eig_check(0, prec, Q.SOLVER_RANGE, G, tol=1e-18, cap=n)
    assert 1 <= k <= n
    assert np.max(np.abs(U.conj().T @ U - np.eye(k))) <= 40 * n * EPS[prec]
    left = np.trace(G).real - np.trace(U.conj().T @ G @ U).real
    assert left <= 40 * n * EPS[prec] * np.linalg.norm(G), left


@pytest.mark.parametrize("prec", [Q.PREC_F64, Q.PREC_MIXED])
def test_range_basis_hands_a_binding_cap_to_jacobi(prec):
    G = _gram(64, 20, seed=5)
    _, U, k, _ = Q.qlb_eig_check(0, prec, Q.SOLVER_RANGE, G, tol=1e-12, cap=12)
    assert k == -1 and U is None
    _, U, k, _ = Q.qlb_eig_check(0, prec, Q.SOLVER_STEP, G, tol=1e-12, cap=12)
    assert k == 12


def test_check_entry_rejects_bad_arguments():
    G = _gram(8, 8, seed=1)
    with pytest.raises(Q.QlbError):
        Q.qlb_eig_check(0, Q.PREC_MIXED, Q.SOLVER_QL, G)  # QL is FP64 only
    with pytest.raises(Q.QlbError):
        Q.qlb_eig_check(0, Q.PREC_F64, 9, G)
    Gn = G.copy()
    Gn[0, 0] = np.nan
    with pytest.raises(Q.QlbError):
        Q.qlb_eig_check(0, Q.PREC_F64, Q.SOLVER_JACOBI, Gn)
