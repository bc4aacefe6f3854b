"""Quantics tensor trains, written out plainly (test infrastructure only).

* Quantics encoding (Sec. II.A): n(sigma) = sum_{i=1..R} 2^{R-i} sigma_i, with
  sigma_1 the most significant bit.  Several modes are concatenated mode by mode,
  mode 0 first, so the global site order is the bit order of the Kronecker index.
* TT / MPS format (Eq. MPS): Psi_{s1..sR} = M1(s1) M2(s2) ... MR(sR).
* MPOs (Sec. II.B): site tensors W[a, s_out, s_in, b]; built here by TT-SVD of the
  dense operator, the exact rank-revealing SVD construction that the paper lists
  as the first-generation method (Sec. II.A), in place of TCI.
* Ranks (Table I): the maximal bond of the MPO built at a given relative
  Frobenius precision.

Truncation rule of the TT-SVD (Oseledets' bound): at each of the d-1 bonds drop
the smallest singular values whose squared sum is at most eps^2 ||A||_F^2 / (d-1),
so that the whole train is within eps ||A||_F of the tensor.
"""
from __future__ import annotations

import numpy as np


def bits_of(n: int, R: int):
    """sigma_1..sigma_R of n, sigma_1 the most significant (Sec. II.A)."""
    return [(n >> (R - i)) & 1 for i in range(1, R + 1)]


def index_of(bits) -> int:
    """n(sigma) = sum_i 2^{R-i} sigma_i (Sec. II.A)."""
    R = len(bits)
    return int(sum((2 ** (R - i)) * b for i, b in enumerate(bits, start=1)))


def _truncate_rank(s: np.ndarray, budget2: float) -> int:
    """Smallest k such that sum_{i>=k} s_i^2 <= budget2 (s sorted descending)."""
    tail = 0.0
    k = len(s)
    while k > 1 and tail + s[k - 1] ** 2 <= budget2:
        tail += s[k - 1] ** 2
        k -= 1
    return k


def tt_svd(T: np.ndarray, eps: float):
    """TT-SVD of a d-way tensor T (shape n_1 x ... x n_d) at relative
    Frobenius precision eps; returns cores G_k[r_{k-1}, n_k, r_k]."""
    shape = T.shape
    d = len(shape)
    norm2 = float(np.vdot(T, T).real)
    budget2 = (eps ** 2) * norm2 / max(d - 1, 1)
    cores = []
    C = np.asarray(T, np.complex128).reshape(1, -1)
    r = 1
    for k in range(d - 1):
        C = C.reshape(r * shape[k], -1)
        U, s, Vh = np.linalg.svd(C, full_matrices=False)
        rk = _truncate_rank(s, budget2) if eps > 0 else int(np.sum(s > 0)) or 1
        cores.append(U[:, :rk].reshape(r, shape[k], rk))
        C = s[:rk, None] * Vh[:rk]
        r = rk
    cores.append(C.reshape(r, shape[-1], 1))
    return cores


def tt_full(cores) -> np.ndarray:
    """Contract a train back to the full tensor."""
    T = cores[0]
    for G in cores[1:]:
        T = np.tensordot(T, G, axes=([-1], [0]))
    return T.reshape(T.shape[1:-1])


def mps_from_vector(v: np.ndarray, R: int, eps: float = 0.0):
    """Quantics MPS of a length-2^R vector (Sec. II.A): cores [r, 2, r']."""
    return tt_svd(np.asarray(v, np.complex128).reshape((2,) * R), eps)


def mps_to_vector(cores) -> np.ndarray:
    return tt_full(cores).reshape(-1)


def mpo_from_dense(O: np.ndarray, nbits: int, eps: float):
    """Quantics MPO of a 2^nbits x 2^nbits matrix by TT-SVD of the tensor
    O[(s'_1 s_1), (s'_2 s_2), ...]; cores W[a, s_out, s_in, b] (Sec. II.B)."""
    T = np.asarray(O, np.complex128).reshape((2,) * (2 * nbits))
    perm = []
    for i in range(nbits):
        perm += [i, nbits + i]
    T = T.transpose(perm).reshape((4,) * nbits)
    cores = tt_svd(T, eps)
    return [G.reshape(G.shape[0], 2, 2, G.shape[-1]) for G in cores]


def mpo_to_dense(W) -> np.ndarray:
    """Contract an MPO W[a, s_out, s_in, b] back to its 2^L x 2^L matrix."""
    L = len(W)
    T = W[0]
    for G in W[1:]:
        T = np.tensordot(T, G, axes=([-1], [0]))
    T = T.reshape((2, 2) * L)  # (o1, i1, o2, i2, ...)
    perm = [2 * i for i in range(L)] + [2 * i + 1 for i in range(L)]
    return T.transpose(perm).reshape(2 ** L, 2 ** L)


def mpo_rank(W) -> int:
    """Largest bond dimension of an MPO (the 'rank' of Table I)."""
    return max(G.shape[-1] for G in W[:-1]) if len(W) > 1 else 1


def mpo_bonds(W):
    return [G.shape[-1] for G in W[:-1]]
