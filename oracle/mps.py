"""The purified quantics MPS step, written out in numpy (test infrastructure only).

State (Sec. IV, Eqs. for rho = Psi Psi^dag and the MPS of Psi): Psi_{n,mu} is a
matrix product over the quantics sites of all modes (Sec. IV.C), mode 0 first,
sigma_1 (most significant bit) first inside a mode.  The purification index mu
is carried by the first site: core 0 has shape [chi_mu, 2, chi_1].  The paper
lets the mu tensor sit anywhere in the chain (Sec. IV.B); here it is merged into
the first site.  All other cores have shape [chi_{i-1}, 2, chi_i], the last
right bond is 1.

One step, in the order of Sec. V:
  1. Kraus operators K_0 = U_1 = 1 - i h H_eff, K_k = sqrt(h) L_k (Sec. V.B).
  2. Psi_k = K_k Psi, each an MPO.MPS product (Sec. V.B, first paragraph),
     formed exactly.
  3. Matrix addition of the Psi_k (Sec. V.A, Eq. for Psi^(0)(mu)): cores
     block-diagonal, mu ranges concatenated.
  4. Compression after the addition (Sec. V.A, last sentence): left-canonical
     QR sweep, then right-to-left truncated SVD on every bond.
  5. Purification-rank truncation (Sec. IV.A): SVD of Psi as an (mu) x (rest)
     matrix, keep the largest singular values and drop the mu-side unitary.
  6. rho / Tr rho (Sec. V.B, last paragraph).

Truncation rule (readings of the unstated "tolerance"):
  * relative discarded weight: keep the smallest k with
    sum_{i>=k} s_i^2 <= tol * sum_i s_i^2, then cap k at chi_max;
  * degenerate singular values are never split: if the first dropped value is
    within a relative gap `gap` of the last kept one, k grows through the
    cluster while the cap allows, otherwise k falls back to the cluster start.
"""
from __future__ import annotations

import numpy as np

from . import qtt


def keep_count(s: np.ndarray, tol: float, chi_max: int, gap: float = 1e-10) -> int:
    """Number of singular values kept under the rule in the module doc."""
    s = np.asarray(s, np.float64)
    n = len(s)
    if n == 0:
        return 0
    w = s ** 2
    total = float(np.sum(w))
    if total <= 0.0:
        return 1
    k = n
    tail = 0.0
    while k > 1 and tail + w[k - 1] <= tol * total:
        tail += w[k - 1]
        k -= 1
    k = min(k, chi_max)
    if k < n and s[k] >= (1.0 - gap) * s[k - 1]:
        j = k
        while j < n and j < chi_max and s[j] >= (1.0 - gap) * s[j - 1]:
            j += 1
        if j < n and s[j] >= (1.0 - gap) * s[j - 1]:
            # cluster does not fit under the cap: cut at the cluster start
            j = k
            while j > 1 and s[j] >= (1.0 - gap) * s[j - 1]:
                j -= 1
        k = j
    return max(k, 1)


def product_state(vecs, Rs):
    """Pure separable start, chi_mu = chi_e = 1 (Sec. V, first paragraph): each
    mode vector is turned into its quantics MPS and the chains are joined."""
    cores = []
    for v, R in zip(vecs, Rs):
        v = np.asarray(v, np.complex128)
        cores += qtt.mps_from_vector(v / np.linalg.norm(v), R, eps=1e-15)
    return cores


def psi_matrix(cores) -> np.ndarray:
    """Psi as a (Fock index) x (mu) matrix."""
    T = np.transpose(cores[0], (1, 2, 0))  # [s, r, mu]
    T = T.reshape(2, cores[0].shape[2], -1)
    out = T
    for G in cores[1:]:
        # out: [n, r, mu] ; G: [r, s, r']
        out = np.einsum("nrm,rsq->nsqm", out, G).reshape(-1, G.shape[2], out.shape[2])
    return out[:, 0, :]


def density(cores) -> np.ndarray:
    P = psi_matrix(cores)
    return P @ P.conj().T


def apply_mpo(W, cores):
    """Exact MPO.MPS product K Psi; the mu index is untouched."""
    out = []
    for A, Wi in zip(cores, W):
        l, _, r = A.shape
        a, _, _, b = Wi.shape
        if out == []:
            assert a == 1
        C = np.einsum("lsr,aosb->laorb", A, Wi)
        out.append(C.reshape(l * a, 2, r * b))
    return out


def matrix_add(states):
    """rho_1 + rho_2 + ... as one purification (Sec. V.A): block-diagonal cores,
    the mu ranges of the first core concatenated."""
    L = len(states[0])
    out = []
    for i in range(L):
        blocks = [s[i] for s in states]
        ls = [B.shape[0] for B in blocks]
        rs = [B.shape[2] for B in blocks]
        if i == L - 1:
            R = np.zeros((sum(ls), 2, 1), np.complex128)
            o = 0
            for B in blocks:
                R[o:o + B.shape[0]] = B
                o += B.shape[0]
        else:
            R = np.zeros((sum(ls), 2, sum(rs)), np.complex128)
            ol = orr = 0
            for B in blocks:
                R[ol:ol + B.shape[0], :, orr:orr + B.shape[2]] = B
                ol += B.shape[0]
                orr += B.shape[2]
        out.append(R)
    return out


def compress(cores, tol: float, chi_max: int, chi_mu_max: int, gap: float = 1e-10):
    """Steps 4-6 of the module doc.  Returns (cores, info) where info holds the
    bond dimensions and the trace before renormalisation."""
    cores = [c.copy() for c in cores]
    L = len(cores)
    # left-canonical sweep (QR), mu rows kept with the first site
    for i in range(L - 1):
        l, _, r = cores[i].shape
        Q, Rm = np.linalg.qr(cores[i].reshape(l * 2, r))
        cores[i] = Q.reshape(l, 2, Q.shape[1])
        cores[i + 1] = np.einsum("ab,bsr->asr", Rm, cores[i + 1])
    # right-to-left truncated SVD on every inter-site bond
    for i in range(L - 1, 0, -1):
        l, _, r = cores[i].shape
        U, s, Vh = np.linalg.svd(cores[i].reshape(l, 2 * r), full_matrices=False)
        k = keep_count(s, tol, chi_max, gap)
        cores[i] = Vh[:k].reshape(k, 2, r)
        cores[i - 1] = np.einsum("lsa,ak->lsk", cores[i - 1], U[:, :k] * s[:k])
    # purification-rank truncation: drop the mu-side unitary
    m, _, r = cores[0].shape
    U, s, Vh = np.linalg.svd(cores[0].reshape(m, 2 * r), full_matrices=False)
    k = keep_count(s, tol, chi_mu_max, gap)
    cores[0] = (s[:k, None] * Vh[:k]).reshape(k, 2, r)
    tr = float(np.sum(np.abs(cores[0]) ** 2))
    cores[0] = cores[0] / np.sqrt(tr)
    info = {"bonds": [c.shape[2] for c in cores[:-1]], "chi_mu": cores[0].shape[0], "trace": tr}
    return cores, info


def kraus_mpos(K_dense, nbits: int, eps: float = 1e-14):
    """Each dense Kraus operator as a quantics MPO (TT-SVD, Sec. II.B)."""
    return [qtt.mpo_from_dense(K, nbits, eps) for K in K_dense]


def kraus_step(cores, mpos, tol: float, chi_max: int, chi_mu_max: int, gap: float = 1e-10):
    """One step: Psi_k = K_k Psi, matrix addition, compression (module doc)."""
    branches = [apply_mpo(W, cores) for W in mpos]
    return compress(matrix_add(branches), tol, chi_max, chi_mu_max, gap)


def expectation(cores, O_dense: np.ndarray) -> complex:
    """Tr(O rho) with rho = Psi Psi^dag (small sizes: through the dense Psi)."""
    P = psi_matrix(cores)
    return complex(np.trace(P.conj().T @ (O_dense @ P)))
