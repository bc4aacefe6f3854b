"""Dense FP64 density-matrix oracle (test infrastructure only; see package doc).

What it computes is the plain definition the tensor-network step reaches when
nothing is truncated:

    H_eff = H(t_n) - (i/2) sum_k L_k^dag L_k          (Sec. V.B, Eq. for H_eff)
    U_1   = 1 - i h H_eff                              (Sec. V.B, Eq. for U_1)
    rho'  = U_1 rho U_1^dag + h sum_k L_k rho L_k^dag  (K = U + h L, Sec. V.B)
    rho   = rho' / Tr rho'                             (renormalisation, Sec. V.B)

Operators are Fock-truncated dense matrices, products are formed from the
truncated matrices in the order written, and multi-mode operators are sums of
Kronecker products applied mode by mode (Sec. II.B, last paragraph).

Readings of the paper taken here:
  * a^dag is the conjugate transpose of the truncated a (the text's "T^dag B"
    would put sqrt(n') on the wrong side).
  * The shift behind a is open: a|0> = 0 and nothing wraps from N-1 to 0.
  * L^dag L is always formed as (L)^dag (L) of truncated matrices.
  * Inside a first-order step the Hamiltonian is taken at the left end t_n.
  * Mode order: mode 0 is the most significant factor of the Kronecker product.
"""
from __future__ import annotations

import numpy as np

# --------------------------------------------------------------------------
# single-mode operators (Sec. II.B)
# --------------------------------------------------------------------------


def op_a(N: int) -> np.ndarray:
    """<n|a|n'> = delta_{n+1,n'} sqrt(n')  (Sec. II.B, matrix A), truncated to N."""
    a = np.zeros((N, N), dtype=np.complex128)
    for n in range(N - 1):
        a[n, n + 1] = np.sqrt(n + 1.0)
    return a


def op_adag(N: int) -> np.ndarray:
    """a^dag = conjugate transpose of the truncated a."""
    return op_a(N).conj().T.copy()


def op_num(N: int) -> np.ndarray:
    """n = a^dag a (Sec. II), diagonal 0..N-1."""
    return np.diag(np.arange(N, dtype=np.float64)).astype(np.complex128)


def op_parity(N: int) -> np.ndarray:
    """Photon-number parity (-1)^n."""
    return np.diag((-1.0) ** np.arange(N)).astype(np.complex128)


def op_identity(N: int) -> np.ndarray:
    return np.eye(N, dtype=np.complex128)


def op_charge(N: int, offset: int) -> np.ndarray:
    """Transmon charge operator n_t in the charge basis (Sec. VII, Eq. transmon):
    basis state j stands for charge j - offset."""
    return np.diag(np.arange(N, dtype=np.float64) - offset).astype(np.complex128)


def op_cos_phi(N: int) -> np.ndarray:
    """cos(phi_t) = 1/2 sum_n |n><n+1| + |n+1><n| in the charge basis
    (Sec. VII), cut open at both ends of the truncated charge range."""
    c = np.zeros((N, N), dtype=np.complex128)
    for n in range(N - 1):
        c[n, n + 1] = 0.5
        c[n + 1, n] = 0.5
    return c


# --------------------------------------------------------------------------
# multi-mode operators as sums of products (Sec. II.B, last paragraph)
# --------------------------------------------------------------------------


class Operator:
    """sum_t c_t (x)_m O_{t,m}; a missing mode factor is the identity."""

    def __init__(self, dims, terms=None):
        self.dims = tuple(int(d) for d in dims)
        self.terms = []  # list of (complex coeff, {mode: N_m x N_m matrix})
        for c, fac in terms or []:
            self.terms.append((complex(c), {int(m): np.asarray(f, np.complex128) for m, f in fac.items()}))

    @staticmethod
    def local(dims, mode, mat, coeff=1.0):
        return Operator(dims, [(coeff, {mode: mat})])

    @staticmethod
    def identity(dims, coeff=1.0):
        return Operator(dims, [(coeff, {})])

    def __add__(self, other):
        assert self.dims == other.dims
        return Operator(self.dims, self.terms + other.terms)

    def __sub__(self, other):
        return self + other.scale(-1.0)

    def scale(self, c):
        return Operator(self.dims, [(c * t, f) for t, f in self.terms])

    def __matmul__(self, other):
        """Operator product: per mode the matrix product of the factors, in order."""
        assert self.dims == other.dims
        out = []
        for c1, f1 in self.terms:
            for c2, f2 in other.terms:
                fac = {}
                for m in set(f1) | set(f2):
                    A = f1.get(m)
                    B = f2.get(m)
                    if A is None:
                        fac[m] = B
                    elif B is None:
                        fac[m] = A
                    else:
                        fac[m] = A @ B
                out.append((c1 * c2, fac))
        return Operator(self.dims, out)

    def dag(self):
        return Operator(self.dims, [(np.conj(c), {m: f.conj().T for m, f in fac.items()}) for c, fac in self.terms])

    def dense(self) -> np.ndarray:
        """Full matrix; mode 0 is the most significant Kronecker factor."""
        D = int(np.prod(self.dims))
        out = np.zeros((D, D), dtype=np.complex128)
        for c, fac in self.terms:
            M = np.ones((1, 1), dtype=np.complex128)
            for m, N in enumerate(self.dims):
                M = np.kron(M, fac.get(m, np.eye(N, dtype=np.complex128)))
            out += c * M
        return out

    def apply_left(self, X: np.ndarray) -> np.ndarray:
        """O X for a D x K matrix X, applying each mode factor separately."""
        D = int(np.prod(self.dims))
        K = X.shape[1]
        out = np.zeros((D, K), dtype=np.complex128)
        for c, fac in self.terms:
            T = X.reshape(self.dims + (K,))
            for m, f in fac.items():
                T = np.moveaxis(np.tensordot(f, T, axes=([1], [m])), 0, m)
            out += c * T.reshape(D, K)
        return out


# --------------------------------------------------------------------------
# the first-order Kraus step (Sec. V.B)
# --------------------------------------------------------------------------


def h_eff(H: Operator, Ls) -> Operator:
    """H_eff = H - (i/2) sum_k L_k^dag L_k  (Sec. V.B)."""
    out = H
    for L in Ls:
        out = out + (L.dag() @ L).scale(-0.5j)
    return out


def u1(H: Operator, Ls, h: float) -> Operator:
    """U_1 = 1 - i h H_eff  (Sec. V.B)."""
    return Operator.identity(H.dims) + h_eff(H, Ls).scale(-1j * h)


def sandwich(A: Operator, rho: np.ndarray) -> np.ndarray:
    """A rho A^dag for Hermitian rho, using (A rho)^dag = rho A^dag."""
    X = A.apply_left(rho)
    return A.apply_left(X.conj().T)


def kraus_step(rho: np.ndarray, H: Operator, Ls, h: float, normalize: bool = True, order: int = 1) -> np.ndarray:
    """One Kraus step, then rho / Tr rho (Sec. V.B).

    order 1: K = U + h L with U(rho) = U_1 rho U_1^dag.
    order 2: K = U' + (h/2)(U L + L U) + (h^2/2) L^2 with U'(rho) = U_1' rho U_1'^dag,
             U_1' = 1 - i h H_eff - (h^2/2) H_eff^2; the compositions of Kraus maps
             are applied one after the other (Sec. V.B, Kraus algebra)."""
    if order == 1:
        U = u1(H, Ls, h)
        out = sandwich(U, rho)
        for L in Ls:
            out = out + h * sandwich(L, rho)
    elif order == 2:
        He = h_eff(H, Ls)
        U = u1(H, Ls, h)
        Up = U + (He @ He).scale(-0.5 * h * h)

        def jump(r):
            acc = np.zeros_like(r)
            for L in Ls:
                acc = acc + sandwich(L, r)
            return acc

        out = sandwich(Up, rho)
        out = out + (h / 2) * (sandwich(U, jump(rho)) + jump(sandwich(U, rho)))
        out = out + (h * h / 2) * jump(jump(rho))
    else:
        raise ValueError("order must be 1 or 2")
    out = 0.5 * (out + out.conj().T)  # exact Hermiticity; removes rounding skew only
    if normalize:
        out = out / np.trace(out).real
    return out


def evolve(rho0, H0: Operator, Ls, h: float, nsteps: int, H1: Operator | None = None, f_table=None,
           record_every: int = 0, observables=None, order: int = 1):
    """Repeat the step nsteps times.  With a drive, H(t_n) = H0 + f(t_n) H1 with
    f taken from f_table[n] at the left end of step n (Sec. III.A coefficient
    form H0 + f(t) H1; first-order steps use t_n).

    order selects the Kraus scheme of kraus_step.
    Returns (rho, records) where records is a list of (step, [values]).
    """
    rho = np.array(rho0, dtype=np.complex128, copy=True)
    recs = []
    if record_every and observables:
        recs.append((0, [obs(rho) for obs in observables]))
    for n in range(nsteps):
        H = H0 if H1 is None else H0 + H1.scale(float(f_table[n]))
        rho = kraus_step(rho, H, Ls, h, order=order)
        if record_every and observables and ((n + 1) % record_every == 0 or n + 1 == nsteps):
            recs.append((n + 1, [obs(rho) for obs in observables]))
    return rho, recs


# --------------------------------------------------------------------------
# observables (Sec. III.B, Sec. IV.A, Sec. VII)
# --------------------------------------------------------------------------


def expectation(rho: np.ndarray, O: Operator) -> complex:
    """Tr(O rho)."""
    return complex(np.trace(O.apply_left(rho)))


def fidelity(rho: np.ndarray, psi: np.ndarray) -> float:
    """<psi|rho|psi> for a normalised pure target psi."""
    return float(np.real(np.vdot(psi, rho @ psi)))


def purity(rho: np.ndarray) -> float:
    """Tr rho^2 (Sec. IV.A)."""
    return float(np.real(np.sum(rho * rho.T)))


def pure(psi: np.ndarray) -> np.ndarray:
    psi = np.asarray(psi, np.complex128)
    psi = psi / np.linalg.norm(psi)
    return np.outer(psi, psi.conj())


def product_vector(vecs) -> np.ndarray:
    """Kronecker product of per-mode vectors, mode 0 most significant."""
    v = np.ones(1, dtype=np.complex128)
    for x in vecs:
        v = np.kron(v, np.asarray(x, np.complex128))
    return v


def coherent(N: int, alpha: complex) -> np.ndarray:
    """Truncated coherent state, renormalised: c_n = alpha^n / sqrt(n!)."""
    c = np.zeros(N, dtype=np.complex128)
    c[0] = 1.0
    for n in range(1, N):
        c[n] = c[n - 1] * alpha / np.sqrt(n)
    return c / np.linalg.norm(c)


def fock(N: int, n: int) -> np.ndarray:
    v = np.zeros(N, dtype=np.complex128)
    v[n] = 1.0
    return v


# --------------------------------------------------------------------------
# brute-force and continuous-time siblings (used only as pins)
# --------------------------------------------------------------------------


def superoperator(H: Operator, Ls, h: float) -> np.ndarray:
    """The same first-order map written as a matrix on row-major vec(rho):
    vec(A rho B) = (A kron B^T) vec(rho), so
    S = U_1 kron conj(U_1) + h sum_k L_k kron conj(L_k)."""
    U = u1(H, Ls, h).dense()
    S = np.kron(U, U.conj())
    for L in Ls:
        Ld = L.dense()
        S = S + h * np.kron(Ld, Ld.conj())
    return S


def lindbladian(H: Operator, Ls) -> np.ndarray:
    """Generator of Eq. 1 on row-major vec(rho):
    -i[H, rho] + sum_k (L rho L^dag - 1/2 {L^dag L, rho})."""
    Hd = H.dense()
    D = Hd.shape[0]
    I = np.eye(D, dtype=np.complex128)
    G = -1j * (np.kron(Hd, I) - np.kron(I, Hd.T))
    for L in Ls:
        Ld = L.dense()
        LdL = Ld.conj().T @ Ld
        G = G + np.kron(Ld, Ld.conj()) - 0.5 * (np.kron(LdL, I) + np.kron(I, LdL.T))
    return G
