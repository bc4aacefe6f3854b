"""Pins for the dense oracle (CPU only).

Each check compares the oracle with something other than itself: the exact
discrete population recursion of the first-order map for pure loss, the
continuous closed forms n0 e^{-kt} and alpha0 e^{-kt/2}, the two-photon steady
manifold spanned by |+alpha> and |-alpha> (Sec. VI.A), exact parity conservation,
the Lindblad generator of Eq. 1 (local error of a first-order map is O(h^2)),
the vectorised superoperator, and the invariants of a density matrix.  The
planted-mistake tests show that plausible slips in the oracle fail the pins.
"""
import numpy as np
import pytest
import scipy.linalg

from oracle import dense as D
from paper_2605_27515_gb300 import inputs


def _rand_system(dims, n_jumps, seed):
    rng = np.random.default_rng(seed)
    Dm = int(np.prod(dims))

    def rand_local(N):
        return rng.normal(size=(N, N)) + 1j * rng.normal(size=(N, N))

    terms = []
    for m, N in enumerate(dims):
        X = rand_local(N)
        terms.append((0.3, {m: X + X.conj().T}))
    if len(dims) > 1:
        terms.append((0.2, {0: rand_local(dims[0]), 1: rand_local(dims[1])}))
        terms.append((0.2, {0: terms[-1][1][0].conj().T, 1: terms[-1][1][1].conj().T}))
    H = D.Operator(dims, terms)
    Ls = [D.Operator(dims, [(0.5, {m: rand_local(N)}) for m, N in enumerate(dims)]) for _ in range(n_jumps)]
    v = rng.normal(size=(Dm, 3)) + 1j * rng.normal(size=(Dm, 3))
    rho = v @ v.conj().T
    return H, Ls, rho / np.trace(rho).real


def _pure_loss(N, kappa):
    dims = (N,)
    return D.Operator(dims, []), [D.Operator.local(dims, 0, D.op_a(N), np.sqrt(kappa))]


# ---------------------------------------------------------------- machinery


def test_mode_wise_apply_equals_kronecker():
    dims = (3, 2, 4)
    rng = np.random.default_rng(1)
    mats = {m: rng.normal(size=(N, N)) + 1j * rng.normal(size=(N, N)) for m, N in enumerate(dims)}
    O = D.Operator(dims, [(0.7 - 0.2j, {0: mats[0], 2: mats[2]}), (1.3, {1: mats[1]})])
    full = 0.7 - 0.2j
    K = np.kron(np.kron(mats[0], np.eye(2)), mats[2]) * full + 1.3 * np.kron(np.kron(np.eye(3), mats[1]), np.eye(4))
    X = rng.normal(size=(24, 5)) + 1j * rng.normal(size=(24, 5))
    np.testing.assert_allclose(O.dense(), K, atol=1e-13)
    np.testing.assert_allclose(O.apply_left(X), K @ X, atol=1e-12)


def test_fock_operators_textbook():
    N = 12
    a, ad, n = D.op_a(N), D.op_adag(N), D.op_num(N)
    # <n|a|n'> = delta_{n+1,n'} sqrt(n'); a|0> = 0; commutator is 1 except the last level
    assert a[3, 4] == pytest.approx(2.0)
    np.testing.assert_allclose(a @ D.fock(N, 0), 0)
    np.testing.assert_allclose(ad @ a, n, atol=1e-14)
    comm = a @ ad - ad @ a
    np.testing.assert_allclose(np.diag(comm)[:-1], 1.0, atol=1e-13)
    assert np.diag(comm)[-1] == pytest.approx(-(N - 1))


# ---------------------------------------------------------------- brute force


@pytest.mark.parametrize("dims", [(8,), (4, 2)])
def test_superoperator_equals_step(dims):
    H, Ls, rho = _rand_system(dims, 2, seed=7)
    h = 0.013
    S = D.superoperator(H, Ls, h)
    v = S @ rho.reshape(-1)
    ref = v.reshape(rho.shape)
    ref = ref / np.trace(ref).real
    got = D.kraus_step(rho, H, Ls, h)
    np.testing.assert_allclose(got, ref, atol=1e-13)


def _local_error(H, Ls, rho, h):
    """|| K_h(rho) - exp(h G) rho || without renormalisation."""
    G = D.lindbladian(H, Ls)
    exact = (scipy.linalg.expm(h * G) @ rho.reshape(-1)).reshape(rho.shape)
    got = D.kraus_step(rho, H, Ls, h, normalize=False)
    return np.linalg.norm(got - exact)


def test_first_order_local_error_against_eq1():
    """K = U + hL agrees with the flow of Eq. 1 to O(h^2) per step."""
    H, Ls, rho = _rand_system((5,), 2, seed=3)
    e1 = _local_error(H, Ls, rho, 2e-3)
    e2 = _local_error(H, Ls, rho, 1e-3)
    assert 3.5 < e1 / e2 < 4.5


def _local_error2(H, Ls, rho, h):
    G = D.lindbladian(H, Ls)
    exact = (scipy.linalg.expm(h * G) @ rho.reshape(-1)).reshape(rho.shape)
    return np.linalg.norm(D.kraus_step(rho, H, Ls, h, normalize=False, order=2) - exact)


def test_second_order_local_error_against_eq1():
    """K = U' + (h/2)(UL + LU) + (h^2/2) L^2 agrees with the flow of Eq. 1 to O(h^3)."""
    H, Ls, rho = _rand_system((5,), 2, seed=3)
    e1 = _local_error2(H, Ls, rho, 4e-3)
    e2 = _local_error2(H, Ls, rho, 2e-3)
    assert 7.0 < e1 / e2 < 9.0
    # and it is an order better than the first-order map at the same h
    assert e2 < 0.05 * _local_error(H, Ls, rho, 2e-3)


def test_second_order_superoperator():
    """Brute force: the second-order map as a matrix on vec(rho), built from the
    Kraus operators U_1', sqrt(h/2) U_1 L_k, sqrt(h/2) L_k U_1, (h/sqrt 2) L_j L_k."""
    H, Ls, rho = _rand_system((4, 2), 2, seed=21)
    h = 0.01
    U = D.u1(H, Ls, h).dense()
    He = D.h_eff(H, Ls).dense()
    Up = U - 0.5 * h * h * He @ He
    Ld = [L.dense() for L in Ls]
    ks = [Up] + [np.sqrt(h / 2) * U @ L for L in Ld] + [np.sqrt(h / 2) * L @ U for L in Ld]
    ks += [h / np.sqrt(2) * A @ B for A in Ld for B in Ld]
    S = sum(np.kron(K, K.conj()) for K in ks)
    ref = (S @ rho.reshape(-1)).reshape(rho.shape)
    ref /= np.trace(ref).real
    np.testing.assert_allclose(D.kraus_step(rho, H, Ls, h, order=2), ref, atol=1e-13)


# ---------------------------------------------------------------- closed forms


def test_pure_loss_population_recursion():
    """Exact discrete map for L = sqrt(k) a, H = 0, Fock-diagonal rho:
    p'_n = (1 - h k n / 2)^2 p_n + h k (n+1) p_{n+1}, then renormalise."""
    N, kappa, h = 16, 0.7, 0.05
    H, Ls = _pure_loss(N, kappa)
    rng = np.random.default_rng(5)
    p = rng.random(N)
    p /= p.sum()
    rho = np.diag(p).astype(np.complex128)
    for _ in range(4):
        n = np.arange(N)
        q = (1 - h * kappa * n / 2) ** 2 * p
        q[:-1] += h * kappa * (n[:-1] + 1) * p[1:]
        p = q / q.sum()
        rho = D.kraus_step(rho, H, Ls, h)
        np.testing.assert_allclose(np.diag(rho).real, p, atol=1e-15)
        assert np.max(np.abs(rho - np.diag(np.diag(rho)))) < 1e-16


def _loss_run(h, T=1.0, N=40, kappa=1.0, alpha=2.0):
    H, Ls = _pure_loss(N, kappa)
    rho = D.pure(D.coherent(N, alpha))
    for _ in range(int(round(T / h))):
        rho = D.kraus_step(rho, H, Ls, h)
    n = np.trace(D.op_num(N) @ rho).real
    am = np.trace(D.op_a(N) @ rho)
    return n, am


def test_pure_loss_closed_form_first_order_convergence():
    """n(t) = n0 e^{-kt}, <a>(t) = alpha0 e^{-kt/2}; the first-order map converges at O(h)."""
    T, kappa, alpha = 1.0, 1.0, 2.0
    n_ex = alpha ** 2 * np.exp(-kappa * T)
    a_ex = alpha * np.exp(-kappa * T / 2)
    n1, a1 = _loss_run(2e-3)
    n2, a2 = _loss_run(1e-3)
    e1, e2 = abs(n1 - n_ex), abs(n2 - n_ex)
    f1, f2 = abs(a1 - a_ex), abs(a2 - a_ex)
    assert e2 < 2e-3 and f2 < 2e-3
    assert 1.8 < e1 / e2 < 2.2
    assert 1.8 < f1 / f2 < 2.2
    assert abs(a2.imag) < 1e-14


def test_two_photon_manifold_is_fixed():
    """|+alpha>, |-alpha> and the even cat are steady under L = a^2 - alpha^2 (Sec. VI.A)."""
    N, alpha, h = 64, 2.0, 1e-3
    dims = (N,)
    a = D.op_a(N)
    L1 = D.Operator(dims, [(1.0, {0: a @ a}), (-alpha ** 2, {})])
    H = D.Operator(dims, [])
    cp, cm = D.coherent(N, alpha), D.coherent(N, -alpha)
    even = (cp + cm) / np.linalg.norm(cp + cm)
    for psi in (cp, cm, even):
        rho = D.pure(psi)
        out = D.kraus_step(rho, H, [L1], h)
        assert np.max(np.abs(out - rho)) < 1e-12
    # and a state off the manifold is not fixed
    rho = D.pure(D.fock(N, 1))
    assert np.max(np.abs(D.kraus_step(rho, H, [L1], h) - rho)) > 1e-4


def test_two_photon_from_vacuum_reaches_even_cat():
    """k1 = 0: parity is conserved exactly and n -> alpha^2 tanh(alpha^2), the even cat."""
    N, alpha2, h = 32, 4.0, 2e-3
    dims = (N,)
    a = D.op_a(N)
    L1 = D.Operator(dims, [(1.0, {0: a @ a}), (-alpha2, {})])
    H = D.Operator(dims, [])
    rho = D.pure(D.fock(N, 0))
    par = D.op_parity(N)
    for _ in range(int(5.0 / h)):
        rho = D.kraus_step(rho, H, [L1], h)
    assert abs(np.trace(par @ rho).real - 1.0) < 1e-12
    n = np.trace(D.op_num(N) @ rho).real
    assert abs(n - alpha2 * np.tanh(alpha2)) < 2e-3


# ---------------------------------------------------------------- invariants


def test_invariants_along_trajectory():
    H, Ls, rho = _rand_system((3, 4), 2, seed=11)
    for _ in range(20):
        rho = D.kraus_step(rho, H, Ls, 0.01)
        assert abs(np.trace(rho) - 1) < 1e-13
        assert np.max(np.abs(rho - rho.conj().T)) < 1e-15
        w = np.linalg.eigvalsh(rho)
        assert w.min() > -1e-14
        assert D.purity(rho) <= 1 + 1e-13


def test_observables():
    N = 10
    psi = D.coherent(N, 0.8 + 0.3j)
    rho = D.pure(psi)
    assert D.fidelity(rho, psi) == pytest.approx(1.0, abs=1e-14)
    assert D.purity(rho) == pytest.approx(1.0, abs=1e-14)
    nO = D.Operator.local((N,), 0, D.op_num(N))
    assert D.expectation(rho, nO).real == pytest.approx(np.vdot(psi, D.op_num(N) @ psi).real, abs=1e-14)
    mixed = 0.5 * D.pure(D.fock(N, 0)) + 0.5 * D.pure(D.fock(N, 3))
    assert D.purity(mixed) == pytest.approx(0.5, abs=1e-15)


# ---------------------------------------------------------------- planted mistakes


def _pins_pass(step):
    """Run the recursion pin and the Eq. 1 pin against a (possibly broken) step."""
    N, kappa, h = 8, 0.9, 0.05
    H, Ls = _pure_loss(N, kappa)
    p = np.linspace(1, 2, N)
    p /= p.sum()
    n = np.arange(N)
    q = (1 - h * kappa * n / 2) ** 2 * p
    q[:-1] += h * kappa * (n[:-1] + 1) * p[1:]
    q /= q.sum()
    ok1 = np.allclose(np.diag(step(np.diag(p).astype(complex), H, Ls, h)).real, q, atol=1e-14)
    H2, Ls2, rho2 = _rand_system((4,), 1, seed=2)
    G = D.lindbladian(H2, Ls2)

    def err(hh):
        ex = (scipy.linalg.expm(hh * G) @ rho2.reshape(-1)).reshape(rho2.shape)
        got = step(rho2, H2, Ls2, hh, normalize=False)
        return np.linalg.norm(got - ex)

    r = err(2e-3) / err(1e-3)
    ok2 = 3.5 < r < 4.5
    return ok1 and ok2


def test_pins_accept_oracle():
    assert _pins_pass(D.kraus_step)


def test_pins_reject_planted_mistakes(monkeypatch):
    # 1. wrong sign of the anti-Hermitian part of H_eff
    def heff_sign(H, Ls):
        out = H
        for L in Ls:
            out = out + (L.dag() @ L).scale(+0.5j)
        return out

    monkeypatch.setattr(D, "h_eff", heff_sign)
    assert not _pins_pass(D.kraus_step)
    monkeypatch.undo()

    # 2. jump term without the factor h
    def step_noh(rho, H, Ls, h, normalize=True):
        out = D.sandwich(D.u1(H, Ls, h), rho)
        for L in Ls:
            out = out + D.sandwich(L, rho)
        return out / np.trace(out).real if normalize else out

    assert not _pins_pass(step_noh)

    # 3. dagger dropped on the right of the sandwich
    def step_nodag(rho, H, Ls, h, normalize=True):
        def sw(A, r):
            return A.apply_left(A.apply_left(r).T)

        out = sw(D.u1(H, Ls, h), rho)
        for L in Ls:
            out = out + h * sw(L, rho)
        return out / np.trace(out).real if normalize else out

    assert not _pins_pass(step_nodag)

    # 4. factor 1/2 dropped from H_eff
    def heff_half(H, Ls):
        out = H
        for L in Ls:
            out = out + (L.dag() @ L).scale(-1.0j)
        return out

    monkeypatch.setattr(D, "h_eff", heff_half)
    assert not _pins_pass(D.kraus_step)


def test_inputs_module_holds_configs():
    cfg = inputs.config("cat_r5")
    assert cfg["R"] == [5] and cfg["steps"] == 5000
