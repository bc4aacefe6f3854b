"""Pins of the oracle's transmon eigenbasis (Sec. VII, numerical experiment).

The transmon 4 Ec n^2 - Ej cos(phi) is diagonalised on |n| <= 500 charges; the
lowest 2^R_t eigenstates carry the charge operator n_t.  Pinned against the
transmon frequency the paper prints, the eigen-equation itself, the parity
selection rule, convergence in the charge cutoff, the transmon-limit matrix
element and the free-rotor closed form."""
import numpy as np
import pytest

from oracle import systems as OS

EC = 2 * np.pi * 0.28  # rad/ns, Ec/h = 280 MHz (Sec. VII)
EJ = 50.0 * EC


def test_transmon_frequency_matches_the_paper():
    """Sec. VII: w_t / 2pi ~ sqrt(8 Ec Ej) - Ec ~ 5.320 GHz for Ej/Ec = 50."""
    E, _, _ = OS.transmon_eigenbasis(EC, EJ, 8)
    w01 = (E[1] - E[0]) / (2 * np.pi)
    assert abs(w01 - 5.320) < 0.03


def test_states_solve_the_charge_hamiltonian():
    n_cut = 80
    E, nt, Psi = OS.transmon_eigenbasis(EC, EJ, 32, n_cut=n_cut)
    n = np.arange(-n_cut, n_cut + 1)
    H = np.diag(4 * EC * n * n) - 0.5 * EJ * (np.eye(n.size, k=1) + np.eye(n.size, k=-1))
    scale = np.abs(E).max()
    np.testing.assert_allclose(Psi.T @ Psi, np.eye(32), atol=1e-12)
    np.testing.assert_allclose(Psi.T @ H @ Psi, np.diag(E), atol=1e-10 * scale)
    assert np.all(np.diff(E) >= -1e-9 * scale)
    # they are the lowest 32: no eigenvalue of H lies below E[-1] outside them
    w = np.linalg.eigvalsh(H)
    np.testing.assert_allclose(np.sort(E), w[:32], atol=1e-9 * scale)
    np.testing.assert_allclose(nt, Psi.T @ np.diag(n) @ Psi, atol=1e-12)


def test_parity_selection_rule():
    """n is odd under n -> -n: it connects only states of opposite charge parity."""
    n_cut = 500
    E, nt, Psi = OS.transmon_eigenbasis(EC, EJ, 32, n_cut=n_cut)
    flip = Psi[::-1, :]
    par = np.array([1 if np.allclose(flip[:, j], Psi[:, j], atol=1e-12) else -1 for j in range(32)])
    for j in range(32):
        np.testing.assert_allclose(flip[:, j], par[j] * Psi[:, j], atol=1e-12)
    same = par[:, None] == par[None, :]
    assert np.abs(nt[same]).max() < 1e-12
    assert np.abs(nt[~same]).max() > 1.0
    np.testing.assert_allclose(nt, nt.T, atol=1e-12)
    assert par[0] == 1 and par[1] == -1  # ground state even, first excited odd


def test_charge_cutoff_convergence():
    E1, nt1, _ = OS.transmon_eigenbasis(EC, EJ, 32, n_cut=500)
    E2, nt2, _ = OS.transmon_eigenbasis(EC, EJ, 32, n_cut=60)
    np.testing.assert_allclose(E1, E2, rtol=1e-12, atol=1e-12 * np.abs(E1).max())
    np.testing.assert_allclose(nt1, nt2, atol=1e-9)


def test_transmon_limit_matrix_element():
    """Deep transmon regime: |<0|n|1>| ~ (Ej / 8 Ec)^(1/4) / sqrt 2 (harmonic limit)."""
    _, nt, _ = OS.transmon_eigenbasis(EC, EJ, 4)
    assert abs(abs(nt[0, 1]) - (EJ / (8 * EC)) ** 0.25 / np.sqrt(2)) < 0.05 * abs(nt[0, 1])


def test_free_rotor_closed_form():
    """Ej = 0: energies 4 Ec m^2 (m = 0 once, each m >= 1 twice: even then odd state)
    and <e_m| n |o_m> = m between the two partners, nothing else."""
    K = 9
    E, nt, Psi = OS.transmon_eigenbasis(EC, 0.0, K, n_cut=20)
    m = np.array([0, 1, 1, 2, 2, 3, 3, 4, 4])
    np.testing.assert_allclose(E, 4 * EC * m * m, atol=1e-12)
    ref = np.zeros((K, K))
    for k in range(1, 5):
        e, o = 2 * k - 1, 2 * k
        ref[e, o] = ref[o, e] = k
    np.testing.assert_allclose(nt, ref, atol=1e-12)


def test_planted_missing_half_in_cos_phi_is_caught():
    """A plausible slip, cos(phi) written as |n><n+1| + |n+1><n| without the 1/2,
    acts like a doubled Ej and fails the frequency pin."""
    E, _, _ = OS.transmon_eigenbasis(EC, 2 * EJ, 8)
    assert abs((E[1] - E[0]) / (2 * np.pi) - 5.320) > 0.03
