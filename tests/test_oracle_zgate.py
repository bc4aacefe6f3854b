"""Pins of the Z-gate system (Sec. VI): the oracle's own operating point
reproduces the paper's expected error p_Z = pi / (40 |alpha|^3), its cat is the
truncated cat, the buffer is dark on the cat, and its dynamics rotate the cat
qubit by theta = 4 alpha T eps_Z (memory parity cos(theta)).  The product's
parameter derivation is checked against the oracle's."""
import numpy as np
import pytest

from oracle import dense as D
from oracle import systems as OS
from paper_2605_27515_gb300 import inputs
from paper_2605_27515_gb300 import systems as PS


def test_parameters_give_the_expected_error_formula():
    """p_buf = theta^2 / (16 |alpha|^4 T_Z) * kappa_b / (4 g2^2) equals pi / (40 |alpha|^3)
    for g2 = 1, kappa_b = 10 g2, eps_Z = 4 g2^2 / (10 kappa_b), theta = pi (Eq. pZ)."""
    for R in (4, 6, 9, 11):
        cfg = inputs.config("z_gate")
        cfg["R"] = [R, 4]
        zp = OS.z_gate_params(cfg)
        assert zp["alpha2"] == 2 ** R / 3.0
        p_buf = cfg["theta"] ** 2 / (16 * zp["alpha"] ** 4 * zp["t_z"]) * cfg["kb"] / (4 * cfg["g2"] ** 2)
        assert abs(p_buf - np.pi / (40 * zp["alpha"] ** 3)) < 1e-14
        assert abs(4 * zp["alpha"] * zp["t_z"] * zp["eps_z"] - np.pi) < 1e-12  # theta = 4 alpha T_Z eps_Z


def test_cat_state_is_the_truncated_cat():
    """The oracle's cat: even/odd parity exactly, and the closed-form amplitudes
    c_n = 2 e^{-|alpha|^2/2} alpha^n / sqrt(n!) on even (odd) n, normalised."""
    from math import factorial

    v = OS.cat_state(40, 2.0, +1)
    ref = np.array([2 * np.exp(-2.0) * 2.0 ** n / np.sqrt(float(factorial(n))) if n % 2 == 0 else 0.0
                    for n in range(40)])
    np.testing.assert_allclose(v, ref / np.linalg.norm(ref), atol=1e-14)
    assert abs(np.vdot(v, D.op_parity(40) @ v).real - 1.0) < 1e-14
    w = OS.cat_state(40, 2.0, -1)
    assert abs(np.vdot(w, D.op_parity(40) @ w).real + 1.0) < 1e-14


def test_product_operating_point_matches_the_oracle():
    """The product's own derivation of (alpha, eps_d, eps_Z, T_Z, steps) and of the
    initial cat agrees with the oracle's."""
    for R in (3, 5, 9):
        cfg = inputs.config("z_gate")
        cfg["R"] = [R, 4]
        a, b = PS.z_gate_params(cfg), OS.z_gate_params(cfg)
        for k in b:
            assert abs(a[k] - b[k]) <= 1e-14 * max(1.0, abs(b[k])), (k, a[k], b[k])
        np.testing.assert_allclose(PS.cat_vector(2 ** R, b["alpha"], +1), OS.cat_state(2 ** R, b["alpha"], +1),
                                   atol=1e-14)


def _dark_residual(H, Ls, psi):
    """|| H_eff psi || and max_k || L_k psi ||: both vanish iff |psi><psi| is a fixed
    point of the first-order Kraus step with H_eff psi = 0 (U_1 psi = psi)."""
    He = D.h_eff(H, Ls)
    r = np.linalg.norm(He.apply_left(psi[:, None]))
    return r, max(np.linalg.norm(L.apply_left(psi[:, None])) for L in Ls)


def test_buffer_is_dark_on_the_cat():
    """Without the Z drive, |+-alpha> x |0>_b is dark: g2 a^2 b^dag + eps_d b^dag
    vanishes on it when eps_d = -g2 alpha^2, and b |0> = 0 (Sec. VI, Eq. cb), up to
    the Fock tail of |alpha> at N_a = 32 (alpha^2 = 2).  A planted wrong sign of
    eps_d breaks it."""
    cfg = inputs.config("z_gate")
    cfg["R"] = [5, 2]
    cfg["alpha2"] = 2.0
    ds = OS.z_gate(cfg)
    zp = OS.z_gate_params(cfg)
    Hs = D.Operator(ds.dims, [t for t in ds.H0.terms if not (0 in t[1] and len(t[1]) == 1)])  # drop eps_Z (a + a^dag)
    for sgn in (+1, -1):
        psi = D.product_vector([D.coherent(32, sgn * zp["alpha"]), D.fock(4, 0)])
        h, lk = _dark_residual(Hs, ds.Ls, psi)
        assert h < 1e-11 and lk < 1e-14, (h, lk)
    bad = D.Operator(ds.dims, [(-c if (1 in f and len(f) == 1) else c, f) for c, f in Hs.terms])
    h, _ = _dark_residual(bad, ds.Ls, psi)
    assert h > 0.5


def test_gate_rotates_the_parity():
    """Starting in the even cat, the memory parity follows cos(4 alpha eps_Z t): about 0
    at T_Z / 2 and about -1 at T_Z (theta = pi), up to the gate's phase-flip error."""
    cfg = inputs.config("z_gate")
    cfg["R"] = [4, 3]  # N_a = 16 (alpha^2 = 16/3), N_b = 8
    cfg["dt"] = 5e-3  # kappa_b dt = 0.05: the first-order map still tracks the gate
    zp = OS.z_gate_params(cfg)
    ds = OS.z_gate(cfg)
    half = zp["steps"] // 2
    _, recs = ds.evolve(cfg["dt"], 2 * half, half, names=["parity_a", "n_b"])
    (_, (p0, _)), (_, (p_half, _)), (_, (p_end, nb_end)) = recs
    assert abs(p0 - 1.0) < 1e-12
    assert abs(p_half) < 0.05
    assert p_end < -0.9
    assert nb_end < 0.2  # the lossy buffer stays nearly empty
