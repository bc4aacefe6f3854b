"""Pins of the Z-gate system (Sec. VI): the derived parameters reproduce the
paper's expected error p_Z = pi / (40 |alpha|^3), and the oracle's dynamics rotate
the cat qubit by theta = 4 alpha T eps_Z (memory parity cos(theta))."""
import numpy as np

from oracle import dense as D
from oracle import systems as OS
from paper_2605_27515_gb300 import inputs


def test_parameters_give_the_expected_error_formula():
    """p_buf = theta^2 / (16 |alpha|^4 T_Z) * kappa_b / (4 g2^2) equals pi / (40 |alpha|^3)
    for g2 = 1, kappa_b = 10 g2, eps_Z = 4 g2^2 / (10 kappa_b), theta = pi (Eq. pZ)."""
    for R in (4, 6, 9, 11):
        cfg = inputs.config("z_gate")
        cfg["R"] = [R, 4]
        zp = inputs.z_gate_params(cfg)
        assert zp["alpha2"] == 2 ** R / 3.0
        p_buf = cfg["theta"] ** 2 / (16 * zp["alpha"] ** 4 * zp["t_z"]) * cfg["kb"] / (4 * cfg["g2"] ** 2)
        assert abs(p_buf - np.pi / (40 * zp["alpha"] ** 3)) < 1e-14
        assert abs(4 * zp["alpha"] * zp["t_z"] * zp["eps_z"] - np.pi) < 1e-12  # theta = 4 alpha T_Z eps_Z


def test_cat_vector_is_the_truncated_cat():
    v = inputs.cat_vector(40, 2.0, +1)
    ref = D.coherent(40, 2.0) + D.coherent(40, -2.0)
    np.testing.assert_allclose(v, ref / np.linalg.norm(ref), atol=1e-14)
    assert abs(np.vdot(v, D.op_parity(40) @ v).real - 1.0) < 1e-14
    w = inputs.cat_vector(40, 2.0, -1)
    assert abs(np.vdot(w, D.op_parity(40) @ w).real + 1.0) < 1e-14


def test_gate_rotates_the_parity():
    """Starting in the even cat, the memory parity follows cos(4 alpha eps_Z t): about 0
    at T_Z / 2 and about -1 at T_Z (theta = pi), up to the gate's phase-flip error."""
    cfg = inputs.config("z_gate")
    cfg["R"] = [4, 3]  # N_a = 16 (alpha^2 = 16/3), N_b = 8
    cfg["dt"] = 2e-3
    zp = inputs.z_gate_params(cfg)
    init = [inputs.cat_vector(16, zp["alpha"], +1), D.fock(8, 0)]
    ds = OS.z_gate(cfg, init)
    half = zp["steps"] // 2
    _, recs = ds.evolve(cfg["dt"], 2 * half, half, names=["parity_a", "n_b"])
    (_, (p0, _)), (_, (p_half, _)), (_, (p_end, nb_end)) = recs
    assert abs(p0 - 1.0) < 1e-12
    assert abs(p_half) < 0.05
    assert p_end < -0.9
    assert nb_end < 0.2  # the lossy buffer stays nearly empty
