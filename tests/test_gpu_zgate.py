"""GPU parity of the Z-gate system (Sec. VI): a cat qubit with its lossy buffer
at (N_a, N_b) = (8, 4), against the dense FP64 oracle within 1e-6 (truncated form).
Kept in a file of its own, collected after the other GPU parity files."""
import numpy as np
import pytest

from oracle import dense as D
from oracle import mps as MPS
from oracle import systems as OS
from paper_2605_27515_gb300 import inputs
from paper_2605_27515_gb300 import qlb as Q
from paper_2605_27515_gb300 import systems

pytestmark = pytest.mark.gpu


def _compare(b, ds, dt, nsteps, every, names):
    st = b.sys.state(b.init)
    _, recs = ds.evolve(dt, nsteps, every, names=names)
    worst = {n: 0.0 for n in names}
    done = 0
    for step, vals in recs[1:]:
        st.step(dt, step - done)
        done = step
        for n, o in zip(names, vals):
            worst[n] = max(worst[n], abs(st.expectation(b.observables[n]).real - o))
    st.close()
    return worst


def test_z_gate_check_size():
    """Z gate on a cat qubit with its buffer (Sec. VI) at N_a = 8 (alpha^2 = 8/3),
    N_b = 4: memory parity and photon numbers within 1e-6 of the dense oracle over
    the first 600 steps of dt = 1e-3.  The purification cap is the full 32: with
    chi_mu <= 16 the cap itself moves the parity by 1.22e-6 (the oracle's own MPS
    step shows the same 1.22e-6, against 3e-9 at chi_mu <= 32)."""
    cfg = inputs.config("z_gate")
    cfg.update(cfg.pop("check"))
    cfg["tol"] = 1e-12
    cfg["chi_mu_max"] = 32
    c = Q.Ctx(device=0, tol=cfg["tol"], chi_max=cfg["chi_max"], chi_mu_max=cfg["chi_mu_max"])
    b = systems.build(c, cfg)
    ds = OS.z_gate(cfg)
    worst = _compare(b, ds, cfg["dt"], 600, 100, ["parity_a", "n_a", "n_b"])
    assert max(worst.values()) < 1e-6, worst
    c.close()


def test_z_gate_config_settings_match_the_oracle_mps_step():
    """At the configuration's own truncation (tol 1e-8, chi_mu <= 16, chi <= 64),
    where the purification cap binds at (N_a, N_b) = (8, 4): the device step against
    the oracle's own purified-MPS step (exact MPO.MPS products, matrix addition,
    right-to-left SVD truncation, purification truncation) at the same caps and
    tolerance, and both against the dense step, over 600 steps of dt = 1e-3.
    The two are different truncation schemes (the device cuts the zip-up bonds on
    the fly at tol x 1e-6 before its canonical right-to-left truncation), so they
    differ by an amount that scales with tol (6.4e-7 here, 2.6e-9 at tol 1e-12)
    while each sits ~8.5e-5 from the untruncated dense dynamics.  The test keeps
    their difference below 5 % of the oracle's own truncation error, and the
    device's truncation error within 10 % of the oracle's."""
    cfg = inputs.config("z_gate")
    cfg.update(cfg.pop("check"))
    assert cfg["tol"] == 1e-8 and cfg["chi_mu_max"] == 16
    h = cfg["dt"]
    c = Q.Ctx(device=0, tol=cfg["tol"], chi_max=cfg["chi_max"], chi_mu_max=cfg["chi_mu_max"])
    b = systems.build(c, cfg)
    st = b.sys.state(b.init)
    ds = OS.z_gate(cfg)
    Ks = [D.u1(ds.H0, ds.Ls, h).dense()] + [np.sqrt(h) * L.dense() for L in ds.Ls]
    nbits = sum(cfg["R"])
    mpos = MPS.kraus_mpos(Ks, nbits)
    cores = MPS.product_state(ds.init, cfg["R"])
    rho = ds.rho0()
    obs = {n: ds.observables[n].dense() for n in ("parity_a", "n_a", "n_b")}
    dev_or = dev_de = or_de = 0.0
    for k in range(1, 601):
        cores, info = MPS.kraus_step(cores, mpos, cfg["tol"], cfg["chi_max"], cfg["chi_mu_max"])
        rho = D.kraus_step(rho, ds.H0, ds.Ls, h)
        st.step(h, 1)
        if k % 100 == 0:
            for n, O in obs.items():
                g = st.expectation(b.observables[n]).real
                o = MPS.expectation(cores, O).real
                e = np.trace(O @ rho).real
                dev_or, dev_de, or_de = max(dev_or, abs(g - o)), max(dev_de, abs(g - e)), max(or_de, abs(o - e))
    assert info["chi_mu"] == 16  # the cap binds
    assert or_de > 1e-6  # the truncation is visible at this tolerance
    assert dev_or < 0.05 * or_de, (dev_or, or_de)
    assert dev_de < 1.1 * or_de, (dev_de, or_de)
    st.close()
    c.close()
