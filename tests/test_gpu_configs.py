"""GPU parity of the model systems at the oracle's check sizes (truncated form).

Bar: photon numbers, parities and other recorded observables within 1e-6
absolute of the dense FP64 oracle (the truncated-form tolerance).

* large cat mode at its check size N = 128, alpha^2 = 16, Zeno drive, literal
  dt = 5e-4 (recorded before the explicit step's instability takes over, and the
  stable twin dt = 1e-4 over a longer window, in both precision forms);
* the second-order Kraus scheme on the N = 32 cat;
* transmon x resonator at 32 charge states x 64 Fock levels with the ramped drive,
  and with the transmon in its eigenbasis (32 lowest states);
* the two coupled cats with buffers at (N_b, N_a, N_a, N_b) = (4, 8, 8, 4).
"""
import numpy as np
import pytest

from oracle import dense as D
from oracle import systems as OS
from paper_2605_27515_gb300 import inputs
from paper_2605_27515_gb300 import qlb as Q
from paper_2605_27515_gb300 import systems

pytestmark = pytest.mark.gpu


def _compare(b, ds, dt, nsteps, every, names, order=1):
    st = b.sys.state(b.init)
    _, recs = ds.evolve(dt, nsteps, every, names=names, order=order)
    worst = {n: 0.0 for n in names}
    done = 0
    for step, vals in recs[1:]:
        st.step(dt, step - done)
        done = step
        for n, o in zip(names, vals):
            g = st.expectation(b.observables[n]).real
            worst[n] = max(worst[n], abs(g - o))
    st.close()
    return worst


@pytest.mark.parametrize("dt,nsteps,precision", [(5e-4, 100, Q.PREC_F64), (1e-4, 400, Q.PREC_F64),
                                                  (1e-4, 400, Q.PREC_MIXED)])
def test_cat_r9_check_size(dt, nsteps, precision):
    cfg = inputs.config("cat_r9")
    cfg.update(cfg.pop("check"))  # N = 128, alpha^2 = 16
    c = Q.Ctx(device=0, precision=precision, tol=cfg["tol"], chi_max=cfg["chi_max"], chi_mu_max=cfg["chi_mu_max"])
    b = systems.build(c, cfg)
    worst = _compare(b, OS.cat(cfg), dt, nsteps, 20, ["n", "parity"])
    assert max(worst.values()) < 1e-6, worst
    c.close()


def test_cat_r5_second_order():
    """The second-order scheme on the N = 32 cat (truncated form): within 1e-6 of
    the dense oracle's second-order map over 300 steps of dt = 1e-3."""
    cfg = inputs.config("cat_r5")
    c = Q.Ctx(device=0, tol=cfg["tol"], chi_max=cfg["chi_max"], chi_mu_max=cfg["chi_mu_max"])
    b = systems.build(c, cfg)
    b.sys.set_scheme(2)
    worst = _compare(b, OS.cat(cfg), cfg["dt"], 300, 50, ["n", "parity"], order=2)
    assert max(worst.values()) < 1e-6, worst
    c.close()


def test_transmon_check_size():
    cfg = inputs.config("transmon")
    cfg.update(cfg.pop("check"))  # 32 charge states x 64 Fock levels
    nsteps = 20
    dt = 2e-5
    cfg["dt"] = dt
    c = Q.Ctx(device=0, tol=cfg["tol"], chi_max=cfg["chi_max"], chi_mu_max=cfg["chi_mu_max"])
    b = systems.build(c, cfg, nsteps=nsteps)
    ds = OS.transmon(cfg, nsteps)  # the oracle's own drive table and ground state
    worst = _compare(b, ds, dt, nsteps, 5, ["n_c", "n_t2"])
    assert max(worst.values()) < 1e-6, worst
    c.close()


def test_transmon_eigenbasis_check_size():
    """Sec. VII's construction: the transmon in its own eigenbasis (32 lowest states of
    |n| <= 500 charges, dense factors) x 64 Fock levels with the ramped drive."""
    cfg = inputs.config("transmon_eig")
    cfg.update(cfg.pop("check"))  # 32 transmon states x 64 Fock levels
    nsteps = 20
    dt = 2e-5
    cfg["dt"] = dt
    c = Q.Ctx(device=0, tol=cfg["tol"], chi_max=cfg["chi_max"], chi_mu_max=cfg["chi_mu_max"])
    b = systems.build(c, cfg, nsteps=nsteps)
    ds = OS.transmon_eig(cfg, nsteps)
    worst = _compare(b, ds, dt, nsteps, 5, ["n_c", "n_t"])
    assert max(worst.values()) < 1e-6, worst
    c.close()


def test_cat_pair_check_size():
    cfg = inputs.config("cat_pair")
    cfg.update(cfg.pop("check"))  # R = [3, 2, 3, 2] -> modes [4, 8, 8, 4]
    dt = 2e-3
    c = Q.Ctx(device=0, tol=cfg["tol"], chi_max=cfg["chi_max"], chi_mu_max=cfg["chi_mu_max"])
    b = systems.build(c, cfg)
    worst = _compare(b, OS.cat_pair(cfg), dt, 60, 20, ["n_a1", "n_a2", "parity_a1"])
    assert max(worst.values()) < 1e-6, worst
    c.close()
