"""The zip-up range basis through the C-ABI: column-pivoted Gram-Schmidt on the
zip-up Gram matrix (zip_solver = 1, the default), with the Jacobi solve behind it
only when the zip-up cap binds, against the Jacobi zip-up (zip_solver = 0) and the
dense oracle (Sec. III.A zip-up, Sec. V.A).

Both solvers keep the range of M up to the zip-up cutoff (or the rounding level
of the Gram matrix), so the states they produce differ by a gauge on the zip-up
bonds plus directions of relative weight at the rounding level; after the final
right-to-left truncation the observables agree far below the 1e-6 bar.
"""
import numpy as np
import pytest

from oracle import systems as OS
from paper_2605_27515_gb300 import inputs
from paper_2605_27515_gb300 import qlb as Q
from paper_2605_27515_gb300 import systems

pytestmark = pytest.mark.gpu


def _twin(dt):
    cfg = inputs.config("cat_r9")
    cfg.update(cfg["check"])  # N = 128, alpha^2 = 16
    cfg["dt"] = dt
    return cfg


def _run(cfg, nsteps, every, precision=Q.PREC_F64, **opts):
    c = Q.Ctx(device=0, precision=precision, tol=cfg["tol"], chi_max=cfg["chi_max"],
              chi_mu_max=cfg["chi_mu_max"], **opts)
    b = systems.build(c, cfg)
    st = b.sys.state(b.init)
    c.profile_reset()
    rec = []
    for _ in range(nsteps // every):
        st.step(cfg["dt"], every)
        rec.append((st.expectation(b.observables["n"]).real, st.expectation(b.observables["parity"]).real))
    stats = c.solver_stats()
    bonds = st.bond_dims()
    st.close()
    c.close()
    return np.array(rec), stats, bonds


def _oracle(cfg, nsteps, every):
    _, recs = OS.cat(cfg).evolve(cfg["dt"], nsteps, every, names=["n", "parity"])
    return np.array([v for _, v in recs[1:]])


@pytest.mark.parametrize("precision", [Q.PREC_F64, Q.PREC_MIXED])
def test_zip_range_matches_jacobi_zip_and_oracle(precision):
    """N = 128 cat (alpha^2 = 16), dt = 1e-4, 300 steps: the range-basis zip-up
    serves the zip-up bonds (counter) and, like the Jacobi zip-up, stays within 1e-6
    of the dense oracle at every recorded step.  The two zip-up solvers keep
    different rounding-level directions (the range basis stops at the working
    precision's rounding level, the eigen-solve keeps whatever rounds positive);
    in the FP64 form the runs agree within 1e-8, in the double-float form (rounding
    level ~2^-48) within 1e-6 (1.7e-7 measured on GB300)."""
    cfg = _twin(1e-4)
    nsteps, every = 300, 50
    ref = _oracle(cfg, nsteps, every)
    a, sa, _ = _run(cfg, nsteps, every, precision, zip_solver=1)
    b, sb, _ = _run(cfg, nsteps, every, precision, zip_solver=0)
    assert sa["zip_range"] > 0 and sb["zip_range"] == 0
    ea, eb, dab = np.max(np.abs(a - ref)), np.max(np.abs(b - ref)), np.max(np.abs(a - b))
    assert ea < 1e-6 and eb < 1e-6, (ea, eb, dab)
    assert dab < (1e-8 if precision == Q.PREC_F64 else 1e-6), (ea, eb, dab)


def test_zip_range_cap_falls_back_to_jacobi():
    """chi_max = 10 on the N = 128 cat: the zip-up cap binds, the range basis hands
    those bonds to the Jacobi solve (fallback counter), and the run matches the
    Jacobi zip-up within 1e-8 with every bond within the cap."""
    cfg = _twin(1e-4)
    cfg["chi_max"] = 10
    nsteps, every = 200, 50
    a, sa, ba = _run(cfg, nsteps, every, zip_solver=1)
    b, _, _ = _run(cfg, nsteps, every, zip_solver=0)
    assert sa["zip_fallback"] > 0, sa
    assert max(ba) <= 10
    assert np.max(np.abs(a - b)) < 1e-8, np.max(np.abs(a - b))


def test_zip_chi_max_option_is_validated():
    with pytest.raises(Q.QlbError):
        Q.Ctx(device=0, chi_max=64, zip_chi_max=32)  # below chi_max
    with pytest.raises(Q.QlbError):
        Q.Ctx(device=0, zip_solver=2)
