"""Parity at the benchmark's full size, in the configuration bench.py times: the
single cat mode at N = 512 (alpha^2 = 32, Zeno drive eps_Z = 0.1, dt = 5e-4,
chi <= 64, chi_mu <= 16, cutoff 1e-12, stream-ordered context), against the dense
FP64 oracle at N = 512 every 5 steps over the first 30, in both precision forms;
plus properties that hold at any size (trace, purity, parity range, caps, and the
explicit scheme's instability warning for this step size).  With the Jacobi zip-up
(zip_solver = 0) the zip-up bonds reach the cap of 64 within these steps, and the
solver counters show eigen-solves of size 128 on the multi-SM (cluster) path; with
the default range-basis zip-up the counters show the zip-up bonds served by it.
Kept in a file of its own, collected after the other GPU parity files."""
import pytest

from oracle import systems as OS
from paper_2605_27515_gb300 import inputs
from paper_2605_27515_gb300 import qlb as Q
from paper_2605_27515_gb300 import systems

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def oracle_records():
    cfg = inputs.config("cat_r9")
    _, recs = OS.cat(cfg).evolve(cfg["dt"], 30, 5, names=["n", "parity"])
    return recs


@pytest.mark.parametrize("precision,zip_solver", [(Q.PREC_F64, 1), (Q.PREC_MIXED, 1), (Q.PREC_TC, 1),
                                                  (Q.PREC_F64, 0), (Q.PREC_MIXED, 0)])
def test_full_size_first_steps_match_oracle(oracle_records, precision, zip_solver):
    cfg = inputs.config("cat_r9")
    ctx = Q.Ctx(device=0, precision=precision, tol=cfg["tol"], chi_max=cfg["chi_max"],
                chi_mu_max=cfg["chi_mu_max"], stream_ordered=1, zip_solver=zip_solver)
    b = systems.build(ctx, cfg)
    st = b.sys.state(b.init)
    ctx.profile_reset()
    done = 0
    worst = 0.0
    for step, (n_o, p_o) in oracle_records[1:]:
        status = st.step(cfg["dt"], step - done)
        done = step
        assert status == Q.WUNSTABLE  # h * sum ||L_k||^2 > 4 at N = 512: the warning, not an error
        n_g = st.expectation(b.observables["n"]).real
        p_g = st.expectation(b.observables["parity"]).real
        worst = max(worst, abs(n_g - n_o), abs(p_g - p_o))
        assert abs(st.trace() - 1.0) < 1e-12
        assert 0.0 < st.purity() <= 1.0 + 1e-12
        assert -1.0 - 1e-12 <= p_g <= 1.0 + 1e-12 and n_g >= -1e-12
        bd = st.bond_dims()
        assert bd[0] <= cfg["chi_mu_max"] and max(bd[1:]) <= cfg["chi_max"]
    assert worst < 1e-6, worst
    sv = ctx.solver_stats()
    if zip_solver == 0:
        # the zip-up bonds reach the cap of 64, so the eigen-solves run at 2 x 64 = 128,
        # past one CTA's shared memory (the thread-block cluster path)
        assert sv["max_n"] >= 128, sv
        assert sv["global_ws"] >= 1, sv
    else:
        assert sv["zip_range"] >= 8 * 30, sv  # every zip-up bond of every step
    st.close()
    ctx.close()
