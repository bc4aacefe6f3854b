"""The library's continuous-batching server (qlb_server_*, through the C-ABI): each
result is the same alone and in the mix, admission respects the live-slot cap and
the device-memory budget, served results match the dense oracle, and a request
can be cancelled."""
import numpy as np
import pytest

from oracle import systems as OS
from paper_2605_27515_gb300 import inputs
from paper_2605_27515_gb300 import qlb as Q
from paper_2605_27515_gb300 import serving

pytestmark = pytest.mark.gpu


def _requests(n, seed=5):
    """The serving mix at test size: Fock sizes up to N = 64 and a step that the
    explicit scheme keeps stable there (h sum_k ||L_k||^2 < 4)."""
    reqs = inputs.serving_requests(n=n, seed=seed)
    for r in reqs:
        r["R"] = min(r["R"], 6)
        r["dt"] = 2e-4
    return reqs


def _serve(reqs, step_scale, time_scale=0.0, **kw):
    ctx = Q.Ctx(device=0, chi_max=64, chi_mu_max=8, stream_ordered=1)
    srv = Q.Server(ctx, chunk=50, **kw)
    jobs = serving.drive(srv, reqs, step_scale=step_scale, time_scale=time_scale)
    stats = srv.stats()
    srv.close()
    ctx.close()
    return jobs, stats


def test_alone_equals_mixed():
    reqs = _requests(5)
    alone = {}
    for r in reqs:
        (job,), _ = _serve([dict(r, arrival_s=0.0)], 0.02)
        alone[r["id"]] = job.result
    jobs, stats = _serve(reqs, 0.02)
    assert stats["peak_live"] > 1  # they really ran together
    assert stats["completed"] == 5
    for j in jobs:
        a = alone[j.req["id"]]
        assert abs(j.result["n"] - a["n"]) < 1e-12, (j.req["id"], j.result, a)
        assert abs(j.result["parity"] - a["parity"]) < 1e-12


def test_admission_respects_slots_and_budget():
    reqs = _requests(6, seed=9)
    jobs, stats = _serve(reqs, 0.01, max_live=2)
    assert len(jobs) == 6 and stats["peak_live"] <= 2
    jobs, stats = _serve(reqs, 0.01, hbm_budget=1)  # no two requests fit: one at a time
    assert len(jobs) == 6 and stats["peak_live"] == 1
    assert all(np.isfinite([j.done - j.arrival for j in jobs]))


def test_served_results_match_oracle():
    """Each served request, run in the mix, within 1e-6 of the dense oracle at its own
    Fock size (photon number and parity at completion)."""
    reqs = _requests(3, seed=13)
    jobs, _ = _serve(reqs, 0.02)
    for j in jobs:
        r = j.req
        cfg = dict(kind="cat", R=[r["R"]], alpha2=r["alpha2"], k2=1.0, k1=r["k1_over_k2"], eps_z=0.0)
        _, recs = OS.cat(cfg).evolve(r["dt"], j.steps, j.steps, names=["n", "parity"])
        n_o, p_o = recs[-1][1]
        assert abs(j.result["n"] - n_o) < 1e-6, (r["id"], j.result, n_o)
        assert abs(j.result["parity"] - p_o) < 1e-6, (r["id"], j.result, p_o)


def test_cancel():
    r = _requests(1, seed=21)[0]
    ctx = Q.Ctx(device=0, chi_max=64, chi_mu_max=8, stream_ordered=1)
    srv = Q.Server(ctx, chunk=10)
    q = serving.cat_request(r)
    t = srv.submit(q["R"], q["H"], q["jumps"], q["vecs"], q["dt"], 10 ** 7, q["obs"])
    srv.cancel(t)
    import time
    for _ in range(2000):
        try:
            if srv.poll(t) is not None:
                break
        except Q.QlbError as e:
            assert e.status == Q.ESTATE
            break
        time.sleep(0.005)
    else:
        raise AssertionError("the cancelled request never left the server")
    srv.close()
    ctx.close()
