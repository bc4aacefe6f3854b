"""Serving loop: each result is the same alone and in the mix, and admission
respects the device-memory budget (continuous batching of independent solves)."""
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


def test_alone_equals_mixed():
    reqs = _requests(5)
    ctx = Q.Ctx(device=0, chi_max=64, chi_mu_max=8, stream_ordered=1)
    alone = {}
    for r in reqs:
        srv = serving.Server(ctx, chunk=50)
        (job,) = srv.run([dict(r, arrival_s=0.0)], step_scale=0.02)
        alone[r["id"]] = job.result
    srv = serving.Server(ctx, chunk=50)
    jobs = srv.run(reqs, step_scale=0.02, time_scale=0.0)
    assert srv.peak_live > 1  # they really ran together
    for j in jobs:
        a = alone[j.req["id"]]
        assert abs(j.result["n"] - a["n"]) < 1e-9, (j.req["id"], j.result, a)
        assert abs(j.result["parity"] - a["parity"]) < 1e-9
        assert j.result["bonds"] == a["bonds"]
    ctx.close()


def test_admission_respects_budget():
    reqs = _requests(6, seed=9)
    ctx = Q.Ctx(device=0, chi_max=64, chi_mu_max=8, stream_ordered=1)
    one = max(serving.estimate_bytes(r["R"], 64, 8) for r in reqs)
    srv = serving.Server(ctx, hbm_budget=2 * one + 1, chunk=50)
    jobs = srv.run(reqs, step_scale=0.01, time_scale=0.0)
    assert len(jobs) == 6
    assert srv.peak_live <= 2
    lat = [j.done - j.arrival for j in jobs]
    assert all(np.isfinite(lat))
    ctx.close()


def test_served_results_match_oracle():
    """Each served request, run in the mix, within 1e-6 of the dense oracle at its own
    Fock size (photon number and parity at completion)."""
    reqs = _requests(3, seed=13)
    ctx = Q.Ctx(device=0, chi_max=64, chi_mu_max=8, stream_ordered=1)
    srv = serving.Server(ctx, chunk=50)
    jobs = srv.run(reqs, step_scale=0.02, time_scale=0.0)
    for j in jobs:
        r = j.req
        cfg = dict(kind="cat", R=[r["R"]], alpha2=r["alpha2"], k2=1.0, k1=r["k1_over_k2"], eps_z=0.0)
        _, recs = OS.cat(cfg).evolve(r["dt"], j.steps, j.steps, names=["n", "parity"])
        n_o, p_o = recs[-1][1]
        assert abs(j.result["n"] - n_o) < 1e-6, (r["id"], j.result, n_o)
        assert abs(j.result["parity"] - p_o) < 1e-6, (r["id"], j.result, p_o)
    ctx.close()
