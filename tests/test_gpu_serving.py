"""Serving loop: each result is the same alone and in the mix, and admission
respects the device-memory budget (continuous batching of independent solves)."""
import numpy as np
import pytest

from paper_2605_27515_gb300 import inputs
from paper_2605_27515_gb300 import qlb as Q
from paper_2605_27515_gb300 import serving

pytestmark = pytest.mark.gpu


def _requests(n, seed=5):
    reqs = inputs.serving_requests(n=n, seed=seed)
    for r in reqs:
        r["R"] = min(r["R"], 7)  # keep the test quick
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
