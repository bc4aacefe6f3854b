"""Host logic of the serving loop (admission by memory budget and slots, arrival
order, chunked stepping, completion) with stand-in states, no GPU."""
import numpy as np

from paper_2605_27515_gb300 import serving


class _Opts:
    chi_max = 64
    chi_mu_max = 8


class _Ctx:
    opts = _Opts()

    def memory(self):
        return 0


class _Op:
    def close(self):
        pass


class _State:
    """Finishes each enqueued chunk after `lag` polls, like a stream that is busy."""

    def __init__(self, log, rid, lag=2):
        self.log, self.rid, self.lag = log, rid, lag
        self.busy = 0
        self.steps = 0

    def poll(self):
        if self.busy:
            self.busy -= 1
            return False
        return True

    def step(self, dt, n):
        assert self.busy == 0, "a chunk was enqueued on a busy state"
        self.steps += n
        self.busy = self.lag
        self.log.append(("step", self.rid, n))

    def expectation(self, op):
        return complex(self.steps)

    def bond_dims(self):
        return [1]

    def close(self):
        self.log.append(("close", self.rid))


class _Sys:
    def close(self):
        pass


class _Built:
    def __init__(self):
        self.sys = _Sys()
        self.ops = {"L": _Op()}
        self.observables = {"n": _Op(), "parity": _Op()}


def _requests(n, steps):
    return [dict(id=i, arrival_s=0.0, R=6, alpha2=4.0, k1_over_k2=1e-3, steps=steps, dt=1e-3, chi_max=32,
                 chi_mu_max=8, tol=1e-12) for i in range(n)]


def _server(log, **kw):
    def build(ctx, r):
        log.append(("start", r["id"]))
        return _Built(), _State(log, r["id"])

    return serving.Server(_Ctx(), build=build, **kw)


def test_every_request_completes_with_all_its_steps():
    log = []
    srv = _server(log, chunk=7)
    jobs = srv.run(_requests(5, 30), step_scale=1.0, time_scale=0.0)
    assert sorted(j.req["id"] for j in jobs) == list(range(5))
    for j in jobs:
        assert j.result["n"] == 30  # the stand-in reports the steps it took
        chunks = [e[2] for e in log if e[0] == "step" and e[1] == j.req["id"]]
        assert chunks == [7, 7, 7, 7, 2]
    assert srv.peak_live == 5


def test_budget_limits_live_requests():
    log = []
    one = serving.estimate_bytes(6, 64, 8)
    srv = _server(log, hbm_budget=2 * one + 1, chunk=10)
    jobs = srv.run(_requests(6, 25), step_scale=1.0, time_scale=0.0)
    assert len(jobs) == 6 and srv.peak_live == 2
    live = 0
    for e in log:  # never more than two started and not yet closed
        live += {"start": 1, "close": -1}.get(e[0], 0)
        assert live <= 2


def test_slots_and_arrival_order():
    log = []
    srv = _server(log, max_slots=1, chunk=100)
    reqs = _requests(3, 5)
    for r, t in zip(reqs, (0.0, 0.002, 0.004)):
        r["arrival_s"] = t
    jobs = srv.run(reqs, step_scale=1.0, time_scale=1.0)
    starts = [e[1] for e in log if e[0] == "start"]
    assert starts == [0, 1, 2] and srv.peak_live == 1
    assert all(np.isfinite(j.done - j.arrival) and j.done >= j.arrival for j in jobs)


def test_estimate_grows_with_caps():
    assert serving.estimate_bytes(9, 64, 16) > serving.estimate_bytes(9, 32, 8) > 0
