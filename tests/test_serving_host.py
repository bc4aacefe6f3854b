"""Host side of the serving workload (no GPU): the request marshalling into term
lists, the arrival driver (submission at the arrival times, polling until every
request is done, step scaling) against a stand-in server, and the summary."""
import numpy as np

from paper_2605_27515_gb300 import inputs
from paper_2605_27515_gb300 import qlb as Q
from paper_2605_27515_gb300 import serving


class _Clock:
    def __init__(self):
        self.t = 0.0

    def __call__(self):
        return self.t

    def sleep(self, s):
        self.t += s


class _FakeServer:
    """Finishes each request `lag` polls after its submission; records the order."""

    def __init__(self, clock, lag=3):
        self.clock, self.lag = clock, lag
        self.log = []
        self.jobs = {}

    def submit(self, R, H, jumps, vecs, dt, steps, obs, tol=0.0, chi_max=0, chi_mu_max=0):
        t = len(self.log)
        self.log.append((self.clock(), R, steps, len(jumps), len(obs)))
        self.jobs[t] = [self.lag, steps]
        return t

    def poll(self, t):
        j = self.jobs[t]
        if j[0] > 0:
            j[0] -= 1
            return None
        return [complex(j[1]), complex(1.0)], (0.0, 0.0, 0.0)


def test_cat_request_terms():
    r = inputs.serving_requests(n=1)[0]
    q = serving.cat_request(r)
    assert q["R"] == [r["R"]] and q["H"] == [] and len(q["jumps"]) == 2
    (c1, f1), (c0, f0) = q["jumps"][0]
    assert f1 == [(0, Q.F_A, 2)] and f0 == [] and abs(c0 + r["alpha2"]) < 1e-15 and c1 == 1.0
    assert abs(q["jumps"][1][0][0] - np.sqrt(r["k1_over_k2"])) < 1e-15
    assert q["vecs"][0][0] == 1.0 and np.sum(np.abs(q["vecs"][0])) == 1.0
    assert [o[0][1][0][1] for o in q["obs"]] == [Q.F_NUM, Q.F_PARITY]


def test_drive_submits_at_arrival_and_collects_everything():
    reqs = inputs.serving_requests(n=12, seed=3)
    clk = _Clock()
    srv = _FakeServer(clk)
    jobs = serving.drive(srv, reqs, step_scale=0.01, time_scale=1.0, poll_s=1e-3, clock=clk, sleep=clk.sleep)
    assert len(jobs) == 12 and len(srv.log) == 12
    # submitted in arrival order, never before the arrival time
    times = [t for t, *_ in srv.log]
    assert times == sorted(times)
    for j in jobs:
        assert j.submitted >= j.arrival - 1e-12
        assert j.done >= j.submitted
        assert j.steps == max(10, int(j.req["steps"] * 0.01))
        assert j.result["n"] == float(j.steps)  # the stand-in returns the step count
    s = serving.summarize(jobs, clk.t)
    assert s["requests"] == 12 and s["p99_latency_s"] >= s["p50_latency_s"] > 0


class _SlowServer(_FakeServer):
    """Finishes a request after `steps // 1000` polls and records cancellations."""

    def __init__(self, clock):
        super().__init__(clock)
        self.cancelled = []

    def submit(self, R, H, jumps, vecs, dt, steps, obs, tol=0.0, chi_max=0, chi_mu_max=0):
        t = super().submit(R, H, jumps, vecs, dt, steps, obs, tol, chi_max, chi_mu_max)
        self.jobs[t][0] = steps // 1000
        return t

    def cancel(self, t):
        self.cancelled.append(t)


def test_drive_window_stops_at_the_window_and_cancels_the_rest():
    """The stated mix (own step counts) for a fixed window: requests arriving after
    the window are never submitted, unfinished ones are cancelled, and the summary
    counts only completed requests for latency."""
    reqs = inputs.serving_requests(n=40, seed=4)
    clk = _Clock()
    srv = _SlowServer(clk)
    window = reqs[20]["arrival_s"] + 0.01  # about half of the arrivals fall inside
    jobs, used = serving.drive_window(srv, reqs, window, poll_s=2e-3, clock=clk, sleep=clk.sleep)
    assert used >= window
    assert len(jobs) == len(srv.log) and 21 <= len(jobs) < 40
    assert all(j.steps == j.req["steps"] for j in jobs)  # not scaled
    done = [j for j in jobs if j.done > 0]
    assert sorted(srv.cancelled) == sorted(j.ticket for j in jobs if j.done == 0)
    assert all(j.result["n"] == float(j.steps) for j in done)
    s = serving.summarize_window(jobs, used, steps_taken=12345)
    assert s["submitted"] == len(jobs) and s["completed"] == len(done)
    assert s["steps_per_s"] == 12345 / used
    if done:
        assert s["p99_latency_s"] >= s["p50_latency_s"] >= 0


class _FailingServer(_SlowServer):
    """Request 2 fails: its poll raises the library's error."""

    def poll(self, t):
        if t == 2:
            raise Q.QlbError(Q.EINVAL, "request failed")
        return super().poll(t)


def test_drive_window_reports_a_failed_request():
    reqs = inputs.serving_requests(n=10, seed=5)
    clk = _Clock()
    srv = _FailingServer(clk)
    jobs, used = serving.drive_window(srv, reqs, reqs[-1]["arrival_s"] + 0.01, poll_s=2e-3, clock=clk,
                                      sleep=clk.sleep)
    s = serving.summarize_window(jobs, used, steps_taken=1)
    assert s["failed"] == 1 and "request failed" in s["first_failure"]
    assert 2 not in srv.cancelled  # a failed request is not cancelled again
