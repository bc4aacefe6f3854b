"""Serving workload driver over the library's continuous-batching server.

The scheduling itself (admission by device-memory budget and live slots, chunked
stepping of the live states as same-shape groups, completion, release) runs in
libqlb (qlb_server_*, csrc/server.cu).  This module only
  * turns a request of the serving mix (a single cat mode with its own alpha^2,
    Fock size, loss ratio, step count and bond caps) into the term lists of a
    qlb_request (argument marshalling),
  * submits the requests at their arrival times and polls for completions
    (`drive`; `drive_window` runs the mix with its own step counts for a fixed
    wall window and cancels what is left), and
  * summarises latencies (completion - arrival) and throughput.
"""
from __future__ import annotations

import time
from dataclasses import dataclass, field

import numpy as np

from . import qlb as Q


def vacuum(N):
    v = np.zeros(N, dtype=np.complex128)
    v[0] = 1.0
    return v


def cat_request(r: dict):
    """Term lists of one serving request (Sec. VI cat mode): H = 0,
    L1 = sqrt(k2)(a^2 - alpha^2), L2 = sqrt(k1) a with k2 = 1; observables photon
    number and parity; vacuum start.  Returns a dict of qlb_request fields."""
    k2, k1, a2 = 1.0, r["k1_over_k2"], r["alpha2"]
    jumps = [[(np.sqrt(k2), [(0, Q.F_A, 2)]), (-np.sqrt(k2) * a2, [])]]
    if k1:
        jumps.append([(np.sqrt(k1), [(0, Q.F_A)])])
    obs = [[(1.0, [(0, Q.F_NUM)])], [(1.0, [(0, Q.F_PARITY)])]]
    return dict(R=[r["R"]], H=[], jumps=jumps, vecs=[vacuum(2 ** r["R"])], dt=r["dt"], obs=obs,
                tol=r.get("tol", 0.0), chi_max=r.get("chi_max", 0), chi_mu_max=r.get("chi_mu_max", 0))


@dataclass
class Job:
    req: dict
    arrival: float
    steps: int
    ticket: int = -1
    submitted: float = 0.0
    done: float = 0.0
    result: dict = field(default_factory=dict)
    server_times: tuple = ()
    failed: str = ""


def drive(server, requests, step_scale: float = 1.0, time_scale: float = 1.0, min_steps: int = 10,
          poll_s: float = 0.0005, timeout_s: float = 3600.0, clock=time.perf_counter, sleep=time.sleep):
    """Submit each request at its arrival time (arrival_s * time_scale after the start,
    on the host clock) with steps * step_scale steps, poll until every request is done,
    and return the jobs (result = {'n', 'parity'}; latency = done - arrival)."""
    jobs = sorted((Job(req=r, arrival=r["arrival_s"] * time_scale,
                       steps=max(min_steps, int(r["steps"] * step_scale))) for r in requests),
                  key=lambda j: j.arrival)
    t0 = clock()
    nxt = 0
    open_jobs = []
    while nxt < len(jobs) or open_jobs:
        now = clock() - t0
        if now > timeout_s:
            raise TimeoutError(f"serving did not finish within {timeout_s} s")
        while nxt < len(jobs) and jobs[nxt].arrival <= now:
            j = jobs[nxt]
            q = cat_request(j.req)
            j.ticket = server.submit(q["R"], q["H"], q["jumps"], q["vecs"], q["dt"], j.steps, q["obs"],
                                     tol=q["tol"], chi_max=q["chi_max"], chi_mu_max=q["chi_mu_max"])
            j.submitted = now
            open_jobs.append(j)
            nxt += 1
        still = []
        for j in open_jobs:
            r = server.poll(j.ticket)
            if r is None:
                still.append(j)
                continue
            vals, times = r
            j.done = clock() - t0
            j.result = {"n": vals[0].real, "parity": vals[1].real}
            j.server_times = times
        open_jobs = still
        if open_jobs or nxt < len(jobs):
            sleep(poll_s)
    return jobs


def drive_window(server, requests, window_s: float, poll_s: float = 0.0005, clock=time.perf_counter,
                 sleep=time.sleep):
    """The request mix as stated (every request with its own step count) for a fixed
    wall window: submit each request at its arrival time, collect completions until
    window_s has passed, then cancel what is still pending or running.  Returns the
    jobs (done = 0 for the unfinished ones) and the window actually used."""
    jobs = sorted((Job(req=r, arrival=r["arrival_s"], steps=int(r["steps"])) for r in requests),
                  key=lambda j: j.arrival)
    t0 = clock()
    nxt = 0
    open_jobs = []
    while clock() - t0 < window_s:
        now = clock() - t0
        while nxt < len(jobs) and jobs[nxt].arrival <= now:
            j = jobs[nxt]
            q = cat_request(j.req)
            j.ticket = server.submit(q["R"], q["H"], q["jumps"], q["vecs"], q["dt"], j.steps, q["obs"],
                                     tol=q["tol"], chi_max=q["chi_max"], chi_mu_max=q["chi_mu_max"])
            j.submitted = now
            open_jobs.append(j)
            nxt += 1
        still = []
        for j in open_jobs:
            try:
                r = server.poll(j.ticket)
            except Q.QlbError as e:  # a failed request is reported, not fatal to the window
                j.failed = str(e)
                continue
            if r is None:
                still.append(j)
                continue
            vals, times = r
            j.done = clock() - t0
            j.result = {"n": vals[0].real, "parity": vals[1].real}
            j.server_times = times
        open_jobs = still
        sleep(poll_s)
    used = clock() - t0
    for j in open_jobs:
        server.cancel(j.ticket)
    return jobs[:nxt], used


def summarize_window(jobs, window_s: float, steps_taken: int):
    """Completed requests, their latencies, and the steps all requests took in the
    window (finished or not) per second."""
    done = [j for j in jobs if j.done > 0]
    lat = np.array([j.done - j.arrival for j in done])
    failed = [j for j in jobs if j.failed]
    out = {"window_s": window_s, "submitted": len(jobs), "completed": len(done), "failed": len(failed),
           "steps_taken": int(steps_taken), "steps_per_s": steps_taken / window_s if window_s > 0 else None}
    if failed:
        out["first_failure"] = failed[0].failed
    if len(done):
        out.update({"p50_latency_s": float(np.percentile(lat, 50)), "p99_latency_s": float(np.percentile(lat, 99)),
                    "completed_steps": int(sum(j.steps for j in done))})
    return out


def summarize(jobs, wall_s: float):
    lat = np.array([j.done - j.arrival for j in jobs])
    steps = sum(j.steps for j in jobs)
    return {"requests": len(jobs), "steps_total": int(steps), "wall_s": wall_s,
            "steps_per_s": steps / wall_s if wall_s > 0 else None,
            "p50_latency_s": float(np.percentile(lat, 50)), "p99_latency_s": float(np.percentile(lat, 99)),
            "mean_latency_s": float(lat.mean())}
