"""Continuous-batching request loop for many independent Lindblad solves on one GPU.

Requests (single cat modes with their own alpha^2, Fock size, loss ratio, step
count and bond cap) arrive over time.  The loop admits a request when a slot is
free and its estimated device memory fits the budget, builds its system through
the C-ABI (the context caches the MPOs of the built-in factors, so a new request
costs only MPO sums), creates its state on its own CUDA stream, and keeps every
live state busy with chunks of steps.  Steps of different states run
concurrently on the GPU; a finished request releases its slot and memory, and
the next arrival takes them.  Latency = completion - arrival.

All numerical work happens in libqlb; this module is host-side scheduling.
"""
from __future__ import annotations

import time
from dataclasses import dataclass, field

import numpy as np

from . import qlb as Q
from . import systems


def estimate_bytes(R: int, chi: int, chi_mu: int, branches: int = 3, mpo_bond: int = 40) -> int:
    """Upper estimate of the device memory of one cat state (sites + step scratch),
    from the same capacity rules the library uses: zip-up bonds <= chi, purification
    rows chi_mu * branches, MPO bond ~ mpo_bond."""
    z = max(chi, chi_mu * branches)
    sites = R * 2 * z * z
    X = z * mpo_bond * 2 * chi
    M = 2 * z * chi * mpo_bond
    C = 2 * z * chi * mpo_bond
    G = (2 * z) ** 2
    T = 3 * (2 * z) * (2 * z)
    ew = 2 * (2 * z) ** 2
    return 16 * (sites + X + M + C + G + T + ew) + (1 << 20)


@dataclass
class Job:
    req: dict
    arrival: float
    admit: float = 0.0
    done: float = 0.0
    remaining: int = 0
    steps: int = 0
    sysb: object = None
    state: object = None
    est: int = 0
    result: dict = field(default_factory=dict)


def build_request(ctx: Q.Ctx, r: dict):
    """System and state of one request: a single cat mode with its own alpha^2, Fock
    size, loss ratio and bond caps."""
    cfg = dict(kind="cat", R=[r["R"]], alpha2=r["alpha2"], k2=1.0, k1=r["k1_over_k2"], eps_z=0.0,
               dt=r["dt"], tol=r["tol"])
    b = systems.build_cat(ctx, cfg)
    st = b.sys.state(b.init)
    st.truncate(chi_max=r["chi_max"], chi_mu_max=r["chi_mu_max"])
    return b, st


class Server:
    def __init__(self, ctx: Q.Ctx, hbm_budget: int = 2 << 30, max_slots: int = 64, chunk: int = 100,
                 build=build_request):
        self.ctx = ctx
        self.budget = hbm_budget
        self.max_slots = max_slots
        self.chunk = chunk
        self.build = build
        self.peak_live = 0
        self.peak_bytes = 0

    def _start(self, job: Job):
        job.sysb, job.state = self.build(self.ctx, job.req)
        job.remaining = job.steps

    def _finish(self, job: Job, now: float):
        st, b = job.state, job.sysb
        job.result = {"n": st.expectation(b.observables["n"]).real,
                      "parity": st.expectation(b.observables["parity"]).real,
                      "bonds": st.bond_dims()}
        st.close()
        for op in list(b.ops.values()) + list(b.observables.values()):
            op.close()
        b.sys.close()
        job.state = job.sysb = None
        job.done = now

    def run(self, requests, step_scale: float = 1.0, time_scale: float = 1.0, min_steps: int = 10):
        """Serve the requests (dicts from inputs.serving_requests).  Step counts are
        multiplied by step_scale and arrival times by time_scale.  Returns the jobs."""
        pending = sorted(
            (Job(req=r, arrival=r["arrival_s"] * time_scale, steps=max(min_steps, int(r["steps"] * step_scale)))
             for r in requests), key=lambda j: j.arrival)
        live: list[Job] = []
        done: list[Job] = []
        used = 0
        t0 = time.perf_counter()
        while pending or live:
            now = time.perf_counter() - t0
            # admission: arrived, a free slot, and the memory estimate fits the budget
            while pending and pending[0].arrival <= now and len(live) < self.max_slots:
                job = pending[0]
                job.est = estimate_bytes(job.req["R"], self.ctx.opts.chi_max, self.ctx.opts.chi_mu_max)
                if used + job.est > self.budget and live:
                    break
                pending.pop(0)
                job.admit = now
                self._start(job)
                used += job.est
                live.append(job)
            self.peak_live = max(self.peak_live, len(live))
            self.peak_bytes = max(self.peak_bytes, self.ctx.memory())
            progressed = False
            for job in list(live):
                if not job.state.poll():
                    continue
                progressed = True
                if job.remaining > 0:
                    n = min(self.chunk, job.remaining)
                    job.state.step(job.req["dt"], n)  # enqueued on the state's stream
                    job.remaining -= n
                else:
                    self._finish(job, time.perf_counter() - t0)
                    used -= job.est
                    live.remove(job)
                    done.append(job)
            if not progressed:
                time.sleep(0.0002)
        return done


def summarize(jobs, wall_s: float):
    lat = np.array([j.done - j.arrival for j in jobs])
    steps = sum(j.steps for j in jobs)
    return {"requests": len(jobs), "steps_total": int(steps), "wall_s": wall_s,
            "steps_per_s": steps / wall_s if wall_s > 0 else None,
            "p50_latency_s": float(np.percentile(lat, 50)), "p99_latency_s": float(np.percentile(lat, 99)),
            "mean_latency_s": float(lat.mean())}
