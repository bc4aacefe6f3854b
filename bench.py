"""Benchmark of the purified quantics-MPS Lindblad step on GB300.

Workload (the large single cat mode): one bosonic mode of N = 512 Fock levels
(R = 9 quantics sites), L1 = sqrt(k2)(a^2 - alpha^2) with alpha^2 = 32,
L2 = sqrt(k1) a with k1/k2 = 1e-3, Zeno drive H = 0.1 (a + a^dag), dt = 5e-4,
bond cap chi <= 64, purification cap chi_mu <= 16, cutoff 1e-12, from vacuum.
A "step" is one first-order Kraus step (apply + stack + recompress + purify +
renormalise).  W warm-up steps are run first, then K steps are timed with CUDA
events on the library's stream, L2 flushed (256 MiB write) between steps.

Prints one JSON line (rank 0).  --impl reference times the FP64 dense oracle on
the host cores instead (bounded sample).  Under torchrun each rank steps its own
replica (no collective); value = steps of all ranks / max time.
"""
from __future__ import annotations

import argparse
import json
import os
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "Lindblad steps/s at <=1e-6 obs. error vs plain FP64 form; batched p50/p99 latency"
WORKLOAD = "cat_r9"


def _peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            return json.load(f)
    return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "fallback": True}


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled during the timed region."""

    def __init__(self, index=0):
        self.index = index
        self.rows = []
        self.proc = None

    def __enter__(self):
        q = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.hw_slowdown,"
             "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
             "clocks_event_reasons.sw_power_cap")
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), f"--query-gpu={q}",
                                          "--format=csv,noheader,nounits", "-lms", "100"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except Exception:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            parts = [x.strip() for x in line.split(",")]
            if len(parts) >= 7:
                self.rows.append(parts)

    def __exit__(self, *a):
        if self.proc:
            time.sleep(0.25)
            self.proc.terminate()
            try:
                self.proc.wait(timeout=2)
            except Exception:
                self.proc.kill()

    def summary(self):
        if not self.rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}
        sm = [float(r[0]) for r in self.rows if r[0].replace(".", "").isdigit()]
        mx = [float(r[1]) for r in self.rows if r[1].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in self.rows for i in range(4) if r[3 + i] == "Active"})
        return {"sm_mhz": float(np.median(sm)) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(self.rows)}


def _traffic(kernel_class):
    """DRAM bytes per launch of the class's dominant kernel from the committed ncu
    summary (profiles/traffic.json), or None when that summary was taken on another
    version of the kernel's source (its sha256 no longer matches)."""
    import hashlib

    p = os.path.join(ROOT, "profiles", "traffic.json")
    if not os.path.exists(p):
        return None, None
    with open(p) as f:
        tab = json.load(f)
    ent = tab.get(kernel_class)
    if not ent:
        return None, None
    src = os.path.join(ROOT, ent["source"])
    if not os.path.exists(src):
        return None, None
    with open(src, "rb") as f:
        sha = hashlib.sha256(f.read()).hexdigest()
    if sha != ent["source_sha256"]:
        return None, f"{ent['kernel']}: source changed since the ncu capture"
    return ent["dram_bytes_per_launch"], f"{ent['kernel']} ({ent['capture']})"


def dist_info():
    return int(os.environ.get("RANK", 0)), int(os.environ.get("WORLD_SIZE", 1)), int(os.environ.get("LOCAL_RANK", 0))


def replica_throughput(local_ms: float, steps: int, device=None):
    """Whole-job steps/s of independent replicas: every rank ran `steps` steps in
    `local_ms`; the job lasts as long as its slowest rank (max over ranks).
    Returns (steps/s over all ranks, the max time in ms)."""
    import torch
    import torch.distributed as dist

    world = 1
    total_ms = local_ms
    if dist.is_available() and dist.is_initialized():
        world = dist.get_world_size()
        t = torch.tensor([local_ms], dtype=torch.float64, device=device)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        total_ms = float(t.item())
    return world * steps / (total_ms / 1e3), total_ms


def run_reference(args):
    """FP64 dense oracle of the same workload on the host cores (bounded sample)."""
    rank, world, _ = dist_info()
    if rank != 0:
        return
    from oracle import dense as D
    from oracle import systems as OS
    from paper_2605_27515_gb300 import inputs

    cfg = inputs.config(WORKLOAD)
    ds = OS.cat(cfg)
    rho = ds.rho0()
    for _ in range(max(1, args.warmup)):
        rho = D.kraus_step(rho, ds.H0, ds.Ls, cfg["dt"])
    t0 = time.perf_counter()
    n = 0
    budget = 20.0
    while n < args.steps or (time.perf_counter() - t0) < 0.1:
        rho = D.kraus_step(rho, ds.H0, ds.Ls, cfg["dt"])
        n += 1
        if time.perf_counter() - t0 > budget:
            break
    dt = time.perf_counter() - t0
    v = n / dt
    cores = os.cpu_count()
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": "steps/s", "n_gpus": world,
            "steps": n, "warmup": args.warmup, "ms_per_step": 1e3 * dt / n, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": WORKLOAD, "N": 512, "alpha2": 32.0, "dt": cfg["dt"], "form": "dense rho"},
            "cpu_baseline": {"value": v, "unit": "steps/s", "cores": cores, "kind": "oracle",
                             "sample": f"{n} dense FP64 Kraus steps of the N=512 cat after {args.warmup} warm-up steps"},
            "e2e": {"value": v, "unit": "steps/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def cpu_baseline_sample():
    """The dense oracle on a bounded sample of the same workload (rank 0, N=1)."""
    from oracle import dense as D
    from oracle import systems as OS
    from paper_2605_27515_gb300 import inputs

    cfg = inputs.config(WORKLOAD)
    ds = OS.cat(cfg)
    rho = ds.rho0()
    rho = D.kraus_step(rho, ds.H0, ds.Ls, cfg["dt"])
    t0 = time.perf_counter()
    n = 0
    while time.perf_counter() - t0 < 10.0 and n < 200:
        rho = D.kraus_step(rho, ds.H0, ds.Ls, cfg["dt"])
        n += 1
    dt = time.perf_counter() - t0
    return {"value": n / dt, "unit": "steps/s", "cores": os.cpu_count(), "kind": "oracle",
            "sample": f"{n} dense FP64 Kraus steps of the N=512 cat (about {dt:.0f} s of host time)"}


def _measure_form(args, dev, precision, world, flush):
    """One precision form of the cat_r9 workload: W warm-up steps, K timed steps
    (CUDA events on the state's stream, L2 flushed between steps), a replay of the
    same K steps from a snapshot with events around every launch (kernel classes and
    roofline), a later window, and the end-to-end run through the public API."""
    import torch

    from paper_2605_27515_gb300 import inputs, qlb, systems

    cfg = inputs.config(WORKLOAD)
    ctx = qlb.Ctx(device=dev, precision=precision, tol=cfg["tol"], chi_max=cfg["chi_max"],
                  chi_mu_max=cfg["chi_mu_max"], stream_ordered=1, mixed_gemm=args.mixed_gemm)
    tuning = os.path.join(ROOT, "paper_2605_27515_gb300", "tuning", "gram_splitk_gb300.txt")
    if os.path.exists(tuning):
        ctx.load_tuning(tuning)  # the autotuner's split-K table (qlb_autotune on a GB300)
    b = systems.build(ctx, cfg)
    st = b.sys.state(b.init)
    stream = torch.cuda.ExternalStream(st.stream(), device=dev)
    dt = cfg["dt"]
    status = st.step(dt, args.warmup)
    ctx.synchronize()
    bonds_before = st.bond_dims()
    snapshot = st.export()  # the profiled pass below replays exactly these steps
    ctx.profile_reset()
    evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    if world > 1:
        import torch.distributed as dist

        dist.barrier()
    torch.cuda.synchronize()
    with ClockSampler(dev) as clk:
        torch.cuda.nvtx.range_push("timed_steps")
        with torch.cuda.stream(stream):
            for k in range(args.steps):
                flush.fill_(float(k))
                evs[k][0].record(stream)
                status = max(status, st.step(dt, 1))
                evs[k][1].record(stream)
        torch.cuda.synchronize()
        torch.cuda.nvtx.range_pop()
    if world > 1:
        dist.barrier()
    ms = [a.elapsed_time(bb) for a, bb in evs]
    value, total_ms = replica_throughput(float(sum(ms)), args.steps, device=f"cuda:{dev}")
    bonds_after = st.bond_dims()
    obs_end = [st.expectation(b.observables["n"]).real, st.expectation(b.observables["parity"]).real]
    solver = ctx.solver_stats()  # counters of the timed (graph-launched) steps

    # kernel-class breakdown of the same steps: the state is put back to the
    # snapshot taken before the timed window and the same K steps run again with
    # CUDA events around every launch (no graph)
    st.import_(snapshot)
    ctx.profile_enable(True)
    ctx.profile_reset()
    st.step(dt, args.steps)
    ctx.synchronize()
    prof = {qlb.K_NAMES[k]: ctx.profile_read(k) for k in range(qlb.K_COUNT)}
    ctx.profile_enable(False)
    replay_bonds = st.bond_dims()
    launches_per_step = sum(p["launches"] for p in prof.values()) / args.steps
    dom = max(prof, key=lambda k: prof[k]["ms"])
    dp = prof[dom]
    fp64_peak = qlb.qlb_measure_peak(dev, 0)
    fp32_peak = qlb.qlb_measure_peak(dev, 1)
    achieved = dp["flops"] / (dp["ms"] / 1e3) / 1e12 if dp["ms"] > 0 else 0.0
    traffic, traffic_src = _traffic(dom)
    # the truncation solves do FP64-accurate work: their device-counted flops are set
    # against the measured FP64 peak in both forms (the double-float form runs them
    # on the FP32 pipes, each FP64-equivalent operation costing ~10-20 FP32 ones)
    roofline = {"kernel": dom, "bound": "alu", "achieved": achieved, "peak": fp64_peak, "unit": "TFLOP/s",
                "frac": achieved / fp64_peak, "traffic": traffic, "traffic_source": traffic_src,
                "peak_source": "measured FP64 FMA throughput of this GPU (qlb_measure_peak), of measured",
                "frac_of_fp32_peak": achieved / fp32_peak,
                "launches": dp["launches"], "ms_per_launch": dp["ms"] / max(1, dp["launches"]),
                "flops_per_launch": dp["flops"] / max(1, dp["launches"]),
                "class_ms_per_step": dp["ms"] / args.steps, "step_ms": total_ms / args.steps,
                "same_steps_as_timed": replay_bonds == bonds_after}
    nsol = max(1.0, solver["solves"])
    solver_line = {"solves_per_step": solver["solves"] / args.steps, "sweeps_per_solve": solver["sweeps"] / nsol,
                   "mean_n": solver["sum_n"] / nsol, "mean_kept": solver["sum_k"] / nsol,
                   "at_limit": solver["at_limit"],
                   "zip_range_per_step": solver["zip_range"] / args.steps,
                   "zip_fallback_per_step": solver["zip_fallback"] / args.steps}

    # a later window of the same run: after window2 more steps the bonds have grown
    # to their plateau (the literal dt drives the state into the top Fock levels,
    # where the solves are larger); the same K steps timed again
    window2 = None
    if args.window2 > 0:
        st.import_(snapshot)
        st.step(dt, args.steps + args.window2)
        ctx.synchronize()
        b2 = st.bond_dims()
        ctx.profile_reset()
        ev2 = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
        torch.cuda.synchronize()
        with torch.cuda.stream(stream):
            for k in range(args.steps):
                flush.fill_(float(k))
                ev2[k][0].record(stream)
                st.step(dt, 1)
                ev2[k][1].record(stream)
        torch.cuda.synchronize()
        ms2 = [a.elapsed_time(bb) for a, bb in ev2]
        sv2 = ctx.solver_stats()
        n2 = max(1.0, sv2["solves"])
        window2 = {"first_step": args.warmup + args.steps + args.window2, "steps": args.steps,
                   "ms_per_step": sum(ms2) / args.steps, "steps_per_s": args.steps / (sum(ms2) / 1e3),
                   "bonds": b2, "mean_n": sv2["sum_n"] / n2, "sweeps_per_solve": sv2["sweeps"] / n2,
                   "zip_fallback_per_step": sv2["zip_fallback"] / args.steps}

    # end to end through the public API: host mode vector in (init), K steps each
    # followed by a read-back of the photon number; the system's operators and
    # Kraus MPO were built before (setup), as a caller stepping many states would
    # (the same step indices as the device-timed run: W + K steps from the start)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    st2 = b.sys.state(b.init)
    for _ in range(args.warmup + args.steps):
        st2.step(dt, 1)
        n_obs = st2.expectation(b.observables["n"])
    p_obs = st2.expectation(b.observables["parity"])
    e2e_s = time.perf_counter() - t0
    e2e_steps = args.warmup + args.steps
    st2.close()
    out = {"value": value, "total_ms": total_ms, "status": int(status), "bonds_before": bonds_before,
           "bonds_after": bonds_after, "obs_end": obs_end, "roofline": roofline,
           "classes": {k: v["ms"] / args.steps for k, v in prof.items()}, "solver": solver_line,
           "window2": window2, "peaks": {"fp64": fp64_peak, "fp32": fp32_peak},
           "e2e": {"value": e2e_steps / e2e_s, "unit": "steps/s", "h2d_bytes_per_step": 16 * 512 / e2e_steps,
                   "d2h_bytes_per_step": 16 * (e2e_steps + 1) / e2e_steps, "observables": [n_obs.real, p_obs.real]},
           "gpu_launches": int(round(launches_per_step * args.steps)), "clocks": clk.summary(), "dt": dt}
    st.close()
    ctx.close()
    return out


FORM_DTYPE = {0: "f64", 1: "f64+df64", 2: "f64+df64+tf32x3"}
FORM_NAME = {0: "fp64", 1: "mixed (double-float solves and GEMMs, FP64 storage)",
             2: "tensor-core (3xTF32 MPO application)"}


def run_gpu(args):
    """The headline line.  By default both the plain FP64 form and the mixed form
    (double-float truncation solves on the FP32 pipes) are measured on the same
    workload; the line reports the faster one whose photon number and parity at the
    end of the timed window are within 1e-6 of the FP64 form's (the metric's
    "steps/s at <= 1e-6 observable error vs the plain FP64 form"), with both forms
    listed under "forms".  --precision k measures form k alone."""
    import torch

    rank, world, local = dist_info()
    if world > 1:
        import torch.distributed as dist

        dist.init_process_group("nccl" if torch.cuda.is_available() else "gloo")
    dev = local
    torch.cuda.set_device(dev)
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=f"cuda:{dev}")
    forms = [0, 1] if args.precision < 0 else [args.precision]
    res = {p: _measure_form(args, dev, p, world, flush) for p in forms}
    head = forms[0]
    ref = res.get(0)
    errs = {}
    for p in forms:
        if ref is not None and p != 0:
            errs[p] = max(abs(a - c) for a, c in zip(res[p]["obs_end"], ref["obs_end"]))
            if errs[p] <= 1e-6 and res[p]["value"] > res[head]["value"]:
                head = p
    r = res[head]
    line = {
        "metric": METRIC, "value": r["value"], "unit": "steps/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": r["total_ms"] / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": FORM_DTYPE[head], "data": "synthetic",
        "config": {"workload": WORKLOAD, "N": 512, "R": 9, "alpha2": 32.0, "eps_z": 0.1, "dt": r["dt"],
                   "chi_max": 64, "chi_mu_max": 16, "tol": 1e-12, "form": FORM_NAME[head],
                   "mixed_gemm": args.mixed_gemm,
                   "l2": "flushed (256 MiB write) between timed steps",
                   "parallelism": "replicas" if world > 1 else "single", "bonds_before": r["bonds_before"],
                   "bonds_after": r["bonds_after"], "step_status": r["status"]},
        "roofline": r["roofline"],
        "kernel_classes_ms_per_step": r["classes"],
        "solver": r["solver"],
        "window2": r["window2"],
        "peaks_tflops": dict(r["peaks"], source="qlb_measure_peak, this run"),
        "e2e": r["e2e"],
        "gpu_launches": r["gpu_launches"],
        "clocks": r["clocks"],
        "forms": {FORM_DTYPE[p]: {"value": res[p]["value"], "ms_per_step": res[p]["total_ms"] / args.steps,
                                  "e2e": res[p]["e2e"]["value"], "obs_end": res[p]["obs_end"],
                                  "obs_err_vs_f64": errs.get(p, 0.0 if p == 0 else None),
                                  "window2_ms_per_step": (res[p]["window2"] or {}).get("ms_per_step"),
                                  "eig_ms_per_step": res[p]["classes"]["eig"]} for p in forms},
    }
    if args.serving_requests > 0:
        line["serving"] = serving_summary(dev, args.serving_requests, args.serving_step_scale, max(head, 0))
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline_sample()
    if rank == 0:
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()


def run_other_workload(args):
    """The larger configurations at their stated sizes, as separate bench lines
    (the default line is the cat_r9 workload):
      transmon  transmon (128 charge states, R = 7) x resonator (N = 1024, R = 10),
                17 sites, chi <= 128, chi_mu <= 16, ramped drive, dt = 2e-6; a window
                of K steps after W warm-up steps;
      cat_pair  four modes [b1, a1, a2, b2] = [16, 256, 256, 16] levels (24 sites),
                chi <= 256, chi_mu <= 32, dt = 1e-4, the 16 beam-splitter variants
                J = 0.01 linspace(0.5, 2, 16) stepping concurrently, each on its own
                stream: steps/s = 16 K / the window's duration."""
    import torch

    from paper_2605_27515_gb300 import inputs, qlb, systems

    dev = 0
    torch.cuda.set_device(dev)
    cfg = inputs.config(args.workload)
    ctx = qlb.Ctx(device=dev, precision=max(args.precision, 0), tol=cfg["tol"], chi_max=cfg["chi_max"],
                  chi_mu_max=cfg["chi_mu_max"], stream_ordered=1)
    tuning = os.path.join(ROOT, "paper_2605_27515_gb300", "tuning", "gram_splitk_gb300.txt")
    if os.path.exists(tuning):
        ctx.load_tuning(tuning)
    dt = cfg["dt"]
    n_total = args.warmup + args.steps + 1
    t_start = time.perf_counter()

    def progress(what):
        print(f"[bench {args.workload}] {time.perf_counter() - t_start:7.1f} s  {what}", file=sys.stderr, flush=True)

    if args.workload == "transmon":
        builds = [systems.build(ctx, cfg, nsteps=n_total)]
    else:
        builds = [systems.build(ctx, cfg, J=J) for J in inputs.cat_pair_J(cfg["n_variants"], cfg["J"])]
    progress(f"{len(builds)} systems built")
    states = [b.sys.state(b.init) for b in builds]
    for st in states:
        st.step(dt, args.warmup)
    ctx.synchronize()
    progress("warm-up steps done")
    snaps = [st.export() for st in states]
    ctx.profile_reset()
    torch.cuda.synchronize()
    # each state on its own stream (its own CUDA graph per state)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        for st in states:
            st.step(dt, 1)  # enqueued on each state's own stream
    ctx.synchronize()
    wall_streams = time.perf_counter() - t0
    per_stream_end = [st.bond_dims() for st in states]
    progress("per-stream window done")
    # the same steps again from the same snapshots as one group (one launch per
    # phase of the step over all states)
    for st, sn in zip(states, snaps):
        st.import_(sn)
    grp = qlb.Group(ctx, states) if len(states) > 1 else None
    if grp is not None:
        grp.step(dt, 1)  # records and captures the group's graph
        ctx.synchronize()
        progress(f"group captured ({grp.launches()} launches per step)")
        for st, sn in zip(states, snaps):
            st.import_(sn)
        ctx.synchronize()
    ctx.profile_reset()
    torch.cuda.synchronize()
    with ClockSampler(dev) as clk:
        t0 = time.perf_counter()
        if grp is not None:
            for _ in range(args.steps):
                grp.step(dt, 1)
        else:
            for _ in range(args.steps):
                states[0].step(dt, 1)
        ctx.synchronize()
        wall = time.perf_counter() - t0
    progress("timed window done")
    same_as_streams = [st.bond_dims() for st in states] == per_stream_end
    launches = grp.launches() if grp is not None else None
    if grp is not None:
        grp.close()
    sv = ctx.solver_stats()
    ns = max(1.0, sv["solves"])
    value = len(states) * args.steps / wall
    line = {"metric": METRIC, "value": value, "unit": "steps/s", "n_gpus": 1, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": 1e3 * wall / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": FORM_DTYPE[max(args.precision, 0)],
            "data": "synthetic",
            "config": {"workload": args.workload, "R": cfg["R"], "dt": dt, "chi_max": cfg["chi_max"],
                       "chi_mu_max": cfg["chi_mu_max"], "tol": cfg["tol"], "states": len(states),
                       "bonds_after": [st.bond_dims() for st in states[:2]],
                       "timing": "host wall clock around K steps of every state, device synchronised",
                       "engine": "group (one launch per phase over all states)" if grp is not None
                       else "single state, CUDA graph"},
            "per_stream": {"value": len(states) * args.steps / wall_streams,
                           "ms_per_step": 1e3 * wall_streams / args.steps,
                           "engine": "one CUDA graph per state, each on its own stream"},
            "group_launches_per_step": launches, "group_same_bonds_as_streams": same_as_streams,
            "solver": {"solves_per_step": sv["solves"] / (args.steps * len(states)), "mean_n": sv["sum_n"] / ns,
                       "max_n": sv["max_n"], "sweeps_per_solve": sv["sweeps"] / ns},
            "clocks": clk.summary()}
    print(json.dumps(line), flush=True)
    for st in states:
        st.close()
    ctx.close()


def run_z_gate_sweep(args):
    """Z gate on a cat qubit with its buffer (Sec. VI numerical experiment): for
    N_a = 2^R_a memory levels with |alpha|^2 = N_a / 3 (buffer N_b = 16, g2 = 1,
    kappa_b = 10, eps_Z = 0.04, theta = pi, kappa_a = 0), the even cat is driven for
    T_Z = theta / (4 alpha eps_Z) with the second-order Kraus scheme at tol 1e-8,
    chi_mu <= 16.  Reports the phase-flip error p_Z = (1 + <parity>) / 2 (the ideal
    gate ends in parity -1) beside the paper's p_Z = pi / (40 |alpha|^3), the largest
    bond seen (the plateau of Fig. Z_gate b) and the time per step."""
    import torch

    from paper_2605_27515_gb300 import inputs, qlb, systems

    torch.cuda.set_device(0)
    points = []
    for Ra in args.z_ra:
        cfg = inputs.config("z_gate")
        cfg["R"] = [Ra, 4]
        cfg["dt"] = args.z_dt
        ctx = qlb.Ctx(device=0, precision=max(args.precision, 0), tol=cfg["tol"], chi_max=cfg["chi_max"],
                      chi_mu_max=cfg["chi_mu_max"], stream_ordered=1)
        b = systems.build(ctx, cfg)
        b.sys.set_scheme(2)
        zp = systems.z_gate_params(cfg)
        st = b.sys.state(b.init)
        n = zp["steps"]
        peak_q = peak_mu = 0
        t0 = time.perf_counter()
        done = 0
        while done < n:
            k = min(100, n - done)
            st.step(cfg["dt"], k)
            done += k
            bd = st.bond_dims()
            peak_mu, peak_q = max(peak_mu, bd[0]), max(peak_q, max(bd[1:]))
        ctx.synchronize()
        wall = time.perf_counter() - t0
        par = st.expectation(b.observables["parity_a"]).real
        points.append({"R_a": Ra, "alpha2": zp["alpha2"], "steps": n, "dt": cfg["dt"], "parity_end": par,
                       "p_Z": (1.0 + par) / 2.0, "p_Z_paper": float(np.pi / (40.0 * zp["alpha"] ** 3)),
                       "max_chi": peak_q, "max_chi_mu": peak_mu, "ms_per_step": 1e3 * wall / n})
        st.close()
        ctx.close()
    print(json.dumps({"workload": "z_gate_sweep", "scheme": "second-order Kraus", "tol": 1e-8, "chi_mu_max": 16,
                      "chi_max": 64, "points": points}), flush=True)


def run_solver_sweep(args):
    """Device time of one truncation solve by each kernel (qlb_eig_check) on seeded
    Gram matrices of the zip-up's kind: G = M M^dag with M of rank n / 2 and
    singular values graded over 1e-6 (weights over 1e-12), cutoff 1e-18 (the zip-up's
    tol x 1e-6), in FP64 and double-float.  The step's dispatch thresholds come from
    this table."""
    from paper_2605_27515_gb300 import qlb

    names = {qlb.SOLVER_JACOBI: "jacobi_1cta", qlb.SOLVER_CLUSTER8: "jacobi_cluster8",
             qlb.SOLVER_CLUSTER16: "jacobi_cluster16", qlb.SOLVER_QL: "householder_ql",
             qlb.SOLVER_RANGE: "range_basis"}
    rows = []
    for prec in (qlb.PREC_F64, qlb.PREC_MIXED):
        for n in args.solver_n:
            rng = np.random.default_rng(1000 + n)
            r = max(1, n // 2)
            M = (rng.normal(size=(n, r)) + 1j * rng.normal(size=(n, r))) * np.logspace(0, -6, r)[None, :]
            G = M @ M.conj().T
            G = 0.5 * (G + G.conj().T)
            row = {"precision": "fp64" if prec == qlb.PREC_F64 else "df64", "n": n}
            for sv, name in names.items():
                if (sv == qlb.SOLVER_CLUSTER8 and n > 128) or (sv == qlb.SOLVER_CLUSTER16 and n > 256) or \
                        (sv == qlb.SOLVER_QL and (prec != qlb.PREC_F64 or n > 64)):
                    continue
                best = None
                for _ in range(3):
                    _, _, k, ms = qlb.qlb_eig_check(0, prec, sv, G, tol=1e-18, cap=n)
                    best = ms if best is None else min(best, ms)
                row[name] = {"ms": best, "k": k}
            rows.append(row)
    print(json.dumps({"workload": "solvers", "matrix": "G = M M^dag, rank n/2, weights graded over 1e-12",
                      "tol": 1e-18, "timing": "best of 3 single launches (CUDA events)", "rows": rows}), flush=True)


def serving_summary(dev, n_requests, step_scale, precision, budget_gb=4.0):
    """The serving workload (Poisson arrivals at 200/s of single-cat requests,
    seed 20260527) through the library's continuous-batching server (qlb_server_*):
    requests are submitted at their arrival times, step counts scaled by step_scale
    so the run stays short.  Returns p50/p99 latency and steps/s."""
    from paper_2605_27515_gb300 import inputs, qlb, serving

    ctx = qlb.Ctx(device=dev, precision=precision, chi_max=64, chi_mu_max=8, stream_ordered=1)
    reqs = inputs.serving_requests(n=n_requests)
    srv = qlb.Server(ctx, hbm_budget=int(budget_gb * (1 << 30)), max_live=64, chunk=100)
    t0 = time.perf_counter()
    jobs = serving.drive(srv, reqs, step_scale=step_scale)
    wall = time.perf_counter() - t0
    stats = srv.stats()
    srv.close()
    out = serving.summarize(jobs, wall)
    out.update({"workload": "serving", "step_scale": step_scale, "peak_live": stats["peak_live"],
                "peak_device_bytes": stats["peak_bytes"], "hbm_budget_bytes": int(budget_gb * (1 << 30)),
                "arrivals": "Poisson 200/s, seed 20260527", "engine": "qlb_server (C-ABI)"})
    ctx.close()
    return out


def run_serving_window(args):
    """The serving configuration as stated: all 256 requests of the mix (Poisson
    arrivals at 200/s, seed 20260527, their own step counts of 2000-20000, dt =
    1e-3, chi caps 32/48/64, chi_mu <= 8) through the library's server for a fixed
    wall window; reports the requests completed in the window with their p50/p99
    latency and the steps the server enqueued per second (chunks still in flight
    at the end of the window included)."""
    import torch

    from paper_2605_27515_gb300 import inputs, qlb, serving

    torch.cuda.set_device(0)
    budget_gb = 16.0
    ctx = qlb.Ctx(device=0, precision=max(args.precision, 0), chi_max=64, chi_mu_max=8, stream_ordered=1)
    reqs = inputs.serving_requests(n=256)
    srv = qlb.Server(ctx, hbm_budget=int(budget_gb * (1 << 30)), max_live=64, chunk=100)
    try:
        with ClockSampler(0) as clk:
            jobs, used = serving.drive_window(srv, reqs, args.serving_window)
            stats = srv.stats()
    finally:
        srv.close()
        ctx.close()
    out = serving.summarize_window(jobs, used, stats["steps"])
    line = {"metric": METRIC, "value": out["steps_per_s"], "unit": "steps/s", "n_gpus": 1, "steps": stats["steps"],
            "warmup": 0, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": FORM_DTYPE[max(args.precision, 0)], "data": "synthetic",
            "config": {"workload": "serving_window", "requests": 256, "arrivals": "Poisson 200/s, seed 20260527",
                       "steps_per_request": "U{2000..20000}", "dt": 1e-3, "chi_max": "U{32,48,64}", "chi_mu_max": 8,
                       "max_live": 64, "chunk": 100, "hbm_budget_bytes": int(budget_gb * (1 << 30)),
                       "engine": "qlb_server (C-ABI), same-shape buckets stepped as groups"},
            "serving": dict(out, peak_live=stats["peak_live"], peak_device_bytes=stats["peak_bytes"]),
            "clocks": clk.summary()}
    print(json.dumps(line), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    ap.add_argument("--precision", type=int, default=-1,
                    help="0 FP64, 1 mixed, 2 tensor-core; default: FP64 and mixed, headline the faster within 1e-6")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--serving-requests", type=int, default=32)
    ap.add_argument("--window2", type=int, default=200)
    ap.add_argument("--workload", default=WORKLOAD,
                    choices=[WORKLOAD, "transmon", "cat_pair", "z_gate_sweep", "solvers", "serving_window"])
    ap.add_argument("--solver-n", type=int, nargs="+", default=[8, 16, 24, 32, 48, 64, 96, 128, 192, 256])
    ap.add_argument("--z-ra", type=int, nargs="+", default=[4, 5, 6])
    ap.add_argument("--z-dt", type=float, default=4e-3)
    ap.add_argument("--serving-step-scale", type=float, default=0.005)
    ap.add_argument("--serving-window", type=float, default=60.0,
                    help="--workload serving_window: seconds of wall time the full request mix runs")
    ap.add_argument("--mixed-gemm", type=int, default=1, choices=[0, 1, 2],
                    help="GEMMs of the mixed forms in double-float: 0 none, 1 all but the Grams, 2 all")
    args = ap.parse_args()
    args.warmup = max(3, args.warmup)
    if args.impl == "reference":
        run_reference(args)
    elif args.workload == "z_gate_sweep":
        run_z_gate_sweep(args)
    elif args.workload == "solvers":
        run_solver_sweep(args)
    elif args.workload == "serving_window":
        run_serving_window(args)
    elif args.workload != WORKLOAD:
        run_other_workload(args)
    else:
        run_gpu(args)


if __name__ == "__main__":
    main()
