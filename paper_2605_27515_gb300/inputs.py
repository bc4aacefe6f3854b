"""Seeded synthetic workloads shared by the tests, the bench and the oracle leg.

This module holds parameters and random numbers only, none of the method's
arithmetic: it names the physical systems (mode sizes, rates, drive, time step,
truncation settings) and draws the seeded random inputs (request mixes, random
initial vectors).  Each side builds its own operators, derived operating points
and initial states from these parameters.

Systems (all from the paper's applications, Sec. VI and Sec. VII):
  cat_r5        single cat mode, N = 32: L1 = sqrt(k2)(a^2 - alpha^2),
                L2 = sqrt(k1) a, H = 0, vacuum start, dt = 1e-3, 5000 steps,
                cutoff 1e-12, purification cap 8.
  cat_r9        single cat mode, N = 512, alpha^2 = 32, Zeno drive
                H = eps_Z (a + a^dag), dt = 5e-4, 20000 steps, chi <= 64,
                chi_mu <= 16.  Oracle check size: N = 128, alpha^2 = 16.
  transmon      transmon in the charge basis (128 charge states) x resonator
                (N = 1024), coupling g n_t (a + a^dag), ramped drive
                eps(t) cos(w_r t)(a + a^dag), L = sqrt(kappa) a.
  transmon_eig  the same transmon x resonator with the transmon in its
                eigenbasis (|n| <= 500 charges diagonalised, lowest 2^5 states).
  z_gate        memory cat (N_a = 2^R_a) with a lossy buffer (N_b = 16),
                g2 = 1, kappa_b = 10 g2, theta = pi, kappa_a = 0 (Sec. VI numerical
                experiment); the operating point (alpha, eps_d, eps_Z, T_Z) and the
                even-cat start are derived by each side from these.
  cat_pair      two storage cats (N = 256) each with a buffer (N = 16),
                three-wave mixing g2 (a^2 b^dag + h.c.), buffer drive, beam
                splitter J (a1^dag a2 + h.c.), 16 variants of J.
  serving       256 single-cat requests with Poisson arrivals (seeded).
"""
from __future__ import annotations

import copy

import numpy as np

SERVING_SEED = 20260527

_CONFIGS = {
    "cat_r5": dict(
        kind="cat", R=[5], alpha2=4.0, k2=1.0, k1=1e-3, eps_z=0.0, dt=1e-3, steps=5000,
        tol=1e-12, chi_max=64, chi_mu_max=8, record_every=100,
    ),
    "cat_r9": dict(
        kind="cat", R=[9], alpha2=32.0, k2=1.0, k1=1e-3, eps_z=0.1, dt=5e-4, steps=20000,
        tol=1e-12, chi_max=64, chi_mu_max=16, record_every=100,
        check=dict(R=[7], alpha2=16.0),
    ),
    # Units: angular frequency in rad/ns (GHz * 2 pi), time in ns.
    "transmon": dict(
        kind="transmon", R=[7, 10], ec=2 * np.pi * 0.28, ej_over_ec=50.0, ng=0.0,
        wr=2 * np.pi * 7.5, g_over_ec=0.5, kappa=2 * np.pi * 0.02, eps_over_kappa=40.0,
        ramp_kappa_t=200.0, dt=2e-6, steps=10000, tol=1e-12, chi_max=128, chi_mu_max=16,
        record_every=100, check=dict(R=[5, 6]),
    ),
    "transmon_eig": dict(
        kind="transmon_eig", R=[5, 10], ec=2 * np.pi * 0.28, ej_over_ec=50.0, n_cut=500,
        wr=2 * np.pi * 7.5, g_over_ec=0.5, kappa=2 * np.pi * 0.02, eps_over_kappa=40.0,
        ramp_kappa_t=200.0, dt=2e-6, steps=10000, tol=1e-12, chi_max=128, chi_mu_max=16,
        record_every=100, check=dict(R=[5, 6]),
    ),
    "z_gate": dict(
        kind="z_gate", R=[9, 4], g2=1.0, kb=10.0, theta=float(np.pi), ka=0.0,
        dt=1e-3, tol=1e-8, chi_max=64, chi_mu_max=16, record_every=100,
        check=dict(R=[3, 2]),
    ),
    "cat_pair": dict(
        kind="cat_pair", R=[8, 4, 8, 4], alpha2=8.0, g2=0.2, kb=5.0, k1=1e-3, J=0.01,
        dt=1e-4, steps=10000, tol=1e-12, chi_max=256, chi_mu_max=32, n_variants=16,
        record_every=100, check=dict(R=[3, 2, 3, 2]),
    ),
}


def config(name: str) -> dict:
    """A deep copy of the named parameter set."""
    return copy.deepcopy(_CONFIGS[name])


def config_names():
    return list(_CONFIGS)


def cat_pair_J(n_variants: int = 16, J: float = 0.01):
    """J values of the 16 parameter variants: J * linspace(0.5, 2, n)."""
    return list(J * np.linspace(0.5, 2.0, n_variants))


def transmon_drive_table(cfg: dict, nsteps: int, t0: float = 0.0):
    """f(t_n) for the ramped resonator drive eps(t) cos(w_r t), left endpoints
    t_n = t0 + n dt; eps(t) = eps_max * min(1, t kappa / ramp)."""
    t = t0 + cfg["dt"] * np.arange(nsteps)
    eps_max = cfg["eps_over_kappa"] * cfg["kappa"]
    ramp = np.minimum(1.0, t * cfg["kappa"] / cfg["ramp_kappa_t"])
    return eps_max * ramp * np.cos(cfg["wr"] * t)


def serving_requests(n: int = 256, rate: float = 200.0, seed: int = SERVING_SEED):
    """Seeded request mix of the serving workload: Poisson arrivals at `rate`
    per second, alpha^2 ~ U[4, 36], R ~ U{6..9}, k1/k2 ~ logU[1e-4, 1e-2],
    steps ~ U{2000..20000}, dt = 1e-3, chi cap in {32, 48, 64}."""
    rng = np.random.Generator(np.random.PCG64(seed))
    gaps = rng.exponential(1.0 / rate, size=n)
    arrivals = np.cumsum(gaps) - gaps[0]
    out = []
    for i in range(n):
        out.append(dict(
            id=i, arrival_s=float(arrivals[i]),
            alpha2=float(rng.uniform(4.0, 36.0)),
            R=int(rng.integers(6, 10)),
            k1_over_k2=float(10 ** rng.uniform(-4.0, -2.0)),
            steps=int(rng.integers(2000, 20001)),
            dt=1e-3,
            chi_max=int(rng.choice([32, 48, 64])),
            chi_mu_max=8, tol=1e-12,
        ))
    return out


def random_vector(n: int, seed: int) -> np.ndarray:
    """Seeded complex Gaussian vector (not normalised)."""
    rng = np.random.default_rng(seed)
    return rng.normal(size=n) + 1j * rng.normal(size=n)
