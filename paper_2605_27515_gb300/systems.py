"""The paper's model systems as C-ABI term lists (argument marshalling only).

Each builder turns a parameter set from ``inputs`` into qlb operators made of the
library's built-in factors (a, a^dag, n, parity, charge, cos phi) and registers
the Hamiltonian and jump operators on a ``qlb.System``.  The dense matrices are
generated on the device by the library.

  cat        H = eps_z (a + a^dag);  L1 = sqrt(k2) (a^2 - alpha^2);  L2 = sqrt(k1) a
             (cat qubit with two-photon dissipation, Sec. VI, Eq. Hz)
  transmon   H0 = 4 Ec n_t^2 - Ej cos(phi_t) + w_r a^dag a + g n_t (a + a^dag),
             H1 = (a + a^dag) with f(t) = eps(t) cos(w_r t);  L = sqrt(kappa) a
             (Sec. VII, Eq. transmon_cavity with the coupling written as n_t (a + a^dag))
  cat_pair   modes [b1, a1, a2, b2]: H = sum_i g2 (a_i^2 b_i^dag + a_i^dag^2 b_i)
             + eps_b (b_i + b_i^dag) + J (a1^dag a2 + a2^dag a1);
             L = sqrt(kb) b_i, sqrt(k1) a_i  (Sec. VI, Eq. cb, two cats coupled)
"""
from __future__ import annotations

import numpy as np

from . import inputs
from . import qlb as Q


def transmon_ground_charge(Nt: int, offset: int, ec: float, ej: float, ng: float = 0.0) -> np.ndarray:
    """Initial transmon vector of the transmon system (input preparation for the
    C-ABI): the lowest eigenvector of 4 Ec (n - ng)^2 - Ej cos(phi) on the charge
    states n = j - offset (Sec. VII, Eq. transmon), cut open at both ends."""
    n = np.arange(Nt) - offset
    H = np.diag(4 * ec * (n - ng) ** 2).astype(np.complex128)
    for j in range(Nt - 1):
        H[j, j + 1] = H[j + 1, j] = -ej / 2
    w, v = np.linalg.eigh(H)
    return v[:, 0]


def z_gate_params(cfg: dict) -> dict:
    """Derived Z-gate parameters (Sec. VI): alpha^2 = N_a / 3, eps_d = -g2 alpha^2,
    eps_Z = 4 g2^2 / (10 kappa_b), T_Z = theta / (4 alpha eps_Z), steps = T_Z / dt."""
    Na = 2 ** cfg["R"][0]
    alpha2 = cfg.get("alpha2", Na / 3.0)
    alpha = float(np.sqrt(alpha2))
    eps_z = 0.1 * 4.0 * cfg["g2"] ** 2 / cfg["kb"]
    tz = cfg["theta"] / (4.0 * alpha * eps_z)
    return dict(alpha2=alpha2, alpha=alpha, eps_d=-cfg["g2"] * alpha2, eps_z=eps_z, t_z=tz,
                steps=int(round(tz / cfg["dt"])))


def cat_vector(N: int, alpha: float, parity: int = +1) -> np.ndarray:
    """Normalised cat |alpha> + parity |-alpha> in an N-level Fock space, from the
    coherent amplitudes alpha^n / sqrt(n!) (each coherent part truncated)."""
    c = np.zeros(N, dtype=np.complex128)
    c[0] = 1.0
    for n in range(1, N):
        c[n] = c[n - 1] * alpha / np.sqrt(n)
    sign = (-1.0) ** np.arange(N)
    v = c + parity * sign * c
    return v / np.linalg.norm(v)


def vacuum(N):
    v = np.zeros(N, dtype=np.complex128)
    v[0] = 1.0
    return v


class Built:
    def __init__(self, sys, ops, init, observables, cfg, f_table=None):
        self.sys = sys
        self.ops = ops  # name -> Op (keeps them alive)
        self.init = init  # list of mode vectors
        self.observables = observables  # name -> Op
        self.cfg = cfg
        self.f_table = f_table


def build_cat(ctx, cfg):
    R = cfg["R"][0]
    s = Q.System(ctx, [R])
    a2, k2, k1, ez = cfg["alpha2"], cfg["k2"], cfg["k1"], cfg.get("eps_z", 0.0)
    ops = {}
    if ez:
        ops["H"] = s.op([(ez, [(0, Q.F_A)]), (ez, [(0, Q.F_ADAG)])])
        s.set_hamiltonian(ops["H"])
    ops["L1"] = s.op([(np.sqrt(k2), [(0, Q.F_A, 2)]), (-np.sqrt(k2) * a2, [])])
    s.add_jump(ops["L1"])
    if k1:
        ops["L2"] = s.op([(np.sqrt(k1), [(0, Q.F_A)])])
        s.add_jump(ops["L2"])
    obs = {"n": s.op([(1.0, [(0, Q.F_NUM)])]), "parity": s.op([(1.0, [(0, Q.F_PARITY)])])}
    return Built(s, ops, [vacuum(2 ** R)], obs, cfg)


def build_transmon(ctx, cfg, nsteps=None):
    Rt, Rr = cfg["R"]
    Nt = 2 ** Rt
    off = Nt // 2
    s = Q.System(ctx, [Rt, Rr])
    ec = cfg["ec"]
    ej = cfg["ej_over_ec"] * ec
    g = cfg["g_over_ec"] * ec
    ops = {}
    ops["H0"] = s.op([
        (4 * ec, [(0, Q.F_CHARGE, 2, float(off) + cfg.get("ng", 0.0))]),
        (-ej, [(0, Q.F_COSPHI)]),
        (cfg["wr"], [(1, Q.F_NUM)]),
        (g, [(0, Q.F_CHARGE, 1, float(off)), (1, Q.F_A)]),
        (g, [(0, Q.F_CHARGE, 1, float(off)), (1, Q.F_ADAG)]),
    ])
    ops["H1"] = s.op([(1.0, [(1, Q.F_A)]), (1.0, [(1, Q.F_ADAG)])])
    n = nsteps if nsteps is not None else cfg["steps"]
    f = inputs.transmon_drive_table(cfg, n)
    s.set_hamiltonian(ops["H0"], ops["H1"], f)
    ops["L"] = s.op([(np.sqrt(cfg["kappa"]), [(1, Q.F_A)])])
    s.add_jump(ops["L"])
    obs = {"n_c": s.op([(1.0, [(1, Q.F_NUM)])]), "n_t2": s.op([(1.0, [(0, Q.F_CHARGE, 2, float(off))])])}
    init = [transmon_ground_charge(Nt, off, ec, ej, cfg.get("ng", 0.0)), vacuum(2 ** Rr)]
    return Built(s, ops, init, obs, cfg, f)


def transmon_levels(ec, ej, K, n_cut=500, tie=1e-9):
    """Transmon eigenbasis of Sec. VII (numerical experiment) for the operator
    builder: the K lowest eigenstates of 4 Ec n^2 - Ej cos(phi) on the charges
    |n| <= n_cut (ng = 0, cos(phi) cut open), and the charge operator in that basis.

    Found per charge-parity sector as two tridiagonal chains:
      even |0>, (|m> + |-m>)/sqrt 2: diagonal 4 Ec m^2, coupling -Ej/sqrt 2 between
        m = 0 and 1, -Ej/2 further on;
      odd (|m> - |-m>)/sqrt 2, m >= 1: diagonal 4 Ec m^2, couplings -Ej/2.
    n is odd under n -> -n, so [n_t] joins an even state e and an odd state o only:
    <e| n |o> = sum_{m >= 1} e_m o_m m.  Conventions: within a degenerate pair
    (energies equal to `tie` relative) the even state comes first, and each state's
    largest charge amplitude over n >= 0 is positive.
    Returns (energies ascending, n_t as a real K x K array)."""
    from scipy.linalg import eigh_tridiagonal

    m = np.arange(n_cut + 1, dtype=np.float64)
    d_even = 4.0 * ec * m * m
    off_even = np.full(n_cut, -0.5 * ej)
    off_even[0] = -ej / np.sqrt(2.0)
    we, ve = eigh_tridiagonal(d_even, off_even)
    wo, vo = eigh_tridiagonal(d_even[1:], np.full(n_cut - 1, -0.5 * ej))
    # charge amplitudes over n = 0..n_cut of every sector state
    amp_e = ve.copy()
    amp_e[1:, :] *= np.sqrt(0.5)
    amp_o = np.zeros((n_cut + 1, wo.size))
    amp_o[1:, :] = vo * np.sqrt(0.5)
    levels = [(we[j], 0, j) for j in range(we.size)] + [(wo[j], 1, j) for j in range(wo.size)]
    levels.sort(key=lambda t: t[0])
    for i in range(len(levels) - 1):
        a, b = levels[i], levels[i + 1]
        if a[1] == 1 and b[1] == 0 and abs(a[0] - b[0]) <= tie * max(abs(a[0]), abs(b[0])):
            levels[i], levels[i + 1] = b, a
    levels = levels[:K]
    energies = np.array([t[0] for t in levels])
    vecs = []
    for _, parity, j in levels:
        amp = amp_e[:, j] if parity == 0 else amp_o[:, j]
        k = int(np.argmax(np.abs(amp)))
        sgn = -1.0 if amp[k] < 0 else 1.0
        vecs.append((parity, sgn * (ve[:, j] if parity == 0 else vo[:, j])))
    nt = np.zeros((K, K))
    for a, (pa, va) in enumerate(vecs):
        for b, (pb, vb) in enumerate(vecs):
            if pa == 0 and pb == 1:
                nt[a, b] = nt[b, a] = float(np.dot(va[1:] * m[1:], vb))
    return energies, nt


def build_transmon_eig(ctx, cfg, nsteps=None):
    """Transmon x resonator with the transmon in its eigenbasis (Sec. VII): the
    transmon mode carries the 2^R_t lowest transmon states; H0 = diag(eps - eps_0)
    + w_r a^dag a + g n_t (a + a^dag), drive f(t_n)(a + a^dag), L = sqrt(kappa) a.
    Observables N_t = Tr(b^dag b rho) with b^dag b = diag(alpha) and N_c."""
    Rt, Rr = cfg["R"]
    K = 2 ** Rt
    ec = cfg["ec"]
    ej = cfg["ej_over_ec"] * ec
    g = cfg["g_over_ec"] * ec
    E, nt = transmon_levels(ec, ej, K, cfg.get("n_cut", 500))
    s = Q.System(ctx, [Rt, Rr])
    Ht = np.diag(E - E[0]).astype(np.complex128)
    ntc = nt.astype(np.complex128)
    ops = {}
    ops["H0"] = s.op([
        (1.0, [(0, Q.F_DENSE, Ht)]),
        (cfg["wr"], [(1, Q.F_NUM)]),
        (g, [(0, Q.F_DENSE, ntc), (1, Q.F_A)]),
        (g, [(0, Q.F_DENSE, ntc), (1, Q.F_ADAG)]),
    ])
    ops["H1"] = s.op([(1.0, [(1, Q.F_A)]), (1.0, [(1, Q.F_ADAG)])])
    n = nsteps if nsteps is not None else cfg["steps"]
    f = inputs.transmon_drive_table(cfg, n)
    s.set_hamiltonian(ops["H0"], ops["H1"], f)
    ops["L"] = s.op([(np.sqrt(cfg["kappa"]), [(1, Q.F_A)])])
    s.add_jump(ops["L"])
    obs = {"n_c": s.op([(1.0, [(1, Q.F_NUM)])]), "n_t": s.op([(1.0, [(0, Q.F_NUM)])])}
    init = [vacuum(K), vacuum(2 ** Rr)]  # transmon eigenstate 0 x cavity vacuum
    return Built(s, ops, init, obs, cfg, f)


def build_z_gate(ctx, cfg):
    """Z gate on a cat qubit with its buffer (Sec. VI, Eq. cb and Eq. Hz), modes
    [a (memory), b (buffer)]: H = g2 (a^dag^2 b + a^2 b^dag) + eps_d (b + b^dag)
    + eps_Z (a + a^dag), L_b = sqrt(kappa_b) b (and sqrt(kappa_a) a when kappa_a > 0);
    start in the even cat x buffer vacuum.  Observables: memory parity, photon
    numbers."""
    Ra, Rb = cfg["R"]
    zp = z_gate_params(cfg)
    g2 = cfg["g2"]
    s = Q.System(ctx, [Ra, Rb])
    a, b = 0, 1
    ops = {"H": s.op([
        (g2, [(a, Q.F_ADAG, 2), (b, Q.F_A)]), (g2, [(a, Q.F_A, 2), (b, Q.F_ADAG)]),
        (zp["eps_d"], [(b, Q.F_A)]), (zp["eps_d"], [(b, Q.F_ADAG)]),
        (zp["eps_z"], [(a, Q.F_A)]), (zp["eps_z"], [(a, Q.F_ADAG)]),
    ])}
    s.set_hamiltonian(ops["H"])
    ops["Lb"] = s.op([(np.sqrt(cfg["kb"]), [(b, Q.F_A)])])
    s.add_jump(ops["Lb"])
    if cfg.get("ka", 0.0) > 0.0:
        ops["La"] = s.op([(np.sqrt(cfg["ka"]), [(a, Q.F_A)])])
        s.add_jump(ops["La"])
    obs = {"parity_a": s.op([(1.0, [(a, Q.F_PARITY)])]), "n_a": s.op([(1.0, [(a, Q.F_NUM)])]),
           "n_b": s.op([(1.0, [(b, Q.F_NUM)])])}
    init = [cat_vector(2 ** Ra, zp["alpha"], +1), vacuum(2 ** Rb)]
    return Built(s, ops, init, obs, cfg)


def build_cat_pair(ctx, cfg, J=None):
    Rb1, Ra1, Ra2, Rb2 = cfg["R"][1], cfg["R"][0], cfg["R"][2], cfg["R"][3]
    s = Q.System(ctx, [Rb1, Ra1, Ra2, Rb2])
    b1, a1, a2, b2 = 0, 1, 2, 3
    g2, kb, k1 = cfg["g2"], cfg["kb"], cfg["k1"]
    eb = -g2 * cfg["alpha2"]
    J = cfg["J"] if J is None else J
    terms = []
    for a, b in ((a1, b1), (a2, b2)):
        terms += [(g2, [(a, Q.F_A, 2), (b, Q.F_ADAG)]), (g2, [(a, Q.F_ADAG, 2), (b, Q.F_A)]),
                  (eb, [(b, Q.F_A)]), (eb, [(b, Q.F_ADAG)])]
    terms += [(J, [(a1, Q.F_ADAG), (a2, Q.F_A)]), (J, [(a2, Q.F_ADAG), (a1, Q.F_A)])]
    ops = {"H": s.op(terms)}
    s.set_hamiltonian(ops["H"])
    for name, m, k in (("Lb1", b1, kb), ("Lb2", b2, kb), ("La1", a1, k1), ("La2", a2, k1)):
        ops[name] = s.op([(np.sqrt(k), [(m, Q.F_A)])])
        s.add_jump(ops[name])
    obs = {"n_a1": s.op([(1.0, [(a1, Q.F_NUM)])]), "n_a2": s.op([(1.0, [(a2, Q.F_NUM)])]),
           "parity_a1": s.op([(1.0, [(a1, Q.F_PARITY)])])}
    init = [vacuum(2 ** r) for r in s.R]
    return Built(s, ops, init, obs, cfg)


def build(ctx, cfg, **kw):
    kind = cfg["kind"]
    if kind == "cat":
        return build_cat(ctx, cfg)
    if kind == "transmon":
        return build_transmon(ctx, cfg, **kw)
    if kind == "cat_pair":
        return build_cat_pair(ctx, cfg, **kw)
    if kind == "transmon_eig":
        return build_transmon_eig(ctx, cfg, **kw)
    if kind == "z_gate":
        return build_z_gate(ctx, cfg)
    raise ValueError(kind)
