"""Dense oracle versions of the paper's model systems (test infrastructure only).

Each builder takes a raw parameter set (the dicts of the shared input module:
mode sizes, rates, time step) and derives everything else itself from the
paper's formulas: the Z-gate operating point (Sec. VI), the initial cat and
transmon states, the resonator drive schedule (Sec. VII).  Nothing here imports
the product package.  Mode orders: cat_pair is [b1, a1, a2, b2], transmon and
transmon_eig are [transmon, resonator], z_gate is [memory a, buffer b].
"""
from __future__ import annotations

import numpy as np

from . import dense as D


class DenseSystem:
    def __init__(self, dims, H0, Ls, H1=None, f_table=None, observables=None, init=None):
        self.dims = dims
        self.H0, self.Ls, self.H1, self.f_table = H0, Ls, H1, f_table
        self.observables = observables or {}
        self.init = init

    def rho0(self):
        return D.pure(D.product_vector(self.init))

    def evolve(self, h, nsteps, record_every, names=None, order=1):
        names = names or list(self.observables)
        obs = [lambda r, O=self.observables[n]: D.expectation(r, O).real for n in names]
        rho, recs = D.evolve(self.rho0(), self.H0, self.Ls, h, nsteps, H1=self.H1, f_table=self.f_table,
                             record_every=record_every, observables=obs, order=order)
        return rho, recs


def cat(cfg):
    N = 2 ** cfg["R"][0]
    dims = (N,)
    a, ad = D.op_a(N), D.op_adag(N)
    ez = cfg.get("eps_z", 0.0)
    H = D.Operator(dims, [(ez, {0: a}), (ez, {0: ad})] if ez else [])
    Ls = [D.Operator(dims, [(np.sqrt(cfg["k2"]), {0: a @ a}), (-np.sqrt(cfg["k2"]) * cfg["alpha2"], {})])]
    if cfg["k1"]:
        Ls.append(D.Operator.local(dims, 0, a, np.sqrt(cfg["k1"])))
    obs = {"n": D.Operator.local(dims, 0, D.op_num(N)), "parity": D.Operator.local(dims, 0, D.op_parity(N))}
    return DenseSystem(dims, H, Ls, observables=obs, init=[D.fock(N, 0)])


def transmon_charge_hamiltonian(Nt, ec, ej, ng=0.0):
    """H_t = 4 E_C (n_t - n_g)^2 - E_J cos(phi_t) in the charge basis (Sec. VII, Eq.
    transmon), charges j - Nt/2 for j = 0..Nt-1, cos(phi) cut open at both ends."""
    nt = D.op_charge(Nt, Nt // 2) - ng * np.eye(Nt)
    return 4.0 * ec * nt @ nt - ej * D.op_cos_phi(Nt)


def transmon_ground(Nt, ec, ej, ng=0.0):
    """Lowest eigenvector of the charge-basis transmon (the start of Sec. VII's run)."""
    w, v = np.linalg.eigh(transmon_charge_hamiltonian(Nt, ec, ej, ng))
    return v[:, 0].astype(np.complex128)


def drive_table(cfg, nsteps, t0=0.0):
    """Resonator drive f(t_n) = eps(t_n) cos(w_r t_n) at the left ends t_n = t0 + n h,
    eps ramped linearly to eps_max = (eps/kappa) kappa over ramp/kappa (reading of
    Sec. VII, whose drive frequency and ramp the text leaves open)."""
    t = t0 + cfg["dt"] * np.arange(nsteps)
    eps_max = cfg["eps_over_kappa"] * cfg["kappa"]
    return eps_max * np.minimum(1.0, t * cfg["kappa"] / cfg["ramp_kappa_t"]) * np.cos(cfg["wr"] * t)


def transmon(cfg, nsteps, f_table=None, init=None):
    """Transmon (charge basis) x resonator (Sec. VII): H0 = 4 E_C (n_t - n_g)^2
    - E_J cos(phi_t) + w_r a^dag a + g n_t (a + a^dag), H1 = a + a^dag with f(t_n),
    L = sqrt(kappa) a.  The coupling g n_t (a + a^dag) is the paper's
    -i g n_t (a - a^dag) after a -> -i a (a diagonal phase change of the resonator
    basis, which leaves every observable used here unchanged).  Start: the
    transmon ground state x resonator vacuum."""
    Rt, Rr = cfg["R"]
    Nt, Nr = 2 ** Rt, 2 ** Rr
    off = Nt // 2
    dims = (Nt, Nr)
    ec = cfg["ec"]
    ej = cfg["ej_over_ec"] * ec
    g = cfg["g_over_ec"] * ec
    ntc = D.op_charge(Nt, off)
    a, ad = D.op_a(Nr), D.op_adag(Nr)
    Ht = transmon_charge_hamiltonian(Nt, ec, ej, cfg.get("ng", 0.0))
    H0 = D.Operator(dims, [(1.0, {0: Ht}), (cfg["wr"], {1: D.op_num(Nr)}), (g, {0: ntc, 1: a}),
                           (g, {0: ntc, 1: ad})])
    H1 = D.Operator(dims, [(1.0, {1: a}), (1.0, {1: ad})])
    Ls = [D.Operator.local(dims, 1, a, np.sqrt(cfg["kappa"]))]
    obs = {"n_c": D.Operator.local(dims, 1, D.op_num(Nr)), "n_t2": D.Operator.local(dims, 0, ntc @ ntc)}
    if f_table is None:
        f_table = drive_table(cfg, nsteps)
    if init is None:
        init = [transmon_ground(Nt, ec, ej, cfg.get("ng", 0.0)), D.fock(Nr, 0)]
    return DenseSystem(dims, H0, Ls, H1=H1, f_table=f_table, observables=obs, init=init)


def cat_pair(cfg, J=None):
    R = cfg["R"]
    dims = (2 ** R[1], 2 ** R[0], 2 ** R[2], 2 ** R[3])
    b1, a1, a2, b2 = 0, 1, 2, 3
    g2, kb, k1 = cfg["g2"], cfg["kb"], cfg["k1"]
    eb = -g2 * cfg["alpha2"]
    J = cfg["J"] if J is None else J
    A = {m: D.op_a(dims[m]) for m in range(4)}
    Ad = {m: D.op_adag(dims[m]) for m in range(4)}
    terms = []
    for a, b in ((a1, b1), (a2, b2)):
        terms += [(g2, {a: A[a] @ A[a], b: Ad[b]}), (g2, {a: Ad[a] @ Ad[a], b: A[b]}), (eb, {b: A[b]}),
                  (eb, {b: Ad[b]})]
    terms += [(J, {a1: Ad[a1], a2: A[a2]}), (J, {a2: Ad[a2], a1: A[a1]})]
    H = D.Operator(dims, terms)
    Ls = [D.Operator.local(dims, b1, A[b1], np.sqrt(kb)), D.Operator.local(dims, b2, A[b2], np.sqrt(kb)),
          D.Operator.local(dims, a1, A[a1], np.sqrt(k1)), D.Operator.local(dims, a2, A[a2], np.sqrt(k1))]
    obs = {"n_a1": D.Operator.local(dims, a1, D.op_num(dims[a1])),
           "n_a2": D.Operator.local(dims, a2, D.op_num(dims[a2])),
           "parity_a1": D.Operator.local(dims, a1, D.op_parity(dims[a1]))}
    return DenseSystem(dims, H, Ls, observables=obs, init=[D.fock(N, 0) for N in dims])


def transmon_eigenbasis(ec, ej, K, n_cut=500, tie=1e-9):
    """Sec. VII, numerical experiment: diagonalise the transmon alone,
    4 Ec n^2 - Ej cos(phi) on the charges |n| <= n_cut (cos(phi) cut open at both
    ends, ng = 0), keep the K lowest eigenstates Psi_alpha(n) and write
    [n_t]_{alpha beta} = sum_n Psi_alpha(n) n Psi_beta(n).

    Readings: the eigenstates are taken with definite charge parity (n -> -n), so
    that the exactly degenerate pairs above the well give a unique basis; within a
    pair (energies equal to `tie` relative to their size) the even state comes first; each
    eigenvector's largest component over n >= 0 (the first such n on ties) is
    positive.  Returns (energies ascending, n_t, Psi as columns over n)."""
    n = np.arange(-n_cut, n_cut + 1, dtype=np.float64)
    N = n.size
    H = np.diag(4.0 * ec * n * n) - 0.5 * ej * (np.eye(N, k=1) + np.eye(N, k=-1))
    c = n_cut
    # parity sectors as charge-basis columns
    Pe = np.zeros((N, n_cut + 1))
    Po = np.zeros((N, n_cut))
    Pe[c, 0] = 1.0
    for m in range(1, n_cut + 1):
        Pe[c + m, m] = Pe[c - m, m] = np.sqrt(0.5)
        Po[c + m, m - 1] = np.sqrt(0.5)
        Po[c - m, m - 1] = -np.sqrt(0.5)
    states = []
    for P, parity in ((Pe, 0), (Po, 1)):
        w, v = np.linalg.eigh(P.T @ H @ P)
        for j in range(w.size):
            states.append((w[j], parity, P @ v[:, j]))
    states.sort(key=lambda st: st[0])
    # even before odd inside a degenerate pair
    i = 0
    while i + 1 < len(states):
        a, b = states[i], states[i + 1]
        if abs(a[0] - b[0]) <= tie * max(abs(a[0]), abs(b[0])) and a[1] > b[1]:
            states[i], states[i + 1] = b, a
        i += 1
    states = states[:K]
    E = np.array([st[0] for st in states])
    Psi = np.stack([st[2] for st in states], axis=1)
    for j in range(K):
        half = Psi[c:, j]
        k = int(np.argmax(np.abs(half)))
        if half[k] < 0:
            Psi[:, j] = -Psi[:, j]
    nt = Psi.T @ (n[:, None] * Psi)
    return E, nt, Psi


def transmon_eig(cfg, nsteps, f_table=None):
    """Transmon x resonator with the transmon in its eigenbasis (Sec. VII,
    numerical experiment): H0 = diag(eps_alpha - eps_0) + w_r a^dag a
    + g n_t (a + a^dag), drive f(t_n) (a + a^dag), L = sqrt(kappa) a; observables
    N_t = Tr(b^dag b rho) with b^dag b = diag(alpha) and N_c = Tr(a^dag a rho);
    start in transmon eigenstate 0 x vacuum."""
    Rt, Rr = cfg["R"]
    K, Nr = 2 ** Rt, 2 ** Rr
    dims = (K, Nr)
    ec = cfg["ec"]
    ej = cfg["ej_over_ec"] * ec
    g = cfg["g_over_ec"] * ec
    E, nt, _ = transmon_eigenbasis(ec, ej, K, cfg.get("n_cut", 500))
    a, ad = D.op_a(Nr), D.op_adag(Nr)
    Ht = np.diag(E - E[0]).astype(np.complex128)
    ntc = nt.astype(np.complex128)
    H0 = D.Operator(dims, [(1.0, {0: Ht}), (cfg["wr"], {1: D.op_num(Nr)}), (g, {0: ntc, 1: a}),
                           (g, {0: ntc, 1: ad})])
    H1 = D.Operator(dims, [(1.0, {1: a}), (1.0, {1: ad})])
    Ls = [D.Operator.local(dims, 1, a, np.sqrt(cfg["kappa"]))]
    obs = {"n_c": D.Operator.local(dims, 1, D.op_num(Nr)), "n_t": D.Operator.local(dims, 0, D.op_num(K))}
    if f_table is None:
        f_table = drive_table(cfg, nsteps)
    return DenseSystem(dims, H0, Ls, H1=H1, f_table=f_table, observables=obs, init=[D.fock(K, 0), D.fock(Nr, 0)])


def z_gate_params(cfg):
    """The Z-gate operating point of Sec. VI's numerical experiment, from the raw
    parameters (R_a, g2, kappa_b, theta): |alpha|^2 = N_a / 3 (unless given);
    the buffer is dark for g2 a^2 + eps_d = 0 on the cat, so eps_d = -g2 alpha^2
    (reading of alpha = -sqrt(eps_d / g2), Sec. VI, with H_stab as written);
    eps_Z = (1/10) 4 g2^2 / kappa_b; the gate time from theta = 4 alpha T_Z eps_Z."""
    Na = 2 ** cfg["R"][0]
    alpha2 = cfg.get("alpha2", Na / 3.0)
    alpha = float(np.sqrt(alpha2))
    eps_z = 4.0 * cfg["g2"] ** 2 / cfg["kb"] / 10.0
    t_z = cfg["theta"] / (4.0 * alpha * eps_z)
    return dict(alpha2=alpha2, alpha=alpha, eps_d=-cfg["g2"] * alpha2, eps_z=eps_z, t_z=t_z,
                steps=int(round(t_z / cfg["dt"])))


def cat_state(N, alpha, parity=+1):
    """Normalised cat |alpha> + parity |-alpha> from the truncated coherent states."""
    v = D.coherent(N, alpha) + parity * D.coherent(N, -alpha)
    return v / np.linalg.norm(v)


def z_gate(cfg, init=None):
    """Z gate on a cat qubit with its buffer (Sec. VI, Eq. cb and Eq. Hz), modes
    [a, b]: H = g2 (a^dag^2 b + a^2 b^dag) + eps_d (b + b^dag) + eps_Z (a + a^dag),
    L_b = sqrt(kappa_b) b (+ sqrt(kappa_a) a).  Start (unless `init` is given): the
    even cat of amplitude alpha x buffer vacuum."""
    Ra, Rb = cfg["R"]
    Na, Nb = 2 ** Ra, 2 ** Rb
    dims = (Na, Nb)
    zp = z_gate_params(cfg)
    g2 = cfg["g2"]
    A, Ad, B, Bd = D.op_a(Na), D.op_adag(Na), D.op_a(Nb), D.op_adag(Nb)
    H = D.Operator(dims, [(g2, {0: Ad @ Ad, 1: B}), (g2, {0: A @ A, 1: Bd}), (zp["eps_d"], {1: B}),
                          (zp["eps_d"], {1: Bd}), (zp["eps_z"], {0: A}), (zp["eps_z"], {0: Ad})])
    Ls = [D.Operator.local(dims, 1, B, np.sqrt(cfg["kb"]))]
    if cfg.get("ka", 0.0) > 0.0:
        Ls.append(D.Operator.local(dims, 0, A, np.sqrt(cfg["ka"])))
    obs = {"parity_a": D.Operator.local(dims, 0, D.op_parity(Na)), "n_a": D.Operator.local(dims, 0, D.op_num(Na)),
           "n_b": D.Operator.local(dims, 1, D.op_num(Nb))}
    if init is None:
        init = [cat_state(Na, zp["alpha"], +1), D.fock(Nb, 0)]
    return DenseSystem(dims, H, Ls, observables=obs, init=init)
