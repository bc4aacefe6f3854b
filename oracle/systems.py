"""Dense oracle versions of the paper's model systems (test infrastructure only).

Built from the same parameter sets as the product path (paper_2605_27515_gb300.
inputs) but with the oracle's own dense operators, so the two sides share only
the parameters.  See paper_2605_27515_gb300/systems.py for the formulas; the
mode orders are the same (cat_pair: [b1, a1, a2, b2]).
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


def transmon(cfg, nsteps, f_table, init):
    Rt, Rr = cfg["R"]
    Nt, Nr = 2 ** Rt, 2 ** Rr
    off = Nt // 2
    dims = (Nt, Nr)
    ec = cfg["ec"]
    ej = cfg["ej_over_ec"] * ec
    g = cfg["g_over_ec"] * ec
    nt = D.op_charge(Nt, off) - cfg.get("ng", 0.0) * np.eye(Nt)
    ntc = D.op_charge(Nt, off)
    a, ad = D.op_a(Nr), D.op_adag(Nr)
    H0 = D.Operator(dims, [(4 * ec, {0: nt @ nt}), (-ej, {0: D.op_cos_phi(Nt)}), (cfg["wr"], {1: D.op_num(Nr)}),
                           (g, {0: ntc, 1: a}), (g, {0: ntc, 1: ad})])
    H1 = D.Operator(dims, [(1.0, {1: a}), (1.0, {1: ad})])
    Ls = [D.Operator.local(dims, 1, a, np.sqrt(cfg["kappa"]))]
    obs = {"n_c": D.Operator.local(dims, 1, D.op_num(Nr)), "n_t2": D.Operator.local(dims, 0, ntc @ ntc)}
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
