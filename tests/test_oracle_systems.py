"""Pins of the oracle's model systems that the other oracle tests reach only
indirectly: the single cat mode, the four-mode cat pair (Sec. VI, Eq. cb with a
beam splitter) and the charge-basis transmon x resonator (Sec. VII).  Each pin
is a property the physics fixes (a dark state, a conserved charge, a printed
frequency, a unitary equivalence), and each is shown to fail on a planted
mistake in the oracle's operators."""
import numpy as np

from oracle import dense as D
from oracle import systems as OS
from paper_2605_27515_gb300 import inputs


def _norm_apply(op, psi):
    return float(np.linalg.norm(op.apply_left(psi[:, None])))


# ------------------------------------------------------------------ single cat mode


def test_cat_two_photon_dissipator_annihilates_the_cats():
    """L1 = sqrt(k2)(a^2 - alpha^2) kills |+alpha> and |-alpha> (hence both cats)
    up to the Fock tail; with k1 = 0 and no drive the dense step keeps the even
    cat fixed (Sec. VI: the two-photon manifold)."""
    cfg = inputs.config("cat_r5")  # N = 32, alpha^2 = 4
    cfg.update(k1=0.0, eps_z=0.0, alpha2=2.0)
    ds = OS.cat(cfg)
    alpha = np.sqrt(cfg["alpha2"])
    for v in (D.coherent(32, alpha), D.coherent(32, -alpha), OS.cat_state(32, alpha, +1)):
        assert _norm_apply(ds.Ls[0], v) < 1e-11
    rho = D.pure(OS.cat_state(32, alpha, +1))
    out = D.kraus_step(rho, ds.H0, ds.Ls, 1e-3)
    assert np.abs(out - rho).max() < 1e-12
    # planted: the alpha^2 term with the wrong sign
    c, f = ds.Ls[0].terms[1]
    bad = D.Operator(ds.dims, [ds.Ls[0].terms[0], (-c, f)])
    assert _norm_apply(bad, D.coherent(32, alpha)) > 1.0


def test_cat_drive_and_observables():
    """H = eps_Z (a + a^dag) is Hermitian and odd under parity (it anticommutes
    with (-1)^n); the parity observable is the diagonal (-1)^n."""
    cfg = inputs.config("cat_r9")
    cfg["R"] = [5]
    ds = OS.cat(cfg)
    H = ds.H0.dense()
    P = ds.observables["parity"].dense()
    assert np.abs(H - H.conj().T).max() == 0.0
    assert np.abs(P @ H + H @ P).max() < 1e-14
    assert abs(H[1, 0] - cfg["eps_z"]) < 1e-15 and abs(H[0, 1] - cfg["eps_z"]) < 1e-15
    np.testing.assert_array_equal(np.diag(P).real, (-1.0) ** np.arange(32))


# ------------------------------------------------------------------ cat pair


def _pair_cfg(**kw):
    cfg = inputs.config("cat_pair")
    cfg["R"] = [5, 2, 5, 2]  # storages N = 32, buffers N = 4 (modes [b1, a1, a2, b2])
    cfg.update(kw)
    return cfg


def _pair_charge(dims):
    """Q = n_a1 + n_a2 + 2 (n_b1 + n_b2): two-to-one photon conversion and the beam
    splitter both conserve it."""
    b1, a1, a2, b2 = 0, 1, 2, 3
    return (D.Operator.local(dims, a1, D.op_num(dims[a1])) + D.Operator.local(dims, a2, D.op_num(dims[a2]))
            + D.Operator.local(dims, b1, D.op_num(dims[b1])).scale(2.0)
            + D.Operator.local(dims, b2, D.op_num(dims[b2])).scale(2.0))


def test_cat_pair_buffers_are_dark_on_the_cats():
    """At J = 0 and k1 = 0, |+-alpha>_a1 |+-alpha>_a2 with both buffers empty is dark:
    H_eff psi = 0 (g2 alpha^2 + eps_b = 0 with eps_b = -g2 alpha^2, b|0> = 0) and every
    L_k psi = 0, so |psi><psi| is a fixed point of the dense step (Sec. VI, Eq. cb),
    up to the Fock tail (alpha^2 = 2 at N = 32).  Planted: eps_b with the wrong
    sign, or a single a instead of a^2 in the conversion term, breaks it."""
    cfg = _pair_cfg(J=0.0, k1=0.0, alpha2=2.0)
    ds = OS.cat_pair(cfg)
    al = np.sqrt(cfg["alpha2"])
    vac4 = D.fock(4, 0)
    He = D.h_eff(ds.H0, ds.Ls)
    for s1 in (+1, -1):
        for s2 in (+1, -1):
            psi = D.product_vector([vac4, D.coherent(32, s1 * al), D.coherent(32, s2 * al), vac4])
            assert _norm_apply(He, psi) < 1e-11
            assert max(_norm_apply(L, psi) for L in ds.Ls) < 1e-14
    psi = D.product_vector([vac4, D.coherent(32, al), D.coherent(32, al), vac4])
    # planted mistakes in the oracle's Hamiltonian
    flip = D.Operator(ds.dims, [(-c if len(f) == 1 else c, f) for c, f in ds.H0.terms])
    assert _norm_apply(flip, psi) > 1.0
    A = D.op_a(32)
    A2 = A @ A

    def plant(x):
        return A if x.shape == A2.shape and np.array_equal(x, A2) else x

    one_a = D.Operator(ds.dims, [(c, {m: plant(x) for m, x in f.items()}) for c, f in ds.H0.terms])
    assert _norm_apply(one_a, psi) > 0.1


def test_cat_pair_conserves_the_conversion_charge():
    """[H, Q] = 0 exactly (also in the truncated space) when the buffer drives are
    off, for any J; H is Hermitian.  Planted: b instead of b^dag in a conversion
    term breaks the commutation."""
    cfg = _pair_cfg(R=[3, 2, 3, 2], alpha2=0.0, J=0.37)  # eps_b = -g2 alpha^2 = 0
    ds = OS.cat_pair(cfg)
    H = ds.H0.dense()
    Q = _pair_charge(ds.dims).dense()
    assert np.abs(H - H.conj().T).max() < 1e-15
    assert np.abs(H @ Q - Q @ H).max() < 1e-12
    assert np.abs(H).max() > 0.1
    Bd = D.op_adag(4)
    B = D.op_a(4)
    bad = D.Operator(ds.dims, [(c, {m: (B if x.shape[0] == 4 and np.array_equal(x, Bd) else x) for m, x in f.items()})
                               for c, f in ds.H0.terms])
    Hb = bad.dense()
    assert np.abs(Hb @ Q - Q @ Hb).max() > 0.1


def test_cat_pair_beam_splitter():
    """The J term alone moves one photon between the storages: with g2 = 0 and no
    buffer drive, H = J (a1^dag a2 + a2^dag a1) maps |0,1,0,0> to J |0,0,1,0>."""
    cfg = _pair_cfg(R=[3, 2, 3, 2], g2=0.0, alpha2=0.0, J=0.25)
    ds = OS.cat_pair(cfg)
    e = lambda n: D.fock(8, n)
    psi = D.product_vector([D.fock(4, 0), e(1), e(0), D.fock(4, 0)])
    out = ds.H0.apply_left(psi[:, None])[:, 0]
    ref = 0.25 * D.product_vector([D.fock(4, 0), e(0), e(1), D.fock(4, 0)])
    np.testing.assert_allclose(out, ref, atol=1e-15)


# ------------------------------------------------------------------ charge-basis transmon


def _transmon_cfg(R, g_over_ec=None):
    cfg = inputs.config("transmon")
    cfg["R"] = R
    if g_over_ec is not None:
        cfg["g_over_ec"] = g_over_ec
    return cfg


def test_charge_basis_transmon_frequency():
    """E_C / h = 0.28 GHz, E_J / E_C = 50: the lowest transition of
    4 E_C n^2 - E_J cos(phi) on 32 charges is the 5.320 GHz the paper prints for this
    transmon (Sec. VII), within 0.03 GHz; read off the uncoupled transmon x resonator
    H0 (w_r = 7.5 GHz lies above it).  Planted: cos(phi) without its 1/2 (E_J
    doubled), or 8 E_C in place of 4 E_C, moves it far away.  (E_J with the other
    sign is no mistake at n_g = 0: diag((-1)^n) maps one spectrum onto the other.)"""
    cfg = _transmon_cfg([5, 1], g_over_ec=0.0)
    ds = OS.transmon(cfg, 1)
    w = np.linalg.eigvalsh(ds.H0.dense())
    f01 = (w[1] - w[0]) / (2 * np.pi)
    assert abs(f01 - 5.320) < 0.03, f01
    ec = cfg["ec"]
    ej = cfg["ej_over_ec"] * ec
    for Ht in (OS.transmon_charge_hamiltonian(32, ec, 2 * ej), OS.transmon_charge_hamiltonian(32, 2 * ec, ej)):
        ww = np.linalg.eigvalsh(Ht)
        assert abs((ww[1] - ww[0]) / (2 * np.pi) - 5.320) > 0.3


def test_charge_basis_coupling_is_the_papers_up_to_a_phase():
    """g n_t (a + a^dag) = V [-i g n_t (a - a^dag)] V^dag with V = diag((-i)^n) on the
    resonator (a -> -i a), exactly also in the truncated space, so the whole H0 of
    the oracle equals the paper's form of Sec. VII conjugated by V.  Planted: the
    coupling without the i, g n_t (a - a^dag) after the same V, does not match."""
    cfg = _transmon_cfg([4, 3])
    ds = OS.transmon(cfg, 1)
    Nt, Nr = 16, 8
    ec = cfg["ec"]
    ej = cfg["ej_over_ec"] * ec
    g = cfg["g_over_ec"] * ec
    nt = D.op_charge(Nt, Nt // 2)
    a = D.op_a(Nr)
    paper = (np.kron(OS.transmon_charge_hamiltonian(Nt, ec, ej), np.eye(Nr))
             + cfg["wr"] * np.kron(np.eye(Nt), D.op_num(Nr))
             - 1j * g * np.kron(nt, a - a.conj().T))
    V = np.kron(np.eye(Nt), np.diag((-1j) ** np.arange(Nr)))
    np.testing.assert_allclose(V @ paper @ V.conj().T, ds.H0.dense(), atol=1e-12)
    wrong = paper + 1j * g * np.kron(nt, a - a.conj().T) + g * np.kron(nt, a - a.conj().T)
    assert np.abs(V @ wrong @ V.conj().T - ds.H0.dense()).max() > 1.0


def test_transmon_start_and_drive_table():
    """The oracle's start is the charge-basis ground state (an eigenvector of H_t
    at its lowest eigenvalue) and its drive table is eps(t) cos(w_r t) with the
    linear ramp: f(0) = 0, and past the ramp |f| reaches eps_max."""
    cfg = _transmon_cfg([5, 2])
    ds = OS.transmon(cfg, 4)
    ec = cfg["ec"]
    ej = cfg["ej_over_ec"] * ec
    Ht = OS.transmon_charge_hamiltonian(32, ec, ej)
    g0 = ds.init[0]
    e0 = np.linalg.eigvalsh(Ht)[0]
    np.testing.assert_allclose(Ht @ g0, e0 * g0, atol=1e-10)
    assert ds.f_table[0] == 0.0
    late = OS.drive_table(dict(cfg, dt=1e-3), 200000, t0=cfg["ramp_kappa_t"] / cfg["kappa"])
    eps_max = cfg["eps_over_kappa"] * cfg["kappa"]
    assert abs(np.abs(late).max() - eps_max) < 1e-3 * eps_max
