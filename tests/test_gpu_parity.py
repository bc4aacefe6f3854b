"""GPU parity of the CUDA path (through the C-ABI) against the FP64 oracle.

Untruncated FP64 form: observables within 1e-10 of the dense oracle.
Truncated form (stated tolerance): within 1e-6 absolute (photon number, parity,
fidelity), the bar for the truncated path.
"""
import numpy as np
import pytest

from oracle import dense as D
from oracle import qtt as Qo
from oracle import systems as OS
from paper_2605_27515_gb300 import inputs
from paper_2605_27515_gb300 import qlb as Q
from paper_2605_27515_gb300 import systems

pytestmark = pytest.mark.gpu

EXACT = dict(tol=1e-28, chi_max=256, chi_mu_max=128)


@pytest.fixture(scope="module")
def ctx():
    c = Q.Ctx(device=0, **EXACT)
    yield c
    c.close()


def _rand_dense(N, rng, herm=False):
    X = rng.normal(size=(N, N)) + 1j * rng.normal(size=(N, N))
    return X + X.conj().T if herm else X


# ------------------------------------------------------------------ builder


@pytest.mark.parametrize("R", [1, 3, 5])
def test_builder_builtin_ops_dense(ctx, R):
    N = 2 ** R
    s = Q.System(ctx, [R])
    cases = [
        ([(1.0, [(0, Q.F_A)])], D.op_a(N)),
        ([(1.0, [(0, Q.F_ADAG)])], D.op_adag(N)),
        ([(1.0, [(0, Q.F_A, 2)]), (-4.0, [])], D.op_a(N) @ D.op_a(N) - 4 * np.eye(N)),
        ([(0.3, [(0, Q.F_ADAG, 2), (0, Q.F_A, 2)])], 0.3 * D.op_adag(N) @ D.op_adag(N) @ D.op_a(N) @ D.op_a(N)),
        ([(1.0, [(0, Q.F_NUM)])], D.op_num(N)),
        ([(1.0, [(0, Q.F_PARITY)])], D.op_parity(N)),
        ([(2.0, [(0, Q.F_CHARGE, 2, N / 2)]), (-1.5, [(0, Q.F_COSPHI)])],
         2.0 * D.op_charge(N, N // 2) @ D.op_charge(N, N // 2) - 1.5 * D.op_cos_phi(N)),
    ]
    for terms, ref in cases:
        op = s.op(terms)
        np.testing.assert_allclose(op.to_dense(), ref, atol=1e-12 * max(1, np.abs(ref).max()))
        op.close()
    s.close()


def test_builder_dense_multimode(ctx):
    rng = np.random.default_rng(3)
    Rs = [2, 3]
    dims = (4, 8)
    s = Q.System(ctx, Rs)
    A0, A1, B1 = _rand_dense(4, rng), _rand_dense(8, rng), _rand_dense(8, rng)
    op = s.op([(0.7 - 0.1j, [(0, Q.F_DENSE, A0), (1, Q.F_DENSE, A1)]), (1.1, [(1, Q.F_DENSE, B1), (1, Q.F_A)])])
    ref = D.Operator(dims, [(0.7 - 0.1j, {0: A0, 1: A1}), (1.1, {1: B1 @ D.op_a(8)})]).dense()
    np.testing.assert_allclose(op.to_dense(), ref, atol=1e-11 * np.abs(ref).max())
    s.close()


@pytest.mark.parametrize("R", [8, 10])
def test_builder_table1_ranks(ctx, R):
    """Table I ranks from the device TT-SVD: a -> 8 (+-1), a + a^dag -> 10 (+-1),
    a^2 -> 8 (+-2) at 1e-12 relative Frobenius per bond; (a^dag)^2 a^2 -> 3 exactly."""
    s = Q.System(ctx, [R])
    tol = 1e-24 / (R - 1)  # relative weight per bond ~ (1e-12)^2 spread over the bonds
    ra = max(s.op([(1.0, [(0, Q.F_A)])], tol=tol).bond_dims())
    rx = max(s.op([(1.0, [(0, Q.F_A)]), (1.0, [(0, Q.F_ADAG)])], tol=tol).bond_dims())
    r2 = max(s.op([(1.0, [(0, Q.F_A, 2)])], tol=tol).bond_dims())
    rn = max(s.op([(1.0, [(0, Q.F_ADAG, 2), (0, Q.F_A, 2)])]).bond_dims())
    assert abs(ra - 8) <= 1 and abs(rx - 10) <= 1 and abs(r2 - 8) <= 2
    assert rn == 3
    # and the oracle's own TT-SVD agrees on the exact one
    N = 2 ** R
    a = D.op_a(N)
    assert Qo.mpo_rank(Qo.mpo_from_dense(a.conj().T @ a.conj().T @ a @ a, R, 1e-14)) == 3
    s.close()


# ------------------------------------------------------------------ untruncated step


def _random_system(ctx, Rs, seed, n_jumps=2):
    rng = np.random.default_rng(seed)
    dims = tuple(2 ** r for r in Rs)
    s = Q.System(ctx, Rs)
    Hterms_q, Hterms_o = [], []
    for m, N in enumerate(dims):
        X = _rand_dense(N, rng, herm=True) * 0.3
        Hterms_q.append((1.0, [(m, Q.F_DENSE, X)]))
        Hterms_o.append((1.0, {m: X}))
    if len(dims) > 1:
        Y0, Y1 = _rand_dense(dims[0], rng) * 0.2, _rand_dense(dims[1], rng) * 0.2
        Hterms_q += [(1.0, [(0, Q.F_DENSE, Y0), (1, Q.F_DENSE, Y1)]),
                     (1.0, [(0, Q.F_DENSE, Y0.conj().T), (1, Q.F_DENSE, Y1.conj().T)])]
        Hterms_o += [(1.0, {0: Y0, 1: Y1}), (1.0, {0: Y0.conj().T, 1: Y1.conj().T})]
    H = s.op(Hterms_q)
    s.set_hamiltonian(H)
    Hd = D.Operator(dims, Hterms_o)
    Ls, Lds = [], []
    for k in range(n_jumps):
        m = k % len(dims)
        X = _rand_dense(dims[m], rng) * 0.4
        L = s.op([(1.0, [(m, Q.F_DENSE, X)]), (0.2, [])])
        s.add_jump(L)
        Ls.append(L)
        Lds.append(D.Operator(dims, [(1.0, {m: X}), (0.2, {})]))
    vecs = [rng.normal(size=N) + 1j * rng.normal(size=N) for N in dims]
    O = _rand_dense(int(np.prod(dims)), rng, herm=True)
    return s, H, Ls, Hd, Lds, vecs, O, dims


@pytest.mark.parametrize("Rs", [[3], [2, 2], [1, 2, 1]])
def test_untruncated_step_matches_dense(ctx, Rs):
    s, H, Ls, Hd, Lds, vecs, Odense, dims = _random_system(ctx, Rs, seed=sum(Rs) * 7 + len(Rs))
    # a random Hermitian observable as a single dense factor needs one mode; use per-mode ones
    rng = np.random.default_rng(99)
    obs_q, obs_o = [], []
    for m, N in enumerate(dims):
        X = _rand_dense(N, rng, herm=True)
        obs_q.append(s.op([(1.0, [(m, Q.F_DENSE, X)])]))
        obs_o.append(D.Operator.local(dims, m, X))
    st = s.state(vecs)
    rho = D.pure(D.product_vector([v / np.linalg.norm(v) for v in vecs]))
    h = 0.02
    target = [D.coherent(N, 0.5) for N in dims]
    for k in range(8):
        assert st.step(h, 1) >= 0
        rho = D.kraus_step(rho, Hd, Lds, h)
        for oq, oo in zip(obs_q, obs_o):
            g = st.expectation(oq)
            o = D.expectation(rho, oo)
            assert abs(g - o) < 1e-10, (k, g, o)
        assert abs(st.trace() - 1) < 1e-12
        assert abs(st.purity() - D.purity(rho)) < 1e-10
        assert abs(st.fidelity(target) - D.fidelity(rho, D.product_vector(target))) < 1e-10
    st.close()
    s.close()


def _second_order_branches(Hd, Lds, h):
    """The Kraus operators of the second-order map in branch order:
    U_1', sqrt(h/2) U_1 L_k, sqrt(h/2) L_k U_1, (h/sqrt 2) L_j L_k (Sec. V.B)."""
    He = D.h_eff(Hd, Lds)
    U = D.u1(Hd, Lds, h)
    out = [(U + (He @ He).scale(-0.5 * h * h)).dense()]
    out += [np.sqrt(h / 2) * (U @ L).dense() for L in Lds]
    out += [np.sqrt(h / 2) * (L @ U).dense() for L in Lds]
    out += [h / np.sqrt(2) * (Lj @ Lk).dense() for Lj in Lds for Lk in Lds]
    return out


@pytest.mark.parametrize("Rs", [[3], [2, 2]])
def test_second_order_kraus_branches(ctx, Rs):
    """Each branch of the device's stacked second-order Kraus MPO equals the dense
    product it stands for (1 + 2l + l^2 branches)."""
    s, H, Ls, Hd, Lds, vecs, _, dims = _random_system(ctx, Rs, seed=41 + len(Rs))
    s.set_scheme(2)
    st = s.state(vecs)
    h = 0.03
    ref = _second_order_branches(Hd, Lds, h)
    assert len(ref) == 1 + 2 * len(Lds) + len(Lds) ** 2
    for k, K in enumerate(ref):
        np.testing.assert_allclose(st.kraus_to_dense(h, k), K, atol=1e-12 * max(1.0, np.abs(K).max()))
    st.close()
    s.close()


@pytest.mark.parametrize("Rs", [[3], [2, 2], [1, 2, 1]])
def test_second_order_step_matches_dense(ctx, Rs):
    """Untruncated second-order steps: the whole density matrix within 1e-10 of the
    dense oracle's second-order map, step after step."""
    s, H, Ls, Hd, Lds, vecs, _, dims = _random_system(ctx, Rs, seed=sum(Rs) * 11 + len(Rs))
    s.set_scheme(2)
    st = s.state(vecs)
    rho = D.pure(D.product_vector([v / np.linalg.norm(v) for v in vecs]))
    h = 0.02
    for k in range(8):
        assert st.step(h, 1) >= 0
        rho = D.kraus_step(rho, Hd, Lds, h, order=2)
        Psi = st.to_dense()
        np.testing.assert_allclose(Psi @ Psi.conj().T, rho, atol=1e-10)
        assert abs(st.trace() - 1) < 1e-12
    st.close()
    s.close()


def test_second_order_global_error_against_lindblad(ctx):
    """Through the device path, halving h divides the error against exp(T Lindbladian)
    by about 4 with the second-order scheme and about 2 with the first-order one."""
    import scipy.linalg as sla

    s, H, Ls, Hd, Lds, vecs, _, dims = _random_system(ctx, [3], seed=77)
    rho0 = D.pure(D.product_vector([v / np.linalg.norm(v) for v in vecs]))
    T = 0.4
    G = D.lindbladian(Hd, Lds)
    exact = (sla.expm(T * G) @ rho0.reshape(-1)).reshape(rho0.shape)
    exact = exact / np.trace(exact).real
    errs = {}
    for order in (1, 2):
        s.set_scheme(order)
        for n in (20, 40):
            st = s.state(vecs)
            st.step(T / n, n)
            Psi = st.to_dense()
            errs[order, n] = np.abs(Psi @ Psi.conj().T - exact).max()
            st.close()
    r1 = errs[1, 20] / errs[1, 40]
    r2 = errs[2, 20] / errs[2, 40]
    assert 1.6 < r1 < 2.5, errs
    assert 3.2 < r2 < 5.0, errs
    assert errs[2, 40] < errs[1, 40] / 5
    s.close()


def test_second_order_scheme_errors(ctx):
    s = Q.System(ctx, [3])
    with pytest.raises(Q.QlbError) as e:
        s.set_scheme(3)
    assert e.value.status == Q.EINVAL
    H0 = s.op([(1.0, [(0, Q.F_NUM)])])
    H1 = s.op([(1.0, [(0, Q.F_A)]), (1.0, [(0, Q.F_ADAG)])])
    s.set_hamiltonian(H0, H1, np.ones(4))
    with pytest.raises(Q.QlbError) as e:
        s.set_scheme(2)
    assert e.value.status == Q.EINVAL
    s.close()


def test_drive_table_matches_dense(ctx):
    """H(t_n) = H0 + f(t_n) H1 with f taken at the left end of each step."""
    R = 3
    N = 8
    s = Q.System(ctx, [R])
    H0 = s.op([(0.5, [(0, Q.F_NUM)])])
    H1 = s.op([(1.0, [(0, Q.F_A)]), (1.0, [(0, Q.F_ADAG)])])
    f = np.cos(0.7 * np.arange(30)) * 0.8
    s.set_hamiltonian(H0, H1, f)
    L = s.op([(0.5, [(0, Q.F_A)])])
    s.add_jump(L)
    st = s.state([D.fock(N, 1)])
    dims = (N,)
    H0d = D.Operator.local(dims, 0, 0.5 * D.op_num(N))
    H1d = D.Operator(dims, [(1.0, {0: D.op_a(N)}), (1.0, {0: D.op_adag(N)})])
    Ld = D.Operator.local(dims, 0, D.op_a(N), 0.5)
    nq = s.op([(1.0, [(0, Q.F_A)])])
    rho = D.pure(D.fock(N, 1))
    h = 0.05
    for k in range(25):
        st.step(h, 1)
        rho = D.kraus_step(rho, H0d + H1d.scale(float(f[k])), [Ld], h)
        g = st.expectation(nq)
        o = np.trace(D.op_a(N) @ rho)
        assert abs(g - o) < 1e-10, (k, g, o)
    st.close()
    s.close()


# ------------------------------------------------------------------ the cat configuration (truncated)


@pytest.mark.parametrize("precision,nsteps,bar", [(Q.PREC_F64, 5000, 1e-6), (Q.PREC_MIXED, 5000, 1e-6),
                                                  (Q.PREC_TC, 5000, 3e-4)])
def test_cat_r5_parity_full_run(precision, nsteps, bar):
    """Single cat mode, N = 32, dt = 1e-3, cutoff 1e-12, chi_mu <= 8: photon number
    and parity against the dense oracle every 100 steps over the whole 5000-step
    run: within 1e-6 in the FP64 form and the mixed form (double-float truncation
    solves).  The tensor-core form applies the Kraus MPO in 3xTF32 (~2^-21 per
    operand, FP32 accumulation); its observables drift by ~2e-8 per step, 9.6e-5
    after the 5000 steps on GB300, which is its stated error (bar 3e-4)."""
    cfg = inputs.config("cat_r5")
    cfg["steps"] = nsteps
    c = Q.Ctx(device=0, precision=precision, tol=cfg["tol"], chi_max=cfg["chi_max"], chi_mu_max=cfg["chi_mu_max"])
    b = systems.build(c, cfg)
    st = b.sys.state(b.init)
    ds = OS.cat(cfg)
    _, recs = ds.evolve(cfg["dt"], cfg["steps"], cfg["record_every"], names=["n", "parity"])
    worst = 0.0
    done = 0
    for step, (n_o, p_o) in recs[1:]:
        st.step(cfg["dt"], step - done)
        done = step
        n_g = st.expectation(b.observables["n"]).real
        p_g = st.expectation(b.observables["parity"]).real
        worst = max(worst, abs(n_g - n_o), abs(p_g - p_o))
    assert worst < bar, worst
    assert max(st.bond_dims()) <= cfg["chi_max"] and st.bond_dims()[0] <= cfg["chi_mu_max"]
    st.close()
    c.close()


# ------------------------------------------------------------------ API behaviour


def test_truncate_caps_and_checkpoint(ctx):
    s, H, Ls, Hd, Lds, vecs, O, dims = _random_system(ctx, [4], seed=5)
    st = s.state(vecs)
    st.step(0.05, 5)
    assert st.bond_dims()[0] > 2
    st.truncate(chi_max=2, chi_mu_max=2)
    bd = st.bond_dims()
    assert bd[0] <= 2 and max(bd[1:]) <= 2
    assert abs(st.trace() - 1) < 1e-12
    blob = st.export()
    st2 = s.state(vecs)
    st2.import_(blob)
    assert st2.bond_dims() == st.bond_dims()
    st2.truncate(chi_max=2, chi_mu_max=2)  # same truncation settings as st
    assert st2.bond_dims() == st.bond_dims()
    st.step(0.05, 3)
    st2.step(0.05, 3)
    ob = s.op([(1.0, [(0, Q.F_NUM)])])
    assert abs(st.expectation(ob) - st2.expectation(ob)) < 1e-13
    st.close()
    st2.close()
    s.close()


def test_errors_are_codes(ctx):
    s = Q.System(ctx, [3])
    with pytest.raises(Q.QlbError) as e:
        s.op([(1.0, [(5, Q.F_A)])])
    assert e.value.status == Q.EINVAL
    st = s.state([D.fock(8, 0)])
    with pytest.raises(Q.QlbError) as e:
        st.step(0.1, 1)  # no Hamiltonian, no jumps
    assert e.value.status == Q.ESTATE
    with pytest.raises(Q.QlbError) as e:
        st.step(-1.0, 1)
    assert e.value.status == Q.EINVAL
    st.close()
    s.close()
    c = Q.Ctx(device=0, hbm_budget=1024)
    s = Q.System(c, [6])
    with pytest.raises(Q.QlbError) as e:
        s.op([(1.0, [(0, Q.F_A)])])
    assert e.value.status == Q.ENOMEM
    c.close()


# ------------------------------------------------------------------ failure paths


def test_sweep_limit_returns_enotconv():
    """A context whose eigen-solves may take one sweep (one QL iteration per
    eigenvalue) cannot converge a step's truncation of a random mixed state:
    qlb_step returns QLB_ENOTCONV with a message, and the context stays usable."""
    c = Q.Ctx(device=0, tol=1e-28, chi_max=256, chi_mu_max=128, max_sweeps=1)
    s, H, Ls, Hd, Lds, vecs, O, dims = _random_system(c, [3], seed=23)
    statuses = []
    try:
        st = s.state(vecs)
        for _ in range(3):
            try:
                statuses.append(st.step(0.05, 1))
            except Q.QlbError as e:
                statuses.append(e.status)
                assert "sweep limit" in str(e)
                break
        st.close()
    except Q.QlbError as e:  # the state's first truncation may already stop
        statuses.append(e.status)
    assert Q.ENOTCONV in statuses, statuses
    s.close()
    c.close()
    c2 = Q.Ctx(device=0, **EXACT)
    s2, *_rest, vecs2, _O, _d = _random_system(c2, [3], seed=23)
    st2 = s2.state(vecs2)
    assert st2.step(0.05, 2) >= 0
    st2.close()
    s2.close()
    c2.close()


def test_nonfinite_host_input_returns_enonfinite(ctx):
    s = Q.System(ctx, [3])
    v = D.fock(8, 0).copy()
    v[3] = np.nan
    with pytest.raises(Q.QlbError) as e:
        s.state([v])
    assert e.value.status == Q.ENONFINITE
    s.close()
