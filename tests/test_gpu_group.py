"""Groups (qlb_group_*, through the C-ABI): many states stepped with one launch per
phase of the step over all of them.  A member's numbers must be the ones its own
qlb_step computes (Sec. V.B step, Sec. V.A zip-up and compression, Sec. IV.A
purification), so each group run is compared with twins of its members stepped
one by one: bit for bit when the members share one planned shape (the same
kernels, K splits and reduction orders), and within 1e-12 when they do not (a
member may then be served by the kernel variant its largest co-member needs).
The members' results are also checked against the dense oracle."""
import numpy as np
import pytest

from oracle import dense as D
from oracle import systems as OS
from paper_2605_27515_gb300 import inputs
from paper_2605_27515_gb300 import qlb as Q
from paper_2605_27515_gb300 import systems

pytestmark = pytest.mark.gpu


def _cfg(**kw):
    cfg = inputs.config("cat_r5")
    cfg.update(kw)
    return cfg


def _obs(b, st):
    return np.array([st.expectation(b.observables[k]).real for k in ("n", "parity")] + [st.purity()])


def _start(N, k):
    """Distinct product starts of one mode: coherent-like vectors of growing amplitude."""
    c = np.zeros(N, dtype=np.complex128)
    c[0] = 1.0
    a = 0.3 + 0.25 * k
    for n in range(1, N):
        c[n] = c[n - 1] * a / np.sqrt(n)
    return c / np.linalg.norm(c)


@pytest.mark.parametrize("precision", [Q.PREC_F64, Q.PREC_MIXED, Q.PREC_TC])
def test_group_equals_members_alone_bitwise(precision):
    """Four states of one system (one planned shape), different starts: 60 group
    steps give the same bits as 60 steps of each twin alone."""
    cfg = _cfg()
    ctx = Q.Ctx(device=0, precision=precision, tol=cfg["tol"], chi_max=cfg["chi_max"], chi_mu_max=cfg["chi_mu_max"])
    b = systems.build(ctx, cfg)
    N = 2 ** cfg["R"][0]
    members = [b.sys.state([_start(N, k)]) for k in range(4)]
    twins = [b.sys.state([_start(N, k)]) for k in range(4)]
    g = Q.Group(ctx, members)
    for _ in range(3):
        g.step(cfg["dt"], 20)
        for t in twins:
            t.step(cfg["dt"], 20)
    assert g.launches() > 0
    for m, t in zip(members, twins):
        assert m.bond_dims() == t.bond_dims()
        np.testing.assert_array_equal(_obs(b, m), _obs(b, t))
    g.close()
    for st in members + twins:
        st.close()
    ctx.close()


def test_mixed_group_matches_alone_and_oracle():
    """Members of different systems (the same number of sites): alpha^2 in {2, 4, 6}
    and different single-photon loss, one with a bond cap of 8; 300 group steps
    agree with each twin alone within 1e-12 and with the dense oracle within 1e-6."""
    variants = [dict(alpha2=2.0, k1=1e-3), dict(alpha2=4.0, k1=3e-3), dict(alpha2=6.0, k1=1e-4)]
    # caps that do not bind for N = 32 (a binding zip-up cap cuts real weight):
    # only member 2's lowered bond cap truncates
    ctx = Q.Ctx(device=0, tol=1e-12, chi_max=64, chi_mu_max=32)
    builds = [systems.build(ctx, _cfg(**v)) for v in variants]
    members = [b.sys.state(b.init) for b in builds]
    twins = [b.sys.state(b.init) for b in builds]
    members[2].truncate(chi_max=8)
    twins[2].truncate(chi_max=8)
    dt, n = 1e-3, 300
    g = Q.Group(ctx, members)
    g.step(dt, n)
    for t in twins:
        t.step(dt, n)
    for k, (b, m, t) in enumerate(zip(builds, members, twins)):
        om, ot = _obs(b, m), _obs(b, t)
        assert np.max(np.abs(om - ot)) < 1e-12, (k, om, ot)
        ds = OS.cat(_cfg(**variants[k]))
        rho = ds.rho0()
        for _ in range(n):
            rho = D.kraus_step(rho, ds.H0, ds.Ls, dt)
        if k != 2:  # the chi = 8 member is truncated below the exact ranks
            for name in ("n", "parity"):
                o = D.expectation(rho, ds.observables[name]).real
                assert abs(m.expectation(b.observables[name]).real - o) < 1e-6, (k, name)
    g.close()
    for st in members + twins:
        st.close()
    ctx.close()


def test_group_of_multimode_variants_equals_alone():
    """The four-mode cat pair at check size ([b1, a1, a2, b2] = [4, 8, 8, 4] levels,
    five branches, 10 sites): four beam-splitter variants J as one group, 40 steps,
    bit for bit against each variant stepped alone."""
    cfg = inputs.config("cat_pair")
    cfg["R"] = list(cfg["check"]["R"])
    ctx = Q.Ctx(device=0, precision=Q.PREC_MIXED, tol=cfg["tol"], chi_max=32, chi_mu_max=16)
    Js = inputs.cat_pair_J(4, cfg["J"] * 20)
    builds = [systems.build(ctx, cfg, J=J) for J in Js]
    members = [b.sys.state(b.init) for b in builds]
    twins = [b.sys.state(b.init) for b in builds]
    g = Q.Group(ctx, members)
    g.step(cfg["dt"] * 20, 40)
    for t in twins:
        t.step(cfg["dt"] * 20, 40)
    for b, m, t in zip(builds, members, twins):
        assert m.bond_dims() == t.bond_dims()
        for name in ("n_a1", "n_a2", "parity_a1"):
            assert m.expectation(b.observables[name]) == t.expectation(b.observables[name]), name
    g.close()
    for st in members + twins:
        st.close()
    ctx.close()


def test_group_then_members_alone_continue():
    """A member keeps stepping on its own after group steps (the streams are
    ordered both ways): 40 group steps + 40 own steps equal 80 own steps."""
    cfg = _cfg()
    ctx = Q.Ctx(device=0, tol=cfg["tol"], chi_max=cfg["chi_max"], chi_mu_max=cfg["chi_mu_max"])
    b = systems.build(ctx, cfg)
    N = 2 ** cfg["R"][0]
    a, c = b.sys.state([_start(N, 1)]), b.sys.state([_start(N, 2)])
    ta = b.sys.state([_start(N, 1)])
    g = Q.Group(ctx, [a, c])
    g.step(cfg["dt"], 40)
    a.step(cfg["dt"], 40)
    ta.step(cfg["dt"], 80)
    np.testing.assert_array_equal(_obs(b, a), _obs(b, ta))
    g.close()
    for st in (a, c, ta):
        st.close()
    ctx.close()


def test_group_arguments_are_checked():
    ctx = Q.Ctx(device=0, chi_max=16, chi_mu_max=8)
    b1 = systems.build(ctx, _cfg())
    b2 = systems.build(ctx, _cfg(R=[4]))
    s1, s2 = b1.sys.state(b1.init), b2.sys.state(b2.init)
    with pytest.raises(Q.QlbError):
        Q.Group(ctx, [s1, s1])  # twice
    with pytest.raises(Q.QlbError):
        Q.Group(ctx, [s1, s2])  # 5 sites and 4 sites
    ctx2 = Q.Ctx(device=0, chi_max=16, chi_mu_max=8)
    with pytest.raises(Q.QlbError):
        Q.Group(ctx2, [s1])  # another context
    g = Q.Group(ctx, [s1])
    with pytest.raises(Q.QlbError):
        g.step(-1.0, 1)
    g.close()
    s1.close()
    s2.close()
    ctx2.close()
    ctx.close()
