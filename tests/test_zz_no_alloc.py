"""The purity entry point that allocates no device memory (qlb_purity_noalloc).

Callers under a foreign allocator's fixed budget, or in loops that cannot afford
cudaFree's device-wide synchronisation, cannot let the library allocate.  This
file checks, through the C-ABI, that the no-alloc call returns the same purity
as qlb_purity on two calls in a row, before and after the state moves on, and
that the context's allocation counter does not move across it (while it does
across qlb_purity).  It is collected last on purpose.
"""
import ctypes

import numpy as np
import pytest

from paper_2605_27515_gb300 import qlb as Q

pytestmark = pytest.mark.gpu


def _mixed_state(ctx):
    rng = np.random.default_rng(17)
    s = Q.System(ctx, [3, 2])
    X = rng.normal(size=(8, 8)) + 1j * rng.normal(size=(8, 8))
    H = s.op([(0.3, [(0, Q.F_DENSE, X + X.conj().T)]), (0.2, [(0, Q.F_A), (1, Q.F_ADAG)]),
              (0.2, [(0, Q.F_ADAG), (1, Q.F_A)])])
    s.set_hamiltonian(H)
    for m in (0, 1):
        s.add_jump(s.op([(0.6, [(m, Q.F_A)])]))
    vecs = [rng.normal(size=8) + 1j * rng.normal(size=8), rng.normal(size=4) + 1j * rng.normal(size=4)]
    st = s.state(vecs)
    st.step(0.05, 6)
    return s, st


def test_purity_noalloc_matches_purity_twice():
    ctx = Q.Ctx(device=0, tol=1e-28, chi_max=64, chi_mu_max=32)
    s, st = _mixed_state(ctx)
    assert st.bond_dims()[0] > 1  # a mixed state, so purity < 1
    lib = Q.load()
    ref = st.purity()
    assert ref < 1 - 1e-6
    before = ctx.alloc_count()
    for _ in range(2):
        out = ctypes.c_double(-1.0)
        assert lib.qlb_purity_noalloc(st.h, ctypes.byref(out)) == Q.OK
        assert abs(out.value - ref) < 1e-12, (out.value, ref)
    assert ctx.alloc_count() == before  # no device allocation in either call
    st.purity()
    assert ctx.alloc_count() > before  # while the allocating call does allocate
    # and it tracks the state: one more step, two more calls
    st.step(0.05, 2)
    ref2 = st.purity()
    for _ in range(2):
        assert abs(st.purity_noalloc() - ref2) < 1e-12
    st.close()
    s.close()
    ctx.close()


def test_purity_noalloc_rank_limit_is_the_context_cap():
    """The scratch array serves purification ranks up to 128, the largest
    chi_mu_max a context accepts, so its QLB_EINVAL branch for larger ranks is
    unreachable through the public calls: a context asking for 129 is refused."""
    o = Q.qlb_default_options(device=0, chi_mu_max=129)
    h = ctypes.c_void_p()
    assert Q.load().qlb_create(ctypes.byref(o), ctypes.byref(h)) == Q.EINVAL
