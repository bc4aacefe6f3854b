"""Thin ctypes binding of libqlb (include/qlb.h); argument marshalling only.

Every function here has the name of the C call it wraps and does no arithmetic
of the method: it converts numpy arrays and Python lists into the C structures,
calls the library, and raises ``QlbError`` on a negative status.  The library
must have been built (``paper_2605_27515_gb300.build``); there is no fallback.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

_LIB_PATH = os.path.join(os.path.dirname(os.path.abspath(__file__)), "libqlb.so")
_lib = None

# status codes and constants (mirror of include/qlb.h)
OK, WUNSTABLE = 0, 1
QLB_BUSY = 2
EINVAL, ENOMEM, ENOTCONV, ETIMEOUT, ENONFINITE, EDEVICE, ESTATE = -1, -2, -3, -4, -5, -6, -7
PREC_F64, PREC_MIXED, PREC_TC = 0, 1, 2
F_ID, F_A, F_ADAG, F_NUM, F_PARITY, F_CHARGE, F_COSPHI, F_DENSE = range(8)
K_CONTRACT, K_GRAM, K_EIG, K_APPLY, K_OTHER, K_COUNT = range(6)
K_NAMES = ["contract", "gram", "eig", "apply", "other"]


class QlbError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"qlb status {status}: {msg}")
        self.status = status


class qlb_options(C.Structure):
    _fields_ = [
        ("device", C.c_int), ("precision", C.c_int), ("tol", C.c_double), ("chi_max", C.c_int),
        ("chi_mu_max", C.c_int), ("zip_tol_factor", C.c_double), ("degeneracy_gap", C.c_double),
        ("max_sweeps", C.c_int), ("hbm_budget", C.c_size_t), ("stream_ordered", C.c_int),
        ("zip_solver", C.c_int), ("zip_chi_max", C.c_int), ("mixed_gemm", C.c_int),
    ]


class qlb_factor(C.Structure):
    _fields_ = [("mode", C.c_int), ("kind", C.c_int), ("power", C.c_int), ("param", C.c_double),
                ("dense", C.POINTER(C.c_double))]


class qlb_term(C.Structure):
    _fields_ = [("re", C.c_double), ("im", C.c_double), ("factors", C.POINTER(qlb_factor)), ("n_factors", C.c_int)]


class qlb_request(C.Structure):
    _fields_ = [
        ("n_modes", C.c_int), ("R", C.POINTER(C.c_int)), ("H", C.POINTER(qlb_term)), ("n_H", C.c_int),
        ("jumps", C.POINTER(C.POINTER(qlb_term))), ("n_jump_terms", C.POINTER(C.c_int)), ("n_jumps", C.c_int),
        ("mode_vecs", C.POINTER(C.POINTER(C.c_double))), ("dt", C.c_double), ("steps", C.c_int64),
        ("tol", C.c_double), ("chi_max", C.c_int), ("chi_mu_max", C.c_int),
        ("obs", C.POINTER(C.POINTER(qlb_term))), ("n_obs_terms", C.POINTER(C.c_int)), ("n_obs", C.c_int),
    ]


_vp = C.c_void_p
_st = C.c_int32
_SIGS = {
    "qlb_default_options": (None, [C.POINTER(qlb_options)]),
    "qlb_create": (_st, [C.POINTER(qlb_options), C.POINTER(_vp)]),
    "qlb_destroy": (None, [_vp]),
    "qlb_last_error": (C.c_char_p, []),
    "qlb_ctx_stream": (_st, [_vp, C.POINTER(_vp)]),
    "qlb_synchronize": (_st, [_vp]),
    "qlb_state_stream": (_st, [_vp, C.POINTER(_vp)]),
    "qlb_state_poll": (_st, [_vp]),
    "qlb_ctx_memory": (_st, [_vp, C.POINTER(C.c_size_t)]),
    "qlb_ctx_alloc_count": (_st, [_vp, C.POINTER(C.c_int64)]),
    "qlb_profile_solver_stats": (_st, [_vp, C.POINTER(C.c_double), C.c_int]),
    "qlb_measure_peak": (_st, [C.c_int, C.c_int, C.POINTER(C.c_double)]),
    "qlb_autotune": (_st, [_vp, C.c_char_p]),
    "qlb_load_tuning": (_st, [_vp, C.c_char_p]),
    "qlb_tc_zgemm": (_st, [C.c_int, C.c_int, C.c_int, C.c_int, C.POINTER(C.c_double), C.POINTER(C.c_double),
                           C.POINTER(C.c_double)]),
    "qlb_zgemm_check": (_st, [C.c_int, C.c_int, C.c_int, C.c_int, C.c_int, C.POINTER(C.c_double),
                              C.POINTER(C.c_double), C.POINTER(C.c_double), C.POINTER(C.c_double)]),
    "qlb_eig_check": (_st, [C.c_int, C.c_int, C.c_int, C.c_int, C.POINTER(C.c_double), C.c_double, C.c_int,
                            C.POINTER(C.c_double), C.POINTER(C.c_double), C.POINTER(C.c_int),
                            C.POINTER(C.c_double)]),
    "qlb_system_create": (_st, [_vp, C.c_int, C.POINTER(C.c_int), C.POINTER(_vp)]),
    "qlb_system_destroy": (None, [_vp]),
    "qlb_op_build": (_st, [_vp, C.POINTER(qlb_term), C.c_int, C.c_double, C.c_int, C.POINTER(_vp)]),
    "qlb_op_destroy": (None, [_vp]),
    "qlb_op_bond_dims": (_st, [_vp, C.POINTER(C.c_int), C.c_int, C.POINTER(C.c_int)]),
    "qlb_op_to_dense": (_st, [_vp, C.POINTER(C.c_double), C.c_size_t]),
    "qlb_set_hamiltonian": (_st, [_vp, _vp, _vp, C.POINTER(C.c_double), C.c_int64]),
    "qlb_add_jump": (_st, [_vp, _vp]),
    "qlb_set_scheme": (_st, [_vp, C.c_int]),
    "qlb_state_init_product": (_st, [_vp, C.POINTER(C.POINTER(C.c_double)), C.POINTER(_vp)]),
    "qlb_state_destroy": (None, [_vp]),
    "qlb_truncate": (_st, [_vp, C.c_double, C.c_int, C.c_int]),
    "qlb_step": (_st, [_vp, C.c_double, C.c_int64]),
    "qlb_expectation": (_st, [_vp, _vp, C.POINTER(C.c_double)]),
    "qlb_fidelity": (_st, [_vp, C.POINTER(C.POINTER(C.c_double)), C.POINTER(C.c_double)]),
    "qlb_trace": (_st, [_vp, C.POINTER(C.c_double)]),
    "qlb_purity": (_st, [_vp, C.POINTER(C.c_double)]),
    "qlb_purity_noalloc": (_st, [_vp, C.POINTER(C.c_double)]),
    "qlb_bond_dims": (_st, [_vp, C.POINTER(C.c_int), C.c_int, C.POINTER(C.c_int)]),
    "qlb_step_stats": (_st, [_vp, C.POINTER(C.c_double)]),
    "qlb_state_to_dense": (_st, [_vp, C.POINTER(C.c_double), C.c_size_t, C.POINTER(C.c_int)]),
    "qlb_kraus_to_dense": (_st, [_vp, C.c_double, C.c_int, C.POINTER(C.c_double), C.c_size_t]),
    "qlb_state_export": (_st, [_vp, _vp, C.c_size_t, C.POINTER(C.c_size_t)]),
    "qlb_state_import": (_st, [_vp, _vp, C.c_size_t]),
    "qlb_server_create": (_st, [_vp, C.c_size_t, C.c_int, C.c_int, C.POINTER(_vp)]),
    "qlb_server_destroy": (None, [_vp]),
    "qlb_submit": (_st, [_vp, C.POINTER(qlb_request), C.POINTER(C.c_int64)]),
    "qlb_poll": (_st, [_vp, C.c_int64, C.POINTER(C.c_double), C.c_int, C.POINTER(C.c_double)]),
    "qlb_cancel": (_st, [_vp, C.c_int64]),
    "qlb_server_stats": (_st, [_vp, C.POINTER(C.c_double)]),
    "qlb_profile_enable": (_st, [_vp, C.c_int]),
    "qlb_profile_read": (_st, [_vp, C.c_int, C.POINTER(C.c_double), C.POINTER(C.c_int64), C.POINTER(C.c_double),
                               C.POINTER(C.c_double)]),
    "qlb_profile_reset": (_st, [_vp]),
    "qlb_group_create": (_st, [_vp, C.POINTER(_vp), C.c_int, C.POINTER(_vp)]),
    "qlb_group_destroy": (None, [_vp]),
    "qlb_group_step": (_st, [_vp, C.c_double, C.c_int64]),
    "qlb_group_launches": (_st, [_vp, C.POINTER(C.c_int)]),
    "qlb_group_stream": (_st, [_vp, C.POINTER(_vp)]),
}


def load(path: str | None = None):
    """Load libqlb.so (raises if it has not been built)."""
    global _lib
    if _lib is not None:
        return _lib
    p = path or _LIB_PATH
    if not os.path.exists(p):
        raise QlbError(EDEVICE, f"{p} is missing: build it with python -m paper_2605_27515_gb300.build")
    lib = C.CDLL(p)
    for name, (res, args) in _SIGS.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _lib = lib
    return lib


def _check(status, allow_warning=True):
    if status < 0:
        raise QlbError(status, load().qlb_last_error().decode())
    return status


def _cvec(v):
    a = np.ascontiguousarray(np.asarray(v, dtype=np.complex128))
    return a, a.ctypes.data_as(C.POINTER(C.c_double))


# ---------------------------------------------------------------- contexts


def qlb_default_options(**kw) -> qlb_options:
    o = qlb_options()
    load().qlb_default_options(C.byref(o))
    for k, v in kw.items():
        setattr(o, k, v)
    return o


class Ctx:
    def __init__(self, **opts):
        self.lib = load()
        self.opts = qlb_default_options(**opts)
        h = _vp()
        _check(self.lib.qlb_create(C.byref(self.opts), C.byref(h)))
        self.h = h

    def stream(self) -> int:
        s = _vp()
        _check(self.lib.qlb_ctx_stream(self.h, C.byref(s)))
        return s.value or 0

    def synchronize(self):
        _check(self.lib.qlb_synchronize(self.h))

    def memory(self) -> int:
        b = C.c_size_t()
        _check(self.lib.qlb_ctx_memory(self.h, C.byref(b)))
        return b.value

    def autotune(self, path=None):
        """Run the launch-shape autotuner (qlb_autotune); optionally write its table."""
        _check(self.lib.qlb_autotune(self.h, path.encode() if path else None))

    def load_tuning(self, path):
        _check(self.lib.qlb_load_tuning(self.h, path.encode()))

    def alloc_count(self) -> int:
        n = C.c_int64()
        _check(self.lib.qlb_ctx_alloc_count(self.h, C.byref(n)))
        return n.value

    def solver_stats(self):
        out = (C.c_double * 9)()
        _check(self.lib.qlb_profile_solver_stats(self.h, out, 9))
        # global_ws: solves beyond one CTA's shared memory; zip_range: zip-up bonds given
        # to the pivoted Gram-Schmidt range basis, zip_fallback: of those, the ones that
        # reached the cap and went to the Jacobi solve
        return dict(solves=out[0], sweeps=out[1], sum_n=out[2], sum_k=out[3], at_limit=out[4],
                    global_ws=out[5], max_n=out[6], zip_range=out[7], zip_fallback=out[8])

    def profile_enable(self, on=True):
        _check(self.lib.qlb_profile_enable(self.h, int(on)))

    def profile_read(self, kclass):
        ms, n, fl, by = C.c_double(), C.c_int64(), C.c_double(), C.c_double()
        _check(self.lib.qlb_profile_read(self.h, kclass, C.byref(ms), C.byref(n), C.byref(fl), C.byref(by)))
        return dict(ms=ms.value, launches=n.value, flops=fl.value, bytes=by.value)

    def profile_reset(self):
        _check(self.lib.qlb_profile_reset(self.h))

    def close(self):
        if self.h:
            self.lib.qlb_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def qlb_create(**opts) -> Ctx:
    return Ctx(**opts)


def qlb_measure_peak(device: int, kind: int) -> float:
    """Measured FMA throughput in TFLOP/s (kind 0: FP64, 1: FP32)."""
    out = C.c_double()
    _check(load().qlb_measure_peak(int(device), int(kind), C.byref(out)))
    return out.value


# ---------------------------------------------------------------- systems and operators


def _terms_to_c(terms, keep):
    """A term list as a C qlb_term array; the arrays it points at go into `keep`."""
    cterms = (qlb_term * max(1, len(terms)))()
    for t, (coeff, facs) in enumerate(terms):
        cf = (qlb_factor * max(1, len(facs)))()
        for j, f in enumerate(facs):
            mode, kind = int(f[0]), int(f[1])
            cf[j].mode, cf[j].kind, cf[j].power, cf[j].param = mode, kind, 1, 0.0
            if kind == F_DENSE:
                a, p = _cvec(f[2])
                keep.append(a)
                cf[j].dense = p
            else:
                if len(f) > 2:
                    cf[j].power = int(f[2])
                if len(f) > 3:
                    cf[j].param = float(f[3])
        keep.append(cf)
        c = complex(coeff)
        cterms[t].re, cterms[t].im = c.real, c.imag
        cterms[t].factors = C.cast(cf, C.POINTER(qlb_factor))
        cterms[t].n_factors = len(facs)
    keep.append(cterms)
    return cterms


class System:
    def __init__(self, ctx: Ctx, R):
        self.ctx = ctx
        self.lib = ctx.lib
        self.R = [int(r) for r in R]
        arr = (C.c_int * len(self.R))(*self.R)
        h = _vp()
        _check(self.lib.qlb_system_create(ctx.h, len(self.R), arr, C.byref(h)))
        self.h = h
        self._keep = []  # ops referenced by the system stay alive

    @property
    def L(self):
        return sum(self.R)

    def op(self, terms, tol=0.0, chi_max=0) -> "Op":
        """terms: list of (coeff, [factor, ...]) with factor = (mode, kind[, power[, param]])
        or (mode, F_DENSE, matrix)."""
        keep = []
        cterms = _terms_to_c(terms, keep)
        h = _vp()
        _check(self.lib.qlb_op_build(self.h, cterms, len(terms), float(tol), int(chi_max), C.byref(h)))
        return Op(self, h)

    def set_hamiltonian(self, H0, H1=None, f_table=None):
        ft = None
        n = 0
        if H1 is not None:
            ft = np.ascontiguousarray(np.asarray(f_table, dtype=np.float64))
            n = len(ft)
            self._keep.append(ft)
        _check(self.lib.qlb_set_hamiltonian(self.h, H0.h if H0 else None, H1.h if H1 else None,
                                            ft.ctypes.data_as(C.POINTER(C.c_double)) if ft is not None else None, n))
        self._keep += [H0, H1]

    def add_jump(self, L):
        _check(self.lib.qlb_add_jump(self.h, L.h))
        self._keep.append(L)

    def set_scheme(self, order: int):
        """Kraus scheme order of qlb_step: 1 (K = U + hL) or 2 (second-order map)."""
        _check(self.lib.qlb_set_scheme(self.h, int(order)))

    def state(self, mode_vecs) -> "State":
        arrs = [_cvec(v) for v in mode_vecs]
        ptrs = (C.POINTER(C.c_double) * len(arrs))(*[p for _, p in arrs])
        h = _vp()
        _check(self.lib.qlb_state_init_product(self.h, ptrs, C.byref(h)))
        return State(self, h)

    def close(self):
        if self.h:
            self.lib.qlb_system_destroy(self.h)
            self.h = None


class Op:
    def __init__(self, sys: System, h):
        self.sys, self.h, self.lib = sys, h, sys.lib

    def bond_dims(self):
        n = C.c_int()
        buf = (C.c_int * 128)()
        _check(self.lib.qlb_op_bond_dims(self.h, buf, 128, C.byref(n)))
        return list(buf[: n.value])

    def to_dense(self) -> np.ndarray:
        N = 2 ** self.sys.L
        out = np.zeros((N, N), dtype=np.complex128)
        _check(self.lib.qlb_op_to_dense(self.h, out.ctypes.data_as(C.POINTER(C.c_double)), 2 * N * N))
        return out

    def close(self):
        if self.h:
            self.lib.qlb_op_destroy(self.h)
            self.h = None


class State:
    def __init__(self, sys: System, h):
        self.sys, self.h, self.lib = sys, h, sys.lib

    def step(self, dt, n=1) -> int:
        return _check(self.lib.qlb_step(self.h, float(dt), int(n)))

    def stream(self) -> int:
        s = _vp()
        _check(self.lib.qlb_state_stream(self.h, C.byref(s)))
        return s.value or 0

    def poll(self) -> bool:
        """True when the state's enqueued work has finished."""
        return _check(self.lib.qlb_state_poll(self.h)) == OK

    def truncate(self, tol=0.0, chi_max=0, chi_mu_max=0):
        return _check(self.lib.qlb_truncate(self.h, float(tol), int(chi_max), int(chi_mu_max)))

    def expectation(self, op: Op) -> complex:
        out = (C.c_double * 2)()
        _check(self.lib.qlb_expectation(self.h, op.h, out))
        return complex(out[0], out[1])

    def fidelity(self, mode_vecs) -> float:
        arrs = [_cvec(v) for v in mode_vecs]
        ptrs = (C.POINTER(C.c_double) * len(arrs))(*[p for _, p in arrs])
        out = C.c_double()
        _check(self.lib.qlb_fidelity(self.h, ptrs, C.byref(out)))
        return out.value

    def trace(self) -> float:
        out = C.c_double()
        _check(self.lib.qlb_trace(self.h, C.byref(out)))
        return out.value

    def purity(self) -> float:
        out = C.c_double()
        _check(self.lib.qlb_purity(self.h, C.byref(out)))
        return out.value

    def purity_noalloc(self) -> float:
        """Tr rho^2 through the entry point that allocates no device memory."""
        out = C.c_double()
        _check(self.lib.qlb_purity_noalloc(self.h, C.byref(out)))
        return out.value

    def bond_dims(self):
        n = C.c_int()
        buf = (C.c_int * 128)()
        _check(self.lib.qlb_bond_dims(self.h, buf, 128, C.byref(n)))
        return list(buf[: n.value])

    def stats(self):
        out = (C.c_double * 4)()
        _check(self.lib.qlb_step_stats(self.h, out))
        return dict(trace_before=out[0], max_discarded=out[1], unstable_factor=out[2], steps=int(out[3]))

    def to_dense(self) -> np.ndarray:
        """Psi as a 2^L x chi_mu matrix (small systems)."""
        N = 2 ** self.sys.L
        cap = N * 128
        out = np.zeros(cap, dtype=np.complex128)
        mu = C.c_int()
        _check(self.lib.qlb_state_to_dense(self.h, out.ctypes.data_as(C.POINTER(C.c_double)), 2 * cap, C.byref(mu)))
        return out[: N * mu.value].reshape(N, mu.value)

    def kraus_to_dense(self, dt, k) -> np.ndarray:
        N = 2 ** self.sys.L
        out = np.zeros((N, N), dtype=np.complex128)
        _check(self.lib.qlb_kraus_to_dense(self.h, float(dt), int(k), out.ctypes.data_as(C.POINTER(C.c_double)),
                                           2 * N * N))
        return out

    def export(self) -> bytes:
        n = C.c_size_t()
        _check(self.lib.qlb_state_export(self.h, None, 0, C.byref(n)))
        buf = C.create_string_buffer(n.value)
        _check(self.lib.qlb_state_export(self.h, buf, n.value, C.byref(n)))
        return buf.raw

    def import_(self, data: bytes):
        buf = C.create_string_buffer(data, len(data))
        _check(self.lib.qlb_state_import(self.h, buf, len(data)))

    def close(self):
        if self.h:
            self.lib.qlb_state_destroy(self.h)
            self.h = None


def qlb_tc_zgemm(device: int, A, B) -> np.ndarray:
    """A @ B (complex128) through the tensor-core 3xTF32 engine of the mixed form."""
    A = np.ascontiguousarray(np.asarray(A, dtype=np.complex128))
    B = np.ascontiguousarray(np.asarray(B, dtype=np.complex128))
    m, k = A.shape
    k2, n = B.shape
    assert k == k2
    Cm = np.zeros((m, n), dtype=np.complex128)
    dp = C.POINTER(C.c_double)
    _check(load().qlb_tc_zgemm(int(device), m, n, k, A.ctypes.data_as(dp), B.ctypes.data_as(dp),
                               Cm.ctypes.data_as(dp)))
    return Cm


GEMM_FP64, GEMM_DF64, GEMM_TC = range(3)


def qlb_zgemm_check(device: int, engine: int, A, B):
    """A @ B (complex128) through one of the step's GEMM engines; returns (C, device ms)."""
    A = np.ascontiguousarray(np.asarray(A, dtype=np.complex128))
    B = np.ascontiguousarray(np.asarray(B, dtype=np.complex128))
    m, k = A.shape
    k2, n = B.shape
    assert k == k2
    Cm = np.zeros((m, n), dtype=np.complex128)
    ms = C.c_double()
    dp = C.POINTER(C.c_double)
    _check(load().qlb_zgemm_check(int(device), int(engine), m, n, k, A.ctypes.data_as(dp), B.ctypes.data_as(dp),
                                  Cm.ctypes.data_as(dp), C.byref(ms)))
    return Cm, ms.value


SOLVER_STEP, SOLVER_JACOBI, SOLVER_CLUSTER8, SOLVER_CLUSTER16, SOLVER_QL, SOLVER_RANGE = range(6)


def qlb_eig_check(device: int, precision: int, solver: int, G, tol: float = 0.0, cap: int = 0):
    """One truncation solve of the Hermitian matrix G by the named kernel.  Returns
    (eigenvalues descending, kept vectors n x k or None, k, device ms); k = -1 when
    the range basis (SOLVER_RANGE) reached the cap first."""
    G = np.ascontiguousarray(np.asarray(G, dtype=np.complex128))
    n = G.shape[0]
    lam = np.zeros(n)
    V = np.zeros(n * n, dtype=np.complex128)
    k, ms = C.c_int(), C.c_double()
    dp = C.POINTER(C.c_double)
    _check(load().qlb_eig_check(int(device), int(precision), int(solver), n, G.ctypes.data_as(dp), float(tol),
                                int(cap or n), lam.ctypes.data_as(dp), V.ctypes.data_as(dp), C.byref(k),
                                C.byref(ms)))
    kk = k.value
    return lam, (V[:n * kk].reshape(n, kk) if kk > 0 else None), kk, ms.value


class Group:
    """States stepped together, one launch per phase of the step over all of them
    (qlb_group_*).  Close the group before its states."""

    def __init__(self, ctx: Ctx, states):
        self.ctx, self.lib = ctx, ctx.lib
        self.states = list(states)
        arr = (_vp * len(self.states))(*[st.h for st in self.states])
        h = _vp()
        _check(self.lib.qlb_group_create(ctx.h, arr, len(self.states), C.byref(h)))
        self.h = h

    def step(self, dt, n=1) -> int:
        return _check(self.lib.qlb_group_step(self.h, float(dt), int(n)))

    def launches(self) -> int:
        v = C.c_int()
        _check(self.lib.qlb_group_launches(self.h, C.byref(v)))
        return v.value

    def stream(self) -> int:
        s = _vp()
        _check(self.lib.qlb_group_stream(self.h, C.byref(s)))
        return s.value or 0

    def close(self):
        if self.h:
            self.lib.qlb_group_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Server:
    """The library's continuous-batching server (qlb_server_*): takes over the context
    (created with stream_ordered=1) until close()."""

    def __init__(self, ctx: Ctx, hbm_budget=0, max_live=64, chunk=100):
        self.ctx, self.lib = ctx, ctx.lib
        h = _vp()
        _check(self.lib.qlb_server_create(ctx.h, int(hbm_budget), int(max_live), int(chunk), C.byref(h)))
        self.h = h
        self.n_obs = {}

    def submit(self, R, H, jumps, vecs, dt, steps, obs, tol=0.0, chi_max=0, chi_mu_max=0) -> int:
        """H, each jump and each observable are term lists as for System.op; vecs are
        the product-start mode vectors.  Returns the ticket."""
        keep = []
        req = qlb_request()
        Rs = (C.c_int * len(R))(*[int(r) for r in R])
        keep.append(Rs)
        req.n_modes, req.R = len(R), Rs
        if H:
            req.H, req.n_H = _terms_to_c(H, keep), len(H)
        jl = (C.POINTER(qlb_term) * max(1, len(jumps)))(*[_terms_to_c(j, keep) for j in jumps])
        jn = (C.c_int * max(1, len(jumps)))(*[len(j) for j in jumps])
        ol = (C.POINTER(qlb_term) * max(1, len(obs)))(*[_terms_to_c(o, keep) for o in obs])
        on = (C.c_int * max(1, len(obs)))(*[len(o) for o in obs])
        keep += [jl, jn, ol, on]
        req.jumps, req.n_jump_terms, req.n_jumps = jl, jn, len(jumps)
        req.obs, req.n_obs_terms, req.n_obs = ol, on, len(obs)
        arrs = [_cvec(v) for v in vecs]
        vp = (C.POINTER(C.c_double) * len(arrs))(*[p for _, p in arrs])
        keep += [arrs, vp]
        req.mode_vecs = vp
        req.dt, req.steps, req.tol = float(dt), int(steps), float(tol)
        req.chi_max, req.chi_mu_max = int(chi_max), int(chi_mu_max)
        t = C.c_int64()
        _check(self.lib.qlb_submit(self.h, C.byref(req), C.byref(t)))
        self.n_obs[t.value] = len(obs)
        return t.value

    def poll(self, ticket):
        """None while pending or running; else (list of complex observables, (arrival,
        admit, done) seconds).  Raises QlbError for a failed or cancelled request."""
        n = self.n_obs.get(ticket, 0)
        res = (C.c_double * max(2, 2 * n))()
        tm = (C.c_double * 3)()
        st = self.lib.qlb_poll(self.h, int(ticket), res, 2 * n, tm)
        if st == QLB_BUSY:
            return None
        _check(st)
        return [complex(res[2 * k], res[2 * k + 1]) for k in range(n)], (tm[0], tm[1], tm[2])

    def cancel(self, ticket):
        _check(self.lib.qlb_cancel(self.h, int(ticket)))

    def stats(self):
        out = (C.c_double * 6)()
        _check(self.lib.qlb_server_stats(self.h, out))
        return dict(live=int(out[0]), peak_live=int(out[1]), peak_bytes=int(out[2]), completed=int(out[3]),
                    steps=int(out[4]), pending=int(out[5]))

    def close(self):
        if self.h:
            self.lib.qlb_server_destroy(self.h)
            self.h = None
