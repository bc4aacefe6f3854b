"""Host-side behaviour of the C-ABI that needs no GPU: documented defaults,
argument checks that return status codes before any device work, and a clean
QLB_EDEVICE when no device is present."""
import ctypes as C

import pytest

from paper_2605_27515_gb300 import qlb as Q


@pytest.fixture(scope="module")
def lib():
    from paper_2605_27515_gb300 import build

    build.build()
    return Q.load()


def test_default_options_match_the_header(lib):
    o = Q.qlb_options()
    lib.qlb_default_options(C.byref(o))
    assert o.device == 0 and o.precision == Q.PREC_F64
    assert o.tol == 1e-12 and o.chi_max == 64 and o.chi_mu_max == 16
    assert o.zip_tol_factor == 1e-6 and o.degeneracy_gap == 1e-10 and o.max_sweeps == 40
    assert o.hbm_budget == 0 and o.stream_ordered == 0


@pytest.mark.parametrize("field,value", [("precision", 7), ("tol", 1.5), ("chi_max", 0), ("chi_max", 1000),
                                         ("chi_mu_max", 0), ("max_sweeps", 0)])
def test_create_rejects_bad_options(lib, field, value):
    o = Q.qlb_options()
    lib.qlb_default_options(C.byref(o))
    setattr(o, field, value)
    h = C.c_void_p()
    assert lib.qlb_create(C.byref(o), C.byref(h)) == Q.EINVAL
    assert not h.value
    assert lib.qlb_last_error()  # a message is left for the caller


def test_null_handles_are_codes_not_crashes(lib):
    assert lib.qlb_create(None, None) == Q.EINVAL
    assert lib.qlb_step(None, 1e-3, 1) == Q.EINVAL
    assert lib.qlb_set_scheme(None, 2) == Q.EINVAL
    assert lib.qlb_add_jump(None, None) == Q.EINVAL
    out = C.c_double()
    assert lib.qlb_purity(None, C.byref(out)) == Q.EINVAL
    assert lib.qlb_purity_noalloc(None, C.byref(out)) == Q.EINVAL


def test_no_device_gives_a_status(lib):
    import torch

    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    h = C.c_void_p()
    assert lib.qlb_create(None, C.byref(h)) == Q.EDEVICE
    assert b"device" in lib.qlb_last_error()


def test_group_calls_check_their_arguments(lib):
    """The group calls return QLB_EINVAL for missing handles and impossible sizes
    before touching a device."""
    out = C.c_void_p()
    arr = (C.c_void_p * 1)(None)
    assert lib.qlb_group_create(None, arr, 1, C.byref(out)) == Q.EINVAL
    fake_ctx = C.c_void_p(1)  # never dereferenced: the size check comes first
    assert lib.qlb_group_create(fake_ctx, arr, 0, C.byref(out)) == Q.EINVAL
    assert lib.qlb_group_create(fake_ctx, arr, 5000, C.byref(out)) == Q.EINVAL
    assert lib.qlb_group_create(fake_ctx, arr, 1, C.byref(out)) == Q.EINVAL  # null state
    assert not out.value
    assert lib.qlb_group_step(None, 1e-3, 1) == Q.EINVAL
    n = C.c_int()
    assert lib.qlb_group_launches(None, C.byref(n)) == Q.EINVAL
    s = C.c_void_p()
    assert lib.qlb_group_stream(None, C.byref(s)) == Q.EINVAL
    lib.qlb_group_destroy(None)  # a no-op
