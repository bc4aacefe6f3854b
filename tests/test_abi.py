"""The C-ABI library builds, loads without a GPU and exports every symbol that
include/qlb.h declares (no compute calls)."""
import ctypes
import os
import re

import pytest


def _declared(root):
    with open(os.path.join(root, "include", "qlb.h")) as f:
        text = f.read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(qlb_[a-z0-9_]+)\s*\(", text)))


def test_header_declares_the_boundary(repo_root):
    names = _declared(repo_root)
    for n in ["qlb_create", "qlb_system_create", "qlb_op_build", "qlb_state_init_product", "qlb_truncate",
              "qlb_step", "qlb_expectation", "qlb_fidelity"]:
        assert n in names


def test_library_exports_every_declared_symbol(repo_root):
    from paper_2605_27515_gb300 import build

    lib_path = build.build()
    lib = ctypes.CDLL(lib_path)
    missing = [n for n in _declared(repo_root) if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_covers_the_header(repo_root):
    from paper_2605_27515_gb300 import qlb

    assert set(_declared(repo_root)) <= set(qlb._SIGS)


def test_binding_fails_loudly_without_library(tmp_path):
    from paper_2605_27515_gb300 import qlb

    with pytest.raises(qlb.QlbError):
        qlb._lib_backup = qlb._lib
        qlb._lib = None
        try:
            qlb.load(str(tmp_path / "missing.so"))
        finally:
            qlb._lib = qlb._lib_backup
