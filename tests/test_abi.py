"""The C-ABI library builds for sm_103a, loads, and exports every entry point
that include/kp.h declares (no GPU needed: nothing here launches work)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    src = open(os.path.join(ROOT, "include", "kp.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(kp_[a-z_0-9]+)\s*\(", src)))


def test_header_declares_the_boundary():
    names = _declared()
    for f in ("kp_seed_solve", "kp_store_basis", "kp_project_targets", "kp_refine", "kp_apply",
              "kp_rhs", "kp_create", "kp_destroy"):
        assert f in names


def test_library_builds_loads_and_exports_all_symbols():
    from paper_2511_17634_gb300 import build
    path = build.build()
    lib = ctypes.CDLL(path)
    for name in _declared():
        assert hasattr(lib, name), name
    lib.kp_version.restype = ctypes.c_char_p
    assert b"sm_103a" in lib.kp_version()


def test_binding_fails_loudly_without_library(monkeypatch, tmp_path):
    from paper_2511_17634_gb300 import kp
    monkeypatch.setattr(kp, "LIB_PATH", str(tmp_path / "missing.so"))
    monkeypatch.setattr(kp, "_lib", None)
    with pytest.raises(ImportError):
        kp.lib()
