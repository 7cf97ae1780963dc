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


def test_solver_shape_options_validated():
    # (threads per system, blocks per SM) pairs without a compiled solver are refused
    from paper_2511_17634_gb300 import kp as K
    L = K.lib()
    import ctypes
    for bt, mb, ok in [(0, 0, True), (256, 3, True), (128, 4, True), (64, 4, True),
                       (256, 4, False), (64, 2, False), (96, 0, False), (128, -1, False)]:
        o = K._Options()
        L.kp_options_default(ctypes.byref(o))
        o.block_threads, o.blocks_per_sm = bt, mb
        h = ctypes.c_void_p()
        st = L.kp_create(ctypes.byref(h), ctypes.byref(o), None)
        if ok:
            # no GPU here: creation may fail later at the CUDA step, never at validation
            assert st != K.ERR_ARG, (bt, mb)
        else:
            assert st == K.ERR_ARG, (bt, mb)
        if h:
            L.kp_destroy(h)


def test_cluster_size_option_validated():
    # CTAs per system for mixed precision: 0 (automatic), 2, 4, 8 or 16
    from paper_2511_17634_gb300 import kp as K
    L = K.lib()
    import ctypes
    for cs, ok in [(0, True), (2, True), (4, True), (8, True), (16, True), (3, False), (32, False),
                   (-2, False)]:
        o = K._Options()
        L.kp_options_default(ctypes.byref(o))
        assert o.cluster_size == 0
        o.cluster_size = cs
        h = ctypes.c_void_p()
        st = L.kp_create(ctypes.byref(h), ctypes.byref(o), None)
        if ok:
            assert st != K.ERR_ARG, cs
        else:
            assert st == K.ERR_ARG, cs
        if h:
            L.kp_destroy(h)


def test_ctypes_structs_match_the_header_layout(tmp_path):
    # the binding's ctypes structures against the C compiler's layout of the
    # same structs in include/kp.h: size and the offset of every field
    import ctypes
    import subprocess
    from paper_2511_17634_gb300 import kp as K
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    pairs = {"kp_options": K._Options, "kp_group": K._Group, "kp_march_opts": K._MarchOpts,
             "kp_step_stats": K.StepStats, "kp_march_timing": K.MarchTiming}
    lines = ['#include <stddef.h>', '#include <stdio.h>', '#include "kp.h"', 'int main(void) {']
    for cname, py in pairs.items():
        lines.append(f'  printf("{cname} size %zu\\n", sizeof({cname}));')
        for fname, _ in py._fields_:
            lines.append(f'  printf("{cname} {fname} %zu\\n", offsetof({cname}, {fname}));')
    cfields = {"H": "H", "W": "W", "dt": "dt", "g2": "g2", "h": "h", "mt": "mtilde", "fx": "fx",
               "fy": "fy"}
    lines.append('  printf("kp_op size %zu\\n", sizeof(kp_op));')
    for name, cf in cfields.items():
        lines.append(f'  printf("kp_op {name} %zu\\n", offsetof(kp_op, {cf}));')
    lines += ['  return 0;', '}']
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines) + "\n")
    exe = tmp_path / "layout"
    subprocess.run(["gcc", "-std=c11", "-I", os.path.join(root, "include"), str(src), "-o", str(exe)],
                   check=True, capture_output=True)
    out = subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout.split("\n")
    got = {}
    for ln in out:
        if ln:
            parts = ln.split()
            got[(parts[0], parts[1])] = int(parts[2])
    for cname, py in pairs.items():
        assert got[(cname, "size")] == ctypes.sizeof(py), cname
        for fname, _ in py._fields_:
            assert got[(cname, fname)] == getattr(py, fname).offset, (cname, fname)
    assert got[("kp_op", "size")] == K.OP_DTYPE.itemsize
    for name in cfields:
        assert got[("kp_op", name)] == K.OP_DTYPE.fields[name][1], name
