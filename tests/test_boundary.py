"""The C ABI library builds for sm_103a, loads, and exports every function
include/*.h declares (no GPU needed: no compute call is made)."""
import ctypes
import glob
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    names = set()
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        src = open(h).read()
        src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
        src = re.sub(r"//[^\n]*", "", src)
        for m in re.finditer(r"\b(hg_[a-z0-9_]+)\s*\(", src):
            names.add(m.group(1))
    return sorted(names)


@pytest.fixture(scope="module")
def libpath():
    from paper_2606_00352_gb300 import build
    return build.build()


def test_header_declares_entry_points():
    names = declared_functions()
    for must in ("hg_create_scene", "hg_render", "hg_render_backward", "hg_ctx_create", "hg_state_read"):
        assert must in names


def test_library_exports_every_declared_symbol(libpath):
    lib = ctypes.CDLL(libpath)
    missing = [n for n in declared_functions() if not hasattr(lib, n)]
    assert not missing, f"not exported: {missing}"


def test_status_strings_without_gpu(libpath):
    lib = ctypes.CDLL(libpath)
    lib.hg_status_str.restype = ctypes.c_char_p
    assert lib.hg_status_str(0) == b"ok"
    assert b"capacity" in lib.hg_status_str(-4)
    lib.hg_version.restype = ctypes.c_char_p
    assert b"sm_103a" in lib.hg_version()


def test_binding_refuses_missing_library(tmp_path):
    from paper_2606_00352_gb300 import higs
    saved = higs._lib
    higs._lib = None
    try:
        with pytest.raises(RuntimeError):
            higs.load(str(tmp_path / "nope.so"))
    finally:
        higs._lib = saved
