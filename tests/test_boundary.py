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


def test_noalloc_sort_argument_checks_without_gpu():
    """The binding rejects malformed tensors before it calls the library."""
    import torch
    from paper_2606_00352_gb300 import higs
    n = 16
    off = torch.tensor([0, n], dtype=torch.int32)
    k = torch.zeros(n, dtype=torch.int32)
    good = (off, k, k.clone(), k.clone(), k.clone())
    higs.check_sort_args(*good, require_cuda=False)
    with pytest.raises(ValueError, match="CUDA"):
        higs.check_sort_args(*good)
    bad_cases = [
        ((off.to(torch.int64),) + good[1:], "seg_off must be int32"),
        ((off[:1],) + good[1:], "at least 2"),
        ((off, k.to(torch.int64)) + good[2:], "4-byte"),
        ((off, k, k[:n - 1].clone(), k.clone(), k.clone()), "elements"),
        ((off, k, k.clone(), torch.zeros(2 * n, dtype=torch.int32)[::2], k.clone()), "contiguous"),
        ((off, k, k.clone(), k.clone(), k[:4].clone()), "elements"),
    ]
    for args, msg in bad_cases:
        with pytest.raises(ValueError, match=msg):
            higs.check_sort_args(*args, require_cuda=False)
