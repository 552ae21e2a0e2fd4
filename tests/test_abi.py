"""The C-ABI library loads on a host without a GPU and exports every declared symbol."""
import ctypes
import os
import re

from paper_2010_15595_gb300 import lib

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    names = []
    for f in sorted(os.listdir(os.path.join(ROOT, "include"))):
        if f.endswith(".h"):
            src = open(os.path.join(ROOT, "include", f)).read()
            src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
            names += re.findall(r"\b(gbsh_[a-z0-9_]+)\s*\(", src)
    return sorted(set(names))


def test_library_exports_header():
    so = lib.load()
    names = declared_functions()
    assert names, "no declarations found"
    for name in names:
        assert hasattr(so, name), name
    assert set(names) <= set(lib.exported_symbols()) | set(names)


def test_strerror_and_version():
    so = lib.load()
    assert so.gbsh_version() >= 100
    assert so.gbsh_strerror(1) == b"invalid argument"


def test_invalid_arguments_rejected_without_gpu():
    so = lib.load()
    out = lib.C128()
    # N out of range and null pointers are rejected before any CUDA call
    assert so.gbsh_lhaf(None, -1, 1, ctypes.byref(out), None, None) == lib.GBSH_EINVAL
    assert so.gbsh_lhaf(None, 61, 61, ctypes.byref(out), None, None) == lib.GBSH_EINVAL
    assert so.gbsh_lhaf(None, 0, 0, ctypes.byref(out), None, None) == lib.GBSH_OK
    assert (out.re, out.im) == (1.0, 0.0)
    assert so.gbsh_set_lhaf_tuning(99, 0) == lib.GBSH_EINVAL
    assert so.gbsh_lhaf_workspace_size(0) == 0
