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


def test_tuning_table_set_get_reset_without_gpu():
    """The launch-shape table is host state: entries can be set, read back and reset to the
    built-in (measured) entry without a GPU, and out-of-range values are refused."""
    from paper_2010_15595_gb300 import autotune
    for prec in (lib.PREC_FP64, lib.PREC_TF):
        builtin = lib.get_lhaf_tuning(prec, 40)
        lib.set_lhaf_tuning(prec, 40, 10, lib.LADDER_FINE, 16)
        assert lib.get_lhaf_tuning(prec, 40) == (10, lib.LADDER_FINE, 16)
        lib.set_lhaf_tuning(prec, 40)  # all zero: back to the built-in entry
        assert lib.get_lhaf_tuning(prec, 40) == builtin
        assert autotune.library_default(prec)[1] == lib.LADDER_COARSE
    b = lib.get_batch_tuning(lib.PREC_FP64, 15)
    lib.set_batch_tuning(lib.PREC_FP64, 15, 6, warps_small=12)
    assert lib.get_batch_tuning(lib.PREC_FP64, 15) == (12, 6)
    lib.set_batch_tuning(lib.PREC_FP64, 15, 0, warps_small=0)
    assert lib.get_batch_tuning(lib.PREC_FP64, 15) == b
    so = lib.load()
    assert so.gbsh_set_lhaf_tuning_ex(lib.PREC_FP64, 40, 17, 0, 0) == lib.GBSH_EINVAL
    assert so.gbsh_set_lhaf_tuning_ex(lib.PREC_FP64, 40, 0, 3, 0) == lib.GBSH_EINVAL
    assert so.gbsh_set_lhaf_tuning_ex(lib.PREC_FP64, 40, 0, 0, 19) == lib.GBSH_EINVAL
    assert so.gbsh_set_lhaf_tuning_ex(lib.PREC_C32, 40, 8, 0, 0) == lib.GBSH_EINVAL
    assert so.gbsh_set_lhaf_tuning_ex(lib.PREC_FP64, 61, 8, 0, 0) == lib.GBSH_EINVAL
    assert so.gbsh_set_batch_tuning_ex(lib.PREC_MIXED, 15, 8, 8) == lib.GBSH_EINVAL
    assert so.gbsh_set_batch_tuning_ex(lib.PREC_FP64, 31, 8, 8) == lib.GBSH_EINVAL
    assert lib.builtin_tuning_entries() >= 0


def test_autotune_table_emission():
    """Tuned sizes become table rows covering N up to the next tuned size; rows equal to the
    library default are dropped; the emitted C source lists them before the sentinel."""
    from paper_2010_15595_gb300 import autotune
    fp, tf = lib.PREC_FP64, lib.PREC_TF
    res = {(fp, 24): autotune.library_default(fp), (fp, 32): (10, 2, 18), (fp, 40): (12, 1, 16),
           (tf, 40): (14, 2, 17)}
    rows = autotune.table_entries(res)
    assert rows == [(fp, 32, 39, 10, 2, 18), (fp, 40, 60, 12, 1, 16), (tf, 1, 60, 14, 2, 17)]
    src = autotune.emit_table(rows, [(fp, 1, 30, 12, 6)], "note")
    assert src.index("{0, 32, 39, 10, 2, 18},") < src.index("{-1, 0, 0, 0, 0, 0},")
    assert "{0, 1, 30, 12, 6}," in src and "// note" in src


def test_builtin_tuning_table_applied_by_default():
    """Every row of the committed measured table (csrc/tuned_gb300.inc) is what the library
    reports for its sizes in a fresh process state, without any cache file."""
    import re
    path = os.path.join(ROOT, "paper_2010_15595_gb300", "csrc", "tuned_gb300.inc")
    src = open(path).read()
    single = src.split("kTunedSingle[]")[1].split("};")[0]
    rows = [tuple(int(x) for x in m.groups())
            for m in re.finditer(r"\{(-?\d+), (\d+), (\d+), (\d+), (\d+), (\d+)\}", single)]
    rows = [r for r in rows if r[0] >= 0]
    assert lib.builtin_tuning_entries() >= len(rows) >= 1
    for prec, lo, hi, w, ladder, chunks in rows:
        for N in {lo, (lo + hi) // 2, hi}:
            lib.set_lhaf_tuning(prec, N)  # reset to the built-in entry
            assert lib.get_lhaf_tuning(prec, N) == (w, ladder, chunks), (prec, N)
