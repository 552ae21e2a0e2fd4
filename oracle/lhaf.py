"""ORACLE — test infrastructure only.

ctypes front end of the plain-C loop-hafnian oracle (lhaf_oracle.c). Every function takes
a numpy complex128 square matrix and returns Python complex numbers.

  lhaf_brute(A)        definition: sum over single-pair matchings (Sec. II, Eq. defhaf and
                       the loop-hafnian text after Eq. lhaf); N <= 20.
  haf_brute(A)         same over perfect matchings only (Eq. defhaf); diagonal ignored.
  lhaf_dp(A)           the definition as a memoised subset recursion; N <= 24.
  lhaf_subset(A)       the subset formula of the cited O(N^3 2^{N/2}) algorithm with power
                       traces from explicit matrix powers (Sec. II; benchmarked in Sec. IV).
  lhaf_subset_ld(A)    the same in long double, to estimate the double version's error.
  subset_terms(A, zs)  p_Z of individual subsets z, for sampled parity at large N.
"""
import ctypes
import os

import numpy as np

from . import build as _build

_lib = None


def _load():
    global _lib
    if _lib is None:
        path = _build.build()
        lib = ctypes.CDLL(path)
        dp = ctypes.POINTER(ctypes.c_double)
        for name in ("orc_lhaf_brute", "orc_lhaf_dp"):
            f = getattr(lib, name)
            f.argtypes = [dp, ctypes.c_int, ctypes.c_int, dp]
            f.restype = ctypes.c_int
        for name in ("orc_lhaf_subset", "orc_lhaf_subset_ld"):
            f = getattr(lib, name)
            f.argtypes = [dp, ctypes.c_int, ctypes.c_int, dp, dp]
            f.restype = ctypes.c_int
        lib.orc_lhaf_subset_stats.argtypes = [dp, ctypes.c_int, ctypes.c_int, dp, dp, dp]
        lib.orc_lhaf_subset_stats.restype = ctypes.c_int
        lib.orc_subset_terms.argtypes = [dp, ctypes.c_int,
                                         ctypes.POINTER(ctypes.c_uint64), ctypes.c_int,
                                         ctypes.c_int, dp]
        lib.orc_subset_terms.restype = ctypes.c_int
        _lib = lib
    return _lib


def _mat(A):
    A = np.ascontiguousarray(A, dtype=np.complex128)
    if A.ndim != 2 or A.shape[0] != A.shape[1]:
        raise ValueError("square matrix expected")
    return A


def _ptr(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _threads(nthreads):
    if nthreads is None:
        nthreads = int(os.environ.get("ORACLE_THREADS", "0")) or (os.cpu_count() or 1)
    return int(nthreads)


def lhaf_brute(A):
    A = _mat(A)
    out = np.zeros(2)
    if _load().orc_lhaf_brute(_ptr(A), A.shape[0], 1, _ptr(out)):
        raise ValueError("N too large for brute force")
    return complex(out[0], out[1])


def haf_brute(A):
    A = _mat(A)
    out = np.zeros(2)
    if _load().orc_lhaf_brute(_ptr(A), A.shape[0], 0, _ptr(out)):
        raise ValueError("N too large for brute force")
    return complex(out[0], out[1])


def lhaf_dp(A, with_loops=True):
    A = _mat(A)
    out = np.zeros(2)
    if _load().orc_lhaf_dp(_ptr(A), A.shape[0], 1 if with_loops else 0, _ptr(out)):
        raise ValueError("N too large for the subset recursion")
    return complex(out[0], out[1])


def lhaf_subset(A, nthreads=None, return_abs_sum=False):
    A = _mat(A)
    out = np.zeros(2)
    asum = np.zeros(1)
    if _load().orc_lhaf_subset(_ptr(A), A.shape[0], _threads(nthreads), _ptr(out), _ptr(asum)):
        raise ValueError("bad size")
    val = complex(out[0], out[1])
    return (val, float(asum[0])) if return_abs_sum else val


def lhaf_subset_stats(A, nthreads=None):
    """(lhaf, sum_Z |p_Z|, sum_Z |p_Z|^2) by the subset formula in double."""
    A = _mat(A)
    out = np.zeros(2)
    asum = np.zeros(1)
    sq = np.zeros(1)
    if _load().orc_lhaf_subset_stats(_ptr(A), A.shape[0], _threads(nthreads), _ptr(out),
                                     _ptr(asum), _ptr(sq)):
        raise ValueError("bad size")
    return complex(out[0], out[1]), float(asum[0]), float(sq[0])


def lhaf_subset_ld(A, nthreads=None, return_abs_sum=False):
    A = _mat(A)
    out = np.zeros(2)
    asum = np.zeros(1)
    if _load().orc_lhaf_subset_ld(_ptr(A), A.shape[0], _threads(nthreads), _ptr(out),
                                  _ptr(asum)):
        raise ValueError("bad size")
    val = complex(out[0], out[1])
    return (val, float(asum[0])) if return_abs_sum else val


def subset_terms(A, zs, nthreads=None):
    """p_Z for each subset z (bit j <=> pair (j, j+n) of the matrix padded to even size)."""
    A = _mat(A)
    zs = np.ascontiguousarray(zs, dtype=np.uint64)
    out = np.zeros(2 * len(zs))
    if _load().orc_subset_terms(_ptr(A), A.shape[0],
                                zs.ctypes.data_as(ctypes.POINTER(ctypes.c_uint64)),
                                len(zs), _threads(nthreads), _ptr(out)):
        raise ValueError("bad size")
    return out[0::2] + 1j * out[1::2]


def haf(A, nthreads=None):
    """Hafnian (diagonal ignored) through the subset formula with zero loop weights."""
    A = _mat(A).copy()
    np.fill_diagonal(A, 0)
    if A.shape[0] % 2:
        return 0j
    return lhaf_subset(A, nthreads)
