"""Python binding of the loop-hafnian engine's C ABI (include/gbsh.h).

Argument marshalling only: every step of the computation runs in the CUDA kernels of
libgbsh.so. Matrices may be numpy arrays (host memory) or torch tensors (host or CUDA);
PyTorch serves as the device-memory and stream provider. The binding raises if the
compiled library is missing -- there is no fallback implementation.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_build", "libgbsh.so")

GBSH_OK, GBSH_EINVAL, GBSH_ENOMEM, GBSH_ECUDA, GBSH_ETIMEOUT, GBSH_PENDING, GBSH_ENOTFOUND = range(7)
MAX_N = 60
NOALLOC_SCRATCH_BYTES = 8 << 20  # GBSH_NOALLOC_SCRATCH_BYTES
PREC_FP64, PREC_C32, PREC_MIXED, PREC_DD, PREC_TF = 0, 1, 2, 3, 4
# Largest N for which the complex-FP32 per-subset variant is enabled (GBSH_C32_MAX_N): its
# measured error against the FP64 path stays <= 1e-5 relative up to this size.
C32_MAX_N = 4


class GbshError(RuntimeError):
    def __init__(self, code: int, what: str):
        self.code = code
        super().__init__(f"{what}: {_strerror(code)} (status {code})")


class C128(ctypes.Structure):
    _fields_ = [("re", ctypes.c_double), ("im", ctypes.c_double)]


_lib = None


def load() -> ctypes.CDLL:
    """Loads libgbsh.so (built by paper_2010_15595_gb300.build); raises if it is absent."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise ImportError(f"{LIB_PATH} is missing: build it with "
                          "`python -c 'import __graft_entry__ as g; g.build()'`")
    lib = ctypes.CDLL(LIB_PATH)
    vp, i, d, sz = ctypes.c_void_p, ctypes.c_int, ctypes.c_double, ctypes.c_size_t
    pc = ctypes.POINTER(C128)
    pd = ctypes.POINTER(ctypes.c_double)
    sig = {
        "gbsh_strerror": ([i], ctypes.c_char_p),
        "gbsh_version": ([], i),
        "gbsh_lhaf": ([vp, i, i, pc, pd, vp], i),
        "gbsh_lhaf_workspace_size": ([i], sz),
        "gbsh_lhaf_async": ([vp, i, i, vp, vp, vp, sz, vp], i),
        "gbsh_gbs_prob": ([vp, i, i, vp, ctypes.POINTER(ctypes.c_int), d, pd, pc, vp], i),
        "gbsh_subset_terms": ([vp, i, i, vp, i, vp, vp], i),
        "gbsh_visit_counts": ([i, vp, vp], i),
        "gbsh_set_lhaf_tuning": ([i, i], i),
        "gbsh_lhaf_plan": ([i] + [ctypes.POINTER(ctypes.c_int)] * 5, i),
        "gbsh_lhaf_ex": ([vp, i, i, i, pc, pd, vp], i),
        "gbsh_lhaf_async_ex": ([vp, i, i, i, vp, vp, vp, sz, vp], i),
        "gbsh_lhaf_workspace_size_ex": ([i, i], sz),
        "gbsh_subset_terms_ex": ([vp, i, i, i, vp, i, vp, vp], i),
        "gbsh_lhaf_plan_ex": ([i, i] + [ctypes.POINTER(ctypes.c_int)] * 5, i),
        "gbsh_lhaf_noalloc": ([vp, i, i, vp, vp, vp], i),
        "gbsh_lhaf_noalloc_plan": ([i, ctypes.POINTER(ctypes.c_int)], i),
        "gbsh_lhaf_range_async": ([vp, i, i, i, ctypes.c_uint64, ctypes.c_uint64, vp, vp, sz, vp], i),
        "gbsh_combine_partials": ([vp, i, vp], i),
        "gbsh_lhaf_batch": ([vp, vp, vp, i, vp, vp, i, vp], i),
        "gbsh_gbs_prob_batch": ([vp, i, i, vp, ctypes.c_int64, vp, i, vp, vp, vp, i, vp], i),
        "gbsh_set_batch_tuning": ([i, i, i], i),
        "gbsh_set_batch_tuning_ex": ([i, i, i, i], i),
        "gbsh_set_lhaf_tuning_ex": ([i, i, i, i, i], i),
        "gbsh_get_lhaf_tuning": ([i, i] + [ctypes.POINTER(ctypes.c_int)] * 3, i),
        "gbsh_get_batch_tuning": ([i, i] + [ctypes.POINTER(ctypes.c_int)] * 2, i),
        "gbsh_builtin_tuning_entries": ([], i),
        "gbsh_set_batch_graphs": ([i], i),
        "gbsh_batch_graph_stats": ([ctypes.POINTER(ctypes.c_longlong), ctypes.POINTER(ctypes.c_longlong)], i),
    }
    for name, (args, res) in sig.items():
        f = getattr(lib, name)
        f.argtypes = args
        f.restype = res
    _lib = lib
    return lib


def exported_symbols():
    return ["gbsh_strerror", "gbsh_version", "gbsh_lhaf", "gbsh_lhaf_workspace_size",
            "gbsh_lhaf_async", "gbsh_gbs_prob", "gbsh_subset_terms", "gbsh_visit_counts",
            "gbsh_set_lhaf_tuning", "gbsh_lhaf_plan", "gbsh_lhaf_noalloc", "gbsh_lhaf_batch",
            "gbsh_gbs_prob_batch", "gbsh_set_batch_tuning", "gbsh_set_batch_graphs",
            "gbsh_batch_graph_stats", "gbsh_lhaf_ex", "gbsh_lhaf_async_ex",
            "gbsh_lhaf_workspace_size_ex", "gbsh_subset_terms_ex", "gbsh_lhaf_plan_ex",
            "gbsh_lhaf_noalloc_plan", "gbsh_lhaf_range_async", "gbsh_combine_partials",
            "gbsh_set_batch_tuning_ex", "gbsh_set_lhaf_tuning_ex", "gbsh_get_lhaf_tuning",
            "gbsh_get_batch_tuning", "gbsh_builtin_tuning_entries"]


def _strerror(code: int) -> str:
    try:
        return load().gbsh_strerror(code).decode()
    except Exception:  # library not loadable: keep the numeric code
        return "status"


def _check(rc: int, what: str):
    if rc != GBSH_OK:
        raise GbshError(rc, what)


def _stream_handle(stream) -> int:
    if stream is None:
        import torch
        if torch.cuda.is_available():
            return torch.cuda.current_stream().cuda_stream
        return 0
    return int(getattr(stream, "cuda_stream", stream))


def _as_matrix(A):
    """(pointer, N, ld, keepalive) for a square complex128 numpy array or torch tensor."""
    try:
        import torch
        if isinstance(A, torch.Tensor):
            if A.dtype != torch.complex128 or A.dim() != 2 or A.shape[0] != A.shape[1]:
                raise ValueError("square complex128 tensor expected")
            if A.stride(1) != 1:
                A = A.contiguous()
            return A.data_ptr(), A.shape[0], A.stride(0), A
    except ImportError:
        pass
    A = np.ascontiguousarray(A, dtype=np.complex128)
    if A.ndim != 2 or A.shape[0] != A.shape[1]:
        raise ValueError("square matrix expected")
    return A.ctypes.data, A.shape[0], A.shape[0], A


def version() -> int:
    return load().gbsh_version()


def set_tuning(warps_per_cta: int = 0, kcap: int = 0):
    """Process-wide launch-shape override of single evaluations ((0, 0) = tuning table)."""
    _check(load().gbsh_set_lhaf_tuning(warps_per_cta, kcap), "gbsh_set_lhaf_tuning")


LADDER_COARSE, LADDER_FINE = 1, 2


def set_lhaf_tuning(precision: int, N: int, warps_cap: int = 0, ladder: int = 0,
                    log2_chunks: int = 0):
    """Tuning-table entry of single evaluations of size N (all zero = built-in entry)."""
    _check(load().gbsh_set_lhaf_tuning_ex(precision, N, warps_cap, ladder, log2_chunks),
           "gbsh_set_lhaf_tuning_ex")


def get_lhaf_tuning(precision: int, N: int):
    """(warps_cap, ladder, log2_chunks) of the current entry; 0 = library default."""
    v = [ctypes.c_int(0) for _ in range(3)]
    _check(load().gbsh_get_lhaf_tuning(precision, N, *[ctypes.byref(x) for x in v]),
           "gbsh_get_lhaf_tuning")
    return tuple(x.value for x in v)


def get_batch_tuning(precision: int, n_max: int):
    """(warps_small, warps_large) of the current batched entry; 0 = library default."""
    v = [ctypes.c_int(0) for _ in range(2)]
    _check(load().gbsh_get_batch_tuning(precision, n_max, *[ctypes.byref(x) for x in v]),
           "gbsh_get_batch_tuning")
    return tuple(x.value for x in v)


def builtin_tuning_entries() -> int:
    return load().gbsh_builtin_tuning_entries()


def lhaf(A, stream=None, return_error=False, precision=None):
    """Loop hafnian of a square complex matrix (numpy array or torch tensor, host or CUDA).
    precision: None (gbsh_lhaf, FP64), PREC_FP64 or PREC_TF (gbsh_lhaf_ex)."""
    ptr, N, ld, keep = _as_matrix(A)
    out = C128()
    err = ctypes.c_double()
    st = ctypes.c_void_p(_stream_handle(stream))
    if precision is None:
        rc = load().gbsh_lhaf(ctypes.c_void_p(ptr if N else 0), N, max(ld, N), ctypes.byref(out),
                              ctypes.byref(err), st)
        _check(rc, "gbsh_lhaf")
    else:
        rc = load().gbsh_lhaf_ex(ctypes.c_void_p(ptr if N else 0), N, max(ld, N), int(precision),
                                 ctypes.byref(out), ctypes.byref(err), st)
        _check(rc, "gbsh_lhaf_ex")
    val = complex(out.re, out.im)
    return (val, err.value) if return_error else val


def plan(N: int, precision=None) -> dict:
    """Launch plan of an N x N evaluation on the current device (see gbsh_lhaf_plan)."""
    vals = [ctypes.c_int() for _ in range(5)]
    refs = [ctypes.byref(v) for v in vals]
    if precision is None:
        _check(load().gbsh_lhaf_plan(N, *refs), "gbsh_lhaf_plan")
    else:
        _check(load().gbsh_lhaf_plan_ex(N, int(precision), *refs), "gbsh_lhaf_plan_ex")
    keys = ["nclass", "kernels", "warps", "kcap", "nchunks"]
    return {k: v.value for k, v in zip(keys, vals)}


def workspace_size(N: int, precision=None) -> int:
    if precision is None:
        return int(load().gbsh_lhaf_workspace_size(N))
    return int(load().gbsh_lhaf_workspace_size_ex(N, int(precision)))


def lhaf_async(dA, d_out, workspace, d_abs_sum=None, stream=None, precision=None):
    """Device-only variant: dA (CUDA complex128 N x N), d_out (CUDA complex128, >= 1 entry),
    workspace (CUDA uint8 tensor of >= workspace_size(N, precision) bytes). No
    synchronisation. precision: None (gbsh_lhaf_async), PREC_FP64 or PREC_TF."""
    ptr, N, ld, _ = _as_matrix(dA)
    args = (ctypes.c_void_p(d_out.data_ptr()),
            ctypes.c_void_p(d_abs_sum.data_ptr() if d_abs_sum is not None else 0),
            ctypes.c_void_p(workspace.data_ptr()), workspace.numel() * workspace.element_size(),
            ctypes.c_void_p(_stream_handle(stream)))
    if precision is None:
        rc = load().gbsh_lhaf_async(ctypes.c_void_p(ptr), N, ld, *args)
        _check(rc, "gbsh_lhaf_async")
    else:
        rc = load().gbsh_lhaf_async_ex(ctypes.c_void_p(ptr), N, ld, int(precision), *args)
        _check(rc, "gbsh_lhaf_async_ex")


def lhaf_noalloc(dA, d_out, d_abs_sum=None, stream=None):
    """gbsh_lhaf_noalloc: like lhaf_async, but the scratch memory is a fixed array inside
    the library, for callers that must not allocate device memory. No synchronisation."""
    ptr, N, ld, _ = _as_matrix(dA)
    rc = load().gbsh_lhaf_noalloc(
        ctypes.c_void_p(ptr), N, ld, ctypes.c_void_p(d_out.data_ptr()),
        ctypes.c_void_p(d_abs_sum.data_ptr() if d_abs_sum is not None else 0),
        ctypes.c_void_p(_stream_handle(stream)))
    _check(rc, "gbsh_lhaf_noalloc")


def lhaf_range(dA, i_begin: int, i_end: int, precision=PREC_FP64, stream=None):
    """Compensated partial (re_hi, re_lo, im_hi, im_lo, sum|p|) of the subsets with
    enumeration indices in [i_begin, i_end) (gbsh_lhaf_range_async), as a numpy array;
    synchronises the stream."""
    import torch
    ptr, N, ld, _ = _as_matrix(dA)
    ws = torch.empty(workspace_size(N, precision), dtype=torch.uint8, device=dA.device)
    part = torch.empty(5, dtype=torch.float64, device=dA.device)
    st = ctypes.c_void_p(_stream_handle(stream))
    rc = load().gbsh_lhaf_range_async(ctypes.c_void_p(ptr), N, ld, int(precision), int(i_begin),
                                      int(i_end), ctypes.c_void_p(part.data_ptr()),
                                      ctypes.c_void_p(ws.data_ptr()), ws.numel(), st)
    _check(rc, "gbsh_lhaf_range_async")
    out = part.cpu().numpy()
    return out


def combine_partials(partials) -> np.ndarray:
    """gbsh_combine_partials: fixed-order compensated sum of range partials (k x 5)."""
    p = np.ascontiguousarray(partials, dtype=np.float64).reshape(-1, 5)
    out = np.zeros(5)
    _check(load().gbsh_combine_partials(ctypes.c_void_p(p.ctypes.data), p.shape[0],
                                        ctypes.c_void_p(out.ctypes.data)), "gbsh_combine_partials")
    return out


def partial_value(p) -> complex:
    """The complex value (re_hi + re_lo) + i (im_hi + im_lo) of a (combined) partial."""
    return complex(p[0] + p[1], p[2] + p[3])


def range_bounds(N: int, rank: int, world: int):
    """[i_begin, i_end) of rank `rank` when the 2^n enumeration indices of an N x N loop
    hafnian are split into `world` contiguous ranges of (nearly) equal length."""
    n = (N + (N & 1)) // 2
    total = 1 << n
    return total * rank // world, total * (rank + 1) // world


def noalloc_chunks(N: int) -> int:
    """Chunks gbsh_lhaf_noalloc uses for size N (raises GbshError(GBSH_ENOMEM) when none fit)."""
    c = ctypes.c_int()
    _check(load().gbsh_lhaf_noalloc_plan(N, ctypes.byref(c)), "gbsh_lhaf_noalloc_plan")
    return c.value


def gbs_prob(B, gamma, pattern, p_vac=1.0, stream=None, return_lhaf=False):
    """Eq. lhaf-pure: p_vac |lhaf(filldiag(B_S, gamma_S))|^2 / prod s_i!."""
    bptr, M, ld, keepB = _as_matrix(B)
    try:
        import torch
        is_t = isinstance(gamma, torch.Tensor)
    except ImportError:
        is_t = False
    if is_t:
        g = gamma.contiguous()
        gptr = g.data_ptr()
    else:
        g = np.ascontiguousarray(gamma, dtype=np.complex128)
        gptr = g.ctypes.data
    pat = np.ascontiguousarray(pattern, dtype=np.int32)
    if pat.shape != (M,):
        raise ValueError("pattern must have one entry per mode")
    prob = ctypes.c_double()
    lh = C128()
    rc = load().gbsh_gbs_prob(ctypes.c_void_p(bptr), M, ld, ctypes.c_void_p(gptr),
                              pat.ctypes.data_as(ctypes.POINTER(ctypes.c_int)), float(p_vac),
                              ctypes.byref(prob), ctypes.byref(lh),
                              ctypes.c_void_p(_stream_handle(stream)))
    _check(rc, "gbsh_gbs_prob")
    return (prob.value, complex(lh.re, lh.im)) if return_lhaf else prob.value


def subset_terms(dA, d_z, stream=None, precision=None):
    """p_Z for the subsets in d_z (CUDA uint64/int64 tensor); returns a CUDA complex128 tensor.
    precision: None (gbsh_subset_terms, FP64), PREC_FP64 or PREC_TF."""
    import torch
    ptr, N, ld, _ = _as_matrix(dA)
    out = torch.empty(d_z.numel(), dtype=torch.complex128, device=d_z.device)
    st = ctypes.c_void_p(_stream_handle(stream))
    if precision is None:
        rc = load().gbsh_subset_terms(ctypes.c_void_p(ptr), N, ld, ctypes.c_void_p(d_z.data_ptr()),
                                      d_z.numel(), ctypes.c_void_p(out.data_ptr()), st)
        _check(rc, "gbsh_subset_terms")
    else:
        rc = load().gbsh_subset_terms_ex(ctypes.c_void_p(ptr), N, ld, int(precision),
                                         ctypes.c_void_p(d_z.data_ptr()), d_z.numel(),
                                         ctypes.c_void_p(out.data_ptr()), st)
        _check(rc, "gbsh_subset_terms_ex")
    return out


def visit_counts(N: int, stream=None):
    """Visit count of every subset z under the enumeration used by lhaf (CUDA int32 tensor)."""
    import torch
    n = (N + (N & 1)) // 2
    counts = torch.zeros(1 << n, dtype=torch.int32, device="cuda")
    rc = load().gbsh_visit_counts(N, ctypes.c_void_p(counts.data_ptr()),
                                  ctypes.c_void_p(_stream_handle(stream)))
    _check(rc, "gbsh_visit_counts")
    return counts


def _ptr_of(x):
    """Data pointer of a numpy array or torch tensor (host or CUDA)."""
    try:
        import torch
        if isinstance(x, torch.Tensor):
            return x.data_ptr()
    except ImportError:
        pass
    return x.ctypes.data


def lhaf_batch(mats, precision=PREC_FP64, stream=None, return_abs_sum=False):
    """Loop hafnians of a list of square complex128 numpy matrices (uneven sizes) in one
    batched launch. Returns a complex128 numpy array (and the sums |p_Z| if asked)."""
    Ns = np.array([m.shape[0] for m in mats], dtype=np.int32)
    offs = np.zeros(len(mats), dtype=np.int64)
    if len(mats) > 1:
        offs[1:] = np.cumsum(Ns.astype(np.int64) ** 2)[:-1]
    packed = np.concatenate([np.ascontiguousarray(m, dtype=np.complex128).ravel() for m in mats]
                            + [np.zeros(1, np.complex128)])
    outs = np.zeros(len(mats), dtype=np.complex128)
    sums = np.zeros(len(mats), dtype=np.float64)
    rc = load().gbsh_lhaf_batch(ctypes.c_void_p(packed.ctypes.data), ctypes.c_void_p(offs.ctypes.data),
                                ctypes.c_void_p(Ns.ctypes.data), len(mats),
                                ctypes.c_void_p(outs.ctypes.data), ctypes.c_void_p(sums.ctypes.data),
                                int(precision), ctypes.c_void_p(_stream_handle(stream)))
    _check(rc, "gbsh_lhaf_batch")
    return (outs, sums) if return_abs_sum else outs


def gbs_prob_batch(B, gammas, patterns, p_vacs=None, precision=PREC_FP64, stream=None):
    """Eq. lhaf-pure for many patterns of one kernel matrix B. `gammas`: one fill vector
    (shared) or a (count, M) array; `patterns`: (count, M) photon numbers.
    Returns (probs, lhafs) as numpy arrays."""
    bptr, M, ld, keepB = _as_matrix(B)
    pats = np.ascontiguousarray(patterns, dtype=np.int32)
    if pats.ndim != 2 or pats.shape[1] != M:
        raise ValueError("patterns must be (count, M)")
    count = pats.shape[0]
    try:
        import torch
        is_t = isinstance(gammas, torch.Tensor)
    except ImportError:
        is_t = False
    g = gammas.contiguous() if is_t else np.ascontiguousarray(gammas, dtype=np.complex128)
    stride = 0 if g.ndim == 1 else M
    pv = None if p_vacs is None else np.ascontiguousarray(p_vacs, dtype=np.float64)
    probs = np.zeros(count, dtype=np.float64)
    lh = np.zeros(count, dtype=np.complex128)
    rc = load().gbsh_gbs_prob_batch(ctypes.c_void_p(bptr), M, ld, ctypes.c_void_p(_ptr_of(g)),
                                    stride, ctypes.c_void_p(pats.ctypes.data), count,
                                    ctypes.c_void_p(pv.ctypes.data if pv is not None else 0),
                                    ctypes.c_void_p(probs.ctypes.data),
                                    ctypes.c_void_p(lh.ctypes.data), int(precision),
                                    ctypes.c_void_p(_stream_handle(stream)))
    _check(rc, "gbsh_gbs_prob_batch")
    return probs, lh


def set_batch_tuning(precision: int, n_max: int, warps_per_cta: int,
                     warps_small: int | None = None):
    """Warps per CTA of the batched kernel's large-popcount class (and, if given, of its
    small-popcount class) for batches with largest size n_max pairs."""
    if warps_small is None:
        _check(load().gbsh_set_batch_tuning(precision, n_max, warps_per_cta),
               "gbsh_set_batch_tuning")
    else:
        _check(load().gbsh_set_batch_tuning_ex(precision, n_max, warps_small, warps_per_cta),
               "gbsh_set_batch_tuning_ex")


def set_batch_graphs(enable: bool):
    """CUDA-graph replay of repeated batched launch shapes (on by default)."""
    _check(load().gbsh_set_batch_graphs(1 if enable else 0), "gbsh_set_batch_graphs")


def batch_graph_stats() -> dict:
    """{"captures": graphs captured, "replays": graph launches} of the batched path so far."""
    c, r = ctypes.c_longlong(), ctypes.c_longlong()
    _check(load().gbsh_batch_graph_stats(ctypes.byref(c), ctypes.byref(r)), "gbsh_batch_graph_stats")
    return {"captures": c.value, "replays": r.value}
