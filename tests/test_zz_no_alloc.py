"""gbsh_lhaf_noalloc: the loop-hafnian entry point for callers that cannot allocate device
memory (plugins inside another framework's memory-managed region, latency-critical loops
that cannot absorb an allocation's implicit synchronisation). Its scratch is a fixed array
inside the library. Checked through the C ABI against gbsh_lhaf_async (caller-provided
workspace) on two calls in a row, with different sizes and matrices, so that a second call
sees the first call's leftovers in the shared array.

This file is collected last on purpose."""
import numpy as np
import pytest

from paper_2010_15595_gb300 import workloads as W

pytestmark = pytest.mark.gpu

U = 2.0 ** -53


def _run_both(lib, A):
    import torch
    dA = torch.from_numpy(A).cuda()
    N = A.shape[0]
    out_ref = torch.zeros(1, dtype=torch.complex128, device="cuda")
    abs_ref = torch.zeros(1, dtype=torch.float64, device="cuda")
    ws = torch.empty(lib.workspace_size(N), dtype=torch.uint8, device="cuda")
    lib.lhaf_async(dA, out_ref, ws, d_abs_sum=abs_ref)
    out_na = torch.full((1,), complex(np.nan, np.nan), dtype=torch.complex128, device="cuda")
    abs_na = torch.full((1,), np.nan, dtype=torch.float64, device="cuda")
    lib.lhaf_noalloc(dA, out_na, d_abs_sum=abs_na)
    torch.cuda.synchronize()
    return complex(out_ref.item()), float(abs_ref.item()), complex(out_na.item()), float(abs_na.item())


def test_noalloc_matches_workspace_entry_two_calls(gbsh):
    from oracle import lhaf as L
    cases = [W.single_lhaf_mid(32), W.single_lhaf_mid(26, seed=3)]
    for A in cases:  # two calls in a row on the shared scratch
        ref, aref, got, agot = _run_both(gbsh, A)
        v, _, sq = L.lhaf_subset_stats(A)
        tol = max(1e-9, 512 * U * sq ** 0.5 / abs(v))  # same gate as the parity tests
        assert abs(got - ref) <= tol * abs(ref), (A.shape, got, ref)
        assert abs(agot - aref) <= 1e-12 * aref


def test_noalloc_chunk_halving_n40(gbsh):
    """N = 40: the default plan's scratch (2^18 chunk partial sums per popcount class)
    exceeds the fixed array, so the no-alloc entry halves the chunk count until it fits.
    The terms are the same; only the grouping of the compensated sum differs, so the result
    agrees with the workspace entry to rounding. Checked against the long-double oracle too."""
    import json
    import os
    from tests.golden.make_golden import read_matrix
    assert gbsh.workspace_size(40) > gbsh.NOALLOC_SCRATCH_BYTES
    assert gbsh.noalloc_chunks(40) < gbsh.plan(40)["nchunks"]  # the halving branch runs
    here = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")
    A = read_matrix(os.path.join(here, "lhaf_n40.matrix.txt"))
    with open(os.path.join(here, "lhaf_n40.json")) as f:
        rec = json.load(f)
    for _ in range(2):
        ref, aref, got, agot = _run_both(gbsh, A)
        assert abs(got - ref) <= 1e-12 * abs(ref), (got, ref)
        assert abs(agot - aref) <= 1e-12 * aref
    ld = complex(*rec["lhaf_ld"])
    assert abs(got - ld) <= max(1e-9, 512 * U * rec["sq_sum"] ** 0.5 / abs(ld)) * abs(ld)


def test_noalloc_largest_size_plan(gbsh):
    """N = GBSH_MAX_N = 60: the no-alloc plan either fits the fixed array (with fewer
    chunks than the default plan) or is refused cleanly with GBSH_ENOMEM. (A full N = 60
    evaluation, 2^30 subsets, takes minutes, so the plan query stands in for it.) A call
    at a size that fits still works afterwards."""
    try:
        c = gbsh.noalloc_chunks(60)
        assert 1 <= c <= gbsh.plan(60)["nchunks"]
    except gbsh.GbshError as e:
        assert e.code == gbsh.GBSH_ENOMEM
    ref, _, got, _ = _run_both(gbsh, W.single_lhaf_mid(20))
    assert abs(got - ref) <= 1e-12 * abs(ref)


def test_noalloc_empty_matrix(gbsh):
    """N = 0 writes lhaf = 1 and sum |p_Z| = 0 on the stream."""
    import torch
    out = torch.full((1,), complex(np.nan, np.nan), dtype=torch.complex128, device="cuda")
    asum = torch.full((1,), np.nan, dtype=torch.float64, device="cuda")
    gbsh.lhaf_noalloc(torch.zeros((0, 0), dtype=torch.complex128, device="cuda"), out,
                      d_abs_sum=asum)
    torch.cuda.synchronize()
    assert complex(out.item()) == 1 and float(asum.item()) == 0.0


def test_noalloc_rejects_bad_sizes(gbsh):
    import torch
    out = torch.zeros(1, dtype=torch.complex128, device="cuda")
    A = torch.zeros((61, 61), dtype=torch.complex128, device="cuda")
    with pytest.raises(gbsh.GbshError) as e:
        gbsh.lhaf_noalloc(A, out)
    assert e.value.code == gbsh.GBSH_EINVAL
