"""GPU loop hafnian (C ABI, CUDA kernels) against the CPU oracle."""
import math

import numpy as np
import pytest

from oracle import lhaf as L
from paper_2010_15595_gb300 import workloads as W

pytestmark = pytest.mark.gpu

# Relative tolerance of the GPU result against the FP64 oracle for N <= 40 and above.
TOL_40 = 1e-9
TOL_50 = 1e-7


def rel(a, b):
    return abs(a - b) / abs(b)


def _dev(A):
    import torch
    return torch.from_numpy(np.ascontiguousarray(A)).to("cuda")


@pytest.mark.parametrize("N", list(range(0, 25)))
def test_random_small_vs_definition(gbsh, N):
    """Every size up to 24 (odd sizes padded), against the definition (brute force / DP);
    several tiles of the Hessenberg and La Budde loops and ragged shapes."""
    rng = np.random.default_rng(1000 + N)
    A = W.random_complex_symmetric(N, rng)
    ref = L.lhaf_brute(A) if N <= 12 else L.lhaf_dp(A)
    got = gbsh.lhaf(_dev(A)) if N else gbsh.lhaf(A)
    _, asum = L.lhaf_subset(A, return_abs_sum=True) if N else (1, 1)
    assert abs(got - ref) <= 1e-12 * max(asum, abs(ref)), (N, got, ref)


@pytest.mark.parametrize("N", [1, 2, 3, 8, 15, 22, 29, 30])
def test_all_ones(gbsh, N):
    """lhaf(all-ones) = telephone number T(N)."""
    t = [1, 1]
    for k in range(2, N + 1):
        t.append(t[-1] + (k - 1) * t[-2])
    got = gbsh.lhaf(_dev(W.all_ones(N)))
    _, asum = L.lhaf_subset(W.all_ones(N), return_abs_sum=True)
    assert abs(got - t[N]) <= 1e-13 * N * asum


def test_haf_mode(gbsh):
    """Zero loop weights give the hafnian; haf(all-ones 2n) = (2n-1)!!."""
    for n in (1, 4, 9, 13):
        A = W.all_ones(2 * n)
        np.fill_diagonal(A, 0)
        dfac = math.prod(range(1, 2 * n, 2))
        got = gbsh.lhaf(_dev(A))
        _, asum = L.lhaf_subset(A, return_abs_sum=True)
        assert abs(got - dfac) <= 1e-13 * n * asum


def test_config_n16(gbsh):
    A = W.single_lhaf_n16()
    ref = L.lhaf_subset(A)
    got, err = gbsh.lhaf(_dev(A), return_error=True)
    assert rel(got, ref) <= TOL_40
    assert err < 1e-9


def test_host_pointer_and_lda(gbsh):
    """Host input is copied in; a leading dimension > N is honoured."""
    A = W.single_lhaf_mid(20)
    ref = L.lhaf_subset(A)
    assert rel(gbsh.lhaf(A), ref) <= TOL_40
    import torch
    big = torch.zeros((20, 27), dtype=torch.complex128, device="cuda")
    big[:, :20] = torch.from_numpy(A).cuda()
    assert rel(gbsh.lhaf(big[:, :20]), ref) <= TOL_40


def test_config_n32(gbsh):
    A = W.single_lhaf_mid(32)
    ref, asum = L.lhaf_subset(A, return_abs_sum=True)
    got = gbsh.lhaf(_dev(A))
    assert rel(got, ref) <= TOL_40, (got, ref, asum / abs(ref))


def test_deterministic(gbsh):
    A = _dev(W.single_lhaf_mid(28))
    vals = {gbsh.lhaf(A) for _ in range(3)}
    assert len(vals) == 1


def test_launch_shape_independent(gbsh):
    """The chunked sum does not depend on warps per CTA or the popcount split."""
    A = _dev(W.single_lhaf_mid(26))
    try:
        gbsh.set_tuning(8, 0)
        a = gbsh.lhaf(A)
        gbsh.set_tuning(4, 0)
        b = gbsh.lhaf(A)
        gbsh.set_tuning(8, 7)  # forces a second, many-popcount class
        c = gbsh.lhaf(A)
    finally:
        gbsh.set_tuning(0, 0)
    assert a == b
    assert rel(c, a) < 1e-13


@pytest.mark.parametrize("N", [4, 11, 20, 31])
def test_visit_each_subset_once(gbsh, N):
    """Bit-exact enumeration: every nonempty subset z of the pairs visited exactly once."""
    try:
        gbsh.set_tuning(8, 3)  # two classes, to cover the split as well
        c = gbsh.visit_counts(N).cpu().numpy()
    finally:
        gbsh.set_tuning(0, 0)
    assert c[0] == 0
    assert (c[1:] == 1).all()


def test_subset_terms_match_oracle(gbsh):
    """Individual terms p_Z at N=40 for a seeded sample of subsets of every popcount."""
    import torch
    A = W.single_lhaf_mid(40)
    rng = np.random.default_rng(7)
    zs = np.unique(np.concatenate([rng.integers(1, 1 << 20, 200), [1, (1 << 20) - 1]]))
    zs = zs.astype(np.uint64)
    ref = L.subset_terms(A, zs)
    got = gbsh.subset_terms(_dev(A), torch.from_numpy(zs.astype(np.int64)).cuda()).cpu().numpy()
    scale = np.maximum(np.abs(ref), 1e-300)
    assert (np.abs(got - ref) / scale).max() < 1e-9


def test_errors(gbsh):
    with pytest.raises(gbsh.GbshError):
        gbsh.lhaf(np.ones((61, 61), complex))
