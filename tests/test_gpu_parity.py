"""GPU loop hafnian (C ABI, CUDA kernels) against the CPU oracle."""
import math

import numpy as np
import pytest

from oracle import lhaf as L
from paper_2010_15595_gb300 import workloads as W

pytestmark = pytest.mark.gpu

U = 2.0 ** -53
# Targets for the relative error: 1e-9 for N <= 40, 1e-7 above.
TOL_40 = 1e-9
TOL_50 = 1e-7
# Per-subset relative rounding error of the FP64 kernel, in units of U, with margin. The
# subset terms p_Z are computed with independent rounding errors of rms ~20-90 U (measured
# against long-double evaluations of the same terms), so the signed sum's error behaves
# like a random walk: |error| ~ eps_rms * sqrt(sum_Z |p_Z|^2). Gate = 512 U that scale.
FP64_TERM_ERR = 512 * U


def rel(a, b):
    return abs(a - b) / abs(b)


def ns_tol(N):
    return TOL_40 if N <= 40 else TOL_50


def fp64_tol(N, lhaf_ref, sq_sum):
    """Tolerance of the FP64 path: the stated target, or the rounding floor of an FP64
    evaluation of this matrix if that is larger (derived above)."""
    return max(ns_tol(N), FP64_TERM_ERR * (sq_sum ** 0.5) / abs(lhaf_ref))


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
    if N == 0:
        assert got == 1
        return
    _, _, sq = L.lhaf_subset_stats(A)
    assert rel(got, ref) <= fp64_tol(N, ref, sq), (N, got, ref)


@pytest.mark.parametrize("scale", [1e-9, 1e9])
def test_extreme_entry_scale(gbsh, scale):
    """The unit-subdiagonal Hessenberg reduction makes each pivot a running product of the
    earlier ones, so at N = 24 with entries near 1e-9 (1e9) |pivot|^2 would leave the double
    exponent range; the complex reciprocal pre-scales by a power of two. Against the
    definition (subset DP)."""
    rng = np.random.default_rng(77)
    A = W.random_complex_symmetric(24, rng) * scale
    ref = L.lhaf_dp(A)
    got = gbsh.lhaf(_dev(A))
    _, _, sq = L.lhaf_subset_stats(A)
    assert np.isfinite(got.real) and np.isfinite(got.imag)
    assert rel(got, ref) <= fp64_tol(24, ref, sq), (scale, got, ref)


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
    ref = L.lhaf_subset_ld(A)
    got, err = gbsh.lhaf(_dev(A), return_error=True)
    assert rel(got, ref) <= TOL_40
    assert err < 1e-9


def test_host_pointer_and_lda(gbsh):
    """Host input is copied in; a leading dimension > N is honoured (same bits)."""
    A = W.single_lhaf_mid(20)
    ref = L.lhaf_subset_ld(A)
    on_dev = gbsh.lhaf(_dev(A))
    assert rel(on_dev, ref) <= TOL_40
    assert gbsh.lhaf(A) == on_dev
    import torch
    big = torch.zeros((20, 27), dtype=torch.complex128, device="cuda")
    big[:, :20] = torch.from_numpy(A).cuda()
    assert gbsh.lhaf(big[:, :20]) == on_dev


def test_config_n32(gbsh):
    """N=32 config matrix. The double oracle's own error here is ~6e-11 (vs long double)."""
    A = W.single_lhaf_mid(32)
    ref, asum, sq = L.lhaf_subset_stats(A)
    got = gbsh.lhaf(_dev(A))
    assert rel(got, ref) <= fp64_tol(32, ref, sq), (got, ref, asum / abs(ref))


def _golden(name):
    import json
    import os
    here = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")
    from tests.golden.make_golden import read_matrix
    with open(os.path.join(here, name + ".json")) as f:
        rec = json.load(f)
    return read_matrix(os.path.join(here, name + ".matrix.txt")), rec


@pytest.mark.parametrize("name", ["lhaf_n40", "lhaf_n40_repeated"])
def test_golden_n40(gbsh, name):
    """N=40 against the long-double oracle (the double oracle is itself ~3e-9 off here)."""
    A, rec = _golden(name)
    ref = complex(*rec["lhaf_ld"])
    got = gbsh.lhaf(_dev(A))
    assert rel(got, ref) <= fp64_tol(40, ref, rec["sq_sum"]), (got, ref)


def test_golden_n50(gbsh):
    """N=50 (2^25 subsets), FP64 path, against the double oracle, at the FP64 gate: the
    oracle's own sum of |p_Z|^2 sets it (no GPU output enters it)."""
    A, rec = _golden("lhaf_n50")
    ref = complex(*rec.get("lhaf_ld", rec["lhaf_d"]))
    got = gbsh.lhaf(_dev(A))
    assert rel(got, ref) <= fp64_tol(50, ref, rec["sq_sum"]), (got, ref, rel(got, ref))


# The FP64 path held to the stated tolerance: it misses it at N >= 40 (measured 4.7e-8 at
# N=40, 2.5e-7 for the repeated-mode N=40 matrix and 1.7e-5 at N=50), which is why the
# triple-float path exists (tests/test_gpu_accurate.py carries the stated-tolerance claim).
# strict: an FP64 result that unexpectedly met the tolerance would fail the suite too.
@pytest.mark.xfail(strict=True, reason="FP64 per subset is above the stated tolerance at N >= 40")
@pytest.mark.parametrize("name", ["lhaf_n40", "lhaf_n40_repeated"])
def test_fp64_at_stated_tolerance_n40(gbsh, name):
    A, rec = _golden(name)
    ref = complex(*rec["lhaf_ld"])
    assert rel(gbsh.lhaf(_dev(A)), ref) <= TOL_40


@pytest.mark.parametrize("name", ["lhaf_n40", "lhaf_n50", "lhaf_n56"])
def test_golden_sampled_terms(gbsh, name):
    """Per-subset terms at full size (N=56: 2^28 subsets, too many for the oracle) on a
    seeded sample of subsets including the full set."""
    import torch
    A, rec = _golden(name)
    zs = np.array([t[0] for t in rec["terms"]], dtype=np.int64)
    ref = np.array([complex(t[1], t[2]) for t in rec["terms"]])
    got = gbsh.subset_terms(_dev(A), torch.from_numpy(zs).cuda()).cpu().numpy()
    err = np.abs(got - ref) / np.abs(ref)
    assert err.max() < 1e-10, err.max()


def test_scaling_property_n56(gbsh):
    """p_Z(filldiag(c^2 A0, c v)) = c^N p_Z(A) for every subset (homogeneity), at N=56."""
    import torch
    A, rec = _golden("lhaf_n56")
    c = 0.75
    As = c * c * A
    As[np.diag_indices(56)] = c * np.diag(A)
    zs = torch.tensor([t[0] for t in rec["terms"]][:64], dtype=torch.int64, device="cuda")
    a = gbsh.subset_terms(_dev(A), zs).cpu().numpy()
    b = gbsh.subset_terms(_dev(As), zs).cpu().numpy()
    assert (np.abs(b - c ** 56 * a) / np.abs(c ** 56 * a)).max() < 1e-10


def test_gbs_prob_pattern_expansion_bit_exact(gbsh):
    """The device pattern expansion (repeated rows/columns, filldiag) gives bit-identical
    results to the same matrix expanded on the host (Sec. II, B_S and gamma_S)."""
    from oracle import gbs as G
    B, gamma, pattern = W.repeated_mode_state()
    pattern = pattern.copy()
    pattern[::3] = 1  # N = 34: mixes 1- and 2-photon modes
    AS = G.expand_pure(B, gamma, pattern)
    direct = gbsh.lhaf(_dev(AS))
    import torch
    prob, via_pattern = gbsh.gbs_prob(_dev(B), torch.from_numpy(gamma).cuda(), pattern,
                                      p_vac=0.5, return_lhaf=True)
    assert via_pattern == direct
    fact = np.prod([math.factorial(int(s)) for s in pattern])
    assert prob == pytest.approx(0.5 * abs(direct) ** 2 / fact, rel=1e-15)


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


def test_visit_each_subset_once_default_ladder(gbsh):
    """N = 40 with the default launch plan (three popcount classes on the warps-per-CTA
    ladder, 2^18 chunks, classes overlapped on side streams): every nonempty subset once."""
    assert gbsh.plan(40)["nclass"] >= 3
    c = gbsh.visit_counts(40).cpu().numpy()
    assert c[0] == 0
    assert (c[1:] == 1).all()


def test_async_on_user_stream_is_ordered(gbsh):
    """gbsh_lhaf_async on a non-default stream: the popcount classes that run on the
    library's side streams are joined back into the caller's stream, so work queued on that
    stream after the call sees the finished result (the output is cleared before each call)."""
    import torch
    A = W.single_lhaf_mid(34)
    assert gbsh.plan(34)["nclass"] >= 2
    ref = gbsh.lhaf(A)
    s = torch.cuda.Stream()
    dA = torch.from_numpy(A).cuda()
    ws = torch.empty(gbsh.workspace_size(34), dtype=torch.uint8, device="cuda")
    out = torch.zeros(1, dtype=torch.complex128, device="cuda")
    copies = []
    torch.cuda.synchronize()
    with torch.cuda.stream(s):
        for _ in range(3):
            out.zero_()
            gbsh.lhaf_async(dA, out, ws, stream=s)
            copies.append(out.clone())
    s.synchronize()
    for c in copies:
        assert complex(c.item()) == ref


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
