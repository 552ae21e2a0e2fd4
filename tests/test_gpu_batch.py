"""Batched loop hafnians (gbsh_lhaf_batch, gbsh_gbs_prob_batch) against the oracle and
against the single-matrix path."""
import math

import numpy as np
import pytest

from oracle import gbs as G
from oracle import lhaf as L
from paper_2010_15595_gb300 import workloads as W

pytestmark = pytest.mark.gpu

U = 2.0 ** -53


def fp64_tol(ref, sq):
    return max(1e-9, 512 * U * sq ** 0.5 / abs(ref))


def test_batch_uneven_vs_definition(gbsh):
    rng = np.random.default_rng(77)
    sizes = [0, 1, 2, 3, 5, 8, 11, 12, 16, 17, 20, 7, 4, 19]
    mats = [W.random_complex_symmetric(N, rng) for N in sizes]
    got = gbsh.lhaf_batch(mats)
    for A, g in zip(mats, got):
        N = A.shape[0]
        if N == 0:
            assert g == 1
            continue
        ref = L.lhaf_brute(A) if N <= 12 else L.lhaf_dp(A)
        _, _, sq = L.lhaf_subset_stats(A)
        assert abs(g - ref) <= fp64_tol(ref, sq) * abs(ref), (N, g, ref)


def test_batch_same_alone_and_in_mix(gbsh):
    """Each result is bit-identical alone (batch of one) and inside a mixed batch."""
    B, gamma = W.batch_state()
    pats = W.batch_patterns(64, seed=3)
    mats = [G.expand_pure(B, gamma, p) for p in pats]
    mix = gbsh.lhaf_batch(mats)
    for i in (0, 17, 40, 63):
        alone = gbsh.lhaf_batch([mats[i]])
        assert alone[0] == mix[i]
    # shuffled order gives the same bits too
    perm = np.random.default_rng(1).permutation(len(mats))
    mix2 = gbsh.lhaf_batch([mats[i] for i in perm])
    assert np.array_equal(mix2, mix[perm])


def test_batch_matches_single_path(gbsh):
    B, gamma = W.batch_state()
    pats = W.batch_patterns(24, seed=5)
    mats = [G.expand_pure(B, gamma, p) for p in pats]
    got = gbsh.lhaf_batch(mats)
    for A, g in zip(mats, got):
        single = gbsh.lhaf(A)
        _, asum = L.lhaf_subset(A, return_abs_sum=True) if A.shape[0] <= 24 else (0, 0)
        # different chunking: agree to rounding (compensated sums of the same terms)
        assert abs(g - single) <= 1e-12 * max(abs(single), 1e-300) or abs(g - single) <= 64 * U * asum


def test_gbs_prob_batch_vs_single_and_oracle(gbsh):
    """Batched Eq. lhaf-pure from (B, gamma, pattern) equals the single-pattern entry point
    bit for bit, and the oracle's expansion + loop hafnian within tolerance."""
    B, gamma = W.batch_state()
    pats = W.batch_patterns(32, seed=9, n_max=22)
    pv = 0.25
    probs, lh = gbsh.gbs_prob_batch(B, gamma, pats, p_vacs=np.full(len(pats), pv))
    for p, pr, l in zip(pats, probs, lh):
        single_prob, single_l = gbsh.gbs_prob(B, gamma, p, p_vac=pv, return_lhaf=True)
        ref = L.lhaf_dp(G.expand_pure(B, gamma, p)) if p.sum() <= 22 else None
        fact = np.prod([math.factorial(int(s)) for s in p])
        assert pr == pytest.approx(pv * abs(l) ** 2 / fact, rel=1e-14)
        assert abs(l - single_l) <= 1e-12 * abs(single_l)
        if ref is not None:
            _, _, sq = L.lhaf_subset_stats(G.expand_pure(B, gamma, p))
            assert abs(l - ref) <= fp64_tol(ref, sq) * abs(ref)


def test_gbs_prob_batch_per_problem_gamma(gbsh):
    """Per-problem fill vectors (the sampler's case)."""
    B, gamma = W.batch_state()
    rng = np.random.default_rng(4)
    pats = W.batch_patterns(8, seed=2, n_max=16)
    gams = np.stack([gamma + 0.05 * (rng.normal(size=100) + 1j * rng.normal(size=100))
                     for _ in range(8)])
    probs, lh = gbsh.gbs_prob_batch(B, gams, pats)
    for p, g, l in zip(pats, gams, lh):
        ref = L.lhaf_dp(G.expand_pure(B, g, p))
        _, _, sq = L.lhaf_subset_stats(G.expand_pure(B, g, p))
        assert abs(l - ref) <= fp64_tol(ref, sq) * abs(ref)


def test_c32_variant_error_map(gbsh):
    """Complex-FP32 per-subset variant: within 1e-5 relative of FP64 at the sizes where the
    mixed mode enables it (N <= C32_MAX_N); larger sizes exceed it (why it is not enabled
    there), and the mixed mode returns the FP64 bits for them."""
    from paper_2010_15595_gb300.lib import C32_MAX_N, PREC_C32, PREC_MIXED
    B, gamma = W.batch_state()
    small = [G.expand_pure(B, gamma, p) for p in W.batch_patterns(64, seed=11, n_min=2, n_max=C32_MAX_N)]
    large = [G.expand_pure(B, gamma, p) for p in W.batch_patterns(16, seed=12, n_min=12, n_max=12)]
    f64 = gbsh.lhaf_batch(small + large)
    c32 = gbsh.lhaf_batch(small + large, precision=PREC_C32)
    mixed = gbsh.lhaf_batch(small + large, precision=PREC_MIXED)
    err = np.abs(c32 - f64) / np.abs(f64)
    ns = len(small)
    assert err[:ns].max() <= 1e-5, err[:ns].max()
    assert err[ns:].max() > 1e-5  # measured: ~5e-4 at N=12
    assert np.array_equal(mixed[:ns], c32[:ns])
    assert np.array_equal(mixed[ns:], f64[ns:])


def test_c32_finite_at_batched_workload_sizes(gbsh):
    """The complex-FP32 variant stays finite across the batched workload's sizes (N = 10..30):
    pivots are running products whose squares would leave FP32's exponent range without the
    power-of-two pre-scaling in the complex reciprocal."""
    from paper_2010_15595_gb300.lib import PREC_C32
    B, gamma = W.batch_state()
    mats = [G.expand_pure(B, gamma, p) for p in W.batch_patterns(48, seed=13, n_min=10, n_max=30)]
    c32 = gbsh.lhaf_batch(mats, precision=PREC_C32)
    assert np.all(np.isfinite(c32.real)) and np.all(np.isfinite(c32.imag))


def test_batch_graph_replay_bit_identical(gbsh):
    """A repeated launch shape is captured into a CUDA graph on its second use and replayed
    afterwards; replays give the direct launch's bits, also for new values of the same shape
    (the per-call tables are uploaded before each launch)."""
    rng = np.random.default_rng(21)
    sizes = [12, 26, 8, 22, 30, 16]
    mats_a = [W.random_complex_symmetric(N, rng) for N in sizes]
    mats_b = [W.random_complex_symmetric(N, rng) for N in sizes]
    try:
        gbsh.set_batch_graphs(False)
        direct_a = gbsh.lhaf_batch(mats_a)
        direct_b = gbsh.lhaf_batch(mats_b)
        gbsh.set_batch_graphs(True)
        s0 = gbsh.batch_graph_stats()
        runs = [gbsh.lhaf_batch(m) for m in (mats_a, mats_a, mats_b, mats_a)]
        s1 = gbsh.batch_graph_stats()
    finally:
        gbsh.set_batch_graphs(True)
    assert s1["captures"] >= s0["captures"] + 1
    assert s1["replays"] >= s0["replays"] + 3
    assert np.array_equal(runs[0], direct_a) and np.array_equal(runs[1], direct_a)
    assert np.array_equal(runs[2], direct_b) and np.array_equal(runs[3], direct_a)


def test_batch_graph_same_count_other_layout(gbsh):
    """Two batches with equal count, largest size and chunk total but another size mix (so
    other workspace offsets) must not share a graph: alternating them keeps direct results."""
    rng = np.random.default_rng(22)
    # chunk totals: 2^n / chunk(n) summed; {14, 14, 6, 6} and {14, 14, 4, 8} differ in the
    # small problems' sizes, which moves the expanded-matrix area and everything after it
    sizes_a, sizes_b = [14, 14, 6, 6], [14, 14, 4, 8]
    mats_a = [W.random_complex_symmetric(N, rng) for N in sizes_a]
    mats_b = [W.random_complex_symmetric(N, rng) for N in sizes_b]
    try:
        gbsh.set_batch_graphs(False)
        da, db = gbsh.lhaf_batch(mats_a), gbsh.lhaf_batch(mats_b)
        gbsh.set_batch_graphs(True)
        runs = [gbsh.lhaf_batch(m) for m in (mats_a, mats_b, mats_a, mats_b, mats_a, mats_b)]
    finally:
        gbsh.set_batch_graphs(True)
    for i, r in enumerate(runs):
        assert np.array_equal(r, da if i % 2 == 0 else db), i


def test_batch_rejects_bad_input(gbsh):
    with pytest.raises(gbsh.GbshError):
        gbsh.lhaf_batch([np.ones((61, 61), complex)])
    with pytest.raises(gbsh.GbshError):
        gbsh.gbs_prob_batch(np.eye(3, dtype=complex), np.zeros(3, complex), np.array([[1, -1, 0]]))


def test_double_double_meets_stated_tolerance(gbsh):
    """Double-double per-subset arithmetic (GBSH_PREC_DD) removes the FP64 rounding floor:
    within 1e-9 of the long-double oracle where FP64 cannot get there (N=32..40)."""
    from paper_2010_15595_gb300.lib import PREC_DD
    from tests.test_gpu_parity import _golden
    A40, rec = _golden("lhaf_n40")
    mats = [W.single_lhaf_mid(32), A40]
    refs = [L.lhaf_subset_ld(mats[0]), complex(*rec["lhaf_ld"])]
    got = gbsh.lhaf_batch(mats, precision=PREC_DD)
    for g, ref in zip(got, refs):
        assert abs(g - ref) <= 1e-9 * abs(ref), (g, ref, abs(g - ref) / abs(ref))


def test_double_double_small_vs_definition(gbsh):
    """Against the long-double oracle; the gate is that oracle's own rounding floor
    (64-bit significand, same random-walk model as the FP64 gate), not the GPU's."""
    from paper_2010_15595_gb300.lib import PREC_DD
    rng = np.random.default_rng(21)
    mats = [W.random_complex_symmetric(N, rng) for N in (1, 2, 5, 9, 14, 20)]
    got = gbsh.lhaf_batch(mats, precision=PREC_DD)
    for A, g in zip(mats, got):
        ref = L.lhaf_subset_ld(A)
        _, _, sq = L.lhaf_subset_stats(A)
        tol = max(1e-14, 512 * 2.0 ** -64 * sq ** 0.5 / abs(ref))
        assert abs(g - ref) <= tol * abs(ref), (A.shape, g, ref)


def test_double_double_all_ones_telephone(gbsh):
    """Fig. 2's accuracy pin: lhaf(all-ones) = T(n). In double-double (terms accumulated
    without rounding their low parts) the error stays at the final rounding, far below the
    paper's long-double values (3.6e-12 at n=30, 3.4e-10 at n=36)."""
    from paper_2010_15595_gb300.lib import PREC_DD
    from fractions import Fraction
    import bench
    for n in (30, 36):
        v = gbsh.lhaf_batch([W.all_ones(n)], precision=PREC_DD)[0]
        T = bench.telephone(n)
        assert float(abs(Fraction(v.real) - T) / T) <= 1e-13, (n, v, T)


def test_autotuner_picks_a_candidate_and_keeps_results(gbsh, tmp_path, monkeypatch):
    from paper_2010_15595_gb300 import autotune
    monkeypatch.setenv("GBSH_TUNE_CACHE", str(tmp_path / "tune.json"))
    mats = autotune.synthetic_batch(9, count=64, seed=3)
    before = gbsh.lhaf_batch(mats)
    res = autotune.tune_batch(9, count=64)
    assert res["best"] in autotune.CANDIDATES and res["seconds"]
    after = gbsh.lhaf_batch(mats)
    assert np.array_equal(before, after)  # launch shape never changes the bits
    assert autotune.apply_cache() == 1
    gbsh.set_batch_tuning(0, 9, 0, warps_small=0)
