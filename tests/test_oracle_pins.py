"""Pins of the CPU oracle against facts that do not come from the oracle itself:
brute force over matchings, closed forms (telephone numbers, double factorials),
block-diagonal products, invariances, and the paper's probability formulas reduced to
textbook cases. CPU only."""
import math

import numpy as np
import pytest

from oracle import lhaf as L
from paper_2010_15595_gb300 import workloads as W


def telephone(n):
    """T(n): number of matchings with loops of the complete graph = lhaf(all-ones n x n)
    (Sec. IV, caption of Fig. 2). T(0)=T(1)=1, T(n)=T(n-1)+(n-1)T(n-2)."""
    t = [1, 1]
    for k in range(2, n + 1):
        t.append(t[-1] + (k - 1) * t[-2])
    return t[n]


def double_factorial_odd(n):
    r = 1
    for k in range(1, 2 * n, 2):
        r *= k
    return r


def rel(a, b):
    return abs(a - b) / max(abs(b), 1e-300)


@pytest.mark.parametrize("N", range(0, 13))
def test_brute_vs_dp(N):
    rng = np.random.default_rng(100 + N)
    A = W.random_complex_symmetric(N, rng)
    assert rel(L.lhaf_dp(A), L.lhaf_brute(A)) < 1e-12
    assert rel(L.lhaf_dp(A, with_loops=False) if N else 1, L.haf_brute(A) if N else 1) < 1e-12


def test_brute_counts_matchings():
    for N in range(0, 11):
        assert L.lhaf_brute(np.ones((N, N))) == telephone(N)
    for n in range(0, 6):
        assert L.haf_brute(np.ones((2 * n, 2 * n))) == double_factorial_odd(n)


@pytest.mark.parametrize("N", list(range(0, 21)))
def test_subset_formula_vs_definition(N):
    rng = np.random.default_rng(200 + N)
    A = W.random_complex_symmetric(N, rng)
    ref = L.lhaf_brute(A) if N <= 12 else L.lhaf_dp(A)
    val, asum = L.lhaf_subset(A, return_abs_sum=True)
    # rounding of the formula is bounded by a few ulps times the cancellation scale
    assert abs(val - ref) <= 1e-12 * max(asum, abs(ref))


@pytest.mark.parametrize("N", [2, 5, 9, 16])
def test_subset_formula_haf_mode(N):
    """With zero loop weights the formula gives the hafnian (odd sizes give 0)."""
    rng = np.random.default_rng(300 + N)
    A = W.random_complex_symmetric(N, rng)
    h = L.haf(A)
    ref = L.lhaf_dp(A, with_loops=False)
    assert abs(h - ref) <= 1e-12 * max(1.0, abs(ref))


@pytest.mark.parametrize("N", list(range(1, 31)))
def test_all_ones_telephone(N):
    """lhaf(all-ones N x N) = T(N) (Fig. 2 caption). Exact integers; the tolerance grows with
    the cancellation of the signed subset sum, as the paper's Fig. 2 shows for its own code."""
    val, asum = L.lhaf_subset(W.all_ones(N), return_abs_sum=True)
    T = telephone(N)
    assert abs(val.imag) <= 1e-13 * asum
    assert abs(val.real - T) <= 4e-14 * N * asum, (N, val, T)


@pytest.mark.parametrize("n", list(range(1, 13)))
def test_all_ones_double_factorial(n):
    """haf(all-ones 2n x 2n) = (2n-1)!! (number of perfect matchings, Eq. defhaf)."""
    A = W.all_ones(2 * n)
    np.fill_diagonal(A, 0)
    val, asum = L.lhaf_subset(A, return_abs_sum=True)
    assert abs(val.real - double_factorial_odd(n)) <= 4e-14 * n * asum
    assert abs(val.imag) <= 1e-13 * asum


@pytest.mark.parametrize("n1,n2", [(3, 4), (7, 9), (10, 12)])
def test_block_diagonal_product(n1, n2):
    """lhaf(A1 (+) A2) = lhaf(A1) lhaf(A2): a matching of a disconnected graph is a pair of
    matchings. Checks the formula beyond the sizes brute force reaches."""
    rng = np.random.default_rng(400 + n1 + n2)
    A1 = W.random_complex_symmetric(n1, rng)
    A2 = W.random_complex_symmetric(n2, rng)
    A = np.zeros((n1 + n2, n1 + n2), complex)
    A[:n1, :n1] = A1
    A[n1:, n1:] = A2
    val, asum = L.lhaf_subset(A, return_abs_sum=True)
    ref = L.lhaf_dp(A1) * L.lhaf_dp(A2)
    assert abs(val - ref) <= 1e-12 * max(asum, abs(ref))


def test_block_diagonal_product_large():
    rng = np.random.default_rng(401)
    A1 = W.random_complex_symmetric(12, rng, 0.5)
    A2 = W.random_complex_symmetric(14, rng, 0.5)
    A = np.zeros((26, 26), complex)
    A[:12, :12] = A1
    A[12:, 12:] = A2
    P = np.random.default_rng(5).permutation(26)
    val, asum = L.lhaf_subset(A[np.ix_(P, P)], return_abs_sum=True)
    ref = L.lhaf_dp(A1) * L.lhaf_dp(A2)
    assert abs(val - ref) <= 1e-12 * max(asum, abs(ref))


@pytest.mark.parametrize("N", [6, 11, 18])
def test_permutation_invariance(N):
    """lhaf(P A P^T) = lhaf(A): catches a wrong pairing or a transposed operand."""
    rng = np.random.default_rng(500 + N)
    A = W.random_complex_symmetric(N, rng)
    P = rng.permutation(N)
    v1, s1 = L.lhaf_subset(A, return_abs_sum=True)
    v2, s2 = L.lhaf_subset(A[np.ix_(P, P)], return_abs_sum=True)
    assert abs(v1 - v2) <= 1e-12 * max(s1, s2)


@pytest.mark.parametrize("N", [8, 13])
def test_diagonal_scaling(N):
    """lhaf(filldiag(D A0 D, D v)) = det(D) lhaf(filldiag(A0, v)): every vertex appears in
    exactly one loop or edge. Catches a dropped loop term or a wrong power of a weight."""
    rng = np.random.default_rng(600 + N)
    A = W.random_complex_symmetric(N, rng)
    d = rng.normal(size=N) + 1j * rng.normal(size=N)
    A0 = A.copy()
    np.fill_diagonal(A0, 0)
    As = (d[:, None] * A0 * d[None, :])
    As[np.diag_indices(N)] = d * np.diag(A)
    v1, s1 = L.lhaf_subset(A, return_abs_sum=True)
    v2, s2 = L.lhaf_subset(As, return_abs_sum=True)
    assert abs(v2 - np.prod(d) * v1) <= 1e-11 * max(s2, abs(np.prod(d)) * s1)


def test_odd_padding_brute():
    for N in (1, 3, 7, 11):
        rng = np.random.default_rng(700 + N)
        A = W.random_complex_symmetric(N, rng)
        assert rel(L.lhaf_subset(A), L.lhaf_brute(A)) < 1e-12


def test_small_closed_forms():
    """N=2: lhaf = A01 + A00 A11 ; N=0: 1."""
    A = np.array([[2 + 1j, 3 - 1j], [3 - 1j, -1 + 0.5j]])
    assert abs(L.lhaf_subset(A) - (A[0, 1] + A[0, 0] * A[1, 1])) < 1e-15
    assert L.lhaf_subset(np.zeros((0, 0))) == 1


def test_subset_terms_sum_to_lhaf():
    """The per-subset terms, signed and summed, give the loop hafnian (used for sampled
    parity at large N)."""
    rng = np.random.default_rng(800)
    A = W.random_complex_symmetric(14, rng)
    n = 7
    zs = np.arange(1 << n, dtype=np.uint64)
    pz = L.subset_terms(A, zs)
    sgn = np.array([(-1) ** (n - bin(int(z)).count("1")) for z in zs])
    assert rel((sgn * pz).sum(), L.lhaf_dp(A)) < 1e-12


def test_long_double_agrees():
    A = W.single_lhaf_n16()
    v, s = L.lhaf_subset(A, return_abs_sum=True)
    vl = L.lhaf_subset_ld(A)
    assert abs(v - vl) <= 1e-13 * s
