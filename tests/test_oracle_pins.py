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


# ---------------------------------------------------------------- probability layer

def _fock_state(U, r, alpha, D=40):
    """Fock amplitudes of D(alpha) U S(r) |0> built from matrix exponentials of the
    generators in a truncated Fock space (no Gaussian-state formulas involved)."""
    import scipy.linalg as sl
    m = len(r)
    a1 = np.diag(np.sqrt(np.arange(1, D)), 1).astype(complex)
    eye = np.eye(D)

    def op(k):
        mats = [eye] * m
        mats[k] = a1
        out = mats[0]
        for x in mats[1:]:
            out = np.kron(out, x)
        return out
    a = [op(k) for k in range(m)]
    ad = [x.conj().T for x in a]
    sq = sum(0.5 * r[k] * (a[k] @ a[k] - ad[k] @ ad[k]) for k in range(m))
    K = sl.logm(U)
    pas = sum(ad[i] @ a[j] * K[i, j] for i in range(m) for j in range(m))
    dis = sum(alpha[k] * ad[k] - np.conj(alpha[k]) * a[k] for k in range(m))
    v = np.zeros(D ** m, complex)
    v[0] = 1
    for gen in (sq, pas, dis):
        v = sl.expm(gen) @ v
    return v.reshape([D] * m)


@pytest.mark.parametrize("m,seed", [(1, 0), (2, 1), (2, 2)])
def test_pure_probabilities_match_fock_construction(m, seed):
    """Eq. lhaf-pure with the Sec. II quantities reproduces |<S|psi>|^2 of displaced
    squeezed states built directly in Fock space, with rotated squeezing and complex
    displacement (the phase-sensitive case). Pins the reading A = conj(X (I - Q^{-1}))."""
    from oracle import gbs as G
    rng = W.rng_for(90, seed)
    U = W.haar_unitary(m, rng)
    r = rng.uniform(0.2, 0.6, m)
    al = W.complex_normal(m, 0.7, rng)
    psi = _fock_state(U, r, al, D=40 if m == 2 else 80)
    V, R = G.pure_state_covariance(U, r), G.means_from_alpha(al)
    B, g, pv = G.pure_B_gamma(V, R)
    import itertools
    for S in itertools.product(range(5), repeat=m):
        assert G.prob_pure(B, g, pv, list(S)) == pytest.approx(abs(psi[S]) ** 2, abs=1e-12)


def test_probability_normalisation_3_modes():
    """sum_S p(S) over s_i <= 8 equals 1 minus the truncated tail (Sec. II)."""
    from oracle import gbs as G
    rng = W.rng_for(91, 0)
    U = W.haar_unitary(3, rng)
    r = np.array([0.5, 0.3, 0.2])
    al = W.complex_normal(3, 0.4, rng)
    V, R = G.pure_state_covariance(U, r), G.means_from_alpha(al)
    B, g, pv = G.pure_B_gamma(V, R)
    total = sum(G.prob_table(B, g, pv, 3, 8).values())
    mean_n = (np.trace(V) / 2 - 3) / 2 + (np.abs(al) ** 2).sum()  # <n> (hbar = 2)
    assert 1 - mean_n / 9 <= total <= 1 + 1e-12


def test_pure_equals_mixed_form():
    """Eq. lhaf (2N-size, Sec. II) equals Eq. lhaf-pure for a pure displaced state."""
    from oracle import gbs as G
    rng = W.rng_for(92, 0)
    U = W.haar_unitary(3, rng)
    r = np.array([0.5, 0.3, 0.2])
    al = W.complex_normal(3, 0.4, rng)
    V, R = G.pure_state_covariance(U, r), G.means_from_alpha(al)
    q = G.gbs_quantities(V, R)
    B, g, pv = G.pure_B_gamma(V, R)
    for S in [(1, 0, 0), (1, 1, 0), (2, 1, 1), (0, 2, 3)]:
        assert G.prob_pure(B, g, pv, S) == pytest.approx(G.prob_mixed(q["A"], q["gamma"], pv, S),
                                                         rel=1e-10)


def test_single_mode_closed_forms():
    """Squeezed vacuum: p(2n) = tanh^{2n} r (2n)!/(2^n n!)^2 / cosh r, odd p = 0;
    coherent state: Poisson with mean |alpha|^2 (fill vector = alpha)."""
    import math as _m
    from oracle import gbs as G
    r = 0.7
    V = G.pure_state_covariance(np.eye(1, dtype=complex), np.array([r]))
    B, g, pv = G.pure_B_gamma(V, np.zeros(2))
    for n in range(8):
        want = 0 if n % 2 else np.tanh(r) ** n * _m.factorial(n) / (2 ** (n // 2) * _m.factorial(n // 2)) ** 2 / np.cosh(r)
        assert G.prob_pure(B, g, pv, [n]) == pytest.approx(want, abs=1e-15)
    a = 0.6 + 0.3j
    B, g, pv = G.pure_B_gamma(np.eye(2), G.means_from_alpha(np.array([a])))
    assert g[0] == pytest.approx(a)
    for n in range(6):
        assert G.prob_pure(B, g, pv, [n]) == pytest.approx(np.exp(-abs(a) ** 2) * abs(a) ** (2 * n) / _m.factorial(n), rel=1e-12)


def test_mixed_form_thermal_closed_form():
    """Eq. lhaf for a mixed state: single-mode thermal state, p(n) = nbar^n/(nbar+1)^(n+1)."""
    from oracle import gbs as G
    nbar = 0.7
    q = G.gbs_quantities((2 * nbar + 1) * np.eye(2), np.zeros(2))
    for n in range(6):
        assert G.prob_mixed(q["A"], q["gamma"], q["pvac"], [n]) == pytest.approx(
            nbar ** n / (nbar + 1) ** (n + 1), rel=1e-12)


# ---------------------------------------------------------------- long-double oracle

@pytest.mark.parametrize("n", [24, 26, 28])
def test_long_double_more_accurate_all_ones(n):
    """The long-double subset formula (the reference of every stated-tolerance gate at
    N >= 32) carries more precision than the double one: against the exact T(n), its error
    is at least 100x smaller (11 more significand bits, ~2000x nominally)."""
    from fractions import Fraction
    A = W.all_ones(n)
    T = telephone(n)
    err_d = float(abs(Fraction(L.lhaf_subset(A).real) - T) / T)
    err_ld = float(abs(Fraction(L.lhaf_subset_ld(A).real) - T) / T)
    assert err_d > 0
    assert 100 * err_ld <= err_d, (n, err_d, err_ld)


@pytest.mark.parametrize("n", [12, 14])
def test_long_double_more_accurate_double_factorial(n):
    """haf(all-ones 2n) = (2n-1)!! through the long-double formula, 100x closer than double."""
    from fractions import Fraction
    A = W.all_ones(2 * n)
    np.fill_diagonal(A, 0)
    df = double_factorial_odd(n)
    err_d = float(abs(Fraction(L.lhaf_subset(A).real) - df) / df)
    err_ld = float(abs(Fraction(L.lhaf_subset_ld(A).real) - df) / df)
    assert err_d > 0
    assert 100 * err_ld <= err_d, (n, err_d, err_ld)


# ---------------------------------------------------------------- Eq. GBS (zero displacement)

def test_zero_displacement_formula_single_mode():
    """Eq. GBS, p(S) = haf(A_S) / (sqrt(det Q) prod s_i!), on squeezed vacuum equals the
    closed form p(2n) = tanh^{2n} r (2n)! / (2^n n!)^2 / cosh r, and 0 for odd counts."""
    import math as _m
    from oracle import gbs as G
    r = 0.55
    q = G.gbs_quantities(G.pure_state_covariance(np.eye(1, dtype=complex), np.array([r])),
                         np.zeros(2))
    for n in range(9):
        want = 0 if n % 2 else np.tanh(r) ** n * _m.factorial(n) / (2 ** (n // 2) * _m.factorial(n // 2)) ** 2 / np.cosh(r)
        assert G.prob_zero_displacement(q["A"], q["Q"], [n]) == pytest.approx(want, abs=1e-15)


def test_zero_displacement_formula_equals_loop_form_mixed():
    """On a lossy (mixed) 3-mode state with zero displacement, Eq. GBS equals Eq. lhaf
    (whose fill vector is then zero, so the loop hafnian is the hafnian)."""
    from oracle import gbs as G
    rng = W.rng_for(93, 0)
    U = W.haar_unitary(3, rng)
    V = G.pure_state_covariance(U, np.array([0.6, 0.4, 0.3]))
    eta = 0.7  # loss channel: V -> eta V + (1 - eta) hbar/2 I
    V = eta * V + (1 - eta) * (G.HBAR / 2) * np.eye(6)
    q = G.gbs_quantities(V, np.zeros(6))
    assert np.allclose(q["gamma"], 0)
    for S in [(0, 0, 0), (1, 1, 0), (2, 0, 0), (1, 2, 1), (2, 2, 2)]:
        assert G.prob_zero_displacement(q["A"], q["Q"], S) == pytest.approx(
            G.prob_mixed(q["A"], q["gamma"], q["pvac"], S), rel=1e-12, abs=1e-18)
