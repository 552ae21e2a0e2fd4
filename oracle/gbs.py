"""ORACLE — test infrastructure only.

Plain numpy restatement of the Gaussian-state algebra of Sec. II and of the chain-rule
sampler of Sec. III, used to pin the conventions of the GPU path (pattern expansion,
filldiag, the fill vector gamma, the conditional fill vector of the sampler) and to give
exact probabilities for small systems. hbar = 2 throughout (results do not depend on it).

Quadrature ordering is (q_1..q_m, p_1..p_m); complex amplitudes alpha = (q + i p)/sqrt(2 hbar).
"""
from __future__ import annotations

import itertools
import math

import numpy as np

from . import lhaf as _lh

HBAR = 2.0


# ------------------------------------------------------------ states (Sec. II)

def pure_state_covariance(U: np.ndarray, r: np.ndarray):
    """Quadrature covariance V = (hbar/2) S S^T of squeezed vacuum (squeezing r_i, q
    quadrature squeezed) sent through the interferometer U (a -> U a)."""
    m = len(r)
    Sr = np.diag(np.concatenate([np.exp(-r), np.exp(r)]))
    SU = np.block([[U.real, -U.imag], [U.imag, U.real]])
    S = SU @ Sr
    return (HBAR / 2.0) * S @ S.T


def means_from_alpha(alpha: np.ndarray) -> np.ndarray:
    """R = [q; p] with alpha = (q + i p)/sqrt(2 hbar)."""
    s = math.sqrt(2 * HBAR)
    return np.concatenate([s * alpha.real, s * alpha.imag])


def F_matrix(m: int) -> np.ndarray:
    """F of Sec. II (Sigma = F V F^dagger)."""
    I = np.eye(m)
    return np.block([[I, 1j * I], [I, -1j * I]]) / math.sqrt(2 * HBAR)


def gbs_quantities(V: np.ndarray, R: np.ndarray):
    """Sec. II: Sigma = F V F^dag, Q = Sigma + I/2, A from X (I - Q^{-1}), alpha_vec = F R,
    gamma_vec = Q^{-1} alpha_vec, p(vac) = exp(-alpha^dag Q^{-1} alpha / 2)/sqrt(det Q).

    Reading of Sec. II (Eq. A_matrix with gamma = Q^{-1} alpha_vec): with F as printed, the
    matrix X (I - Q^{-1}) is the complex conjugate of the kernel that pairs with gamma in
    Eq. lhaf (its top-left block is conj(B) while gamma's first half is the unconjugated
    fill vector), and the pair then gives wrong photon statistics as soon as squeezing
    phase and displacement interact. A is therefore taken as conj(X (I - Q^{-1})); with
    this reading the probabilities equal those of Fock states built explicitly from
    matrix exponentials of the squeezing, interferometer and displacement generators
    (pinned in tests/test_oracle_pins.py)."""
    m = V.shape[0] // 2
    F = F_matrix(m)
    Sigma = F @ V @ F.conj().T
    Q = Sigma + np.eye(2 * m) / 2
    Qinv = np.linalg.inv(Q)
    X = np.block([[np.zeros((m, m)), np.eye(m)], [np.eye(m), np.zeros((m, m))]])
    A = (X @ (np.eye(2 * m) - Qinv)).conj()
    avec = F @ R
    gvec = Qinv @ avec
    pvac = (np.exp(-0.5 * (avec.conj() @ Qinv @ avec)) / np.sqrt(np.linalg.det(Q))).real
    return dict(Sigma=Sigma, Q=Q, A=A, alpha=avec, gamma=gvec, pvac=float(pvac))


def pure_B_gamma(V: np.ndarray, R: np.ndarray):
    """For a pure state A = B (+) B* (Eq. GBS-pure): B is the top-left block of A and the
    fill vector is the first half of gamma_vec."""
    g = gbs_quantities(V, R)
    m = V.shape[0] // 2
    return g["A"][:m, :m], g["gamma"][:m], g["pvac"]


# ------------------------------------------------------------ pattern expansion

def pattern_indices(pattern) -> np.ndarray:
    """Index list of B_S: mode i repeated s_i times, ascending (Sec. II, after Eq. GBS-pure;
    pattern[i] is the photon number of mode i, 0-based)."""
    return np.repeat(np.arange(len(pattern)), np.asarray(pattern, dtype=np.int64))


def expand_pure(B: np.ndarray, gamma: np.ndarray, pattern) -> np.ndarray:
    """filldiag(B_S, gamma_S) (Eq. lhaf-pure)."""
    idx = pattern_indices(pattern)
    A = B[np.ix_(idx, idx)].astype(np.complex128)
    A[np.diag_indices_from(A)] = gamma[idx]
    return A


def expand_mixed(A2: np.ndarray, gvec: np.ndarray, pattern) -> np.ndarray:
    """filldiag(A_S, gamma_S) of Eq. lhaf: rows/columns i and i+m repeated s_i times."""
    m = len(pattern)
    idx = pattern_indices(pattern)
    idx2 = np.concatenate([idx, idx + m])
    A = A2[np.ix_(idx2, idx2)].astype(np.complex128)
    A[np.diag_indices_from(A)] = gvec[idx2]
    return A


def _lhaf_small(A: np.ndarray) -> complex:
    N = A.shape[0]
    if N == 0:
        return 1.0 + 0j
    if N <= 22:
        return _lh.lhaf_dp(A)
    return _lh.lhaf_subset(A)


def _fact_prod(pattern) -> float:
    return float(np.prod([math.factorial(int(s)) for s in pattern]))


def prob_pure(B, gamma, pvac, pattern) -> float:
    """Eq. lhaf-pure: p(S) = p(vac) |lhaf(filldiag(B_S, gamma_S))|^2 / prod s_i!."""
    l = _lhaf_small(expand_pure(B, gamma, pattern))
    return float(pvac * abs(l) ** 2 / _fact_prod(pattern))


def prob_mixed(A2, gvec, pvac, pattern) -> float:
    """Eq. lhaf: p(S) = p(vac) lhaf(filldiag(A_S, gamma_S)) / prod s_i! (2N-size matrix)."""
    l = _lhaf_small(expand_mixed(A2, gvec, pattern))
    return float((pvac * l / _fact_prod(pattern)).real)


def prob_zero_displacement(A2, Q, pattern) -> float:
    """Eq. GBS: p(S) = haf(A_S) / (sqrt(det Q) prod s_i!) for zero displacement."""
    m = len(pattern)
    idx = pattern_indices(pattern)
    idx2 = np.concatenate([idx, idx + m])
    AS = A2[np.ix_(idx2, idx2)]
    h = _lh.lhaf_dp(AS, with_loops=False) if AS.shape[0] else 1.0
    return float((h / np.sqrt(np.linalg.det(Q)) / _fact_prod(pattern)).real)


def prob_table(B, gamma, pvac, m: int, cutoff: int) -> dict:
    """Exact p(S) for every pattern with s_i <= cutoff."""
    return {S: prob_pure(B, gamma, pvac, S)
            for S in itertools.product(range(cutoff + 1), repeat=m)}


# ------------------------------------------------------------ heterodyne (Sec. II)

def conditional_state(V, R, A_modes, B_modes, mu_B):
    """Eqs. condV / condR: state of modes A after heterodyne outcome mu_B (quadratures
    (q_B, p_B)) on modes B."""
    m = V.shape[0] // 2
    qa = list(A_modes) + [i + m for i in A_modes]
    qb = list(B_modes) + [i + m for i in B_modes]
    VAA = V[np.ix_(qa, qa)]
    VAB = V[np.ix_(qa, qb)]
    VBB = V[np.ix_(qb, qb)]
    K = VAB @ np.linalg.inv(VBB + HBAR / 2 * np.eye(len(qb)))
    return VAA - K @ VAB.T, R[qa] + K @ (mu_B - R[qb])


def heterodyne_cov(V, modes):
    """Husimi covariance V_Q = V + hbar/2 I restricted to `modes` (ordering (q, p))."""
    m = V.shape[0] // 2
    q = list(modes) + [i + m for i in modes]
    return (V + HBAR / 2 * np.eye(2 * m))[np.ix_(q, q)]


def alpha_from_mu(mu, nmodes):
    return (mu[:nmodes] + 1j * mu[nmodes:]) / math.sqrt(2 * HBAR)


def mu_from_alpha(alpha):
    s = math.sqrt(2 * HBAR)
    return np.concatenate([s * alpha.real, s * alpha.imag])


# ------------------------------------------------------------ chain rule (Sec. III)

def chain_rule_sample(V, R, cutoff: int, normals: np.ndarray, uniforms: np.ndarray,
                      threshold: bool = False):
    """One sample of the algorithm of Sec. III for a pure state (steps 2-6), with the random
    numbers passed in: `normals` (2(m-1) standard normals for the heterodyne draw of modes
    2..m) and `uniforms` (m numbers in [0, 1) for the draws of s_1..s_m). Conditioning uses
    Eqs. condV/condR at every step. Returns (pattern, per-step probability vectors).
    threshold=True returns the threshold-detector outcome instead of the photon numbers:
    a detector clicks (1) when its mode holds one photon or more (end of Sec. III: threshold
    samples are photon-number samples with every nonzero count replaced by 1); the
    probability vectors are those of the photon-number chain."""
    m = V.shape[0] // 2
    rest = list(range(1, m))
    mu = np.zeros(0)
    if rest:
        VQ = heterodyne_cov(V, rest)
        L = np.linalg.cholesky(VQ)
        q = list(rest) + [i + m for i in rest]
        mu = R[q] + L @ normals[: 2 * len(rest)]
    alpha_rest = alpha_from_mu(mu, len(rest)) if rest else np.zeros(0, complex)
    s = []
    probs = []
    for k in range(1, m + 1):
        A_modes = list(range(k))
        B_modes = list(range(k, m))
        if B_modes:
            # outcomes of modes k+1..m are the last m-k entries of alpha_rest
            aB = alpha_rest[k - 1:]
            Vk, Rk = conditional_state(V, R, A_modes, B_modes, mu_from_alpha(aB))
        else:
            Vk, Rk = V, R
        Bk, gk, pv = pure_B_gamma(Vk, Rk)
        p = np.array([prob_pure(Bk, gk, pv, s + [sk]) for sk in range(cutoff + 1)])
        probs.append(p)
        cdf = np.cumsum(p / p.sum())
        sk = int(np.searchsorted(cdf, uniforms[k - 1], side="right"))
        s.append(min(sk, cutoff))
    if threshold:
        return [1 if x > 0 else 0 for x in s], probs
    return s, probs
