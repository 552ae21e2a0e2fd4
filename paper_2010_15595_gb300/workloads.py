"""Seeded synthetic inputs for the loop-hafnian workloads.

This module only draws inputs; it holds none of the loop-hafnian arithmetic, so both the
GPU path's tests and the CPU oracle can take their inputs from it.

Conventions:
  * CN(0, s^2): complex normal with E|x|^2 = s^2 (real and imaginary parts N(0, s^2/2)).
  * Haar unitary: Q diag(R_ii/|R_ii|) from the QR factorisation of a complex Gaussian
    matrix G_ij = (x + i y)/sqrt(2) (phase-fixed QR).
  * A pure squeezed state through interferometer U has the kernel matrix
    B = U diag(tanh r) U^T (Sec. II, Eq. GBS-pure: A = B (+) B*).
  * Every generator takes a seed; the bit generator is numpy's Philox counter-based
    generator, so a (config, seed) pair always yields the same matrices on any host.
"""
from __future__ import annotations

import numpy as np

_KEY_BASE = 0x20101559


def rng_for(config_id: int, seed: int = 0) -> np.random.Generator:
    return np.random.Generator(np.random.Philox(key=[_KEY_BASE + int(config_id), int(seed)]))


def haar_unitary(M: int, rng: np.random.Generator) -> np.ndarray:
    G = (rng.standard_normal((M, M)) + 1j * rng.standard_normal((M, M))) / np.sqrt(2.0)
    Q, R = np.linalg.qr(G)
    d = np.diag(R)
    return Q * (d / np.abs(d))[None, :]


def complex_normal(size, sigma: float, rng: np.random.Generator) -> np.ndarray:
    s = sigma / np.sqrt(2.0)
    return s * rng.standard_normal(size) + 1j * s * rng.standard_normal(size)


def squeezed_kernel(U: np.ndarray, r: np.ndarray) -> np.ndarray:
    """B = U diag(tanh r) U^T, symmetrised against rounding."""
    B = (U * np.tanh(r)[None, :]) @ U.T
    return 0.5 * (B + B.T)


def with_diagonal(B: np.ndarray, v: np.ndarray) -> np.ndarray:
    """Copy of B whose diagonal is v (the config matrices are defined this way)."""
    A = np.array(B, dtype=np.complex128, copy=True)
    A[np.diag_indices_from(A)] = v
    return A


# ---------------------------------------------------------------- lhaf configs

def single_lhaf_n16(seed: int = 0) -> np.ndarray:
    """N=16: M=16 modes, Haar U, r_i = 0.6, diagonal gamma_i ~ CN(0, 0.3^2), one photon
    per mode (256 pair subsets)."""
    rng = rng_for(1, seed)
    U = haar_unitary(16, rng)
    B = squeezed_kernel(U, np.full(16, 0.6))
    return with_diagonal(B, complex_normal(16, 0.3, rng))


def single_lhaf_mid(N: int, seed: int = 0) -> np.ndarray:
    """N=32 / N=40 family: M=N modes, Haar U, r_i ~ U[0.4, 0.9], gamma ~ CN(0, 0.2^2)."""
    rng = rng_for(2, seed * 1000 + N)
    U = haar_unitary(N, rng)
    r = rng.uniform(0.4, 0.9, N)
    B = squeezed_kernel(U, r)
    return with_diagonal(B, complex_normal(N, 0.2, rng))


def repeated_mode_state(seed: int = 0):
    """N=40 with repeated modes: M=20 modes x 2 photons. Returns (B, gamma, pattern); the
    loop-hafnian matrix is filldiag(B_S, gamma_S) with rows/columns repeated per pattern."""
    rng = rng_for(3, seed)
    U = haar_unitary(20, rng)
    r = rng.uniform(0.4, 0.9, 20)
    B = squeezed_kernel(U, r)
    gamma = complex_normal(20, 0.2, rng)
    return B, gamma, np.full(20, 2, dtype=np.int32)


def large_lhaf(N: int, seed: int = 0) -> np.ndarray:
    """N=50 / N=56: M=N modes, Haar U, r_i = 0.8, gamma ~ CN(0, 0.1^2)."""
    rng = rng_for(5, seed * 1000 + N)
    U = haar_unitary(N, rng)
    B = squeezed_kernel(U, np.full(N, 0.8))
    return with_diagonal(B, complex_normal(N, 0.1, rng))


def block_diagonal_large(N1: int, N2: int, seed: int = 0):
    """An N1+N2 matrix P (A1 (+) A2) P^T made of two independent large-config blocks
    (large_lhaf of sizes N1 and N2, different seeds) under a seeded symmetric permutation P
    of the rows and columns. Returns (A, A1, A2). Its loop hafnian is lhaf(A1) lhaf(A2)
    (a perfect matching with loops of a block-diagonal graph pairs vertices inside blocks
    only, and relabelling vertices leaves the sum unchanged), so a reference at N = 50 or 56
    costs two evaluations of half the size."""
    A1 = large_lhaf(N1, seed=2 * seed + 1)
    A2 = large_lhaf(N2, seed=2 * seed + 2)
    N = N1 + N2
    D = np.zeros((N, N), dtype=np.complex128)
    D[:N1, :N1] = A1
    D[N1:, N1:] = A2
    perm = rng_for(9, seed * 1000 + N).permutation(N)
    return D[np.ix_(perm, perm)], A1, A2


def random_symmetric_uniform(N: int, seed: int = 0) -> np.ndarray:
    """Timing side workload of Sec. IV (Fig. 3): Re and Im of every entry ~ U[0, 1], then
    symmetrised."""
    rng = rng_for(6, seed * 1000 + N)
    X = rng.uniform(0, 1, (N, N)) + 1j * rng.uniform(0, 1, (N, N))
    return 0.5 * (X + X.T)


def all_ones(N: int) -> np.ndarray:
    return np.ones((N, N), dtype=np.complex128)


def random_complex_symmetric(N: int, rng: np.random.Generator, scale: float = 1.0):
    X = scale * (rng.standard_normal((N, N)) + 1j * rng.standard_normal((N, N)))
    return 0.5 * (X + X.T)


# ---------------------------------------------------------------- batched config

def batch_state(seed: int = 0):
    """M=100-mode state for the batched workload: r_i = 0.7, Haar U, gamma ~ CN(0, 0.1^2).
    Returns (B, gamma)."""
    rng = rng_for(4, seed)
    U = haar_unitary(100, rng)
    B = squeezed_kernel(U, np.full(100, 0.7))
    return B, complex_normal(100, 0.1, rng)


def batch_patterns(count: int = 4096, seed: int = 0, M: int = 100, n_min: int = 10,
                   n_max: int = 30, max_per_mode: int = 3):
    """Photon patterns of uneven total N, uniform over even values n_min..n_max: photons are
    added one at a time to a uniformly random mode whose count is below max_per_mode."""
    rng = rng_for(7, seed)
    sizes = rng.choice(np.arange(n_min, n_max + 1, 2), size=count)
    pats = np.zeros((count, M), dtype=np.int32)
    for b, N in enumerate(sizes):
        for _ in range(int(N)):
            free = np.nonzero(pats[b] < max_per_mode)[0]
            pats[b, free[rng.integers(len(free))]] += 1
    return pats


# ---------------------------------------------------------------- serving config

def serving_state(seed: int = 0, M: int = 100, n_squeezed: int = 25, r: float = 0.8,
                  sigma: float = 0.1):
    """Chain-rule sampler state: M modes, Haar U, squeezing r on the first n_squeezed input
    modes (mean photon number ~ n_squeezed sinh^2 r + M sigma^2 ~ 20), output displacement
    alpha ~ CN(0, sigma^2). Returns (U, r_vec, alpha)."""
    rng = rng_for(8, seed)
    U = haar_unitary(M, rng)
    rv = np.zeros(M)
    rv[:n_squeezed] = r
    alpha = complex_normal(M, sigma, rng)
    return U, rv, alpha
