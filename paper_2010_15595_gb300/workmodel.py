"""Algorithmic work of the loop-hafnian kernels, for roofline accounting.

Counts the FP64 floating-point operations the kernel's algorithm needs for one subset of
popcount k (matrix size m = 2k, bordered size S = m + 1) of an N = 2n evaluation, lane by
lane, counting only lanes that do useful work (idle lanes of a warp instruction are not
algorithmic work). Conventions: complex multiply-add = 8 flops, complex multiply = 6,
complex add = 2, complex reciprocal = 7.

  Hessenberg reduction (stabilised elementary similarities), for columns c = 0..S-3:
      multipliers (S-c-2) complex multiplies, one complex reciprocal,
      row update (S-c-2)(S-c-1) and column update S(S-c-2) complex multiply-adds
  La Budde coefficients C(a,b) = H[a][b] prod H[l+1][l]: S(S-1) complex multiplies
  La Budde push recursion truncated at degree D = n+1: one complex multiply-add per
      (target polynomial, coefficient) pair that receives a term
  series: ratio (D^2/2), Newton identities (n^2/2) and exp-polynomial (n^2/2) recursions
  signed compensated accumulation: 14 flops
"""
from __future__ import annotations

from functools import lru_cache
from math import comb


@lru_cache(maxsize=None)
def subset_flops(k: int, n: int) -> int:
    if k == 0:
        return 0
    S = 2 * k + 1
    D = n + 1
    MAC, MUL, ADD, RCP = 8, 6, 2, 7
    f = 0
    for c in range(S - 2):
        r = S - c - 2
        f += r * MUL + RCP + r * (S - c - 1) * MAC + S * r * MAC
    f += S * (S - 1) * MUL
    for s in range(S):
        degs = min(s, D)
        for d in range(0, min(s + 1, D) + 1):
            if d <= degs:
                f += ADD
            if d >= 1:
                f += MAC
        for t in range(s + 2, S + 1):
            emax = min(degs, D - (t - s))
            if emax >= 0:
                f += (emax + 1) * MAC
    f += sum(D - s for s in range(D)) * MAC
    f += n * 2 + sum(n - s for s in range(1, n)) * MAC
    f += n * 4 + sum(n - s for s in range(n)) * MAC + n * 2
    f += 14
    return f


@lru_cache(maxsize=None)
def lhaf_flops(N: int) -> int:
    """Algorithmic FP64 flops of one N x N loop hafnian (odd N padded)."""
    n = (N + (N & 1)) // 2
    return sum(comb(n, k) * subset_flops(k, n) for k in range(1, n + 1))


def subset_count(N: int) -> int:
    n = (N + (N & 1)) // 2
    return 1 << n


# Derived FP64 peak of one GB300: 152 SMs x 2 FP64 FMA lanes per SM per clock x 2 flops
# x 2.070 GHz maximum SM clock.
FP64_PEAK_DERIVED_TFLOPS = 152 * 2 * 2 * 2.070e9 / 1e12
