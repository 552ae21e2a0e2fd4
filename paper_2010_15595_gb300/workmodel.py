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
def subset_ops(k: int, n: int):
    """(complex multiply-adds, complex multiplies, complex adds, complex reciprocals, extra
    real flops) of one subset of popcount k, following the kernel's algorithm."""
    if k == 0:
        return (0, 0, 0, 0, 0)
    S = 2 * k + 1
    D = n + 1
    mac = mul = add = rcp = 0
    for c in range(S - 2):
        r = S - c - 2
        mul += r
        rcp += 1
        mac += r * (S - c - 1) + S * r
    mul += S * (S - 1)
    for s in range(S):
        degs = min(s, D)
        for d in range(0, min(s + 1, D) + 1):
            if d <= degs:
                add += 1
            if d >= 1:
                mac += 1
        for t in range(s + 2, S + 1):
            emax = min(degs, D - (t - s))
            if emax >= 0:
                mac += emax + 1
    mac += sum(D - s for s in range(D))
    mac += sum(n - s for s in range(1, n))
    mac += sum(n - s for s in range(n))
    extra = n * 2 + n * 4 + n * 2 + 14
    return (mac, mul, add, rcp, extra)


@lru_cache(maxsize=None)
def subset_flops(k: int, n: int) -> int:
    mac, mul, add, rcp, extra = subset_ops(k, n)
    return 8 * mac + 6 * mul + 2 * add + 7 * rcp + extra


# FP32 instructions of the triple-float primitives (lhaf_tf.cuh), counted from their code:
# TwoSum 6, TwoProduct 2; one component of the fused multiply-accumulate 108, so a complex
# multiply-accumulate (and a complex multiply, which is one with a zero accumulator) is 216;
# a triple-float add 39 (complex 78); the complex reciprocal (|b|^2, two Newton steps, two
# multiplies) 445. The power-of-two rescalings are exact integer or single-multiply steps and
# are not counted.
TF_INSTR = {"mac": 216, "mul": 216, "add": 78, "rcp": 445}


@lru_cache(maxsize=None)
def subset_tf_instr(k: int, n: int) -> int:
    """FP32 arithmetic instructions of one subset on the triple-float path."""
    mac, mul, add, rcp, _ = subset_ops(k, n)
    # the C(a,b) products are exact power-of-two scalings on this path (S(S-1) of the muls)
    S = 2 * k + 1 if k else 0
    mul_fp = mul - S * (S - 1)
    return TF_INSTR["mac"] * mac + TF_INSTR["mul"] * mul_fp + TF_INSTR["add"] * add + TF_INSTR["rcp"] * rcp


@lru_cache(maxsize=None)
def lhaf_tf_instr(N: int) -> int:
    n = (N + (N & 1)) // 2
    return sum(comb(n, k) * subset_tf_instr(k, n) for k in range(1, n + 1))


def householder_flops(N: int) -> float:
    """The fixed per-subset convention F(m, n) = (40/3) m^3 + (4/3) m^3 + 8 n m^2 + 4 n^2
    (m = 2k: a Householder Hessenberg reduction, La Budde, explicit loop matvecs, the
    exp-polynomial), summed over the subsets. It counts a different algorithm from the
    kernel's (elimination Hessenberg at half the Householder flops, no matvecs), so it is
    reported beside the kernel's own count, not as the roofline numerator."""
    n = (N + (N & 1)) // 2
    tot = 0.0
    for k in range(1, n + 1):
        m = 2 * k
        tot += comb(n, k) * ((40.0 / 3.0) * m ** 3 + (4.0 / 3.0) * m ** 3 + 8.0 * n * m * m + 4.0 * n * n)
    return tot


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
# Derived FP32 instruction issue rate of one GB300: 152 SMs x 128 FP32 lanes per clock x
# 2.070 GHz (one FP32 instruction per lane per clock, an FMA counting once).
FP32_INSTR_PEAK_DERIVED_T = 152 * 128 * 2.070e9 / 1e12
