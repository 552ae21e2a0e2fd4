"""ORACLE — test infrastructure only.

Philox4x32-10 counter-based generator (Salmon, Moraes, Dror, Shaw, "Parallel random
numbers: as easy as 1, 2, 3", SC'11), written from its published definition in plain
numpy/Python integers, plus the mappings the sampler uses: a uniform double from the top
53 bits of two 32-bit words, and standard normals by the Box-Muller transform. Used to give
the oracle sampler the same random numbers as the GPU sampler from the same seed.
"""
import math

import numpy as np

M0, M1 = 0xD2511F53, 0xCD9E8D57
W0, W1 = 0x9E3779B9, 0xBB67AE85
MASK = 0xFFFFFFFF


def philox4x32_10(counter, key):
    c = [int(x) & MASK for x in counter]
    k0, k1 = int(key[0]) & MASK, int(key[1]) & MASK
    for _ in range(10):
        p0 = M0 * c[0]
        p1 = M1 * c[2]
        c = [((p1 >> 32) ^ c[1] ^ k0) & MASK, p1 & MASK,
             ((p0 >> 32) ^ c[3] ^ k1) & MASK, p0 & MASK]
        k0 = (k0 + W0) & MASK
        k1 = (k1 + W1) & MASK
    return c


def uniform53(hi, lo):
    return ((hi << 32 | lo) >> 11) * 2.0 ** -53


def _words(seed, chain, stream, index):
    key = (seed & MASK, (seed >> 32) & MASK)
    return philox4x32_10((chain, stream, index, 0), key)


def chain_normals(seed, chain, count):
    """`count` standard normals of sample `chain` of a request with this seed (stream 0)."""
    z = np.zeros(count)
    for b in range((count + 1) // 2):
        w = _words(seed, chain, 0, b)
        u1, u2 = uniform53(w[0], w[1]), uniform53(w[2], w[3])
        r = math.sqrt(-2.0 * math.log(1.0 - u1))
        z[2 * b] = r * math.cos(2.0 * math.pi * u2)
        if 2 * b + 1 < count:
            z[2 * b + 1] = r * math.sin(2.0 * math.pi * u2)
    return z


def chain_uniforms(seed, chain, count):
    """Uniforms u_1..u_count for the draws of s_1..s_count (stream 1)."""
    out = np.zeros(count)
    for k in range(count):
        w = _words(seed, chain, 1, k)
        out[k] = uniform53(w[0], w[1])
    return out
