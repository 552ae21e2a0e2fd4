"""Writes the stored expected values used by the GPU parity tests at large N.

Calls only the CPU oracle (oracle/) on inputs from the seeded generators. Each fixture
stores the input matrix itself (exact decimal round-trip of every double), so a test on
another host compares against the same bits, plus the oracle's values:
  lhaf_d   subset formula in double, with abs_sum = sum_Z |p_Z| and
           sq_sum = sum_Z |p_Z|^2 (the scales of the cancellation in the signed sum);
  lhaf_ld  the same formula in long double (x86-64 80-bit extended), when requested:
           the reference for sizes where the double oracle's own rounding error is near
           the parity tolerance;
  terms    p_Z of a seeded sample of subsets (double), for sampled per-subset parity.
Usage: python tests/golden/make_golden.py NAME [NAME ...]
       python tests/golden/make_golden.py --add-ld NAME   (adds lhaf_ld to an existing
       fixture, from its stored matrix, keeping every other value)
Block-diagonal fixtures (lhaf_n50_block, lhaf_n56_block) store as lhaf_ld the product of the
long-double oracle's values of their two blocks.
"""
import json
import os
import platform
import sys
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
sys.path.insert(0, ROOT)

from oracle import gbs  # noqa: E402
from oracle import lhaf as L  # noqa: E402
from paper_2010_15595_gb300 import workloads as W  # noqa: E402


def fixtures():
    return {
        "lhaf_n32": lambda: W.single_lhaf_mid(32),
        "lhaf_n40": lambda: W.single_lhaf_mid(40),
        "lhaf_n40_repeated": lambda: gbs.expand_pure(*W.repeated_mode_state()),
        "lhaf_n50": lambda: W.large_lhaf(50),
        "lhaf_n56": lambda: W.large_lhaf(56),
    }


PLAN = {  # name: (full double, full long double, sampled terms)
    "lhaf_n32": (True, True, 256),
    "lhaf_n40": (True, True, 256),
    "lhaf_n40_repeated": (True, True, 256),
    "lhaf_n50": (True, False, 256),
    "lhaf_n56": (False, False, 256),
}


def write_matrix(path, A):
    with open(path, "w") as f:
        f.write(f"{A.shape[0]}\n")
        for row in A:
            f.write(" ".join(f"{repr(float(x.real))} {repr(float(x.imag))}" for x in row) + "\n")


def read_matrix(path):
    with open(path) as f:
        N = int(f.readline())
        vals = np.array([float(t) for t in f.read().split()])
    return (vals[0::2] + 1j * vals[1::2]).reshape(N, N)


def make(name):
    A = fixtures()[name]()
    do_d, do_ld, nterms = PLAN[name]
    mpath = os.path.join(HERE, f"{name}.matrix.txt")
    write_matrix(mpath, A)
    A = read_matrix(mpath)  # use exactly the stored bits
    N = A.shape[0]
    n = (N + 1) // 2
    rec = {"name": name, "N": N, "generator": "paper_2010_15595_gb300.workloads",
           "host": platform.machine(), "oracle": "oracle/lhaf_oracle.c subset formula"}
    rng = np.random.default_rng(12345)
    zs = rng.integers(1, 1 << n, nterms, dtype=np.uint64)
    zs = np.unique(np.concatenate([zs, [np.uint64((1 << n) - 1)]])).astype(np.uint64)
    pz = L.subset_terms(A, zs)
    rec["terms"] = [[int(z), float(p.real), float(p.imag)] for z, p in zip(zs, pz)]
    if do_d:
        t = time.time()
        v, s, sq = L.lhaf_subset_stats(A)
        rec["lhaf_d"] = [v.real, v.imag]
        rec["abs_sum"] = s
        rec["sq_sum"] = sq
        rec["kappa"] = s / abs(v)
        rec["seconds_d"] = time.time() - t
    if do_ld:
        t = time.time()
        v = L.lhaf_subset_ld(A)
        rec["lhaf_ld"] = [v.real, v.imag]
        rec["seconds_ld"] = time.time() - t
        if do_d:
            rec["rel_d_vs_ld"] = abs(complex(*rec["lhaf_d"]) - v) / abs(v)
    with open(os.path.join(HERE, f"{name}.json"), "w") as f:
        json.dump(rec, f, indent=1)
    print(name, {k: rec[k] for k in rec if k not in ("terms",)}, flush=True)


BLOCKS = {  # name: block sizes of W.block_diagonal_large
    "lhaf_n50_block": (22, 28),
    "lhaf_n56_block": (28, 28),
}


def make_block(name):
    """Block-diagonal fixture: the full matrix, and as its reference the product of the
    long-double oracle's values of the two blocks (lhaf of a direct sum is the product of
    the blocks' loop hafnians; the identity and permutation invariance are pinned by the
    oracle tests). The double-oracle values of the blocks are stored too."""
    N1, N2 = BLOCKS[name]
    A, A1, A2 = W.block_diagonal_large(N1, N2)
    mpath = os.path.join(HERE, f"{name}.matrix.txt")
    write_matrix(mpath, A)
    A = read_matrix(mpath)
    rec = {"name": name, "N": A.shape[0], "blocks": [N1, N2],
           "generator": "paper_2010_15595_gb300.workloads.block_diagonal_large",
           "host": platform.machine(), "oracle": "oracle/lhaf_oracle.c subset formula"}
    t = time.time()
    l1, l2 = L.lhaf_subset_ld(A1), L.lhaf_subset_ld(A2)
    d1, d2 = L.lhaf_subset(A1), L.lhaf_subset(A2)
    rec["block_ld"] = [[l1.real, l1.imag], [l2.real, l2.imag]]
    rec["block_d"] = [[d1.real, d1.imag], [d2.real, d2.imag]]
    p = l1 * l2
    rec["lhaf_ld"] = [p.real, p.imag]
    rec["rel_d_vs_ld"] = abs(d1 * d2 - p) / abs(p)
    rec["seconds_ld"] = time.time() - t
    with open(os.path.join(HERE, f"{name}.json"), "w") as f:
        json.dump(rec, f, indent=1)
    print(name, rec, flush=True)


def add_ld(name):
    """Adds the long-double oracle value to an existing fixture, computed from its stored
    matrix; the other stored values are kept as they are."""
    jpath = os.path.join(HERE, f"{name}.json")
    with open(jpath) as f:
        rec = json.load(f)
    A = read_matrix(os.path.join(HERE, f"{name}.matrix.txt"))
    t = time.time()
    v = L.lhaf_subset_ld(A)
    rec["lhaf_ld"] = [v.real, v.imag]
    rec["seconds_ld"] = time.time() - t
    rec["host_ld"] = platform.machine()
    if "lhaf_d" in rec:
        rec["rel_d_vs_ld"] = abs(complex(*rec["lhaf_d"]) - v) / abs(v)
    with open(jpath, "w") as f:
        json.dump(rec, f, indent=1)
    print(name, {k: rec[k] for k in rec if k not in ("terms",)}, flush=True)


if __name__ == "__main__":
    if sys.argv[1:2] == ["--add-ld"]:
        for nm in sys.argv[2:]:
            add_ld(nm)
    else:
        for nm in sys.argv[1:]:
            if nm in BLOCKS:
                make_block(nm)
            else:
                make(nm)
