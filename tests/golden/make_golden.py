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
        "lhaf_n40": lambda: W.single_lhaf_mid(40),
        "lhaf_n40_repeated": lambda: gbs.expand_pure(*W.repeated_mode_state()),
        "lhaf_n50": lambda: W.large_lhaf(50),
        "lhaf_n56": lambda: W.large_lhaf(56),
    }


PLAN = {  # name: (full double, full long double, sampled terms)
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


if __name__ == "__main__":
    for nm in sys.argv[1:]:
        make(nm)
