"""Launch-shape autotuner for the batched loop-hafnian kernel.

For a batch whose largest matrix has n_max index pairs, the tunable is the number of warps
per CTA of the persistent kernel (each warp owns one subset work area in shared memory, so
more warps means more latency hiding but a larger footprint). `tune_batch` times every
candidate on a seeded synthetic batch of the same size range through the C ABI, applies
the fastest with gbsh_set_batch_tuning, and records it in a JSON cache keyed by GPU name,
n_max and precision (path: $GBSH_TUNE_CACHE, default ~/.cache/gbsh/tune.json).
`apply_cache()` re-applies recorded choices in a new process. The choice never changes
results: a problem's subset chunking depends only on its size.
"""
from __future__ import annotations

import json
import os
import time

import numpy as np

from . import lib, workloads

CANDIDATES = (4, 6, 8, 12, 16)


def cache_path() -> str:
    return os.environ.get("GBSH_TUNE_CACHE",
                          os.path.join(os.path.expanduser("~"), ".cache", "gbsh", "tune.json"))


def _gpu_name() -> str:
    import torch
    return torch.cuda.get_device_name() if torch.cuda.is_available() else "none"


def _load() -> dict:
    try:
        with open(cache_path()) as f:
            return json.load(f)
    except (OSError, ValueError):
        return {}


def _store(entries: dict):
    path = cache_path()
    os.makedirs(os.path.dirname(path), exist_ok=True)
    tmp = path + f".tmp{os.getpid()}"
    with open(tmp, "w") as f:
        json.dump(entries, f, indent=1)
    os.replace(tmp, path)


def _key(n_max: int, precision: int) -> str:
    return f"{_gpu_name()}|batch|n_max={n_max}|prec={precision}"


def synthetic_batch(n_max: int, count: int = 512, seed: int = 0):
    """Seeded complex symmetric matrices with N uniform over even values 2..2 n_max."""
    rng = np.random.default_rng(seed)
    sizes = rng.choice(np.arange(2, 2 * n_max + 1, 2), size=count)
    sizes[0] = 2 * n_max
    return [workloads.random_complex_symmetric(int(N), rng, 0.3) for N in sizes]


def tune_batch(n_max: int, precision: int = lib.PREC_FP64, candidates=CANDIDATES, reps: int = 2,
               count: int = 512, record: bool = True) -> dict:
    """Times each candidate warps-per-CTA; applies and (optionally) records the fastest.
    Returns {"best": W, "seconds": {W: t}}. Candidates that do not fit are skipped."""
    mats = synthetic_batch(n_max, count)
    times = {}
    for w in candidates:
        try:
            lib.set_batch_tuning(precision, n_max, w)
            lib.lhaf_batch(mats, precision=precision)  # warm-up
            t0 = time.perf_counter()
            for _ in range(reps):
                lib.lhaf_batch(mats, precision=precision)
            times[w] = (time.perf_counter() - t0) / reps
        except lib.GbshError:
            continue
    if not times:
        lib.set_batch_tuning(precision, n_max, 0)
        return {"best": 0, "seconds": {}}
    best = min(times, key=times.get)
    lib.set_batch_tuning(precision, n_max, best)
    if record:
        entries = _load()
        entries[_key(n_max, precision)] = {"warps": best, "seconds": times}
        _store(entries)
    return {"best": best, "seconds": times}


def apply_cache() -> int:
    """Applies every recorded choice for this GPU; returns how many were applied."""
    prefix = _gpu_name() + "|batch|"
    n = 0
    for key, val in _load().items():
        if not key.startswith(prefix):
            continue
        fields = dict(part.split("=") for part in key[len(prefix):].split("|"))
        lib.set_batch_tuning(int(fields["prec"]), int(fields["n_max"]), int(val["warps"]))
        n += 1
    return n
