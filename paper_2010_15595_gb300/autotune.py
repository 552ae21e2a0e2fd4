"""Launch-shape autotuner of the loop-hafnian kernels.

Two kinds of entries, both timed through the C ABI on seeded synthetic inputs:

* single evaluations of size N (gbsh_lhaf*, per precision FP64 / triple-float): the cap on
  warps per CTA, the popcount-class ladder (coarse or fine steps of warps per CTA) and the
  enumeration chunk count (subsets per chunk = 2^n / chunks: the unit a warp claims from the
  counter, i.e. subsets per warp between claims). Tiles, in this kernel, are the per-warp
  shared-memory work areas, whose size follows from the class's largest popcount, so the
  ladder is what shapes them.
* batched evaluations whose largest problem has n_max pairs: warps per CTA of the
  small-popcount class and of the large-popcount class.

`tune_lhaf` / `tune_batch` search these on the current GPU, apply the winner for this process
and record it in a JSON cache keyed by GPU name (path: $GBSH_TUNE_CACHE, default
~/.cache/gbsh/tune.json); `apply_cache()` re-applies recorded choices. `emit_table()` turns
tuning results into the library's built-in table (csrc/tuned_gb300.inc), which the library
applies by default:

    python -m paper_2010_15595_gb300.autotune --table csrc/tuned_gb300.inc --json out.json

A launch shape never changes which subsets are summed. Batched results are bit-identical
under any entry; for single evaluations the ladder and chunk count regroup the compensated
cross-subset sum, so results agree to its rounding.
"""
from __future__ import annotations

import argparse
import json
import os
import time

import numpy as np

from . import lib, workloads

CANDIDATES = (4, 6, 8, 12, 16)          # warps per CTA, large-popcount batch class
SMALL_CANDIDATES = (8, 12, 16)          # warps per CTA, small-popcount batch class
WARPS_CAPS = (8, 10, 12, 14, 16)        # single evaluation: cap on warps per CTA
LADDERS = (lib.LADDER_COARSE, lib.LADDER_FINE)
LOG2_CHUNKS = (14, 16, 17, 18)
TUNE_SIZES = (24, 28, 32, 36, 40, 44)   # single-evaluation sizes tuned for the built-in table
KEEP_DEFAULT_WITHIN = 0.01              # a candidate must beat the default by more than 1 %


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


def _record(key: str, value: dict):
    entries = _load()
    entries[key] = value
    _store(entries)


def _key(n_max: int, precision: int) -> str:
    return f"{_gpu_name()}|batch|n_max={n_max}|prec={precision}"


def _lhaf_key(N: int, precision: int) -> str:
    return f"{_gpu_name()}|lhaf|N={N}|prec={precision}"


def synthetic_batch(n_max: int, count: int = 512, seed: int = 0):
    """Seeded complex symmetric matrices with N uniform over even values 2..2 n_max."""
    rng = np.random.default_rng(seed)
    sizes = rng.choice(np.arange(2, 2 * n_max + 1, 2), size=count)
    sizes[0] = 2 * n_max
    return [workloads.random_complex_symmetric(int(N), rng, 0.3) for N in sizes]


def _pick(times: dict, default_key):
    """Fastest entry, unless it beats the default by no more than KEEP_DEFAULT_WITHIN."""
    best = min(times, key=times.get)
    if default_key in times and times[best] >= (1.0 - KEEP_DEFAULT_WITHIN) * times[default_key]:
        return default_key
    return best


def tune_batch(n_max: int, precision: int = lib.PREC_FP64, candidates=CANDIDATES,
               small_candidates=(16,), reps: int = 2, count: int = 512,
               record: bool = True) -> dict:
    """Times each (small-class, large-class) warps-per-CTA pair; applies and (optionally)
    records the fastest. Returns {"best": W_large, "best_small": W_small, "seconds": {...}}
    (seconds keyed by W_large when only one small-class value is tried, else by
    "W_small/W_large"). Pairs that do not fit are skipped."""
    mats = synthetic_batch(n_max, count)
    times = {}
    for w0 in small_candidates:
        for w in candidates:
            try:
                lib.set_batch_tuning(precision, n_max, w, warps_small=w0)
                lib.lhaf_batch(mats, precision=precision)  # warm-up
                t0 = time.perf_counter()
                for _ in range(reps):
                    lib.lhaf_batch(mats, precision=precision)
                times[(w0, w)] = (time.perf_counter() - t0) / reps
            except lib.GbshError:
                continue
    if not times:
        lib.set_batch_tuning(precision, n_max, 0, warps_small=0)
        return {"best": 0, "best_small": 0, "seconds": {}}
    w0, best = _pick(times, (16, 8))
    lib.set_batch_tuning(precision, n_max, best, warps_small=w0)
    if len(small_candidates) == 1:
        secs = {w: t for (_, w), t in times.items()}
    else:
        secs = {f"{a}/{b}": t for (a, b), t in times.items()}
    if record:
        _record(_key(n_max, precision), {"warps": best, "warps_small": w0, "seconds": secs})
    return {"best": best, "best_small": w0, "seconds": secs}


def _time_lhaf(A_dev, precision: int, reps: int) -> float:
    lib.lhaf(A_dev, precision=precision)  # warm-up (also builds the plan's scratch)
    best = float("inf")
    for _ in range(reps):
        t0 = time.perf_counter()
        lib.lhaf(A_dev, precision=precision)
        best = min(best, time.perf_counter() - t0)
    return best


def library_default(precision: int):
    """(warps_cap, ladder, log2_chunks) of the library's untuned plan."""
    return (16 if precision == lib.PREC_TF else 12, lib.LADDER_COARSE, 18)


def tune_lhaf(N: int, precision: int = lib.PREC_FP64, warps_caps=WARPS_CAPS, ladders=LADDERS,
              log2_chunks=LOG2_CHUNKS, reps: int = 2, record: bool = True, seed: int = 0) -> dict:
    """Single evaluation of size N: grid over (warps cap, ladder) at 2^18 chunks, then the
    chunk count at the best pair; a candidate replaces the library default only if it is more
    than 1 % faster. Applies the winner for this process; returns {"best": (warps_cap, ladder,
    log2_chunks), "seconds": {"w/l/c": t}, "default": t}."""
    import torch
    rng = np.random.default_rng(seed)
    A = torch.from_numpy(workloads.random_complex_symmetric(N, rng, 0.3)).cuda()
    n = (N + (N & 1)) // 2
    default = library_default(precision)
    times = {}

    def run(cfg):
        if cfg not in times:
            try:
                lib.set_lhaf_tuning(precision, N, *cfg)
                times[cfg] = _time_lhaf(A, precision, reps)
            except lib.GbshError:
                pass
        return times.get(cfg)

    run(default)
    for w in warps_caps:
        for ld in ladders:
            run((w, ld, 18))
    w, ld, _ = _pick(times, default)
    for c in log2_chunks:
        if c <= n:
            run((w, ld, c))
    best = _pick(times, default)
    lib.set_lhaf_tuning(precision, N, *best)
    secs = {"/".join(map(str, k)): v for k, v in times.items()}
    out = {"best": best, "seconds": secs, "default": times[default]}
    if record:
        _record(_lhaf_key(N, precision), {"cfg": list(best), "seconds": secs})
    return out


def apply_cache() -> int:
    """Applies every recorded choice for this GPU; returns how many were applied."""
    prefix = _gpu_name() + "|"
    n = 0
    for key, val in _load().items():
        if not key.startswith(prefix):
            continue
        kind, *rest = key[len(prefix):].split("|")
        fields = dict(part.split("=") for part in rest)
        if kind == "batch":
            lib.set_batch_tuning(int(fields["prec"]), int(fields["n_max"]), int(val["warps"]),
                                 warps_small=int(val.get("warps_small", 0)))
        elif kind == "lhaf":
            lib.set_lhaf_tuning(int(fields["prec"]), int(fields["N"]), *map(int, val["cfg"]))
        else:
            continue
        n += 1
    return n


def emit_table(single: list, batch: list, note: str) -> str:
    """C source of the built-in table. single: [(prec, N_lo, N_hi, warps_cap, ladder,
    log2_chunks)], batch: [(prec, nmax_lo, nmax_hi, warps_small, warps_large)]."""
    lines = ["// Built-in launch-shape table, written by autotune.py (do not edit by hand).",
             *[f"// {ln}" for ln in note.splitlines()],
             "static const TunedSingleEntry kTunedSingle[] = {"]
    lines += [f"    {{{', '.join(map(str, e))}}}," for e in single]
    lines += ["    {-1, 0, 0, 0, 0, 0},", "};", "static const TunedBatchEntry kTunedBatch[] = {"]
    lines += [f"    {{{', '.join(map(str, e))}}}," for e in batch]
    lines += ["    {-1, 0, 0, 0, 0},", "};", ""]
    return "\n".join(lines)


def table_entries(results: dict, max_n: int = 60):
    """Single-evaluation table rows from {(prec, N): (w, ladder, chunks)}: a tuned size N covers
    N up to the next tuned size of the same precision (the first one from N = 1, the last one
    up to max_n). Entries equal to the library default are dropped."""
    rows = []
    for prec in sorted({p for p, _ in results}):
        Ns = sorted(N for p, N in results if p == prec)
        for i, N in enumerate(Ns):
            hi = Ns[i + 1] - 1 if i + 1 < len(Ns) else max_n
            cfg = tuple(results[(prec, N)])
            if cfg != library_default(prec):
                rows.append((prec, N if i else 1, hi, *cfg))
    return rows


def main(argv=None):
    ap = argparse.ArgumentParser(description=__doc__.split("\n\n")[0])
    ap.add_argument("--sizes", default=",".join(map(str, TUNE_SIZES)))
    ap.add_argument("--batch-nmax", type=int, default=15)
    ap.add_argument("--batch-count", type=int, default=4096)
    ap.add_argument("--table", default=None, help="write the built-in table (C source) here")
    ap.add_argument("--json", default=None, help="write every timing here")
    a = ap.parse_args(argv)
    import torch
    torch.cuda.init()
    sizes = [int(s) for s in a.sizes.split(",") if s]
    results, report = {}, {"gpu": _gpu_name(), "single": {}, "batch": {}}
    for prec in (lib.PREC_TF, lib.PREC_FP64):
        for N in sizes:
            t0 = time.time()
            r = tune_lhaf(N, prec, record=False)
            results[(prec, N)] = r["best"]
            report["single"][f"prec={prec}|N={N}"] = {**r, "wall_s": time.time() - t0}
            print(f"lhaf prec={prec} N={N}: best {r['best']} "
                  f"{min(r['seconds'].values()) * 1e3:.2f} ms (default {r['default'] * 1e3:.2f} ms)",
                  flush=True)
    brows = []
    for prec in (lib.PREC_FP64, lib.PREC_TF):
        r = tune_batch(a.batch_nmax, prec, small_candidates=SMALL_CANDIDATES, reps=2,
                       count=a.batch_count, record=False)
        report["batch"][f"prec={prec}|n_max={a.batch_nmax}"] = r
        print(f"batch prec={prec} n_max={a.batch_nmax}: best small {r['best_small']} "
              f"large {r['best']}", flush=True)
        if (r["best_small"], r["best"]) != (16, 8) and r["best"]:
            brows.append((prec, 1, 30, r["best_small"], r["best"]))
    srows = table_entries(results)
    if a.table:
        note = (f"Measured on {report['gpu']} with `python -m paper_2010_15595_gb300.autotune`; "
                f"sizes {a.sizes}, batch n_max {a.batch_nmax} x {a.batch_count}.")
        with open(a.table, "w") as f:
            f.write(emit_table(srows, brows, note))
    if a.json:
        def enc(o):
            if isinstance(o, tuple):
                return list(o)
            raise TypeError
        with open(a.json, "w") as f:
            json.dump(report, f, indent=1, default=enc)


if __name__ == "__main__":
    main()
