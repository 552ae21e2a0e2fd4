#!/usr/bin/env python
"""Benchmark of the loop-hafnian engine (one JSON line on stdout, rank 0).

Workload (one step): the loop hafnian of one N=40 complex symmetric matrix per GPU --
M=40 modes, Haar-random interferometer, squeezing r_i ~ U[0.4, 0.9], B = U diag(tanh r) U^T
with the diagonal replaced by gamma_i ~ CN(0, 0.2^2) -- i.e. the 2^20 pair-subset terms of
the subset formula. Metric: subset-terms per second (whole job). The headline path is the
accurate one (triple-float per subset, which meets the stated relative tolerance), with the
FP32-issue roofline fraction of its subset kernel; the FP64 path is timed beside it with its
FP64 roofline fraction, and each path's error against the oracle's reference is reported.
Each rank evaluates its own seeded matrix (weak scaling, no data-path collective). Shorter
measurements at N=50 (2^25 subsets) are reported under "n50".

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

--impl reference times the CPU oracle (the plain C subset formula) on a bounded sample of
subsets of the same matrix, on the host cores.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "lhaf subset-terms/s at N=40,50 (% FP64 peak); GBS samples/s + p99 vs plain"
UNIT = "subset-terms/s"
WORKLOAD = ("single loop hafnian N=40 complex128 (M=40 Haar U, r_i~U[0.4,0.9], "
            "gamma_i~CN(0,0.2^2)), 2^20 pair subsets per step, one matrix per GPU")
L2_FLUSH_BYTES = 256 << 20


# ------------------------------------------------------------------ distributed helpers

def dist_env():
    """(rank, world, local_rank) from the torchrun environment (1 process if unset)."""
    return (int(os.environ.get("RANK", "0")), int(os.environ.get("WORLD_SIZE", "1")),
            int(os.environ.get("LOCAL_RANK", "0")))


def rank_seed(rank: int) -> int:
    """Each rank evaluates its own matrix: seeds are the rank numbers."""
    return rank


def max_over_ranks(x: float, device=None) -> float:
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return x
    t = torch.tensor([x], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def barrier():
    import torch.distributed as dist
    if dist.is_available() and dist.is_initialized():
        dist.barrier()


# ------------------------------------------------------------------ clocks

class ClockSampler:
    """Samples SM clocks and throttle reasons with nvidia-smi while the timed region runs."""

    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.hw_slowdown,"
              "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
              "clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.lines = []
        self.thread = None

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except (OSError, FileNotFoundError):
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def __exit__(self, *exc):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
            if self.thread:
                self.thread.join(timeout=2)

    def summary(self):
        sm, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in self.lines:
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 7:
                continue
            try:
                sm.append(float(parts[0]))
                mx = float(parts[1])
            except ValueError:
                continue
            for nm, val in zip(names, parts[3:7]):
                if val.lower() == "active":
                    reasons.add(nm)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": mx, "reasons": ["unavailable"]}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": mx, "reasons": sorted(reasons),
                "samples": len(sm)}


# ------------------------------------------------------------------ traffic record

# Sources that define the subset kernel, its launches and its finalize (the sampler and the
# C-ABI wrappers do not change what one evaluation moves through DRAM).
KERNEL_SOURCES = ("lhaf_core.cuh", "lhaf_kernels.cu", "lhaf_kernels.cuh", "lhaf_types.cuh",
                  "lhaf_tf.cuh", "tuned_gb300.inc")


def tuning_block(N: int) -> dict:
    """Launch-shape table entries in force for size N (autotune.py; 0 = library default)."""
    from paper_2010_15595_gb300 import lib
    nb = lib.builtin_tuning_entries()
    return {"source": (f"built-in table measured by autotune.py on a GB300 ({nb} entries)"
                       if nb else "library defaults (no measured entries)"),
            "tf": dict(zip(("warps_cap", "ladder", "log2_chunks"), lib.get_lhaf_tuning(lib.PREC_TF, N))),
            "fp64": dict(zip(("warps_cap", "ladder", "log2_chunks"), lib.get_lhaf_tuning(lib.PREC_FP64, N))),
            "batch_fp64_n15": dict(zip(("warps_small", "warps_large"), lib.get_batch_tuning(lib.PREC_FP64, 15)))}


def kernel_source_hash() -> str:
    h = hashlib.sha256()
    csrc = os.path.join(ROOT, "paper_2010_15595_gb300", "csrc")
    for f in KERNEL_SOURCES:
        with open(os.path.join(csrc, f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def recorded_traffic(N: int, path: str, whole: bool = False):
    """DRAM bytes per evaluation on `path` ("tf" or "fp64") from the committed ncu summary, if
    it was taken on the current kernel sources (else None): the subset kernel's class launches
    (the dominant kernel), or with whole=True every launch of the evaluation (expansion,
    class launches, the two finalize levels)."""
    p = os.path.join(ROOT, "profiles", "lhaf_subsets_dram_traffic.json")
    try:
        with open(p) as f:
            rec = json.load(f)
    except (OSError, ValueError):
        return None
    if rec.get("kernel_source_hash") != kernel_source_hash():
        return None
    key = "bytes_per_evaluation" if whole else "subset_kernel_bytes_per_evaluation"
    return rec.get(key, {}).get(path, {}).get(str(N))


def recorded_probes() -> dict:
    """Throughput probe results committed under profiles/ (context beside derived peaks)."""
    try:
        with open(os.path.join(ROOT, "profiles", "alu_peak_probes.json")) as f:
            return json.load(f)
    except (OSError, ValueError):
        return {}


# ------------------------------------------------------------------ CPU oracle timing

def time_oracle(A, target_s: float, rng_seed: int = 0):
    """Subset-terms/s of the CPU oracle (plain C subset formula, all host cores) on a random
    sample of subsets of A, sized to take about target_s seconds."""
    import numpy as np
    from oracle import lhaf as olhaf
    N = A.shape[0]
    n = (N + (N & 1)) // 2
    rng = np.random.default_rng(rng_seed)
    count = 256
    while True:
        zs = rng.integers(1, 1 << n, count, dtype=np.uint64)
        t = time.perf_counter()
        olhaf.subset_terms(A, zs)
        dt = time.perf_counter() - t
        if dt >= target_s or count >= (1 << n):
            return count / dt, count, dt
        count = int(min(1 << n, max(count * 2, count * target_s / max(dt, 1e-3) * 1.1)))


# ------------------------------------------------------------------ our arm

def golden_reference(name):
    """(matrix, reference value, kind) of a committed oracle fixture, or None. The long-double
    oracle value where the fixture has one, else the double oracle's."""
    import numpy as np
    base = os.path.join(ROOT, "tests", "golden", name)
    try:
        with open(base + ".json") as f:
            rec = json.load(f)
        with open(base + ".matrix.txt") as f:
            n = int(f.readline())
            vals = np.array([float(t) for t in f.read().split()])
    except (OSError, ValueError):
        return None
    A = (vals[0::2] + 1j * vals[1::2]).reshape(n, n)
    if "lhaf_ld" in rec:
        return A, complex(*rec["lhaf_ld"]), "long-double oracle"
    return A, complex(*rec["lhaf_d"]), "double oracle (its own error is estimated at ~2e-7 here)"


def rel_err(v, ref):
    return abs(v - ref) / abs(ref) if ref is not None else None


def host_cpu_model() -> str:
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.lower().startswith("model name"):
                return line.split(":", 1)[1].strip()
    except (OSError, subprocess.SubprocessError):
        pass
    return "unknown"


def run_ours(args, rank, world, local_rank):
    import numpy as np
    import torch
    from paper_2010_15595_gb300 import lib, workloads, workmodel

    if not os.path.exists(lib.LIB_PATH):
        from paper_2010_15595_gb300 import build as pbuild
        pbuild.build()
    torch.cuda.set_device(local_rank)
    dev = torch.device("cuda", local_rank)
    stream = torch.cuda.current_stream()
    N = args.n
    TF, F64 = lib.PREC_TF, lib.PREC_FP64
    A = workloads.single_lhaf_mid(N, seed=rank_seed(rank))
    dA = torch.from_numpy(A).to(dev)
    flush = torch.empty(L2_FLUSH_BYTES, dtype=torch.uint8, device=dev)
    ref40 = golden_reference("lhaf_n40") if (rank == 0 and N == 40) else None

    def timed_path(prec, steps, warmup):
        """Times `steps` evaluations of the step matrix in `prec` (CUDA events on the
        launching stream, L2 flushed between steps outside the events)."""
        ws = torch.empty(lib.workspace_size(N, prec), dtype=torch.uint8, device=dev)
        out = torch.empty(1, dtype=torch.complex128, device=dev)
        asum = torch.empty(1, dtype=torch.float64, device=dev)

        def step():
            lib.lhaf_async(dA, out, ws, d_abs_sum=asum, stream=stream, precision=prec)

        for _ in range(warmup):
            step()
        torch.cuda.synchronize()
        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
              for _ in range(steps)]
        barrier()
        torch.cuda.synchronize()
        with ClockSampler(local_rank) as clocks:
            t0 = time.perf_counter()
            for e0, e1 in ev:
                flush.zero_()
                e0.record(stream)
                step()
                e1.record(stream)
            torch.cuda.synchronize()
            wall = time.perf_counter() - t0
        barrier()
        step_ms = [e0.elapsed_time(e1) for e0, e1 in ev]
        total_s = max_over_ranks(sum(step_ms) / 1e3, dev)
        v = complex(out.item())
        return {"total_s": total_s, "mean_s": statistics.mean(step_ms) / 1e3, "wall": wall,
                "clocks": clocks.summary(), "lhaf": v, "abs_sum": float(asum.item())}

    subsets = workmodel.subset_count(N)
    tf_run = timed_path(TF, args.steps, args.warmup)
    fp_run = timed_path(F64, args.steps, args.warmup)
    ms_per_step = tf_run["total_s"] * 1e3 / args.steps
    value = subsets * world * args.steps / tf_run["total_s"]
    tf_instr = workmodel.lhaf_tf_instr(N)
    tf_ach = tf_instr / tf_run["mean_s"] / 1e12
    tf_peak = workmodel.FP32_INSTR_PEAK_DERIVED_T
    flops = workmodel.lhaf_flops(N)
    sflops = workmodel.householder_flops(N)
    fp_ach = flops / fp_run["mean_s"] / 1e12
    fp_peak = workmodel.FP64_PEAK_DERIVED_TFLOPS
    probes = recorded_probes()
    fp64 = {"value": subsets * world * args.steps / fp_run["total_s"], "unit": UNIT,
            "ms_per_step": fp_run["total_s"] * 1e3 / args.steps,
            "roofline": {"bound": "alu", "achieved": fp_ach, "peak": fp_peak, "unit": "TFLOP/s",
                         "frac": fp_ach / fp_peak, "traffic": recorded_traffic(N, "fp64"),
                         "traffic_whole_evaluation": recorded_traffic(N, "fp64", whole=True),
                         "peak_source": "derived: 152 SM x 2 FP64 FMA/clk x 2 flop x 2.07 GHz",
                         "measured_dfma_probe_tflops": probes.get("dfma_tflops"),
                         "kernel": "lhaf_subsets_kernel<double2>",
                         "flops_per_launch": flops,
                         "flops_convention": "the kernel's own algorithm (elimination Hessenberg, "
                                             "La Budde push form, bordered-matrix loop terms)",
                         "flops_householder_convention": sflops,
                         "frac_householder_convention": sflops / fp_run["mean_s"] / 1e12 / fp_peak},
            "clocks": fp_run["clocks"]}

    # end to end through the public C ABI with host buffers (matrix in, value out)
    def e2e_rate(prec):
        steps_e = max(1, min(args.steps, 5))
        torch.cuda.synchronize()
        barrier()
        t = time.perf_counter()
        for _ in range(steps_e):
            lib.lhaf(A, stream=stream, precision=prec)
        return subsets * world * steps_e / max_over_ranks(time.perf_counter() - t, dev)

    e2e = {"value": e2e_rate(TF), "unit": UNIT, "h2d_bytes_per_step": int(A.nbytes),
           "d2h_bytes_per_step": 24, "api": "gbsh_lhaf_ex, GBSH_PREC_TF (host matrix in, "
                                             "host result out)"}
    fp64["e2e"] = {"value": e2e_rate(F64), "unit": UNIT, "api": "gbsh_lhaf (FP64)"}

    accuracy = None
    if ref40 is not None:
        # the committed fixture matrix (same bits on every host: the generator's QR differs
        # between LAPACK builds in the last bits), one evaluation per path
        dR = torch.from_numpy(ref40[0]).to(dev)
        got = {}
        for pname, prec in (("tf", TF), ("fp64", F64)):
            wsR = torch.empty(lib.workspace_size(N, prec), dtype=torch.uint8, device=dev)
            oR = torch.empty(1, dtype=torch.complex128, device=dev)
            lib.lhaf_async(dR, oR, wsR, stream=stream, precision=prec)
            torch.cuda.synchronize()
            got[pname] = complex(oR.item())
        accuracy = {"N40": {"matrix": "tests/golden/lhaf_n40.matrix.txt (the N=40 configuration "
                                      "generator's matrix, seed 0)",
                            "reference": ref40[2], "tol_stated": 1e-9,
                            "tf_rel_err": rel_err(got["tf"], ref40[1]),
                            "fp64_rel_err": rel_err(got["fp64"], ref40[1])}}

    def large_eval(N_, prec, fixture):
        """One timed evaluation of the large single loop hafnian of size N_ (the kernels are
        warm from the N=40 steps), CUDA events on the launching stream. The matrix is the
        committed fixture's where there is one (so that the error against its oracle value
        can be reported), else the generator's."""
        g = golden_reference(fixture) if fixture else None
        AL = g[0] if g is not None else workloads.large_lhaf(N_)
        dL = torch.from_numpy(AL).to(dev)
        wsL = torch.empty(lib.workspace_size(N_, prec), dtype=torch.uint8, device=dev)
        oL = torch.empty(1, dtype=torch.complex128, device=dev)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        flush.zero_()
        e0.record(stream)
        lib.lhaf_async(dL, oL, wsL, stream=stream, precision=prec)
        e1.record(stream)
        torch.cuda.synchronize()
        sec = e0.elapsed_time(e1) / 1e3
        v = complex(oL.item())
        res = {"seconds": sec, "value": workmodel.subset_count(N_) / sec, "unit": UNIT,
               "plan": lib.plan(N_, prec), "lhaf": [v.real, v.imag]}
        if prec == TF:
            ach = workmodel.lhaf_tf_instr(N_) / sec / 1e12
            res["roofline"] = {"bound": "alu", "achieved": ach, "peak": tf_peak,
                               "unit": "T FP32 instr/s", "frac": ach / tf_peak}
        else:
            ach = workmodel.lhaf_flops(N_) / sec / 1e12
            res["roofline"] = {"bound": "alu", "achieved": ach, "peak": fp_peak,
                               "unit": "TFLOP/s", "frac": ach / fp_peak,
                               "frac_householder_convention": workmodel.householder_flops(N_) / sec / 1e12 / fp_peak}
        if g is not None:
            res["rel_err"] = rel_err(v, g[1])
            res["reference"] = g[2]
        return res

    def large_block(N_, fixture, desc):
        base = {"workload": f"single loop hafnian N={N_}, {desc}, 2^{N_ // 2} subsets, "
                            f"1 timed evaluation per path", "matrix": f"tests/golden/{fixture}.matrix.txt",
                "tol_stated": 1e-7}
        base["tf"] = large_eval(N_, TF, fixture)
        base["fp64"] = large_eval(N_, F64, fixture)
        return base

    n50 = (large_block(50, "lhaf_n50", "M=50 Haar U, r=0.8, gamma~CN(0,0.1^2)")
           if (args.n50 and rank == 0) else None)
    n56 = (large_block(56, "lhaf_n56_block", "two 28-mode blocks of the N=56 configuration "
                                             "(M=28 Haar U, r=0.8, gamma~CN(0,0.1^2)) under a "
                                             "seeded permutation; reference = product of the "
                                             "blocks' long-double oracle values")
           if (args.n56 and rank == 0) else None)

    def small_latency(A_, name, calls=200):
        """Per-call cost of a small evaluation: host wall time of a synchronous gbsh_lhaf with a
        host matrix (copies in and out included), median of `calls`; and device time per
        evaluation of `calls` back-to-back gbsh_lhaf_async on device buffers (CUDA events)."""
        N_ = A_.shape[0]
        res = {"workload": name}
        for pname, prec in (("fp64", F64), ("tf", TF)):
            for _ in range(5):
                lib.lhaf(A_, precision=prec)
            walls = []
            for _ in range(calls):
                t0 = time.perf_counter()
                lib.lhaf(A_, precision=prec)
                walls.append(time.perf_counter() - t0)
            dA_ = torch.from_numpy(A_).to(dev)
            wsS = torch.empty(lib.workspace_size(N_, prec), dtype=torch.uint8, device=dev)
            oS = torch.empty(1, dtype=torch.complex128, device=dev)
            lib.lhaf_async(dA_, oS, wsS, stream=stream, precision=prec)
            torch.cuda.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            for _ in range(calls):
                lib.lhaf_async(dA_, oS, wsS, stream=stream, precision=prec)
            e1.record(stream)
            torch.cuda.synchronize()
            res[pname] = {"sync_call_us_median": 1e6 * statistics.median(walls),
                          "device_us_per_eval": 1e3 * e0.elapsed_time(e1) / calls,
                          "kernels_per_eval": lib.plan(N_, prec)["kernels"]}
        return res

    small = None
    if args.small and rank == 0:
        small = [small_latency(workloads.single_lhaf_n16(), "N=16 (M=16 Haar U, r=0.6, gamma~CN(0,0.3^2)), 256 subsets"),
                 small_latency(workloads.single_lhaf_mid(32), "N=32 (M=32 Haar U, r~U[0.4,0.9], gamma~CN(0,0.2^2)), 65536 subsets", calls=50)]

    batch = None
    if args.batch and rank == 0:
        batch = run_batch_workload(lib, workloads, workmodel, dev, stream)
    serving = None
    if args.serving and rank == 0:
        serving = run_serving_workload(args)

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        cpu = cpu_baseline_block(A, args.cpu_seconds)

    if rank == 0:
        plan = lib.plan(N, TF)
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_per_step,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f32x3", "data": "synthetic (seeded Haar-random GBS kernel matrices)",
            "config": {"workload": WORKLOAD, "N": N, "subsets_per_step_per_gpu": subsets,
                       "path": "triple-float per subset (GBSH_PREC_TF: three FP32 words, "
                               "~72-bit significand), compensated FP64 cross-subset sum",
                       "l2": "flushed between timed steps (256 MiB write, outside the events)",
                       "plan": plan, "tuning": tuning_block(N),
                       "parallelism": f"replicas x{world}"},
            "roofline": {"bound": "alu", "achieved": tf_ach, "peak": tf_peak,
                         "unit": "T FP32 instr/s", "frac": tf_ach / tf_peak,
                         "traffic": recorded_traffic(N, "tf"),
                         "traffic_whole_evaluation": recorded_traffic(N, "tf", whole=True),
                         "traffic_note": "DRAM bytes per evaluation (ncu): the subset kernel's "
                                         "class launches; the whole evaluation adds the chunk "
                                         "partial sums, L2-resident in the timed run",
                         "peak_source": "derived: 152 SM x 128 FP32 lanes/clk x 2.07 GHz",
                         "measured_ffma_probe_t_instr": probes.get("ffma_t_instr"),
                         "kernel": "lhaf_subsets_kernel<tfc> (+expand, finalize in the step time)",
                         "work_per_launch": tf_instr,
                         "work_convention": "FP32 arithmetic instructions of the triple-float "
                                            "algorithm (216 per complex multiply-add)"},
            "fp64": fp64,
            "accuracy": accuracy,
            "cpu_baseline": cpu,
            "e2e": e2e,
            "gpu_launches": plan["kernels"] * args.steps,
            "clocks": tf_run["clocks"],
            "wall_s_timed_region": tf_run["wall"],
            "result": {"lhaf": [tf_run["lhaf"].real, tf_run["lhaf"].imag],
                       "kappa": tf_run["abs_sum"] / abs(tf_run["lhaf"])},
            "n50": n50,
            **({"n56": n56} if n56 is not None else {}),
            "small": small,
            "batch": batch,
            "serving": serving,
            "paper_context": "Fig. 3: N=40 in 44.9 s (23.3k subset-terms/s), N=50 in 2499 s "
                             "(13.4k/s), long double, 96 vCPUs @ 2.345 GHz",
        }
        print(json.dumps(line), flush=True)


def cpu_baseline_block(A40, seconds):
    """The CPU oracle (plain C subset formula, explicit matrix powers, OpenMP over subsets)
    on the host cores: the configuration workloads N=16 (all 256 subsets), N=40 (a random
    sample of the step matrix's subsets, the headline comparison) and N=50 (a random sample),
    each sized to about `seconds`; subset-terms/s per workload and the full-evaluation time
    they imply."""
    from paper_2010_15595_gb300 import workloads
    per = {}
    for name, A_ in (("N16", workloads.single_lhaf_n16()), ("N40", A40),
                     ("N50", workloads.large_lhaf(50))):
        rate, count, dt = time_oracle(A_, seconds if name != "N16" else 1.0)
        n = (A_.shape[0] + 1) // 2
        per[name] = {"value": rate, "subsets_timed": count, "seconds": dt,
                     "full_evaluation_s_implied": (1 << n) / rate}
    cores = int(os.environ.get("ORACLE_THREADS", "0")) or os.cpu_count()
    return {"value": per["N40"]["value"], "unit": UNIT, "cores": cores, "kind": "oracle",
            "cpu_model": host_cpu_model(),
            "sample": f"{per['N40']['subsets_timed']} random pair subsets of the N=40 step matrix "
                      f"({per['N40']['seconds']:.1f} s, plain-C subset formula with explicit "
                      f"matrix powers, OpenMP over subsets); N=16 and N=50 under per_workload",
            "per_workload": per}


def run_batch_workload(lib, workloads, workmodel, dev, stream, count=4096):
    """Batched workload: 4096 loop hafnians of uneven size (N uniform on even 10..30) from
    one M=100-mode state (r=0.7, Haar U, gamma ~ CN(0, 0.1^2)), up to 3 photons per mode,
    through gbsh_gbs_prob_batch (device B and gamma). FP64, triple-float and complex-FP32 per
    subset. Errors: every FP64 and FP32 result against the triple-float result of the same
    problem (the triple-float batch is held within 1e-9 of the oracle by the tests)."""
    import numpy as np
    import torch
    B, gamma = workloads.batch_state()
    pats = workloads.batch_patterns(count, seed=0)
    Ns = pats.sum(axis=1)
    dB = torch.from_numpy(B).to(dev)
    dg = torch.from_numpy(gamma).to(dev)
    subsets = int(sum(workmodel.subset_count(int(n)) for n in Ns))
    flops = float(sum(workmodel.lhaf_flops(int(n)) for n in Ns))
    tfi = float(sum(workmodel.lhaf_tf_instr(int(n)) for n in Ns))
    res = {"workload": f"{count} loop hafnians, N uniform on even 10..30, M=100 Haar state "
                       "r=0.7, gamma~CN(0,0.1^2), <=3 photons/mode (gbsh_gbs_prob_batch, "
                       "host result copy included)", "subset_terms": subsets}
    out = {}
    for name, prec in (("fp64", lib.PREC_FP64), ("tf", lib.PREC_TF), ("c32", lib.PREC_C32)):
        lib.gbs_prob_batch(dB, dg, pats, precision=prec, stream=stream)
        torch.cuda.synchronize()
        t = time.perf_counter()
        reps = 3
        for _ in range(reps):
            probs, lh = lib.gbs_prob_batch(dB, dg, pats, precision=prec, stream=stream)
        dt = (time.perf_counter() - t) / reps
        out[name] = lh
        res[name] = {"seconds": dt, "value": subsets / dt, "unit": UNIT}
    ach = flops / res["fp64"]["seconds"] / 1e12
    res["fp64"]["roofline"] = {"bound": "alu", "achieved": ach,
                               "peak": workmodel.FP64_PEAK_DERIVED_TFLOPS, "unit": "TFLOP/s",
                               "frac": ach / workmodel.FP64_PEAK_DERIVED_TFLOPS}
    ach = tfi / res["tf"]["seconds"] / 1e12
    res["tf"]["roofline"] = {"bound": "alu", "achieved": ach,
                             "peak": workmodel.FP32_INSTR_PEAK_DERIVED_T, "unit": "T FP32 instr/s",
                             "frac": ach / workmodel.FP32_INSTR_PEAK_DERIVED_T}
    for name in ("fp64", "c32"):
        err = np.abs(out[name] - out["tf"]) / np.abs(out["tf"])
        res[name]["rel_err_vs_tf"] = {"median": float(np.median(err)),
                                      "p99": float(np.quantile(err, 0.99)), "max": float(err.max())}
    res["c32"]["enabled_by_mixed_mode_for_N_le"] = lib.C32_MAX_N
    return res


def run_serving_workload(args):
    """Chain-rule sampler (Sec. III) on the serving state: M=100 modes, Haar U, r=0.8 on 25
    input modes (mean ~20 photons), output displacement ~CN(0, 0.1^2), Fock cutoff 4, loop
    hafnians up to N=36. Plain path (one single-evaluation launch sequence and one
    synchronisation per loop hafnian, one sample at a time) vs the served path (continuous
    batching, loop hafnians above --serve-tick-subsets subsets split into subset ranges over
    ticks); Poisson arrivals at 0.5, 1, 2 and 3 times the plain throughput; latencies from
    submission to completion, with n per rate; the fraction of samples that dropped a
    candidate above the N <= 36 cap. --serve-compare also runs the served path without
    splitting and the plain path under the same Poisson arrivals."""
    import numpy as np
    from paper_2010_15595_gb300 import sampler as S, workloads
    U, r, alpha = workloads.serving_state()
    st = S.pure_state(U, r, alpha)
    res = {"workload": "chain-rule GBS sampler, M=100, r=0.8 on 25 modes, alpha~CN(0,0.1^2), "
                       "cutoff 4, N<=36 (candidates above are dropped and counted)",
           "tick_subsets": args.serve_tick_subsets}

    def run_batch(smp, seeds):
        t = time.perf_counter()
        rids = [smp.submit(s_) for s_ in seeds]
        out = [smp.wait(rr, timeout=1800) for rr in rids]
        return time.perf_counter() - t, out

    def poisson(smp, mult, plain_rate):
        lam = mult * plain_rate
        gaps = np.random.default_rng(2 + int(mult * 10)).exponential(1.0 / lam, args.serve_poisson)
        t0 = time.perf_counter()
        rids = []
        for i, gap in enumerate(gaps):
            target = t0 + gaps[: i + 1].sum()
            now = time.perf_counter()
            if target > now:
                time.sleep(target - now)
            rids.append(smp.submit(5000 + 1000 * int(mult * 10) + i))
        outs = [smp.wait(rr, timeout=1800) for rr in rids]
        span = time.perf_counter() - t0
        lats = np.array([o[1]["latency_s"] for o in outs])
        return {"rate_x_plain": mult, "arrival_per_s": lam, "requests": len(outs),
                "samples_per_s": len(outs) / span, "p50_s": float(np.median(lats)),
                "p99_s": float(np.quantile(lats, 0.99)), "max_s": float(lats.max())}

    with S.Sampler(st, cutoff=4, n_cap=36, batching=False) as plain:
        dt, out = run_batch(plain, range(args.serve_plain))
        plain_rate = args.serve_plain / dt
        if args.serve_compare:
            res["plain_poisson"] = [poisson(plain, m, plain_rate) for m in args.serve_rates]
    lat = np.array([o[1]["latency_s"] for o in out])
    res["plain"] = {"samples": args.serve_plain, "samples_per_s": plain_rate,
                    "mean_photons": float(np.mean([o[0].sum() for o in out])),
                    "per_sample_s_p50": float(np.median(np.diff(np.sort(lat), prepend=0.0))),
                    "note": "all submitted at t=0 (saturated), served one at a time"}
    configs = [("", args.serve_tick_subsets)]
    if args.serve_compare and args.serve_tick_subsets:
        configs.append(("_unsplit", 0))
    for suffix, ts in configs:
        with S.Sampler(st, cutoff=4, n_cap=36, max_active=args.serve_slots,
                       tick_subsets=ts) as smp:
            dt, out = run_batch(smp, range(1000, 1000 + args.serve_saturated))
            capped = sum(1 for o in out if o[1]["truncated"] > 0)
            res["served_saturated" + suffix] = {
                "samples": args.serve_saturated, "samples_per_s": args.serve_saturated / dt,
                "truncated_steps": int(sum(o[1]["truncated"] for o in out)),
                "samples_with_capped_candidate": capped,
                "capped_fraction": capped / args.serve_saturated, "slots": args.serve_slots,
                "tick_subsets": ts}
            res["poisson" + suffix] = [poisson(smp, m, plain_rate) for m in args.serve_rates]
    # the plain path under the same arrivals: a queue in front of a single server
    res["plain_queue_model"] = []
    for mult in args.serve_rates:
        lam = mult * plain_rate
        gaps = np.random.default_rng(2 + int(mult * 10)).exponential(1.0 / lam, args.serve_poisson)
        svc = np.random.default_rng(3).choice(np.diff(np.sort(lat), prepend=0.0), args.serve_poisson)
        arr = np.cumsum(gaps)
        done = np.zeros_like(arr)
        free = 0.0
        for i in range(len(arr)):
            start = max(arr[i], free)
            free = done[i] = start + svc[i]
        wl = done - arr
        res["plain_queue_model"].append({"rate_x_plain": mult, "p50_s": float(np.median(wl)),
                                         "p99_s": float(np.quantile(wl, 0.99)),
                                         "note": "FIFO single server with the measured plain "
                                                 "per-sample service times (not run)"})
    res["served_vs_plain_samples_per_s"] = res["served_saturated"]["samples_per_s"] / plain_rate
    return res


def fig1_tvd(modes=(1, 2, 3, 4, 5, 6), unitaries=10, samples=200000, r=0.5, cutoff=6, seed0=0):
    """Sec. III, Fig. 1: percent TVD between exact output probabilities and (a) the served
    chain-rule sampler, (b) exact sampling of the same size, for m modes with squeezing r in
    every mode and Fock cutoff `cutoff`, averaged over Haar-random unitaries. The TVD runs
    over the outputs with at most `cutoff` photons in every mode (those with more than
    2 x cutoff photons in total carry negligible probability at r = 0.5 and are left out).
    Exact probabilities come from the GPU loop hafnians (gbsh_gbs_prob_batch)."""
    import itertools
    import numpy as np
    from paper_2010_15595_gb300 import lib, sampler as S, workloads
    rows = []
    for m in modes:
        pats = [p for p in itertools.product(range(cutoff + 1), repeat=m) if sum(p) <= 2 * cutoff]
        index = {p: i for i, p in enumerate(pats)}
        alg, exp_ = [], []
        for u in range(unitaries):
            rng = workloads.rng_for(70 + m, seed0 + u)
            U = workloads.haar_unitary(m, rng)
            st = S.pure_state(U, np.full(m, r), np.zeros(m, complex))
            probs, _ = lib.gbs_prob_batch(st.B, st.gamma, np.array(pats, dtype=np.int32),
                                          p_vacs=np.full(len(pats), st.p_vac))
            rest = max(0.0, 1.0 - probs.sum())
            per_req = 4000
            with S.Sampler(st, cutoff=cutoff, n_cap=60, max_active=4096) as smp:
                rids = [smp.submit(1_000_000 * m + 1000 * u + q, per_req)
                        for q in range((samples + per_req - 1) // per_req)]
                out = np.concatenate([smp.wait(rr, timeout=1800)[0] for rr in rids])[:samples]
            counts = np.zeros(len(pats))
            for row in out:
                key = tuple(int(x) for x in row)
                if key in index:
                    counts[index[key]] += 1
            alg.append(50.0 * np.abs(counts / samples - probs).sum())
            rs = np.random.default_rng(seed0 + u)
            draw = rs.multinomial(samples, np.append(probs, rest) / (probs.sum() + rest))[:-1]
            exp_.append(50.0 * np.abs(draw / samples - probs).sum())
        rows.append({"modes": m, "algorithm_tvd_pct": [float(np.mean(alg)), float(np.std(alg))],
                     "expected_tvd_pct": [float(np.mean(exp_)), float(np.std(exp_))]})
    return rows


def telephone(n: int) -> int:
    """T(n) = lhaf(all-ones n x n) (number of matchings with loops; Fig. 2 caption)."""
    a, b_ = 1, 1
    for k in range(2, n + 1):
        a, b_ = b_, b_ + (k - 1) * a
    return b_ if n >= 1 else 1


def fig2_allones(sizes_fp64=range(30, 58, 2), sizes_dd=range(30, 48, 2)):
    """Sec. IV, Fig. 2: relative error of lhaf(all-ones n x n) against T(n), with the FP64
    kernels (gbsh_lhaf), the triple-float path (gbsh_lhaf_ex, every size) and the
    double-double per-subset variant (batched entry point, sizes_dd)."""
    from fractions import Fraction
    import numpy as np
    from paper_2010_15595_gb300 import lib

    def rel(v, n):
        T = telephone(n)
        return float(abs(Fraction(v.real) - T) / T), abs(v.imag) / T

    rows = []
    for n in sizes_fp64:
        A = np.ones((n, n), dtype=np.complex128)
        t = time.perf_counter()
        v = lib.lhaf(A)
        dt = time.perf_counter() - t
        row = {"n": n, "fp64_rel_err": rel(v, n)[0], "fp64_seconds": dt}
        t = time.perf_counter()
        vt = lib.lhaf(A, precision=lib.PREC_TF)
        row["tf_rel_err"] = rel(vt, n)[0]
        row["tf_seconds"] = time.perf_counter() - t
        if n in sizes_dd:
            t = time.perf_counter()
            vd = lib.lhaf_batch([A], precision=lib.PREC_DD)[0]
            row["dd_rel_err"] = rel(vd, n)[0]
            row["dd_seconds"] = time.perf_counter() - t
        rows.append(row)
        print(json.dumps(row), flush=True)
    return rows


def accuracy_table():
    """Relative error of both paths (FP64, triple-float) on every committed oracle fixture
    (tests/golden: the configuration matrices N=32/40/50, the repeated-mode N=40 matrix, the
    block-diagonal N=50/56 matrices) and on all-ones matrices (exact T(n)), with each
    evaluation's time."""
    import numpy as np
    import torch
    from fractions import Fraction
    from paper_2010_15595_gb300 import lib
    rows = []
    for name, tol in (("lhaf_n32", 1e-9), ("lhaf_n40", 1e-9), ("lhaf_n40_repeated", 1e-9),
                      ("lhaf_n50", 1e-7), ("lhaf_n50_block", 1e-7), ("lhaf_n56_block", 1e-7)):
        g = golden_reference(name)
        if g is None:
            continue
        dA = torch.from_numpy(g[0]).cuda()
        row = {"fixture": name, "N": g[0].shape[0], "reference": g[2], "tol_stated": tol}
        for pname, prec in (("fp64", lib.PREC_FP64), ("tf", lib.PREC_TF)):
            t = time.perf_counter()
            v = lib.lhaf(dA, precision=prec)
            row[pname + "_seconds"] = time.perf_counter() - t
            row[pname + "_rel_err"] = rel_err(v, g[1])
        rows.append(row)
        print(json.dumps(row), flush=True)
    for n in (40, 56):
        A = np.ones((n, n), dtype=np.complex128)
        T = telephone(n)
        row = {"fixture": f"all-ones {n}", "N": n, "reference": "T(n), exact", "tol_stated": 1e-9 if n <= 40 else 1e-7}
        for pname, prec in (("fp64", lib.PREC_FP64), ("tf", lib.PREC_TF)):
            t = time.perf_counter()
            v = lib.lhaf(A, precision=prec)
            row[pname + "_seconds"] = time.perf_counter() - t
            row[pname + "_rel_err"] = float(abs(Fraction(v.real) - T) / T)
        rows.append(row)
        print(json.dumps(row), flush=True)
    return rows


# ------------------------------------------------------------------ reference arm

def run_reference(args, rank, world):
    if rank != 0:
        return
    from paper_2010_15595_gb300 import workloads
    A = workloads.single_lhaf_mid(args.n, seed=0)
    for _ in range(args.warmup):
        time_oracle(A, 0.05)
    rates = []
    t0 = time.perf_counter()
    counts = 0
    for _ in range(args.steps):
        rate, count, dt = time_oracle(A, args.ref_step_seconds)
        rates.append(rate)
        counts += count
    total = time.perf_counter() - t0
    value = counts / total
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": total * 1e3 / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic (seeded Haar-random GBS kernel matrices)",
        "config": {"workload": WORKLOAD, "N": args.n,
                   "per_step": f"random sample of pair subsets (~{args.ref_step_seconds} s)"},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": os.cpu_count(), "kind": "oracle",
                         "sample": f"{counts} random pair subsets of the N={args.n} matrix over "
                                   f"{args.steps} steps"},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def main(argv=None):
    p = argparse.ArgumentParser(description=__doc__.split("\n")[0])
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=10)
    p.add_argument("--warmup", type=int, default=3)
    p.add_argument("--impl", choices=["ours", "reference"], default="ours")
    p.add_argument("--n", type=int, default=40)
    p.add_argument("--no-n50", dest="n50", action="store_false")
    p.add_argument("--no-small", dest="small", action="store_false")
    p.add_argument("--n56", action="store_true",
                   help="also time one N=56 evaluation (2^28 subsets, about a minute)")
    p.add_argument("--no-batch", dest="batch", action="store_false")
    p.add_argument("--no-serving", dest="serving", action="store_false")
    p.add_argument("--serve-plain", type=int, default=50)
    p.add_argument("--serve-saturated", type=int, default=256)
    p.add_argument("--serve-slots", type=int, default=256)
    p.add_argument("--serve-poisson", type=int, default=60,
                   help="requests per arrival rate (the committed serving profile uses 200)")
    p.add_argument("--serve-rates", type=float, nargs="+", default=[0.5, 1.0, 2.0, 3.0])
    p.add_argument("--serve-tick-subsets", type=int, default=1 << 16,
                   help="split loop hafnians above this many subsets over ticks (0: off)")
    p.add_argument("--serve-compare", action="store_true",
                   help="also serve without splitting and run the plain path under Poisson arrivals")
    p.add_argument("--fig1", action="store_true",
                   help="run the Fig. 1 TVD experiment (Sec. III) instead of the benchmark")
    p.add_argument("--fig1-samples", type=int, default=200000)
    p.add_argument("--fig2", action="store_true",
                   help="run the Fig. 2 all-ones accuracy study (Sec. IV) instead of the benchmark")
    p.add_argument("--fig1-unitaries", type=int, default=10)
    p.add_argument("--accuracy", action="store_true",
                   help="errors of both paths on the committed oracle fixtures, then exit")
    p.add_argument("--no-cpu-baseline", action="store_true")
    p.add_argument("--cpu-seconds", type=float, default=15.0)
    p.add_argument("--ref-step-seconds", type=float, default=4.0)
    args = p.parse_args(argv)
    if args.warmup < 3 and args.impl == "ours":
        args.warmup = 3
    if args.accuracy:
        rows = accuracy_table()
        print(json.dumps({"experiment": "accuracy of both paths on the oracle fixtures", "rows": rows}), flush=True)
        return
    if args.fig2:
        rows = fig2_allones()
        print(json.dumps({"experiment": "Fig. 2 all-ones accuracy", "rows": rows}), flush=True)
        return
    if args.fig1:
        rows = fig1_tvd(samples=args.fig1_samples, unitaries=args.fig1_unitaries)
        print(json.dumps({"experiment": "Fig. 1 TVD", "samples": args.fig1_samples,
                          "unitaries": args.fig1_unitaries, "rows": rows}), flush=True)
        return
    rank, world, local_rank = dist_env()
    if world > 1:
        import torch
        import torch.distributed as dist
        os.environ.setdefault("MASTER_ADDR", "127.0.0.1")
        backend = "nccl" if torch.cuda.is_available() else "gloo"
        if backend == "nccl":
            torch.cuda.set_device(local_rank)
        dist.init_process_group(backend)
    try:
        if args.impl == "reference":
            run_reference(args, rank, world)
        else:
            run_ours(args, rank, world, local_rank)
    finally:
        if world > 1:
            import torch.distributed as dist
            dist.destroy_process_group()


if __name__ == "__main__":
    main()
