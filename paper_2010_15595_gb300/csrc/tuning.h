// Launch-shape tuning of the loop-hafnian kernels: the library's default launch shapes come
// from a table measured by the autotuner on a GB300 (tuned_gb300.inc); callers may override
// entries at run time. Launch shapes never change which subsets are summed, only how the work
// is distributed and, for the single-evaluation chunk count, the grouping of the compensated
// cross-subset sum (results agree to its rounding; a given tuning is deterministic).
#pragma once

namespace gbsh {

// Popcount-class ladders of the single-evaluation plan: the warps-per-CTA steps tried from
// the largest down when popcounts are assigned to classes.
enum Ladder { kLadderDefault = 0, kLadderCoarse = 1, kLadderFine = 2 };

// Single evaluation at size N: 0 in a field selects the library default for that field
// (warps cap 12 FP64 / 16 triple-float, the coarse ladder, 2^18 chunks).
struct SingleTuning {
  int warps_cap;    // 1..16: most warps per CTA of any class
  int ladder;       // Ladder
  int log2_chunks;  // 1..18: enumeration chunks of one evaluation (capped at 2^n)
};

// Batched evaluation whose largest problem has n_max index pairs: 0 selects the default
// (16 warps per CTA for the small-popcount class, 8 for the large-popcount class).
struct BatchTuning {
  int warps_small;  // class of popcounts <= the fixed split
  int warps_large;  // class of larger popcounts
};

// kernel_prec: kPrecFP64 or kPrecTF for single evaluations; any precision for batches.
SingleTuning single_tuning(int kernel_prec, int N);
void set_single_tuning(int kernel_prec, int N, SingleTuning t);  // all-zero t: built-in entry
BatchTuning batch_tuning(int kernel_prec, int n_max);
void set_batch_tuning(int kernel_prec, int n_max, BatchTuning t);  // all-zero t: built-in entry
// Number of built-in (measured) entries, for reporting.
int builtin_tuning_entries(int* single, int* batch);

}  // namespace gbsh
