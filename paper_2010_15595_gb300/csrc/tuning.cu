// Launch-shape tuning tables: built-in entries measured by the autotuner, overlaid by
// run-time overrides (see tuning.h).
#include "tuning.h"

#include <mutex>

#include "lhaf_types.cuh"

namespace gbsh {
namespace {

struct TunedSingleEntry {
  int prec, N_lo, N_hi, warps_cap, ladder, log2_chunks;
};
struct TunedBatchEntry {
  int prec, nmax_lo, nmax_hi, warps_small, warps_large;
};

// kTunedSingle[] and kTunedBatch[], written by autotune.py from measurements on a GB300
// (each ends with a sentinel entry whose prec is -1).
#include "tuned_gb300.inc"

std::mutex g_mu;
SingleTuning g_single[kNumPrec][kMaxN + 1];
BatchTuning g_batch[kNumPrec][kMaxN / 2 + 1];
bool g_init = false;

SingleTuning builtin_single(int prec, int N) {
  for (const TunedSingleEntry& t : kTunedSingle)
    if (t.prec == prec && N >= t.N_lo && N <= t.N_hi)
      return SingleTuning{t.warps_cap, t.ladder, t.log2_chunks};
  return SingleTuning{0, 0, 0};
}

BatchTuning builtin_batch(int prec, int n_max) {
  for (const TunedBatchEntry& t : kTunedBatch)
    if (t.prec == prec && n_max >= t.nmax_lo && n_max <= t.nmax_hi)
      return BatchTuning{t.warps_small, t.warps_large};
  return BatchTuning{0, 0};
}

void init_locked() {
  if (g_init) return;
  for (int p = 0; p < kNumPrec; ++p) {
    for (int N = 0; N <= kMaxN; ++N) g_single[p][N] = builtin_single(p, N);
    for (int n = 0; n <= kMaxN / 2; ++n) g_batch[p][n] = builtin_batch(p, n);
  }
  g_init = true;
}

bool prec_ok(int p) { return p >= 0 && p < kNumPrec; }

}  // namespace

SingleTuning single_tuning(int kernel_prec, int N) {
  if (!prec_ok(kernel_prec) || N < 0 || N > kMaxN) return SingleTuning{0, 0, 0};
  std::lock_guard<std::mutex> lk(g_mu);
  init_locked();
  return g_single[kernel_prec][N];
}

void set_single_tuning(int kernel_prec, int N, SingleTuning t) {
  if (!prec_ok(kernel_prec) || N < 0 || N > kMaxN) return;
  std::lock_guard<std::mutex> lk(g_mu);
  init_locked();
  const bool reset = t.warps_cap == 0 && t.ladder == 0 && t.log2_chunks == 0;
  g_single[kernel_prec][N] = reset ? builtin_single(kernel_prec, N) : t;
}

BatchTuning batch_tuning(int kernel_prec, int n_max) {
  if (!prec_ok(kernel_prec) || n_max < 0 || n_max > kMaxN / 2) return BatchTuning{0, 0};
  std::lock_guard<std::mutex> lk(g_mu);
  init_locked();
  return g_batch[kernel_prec][n_max];
}

void set_batch_tuning(int kernel_prec, int n_max, BatchTuning t) {
  if (!prec_ok(kernel_prec) || n_max < 0 || n_max > kMaxN / 2) return;
  std::lock_guard<std::mutex> lk(g_mu);
  init_locked();
  const bool reset = t.warps_small == 0 && t.warps_large == 0;
  g_batch[kernel_prec][n_max] = reset ? builtin_batch(kernel_prec, n_max) : t;
}

int builtin_tuning_entries(int* single, int* batch) {
  int s = 0, b = 0;
  for (const TunedSingleEntry& t : kTunedSingle) s += t.prec >= 0;
  for (const TunedBatchEntry& t : kTunedBatch) b += t.prec >= 0;
  if (single) *single = s;
  if (batch) *batch = b;
  return s + b;
}

}  // namespace gbsh
