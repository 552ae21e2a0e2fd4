// Host-side launch wrappers for the loop-hafnian kernels (definitions in lhaf_kernels.cu).
#pragma once

#include <cstddef>
#include <cstdint>
#include <cuda_runtime.h>

#include "lhaf_types.cuh"

namespace gbsh {

constexpr int kMaxWarps = 16;          // warps per CTA of the subset kernel
constexpr int kFinalizeThreads = 256;  // threads of the finalize kernels
constexpr int kReduceBlocks = 128;     // CTAs of the first level of the final reduction
constexpr int kMaxClasses = 12;        // popcount classes of one evaluation
constexpr unsigned kTargetChunks = 1u << 18;  // Gray-code chunks of one evaluation (at most)

// One launch of the subset kernel: subsets with popcount in [k_lo, k_hi], `warps` warps per
// CTA, each warp owning `area_elems` double2 of shared memory.
struct ClassPlan {
  int k_lo, k_hi, warps, area_elems, blocks;
};

// Everything needed to evaluate one loop hafnian of padded size Ne.
struct LhafPlan {
  int N, Ne, n;
  int prec;  // kPrecFP64 or kPrecTF: the per-subset arithmetic
  int esz;   // bytes of one complex element of that arithmetic
  int nclass;
  ClassPlan cls[kMaxClasses];
  unsigned nchunks;
  uint64_t chunk_size;
  // workspace layout (byte offsets)
  size_t off_A0, off_v, off_partials, off_counters, off_blocks, off_out, bytes;
};

// Device properties cached per device.
struct DeviceInfo {
  int sm_count;
  int smem_optin;  // max dynamic shared memory per block (bytes)
};

cudaError_t device_info(DeviceInfo* info);
// Uploads constant tables on the current device (once per device).
cudaError_t ensure_constants();
// Builds the launch plan. warps_main = 0 selects the default cap on warps per CTA;
// max_chunks bounds the number of subset chunks (a power of two); prec selects the
// per-subset arithmetic (kPrecFP64 or kPrecTF); ladder is a gbsh::Ladder (tuning.h).
// Returns false if N or prec is out of range for the available shared memory.
bool make_plan(int N, const DeviceInfo& dev, int warps_main, int kcap_override, LhafPlan* plan,
               unsigned max_chunks = kTargetChunks, int prec = kPrecFP64, int ladder = 0);
// make_plan with the launch shape of the tuning table for (prec, N) (tuning.h); max_chunks
// further bounds the chunk count.
bool make_tuned_plan(int N, const DeviceInfo& dev, int prec, LhafPlan* plan,
                     unsigned max_chunks = kTargetChunks);

// Launches expansion + subset classes + finalize for one problem. `base`, `diag`, `idx` as
// in expand_problem_kernel. Writes lhaf (re, im) and sum |p_Z| into ws + off_out.
cudaError_t launch_lhaf(const LhafPlan& plan, const double2* base, int ld, const double2* diag,
                        const int* idx, void* ws, cudaStream_t stream);

// launch_lhaf restricted to the enumeration indices [i_begin, i_end) (expansion from `base`,
// `diag`, `idx` as in launch_lhaf); the range's compensated partial as for launch_lhaf_range.
cudaError_t launch_range(const LhafPlan& plan, const double2* base, int ld, const double2* diag,
                         const int* idx, void* ws, cudaStream_t stream, uint64_t i_begin,
                         uint64_t i_end);

// The subsets of the enumeration indices [i_begin, i_end) only (z = i ^ (i >> 1); any
// partition of [0, 2^n) into such ranges covers every subset once). Writes the range's
// compensated partial (re_hi, re_lo, im_hi, im_lo, sum |p_Z|) to ws + off_out + 3 doubles.
cudaError_t launch_lhaf_range(const LhafPlan& plan, const double2* base, int ld, void* ws,
                              cudaStream_t stream, uint64_t i_begin, uint64_t i_end);

// Writes lhaf = 1 (the empty matrix) to out[0] and 0 to *abs_sum (if not null) with a
// one-thread kernel on `stream`.
cudaError_t launch_write_unit(double2* out, double* abs_sum, cudaStream_t stream);

// Debug: p_Z of `count` subsets (device z list) of an already expanded problem.
cudaError_t launch_subset_terms(const LhafPlan& plan, const double2* base, int ld,
                                const uint64_t* z, int count, double2* out, void* ws,
                                cudaStream_t stream);

// Debug: runs the enumeration of launch_lhaf and counts visits of every subset z into
// counts[2^n] (which must be zeroed by the caller).
cudaError_t launch_visit_count(const LhafPlan& plan, unsigned* counts, void* ws,
                               cudaStream_t stream);

// Batched evaluation: warps per CTA that fit a problem of n_max pairs (0 if none fit).
int batch_warps_for(int n_max, int precision, const DeviceInfo& dev, int warps_pref);

// Popcount boundary of the batched evaluation: subsets with popcount <= kBatchSplitK run in
// one launch with small work areas (many warps per CTA), the rest in a second launch sized
// for n_max (when n_max > kBatchSplitK). Fixed, so a problem's chunk partials do not depend
// on the other problems of its batch.
constexpr int kBatchSplitK = 10;
int batch_classes(int n_max);

// Expands, evaluates and reduces `count` problems. d_in/d_prob: device tables (problem
// order = chunk order, largest first); d_out: 3 doubles per problem (re, im, sum |p_Z|).
// d_counter: 2 counters; d_partials: 2 x total_chunks x 5 doubles. `warps`: warps per CTA of
// the launch whose work areas are sized for n_max. side_stream: stream of the second class
// launch (nullptr: the library's side stream).
cudaError_t launch_batch(const BatchInput* d_in, const BatchProblem* d_prob, int count,
                         unsigned total_chunks, int n_max, int precision, int warps,
                         int warps_small, unsigned* d_counter, double* d_partials, double* d_out,
                         cudaStream_t stream, cudaStream_t side_stream = nullptr);

}  // namespace gbsh
