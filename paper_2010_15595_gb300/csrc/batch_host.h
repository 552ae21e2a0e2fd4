// Host helpers of the batched evaluation, shared by the C ABI and the sampler.
#pragma once

#include <cstddef>
#include <vector>

#include <cuda_runtime.h>

#include "lhaf_types.cuh"

namespace gbsh {

// Workspace layout of a batched evaluation. The first `base_off` bytes belong to the caller
// (staged inputs: matrices, fill vectors, index lists); the tables, expanded matrices,
// chunk partials, counter and results follow. Problems are ordered largest first.
struct BatchLayout {
  size_t off_in, off_prob, off_expanded, off_partials, off_counter, off_out, bytes;
  unsigned total_chunks;
  int n_max;
  std::vector<int> order;  // sorted position -> problem index
  std::vector<BatchProblem> table;
};

BatchLayout batch_layout(const int* Ns, int count, size_t base_off);

// Fills the device tables of `L` (inputs `in` indexed by problem, device pointers into
// memory that is ready on `st`), launches expansion + persistent evaluation + finalize,
// and copies (re, im, sum|p_Z|) per problem into host `out3` in problem order,
// synchronising `st`. warps_pref > 0 sets the warps per CTA of the large-popcount class;
// 0 takes the tuning table's launch shape (tuning.h).
// Returns cudaErrorInvalidValue if no launch shape fits.
cudaError_t batch_run(BatchLayout& L, const std::vector<BatchInput>& in, int count, int precision,
                      int warps_pref, void* ws, cudaStream_t st, double* out3);

// CUDA-graph replay of batch_run's device work for launch shapes seen before (on by default).
void set_batch_graphs(bool enable);
// Graphs captured and graph launches so far (process-wide).
void batch_graph_stats(long long* captures, long long* replays);

}  // namespace gbsh
