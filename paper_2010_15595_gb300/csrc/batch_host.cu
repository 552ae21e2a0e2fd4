// Host helpers of the batched evaluation (see batch_host.h).
#include <algorithm>
#include <numeric>

#include "batch_host.h"
#include "lhaf_kernels.cuh"

namespace gbsh {

namespace {
size_t align_up(size_t x) { return (x + 255) & ~(size_t)255; }
}  // namespace

BatchLayout batch_layout(const int* Ns, int count, size_t base_off) {
  BatchLayout L;
  L.order.resize(count);
  std::iota(L.order.begin(), L.order.end(), 0);
  std::stable_sort(L.order.begin(), L.order.end(),
                   [&](int a, int b) { return Ns[a] > Ns[b]; });
  L.table.resize(count);
  unsigned base = 0;
  size_t exp_elems = 0;
  L.n_max = 0;
  for (int q = 0; q < count; ++q) {
    const int N = Ns[L.order[q]];
    const int Ne = N + (N & 1);
    const int n = Ne / 2;
    BatchProblem& P = L.table[q];
    P.Ne = Ne;
    P.n = n;
    P.chunk_size = n > 0 ? batch_chunk_size(n) : 1;
    P.nchunks = n > 0 ? (unsigned)((1ull << n) / P.chunk_size) : 0u;
    P.chunk_base = base;
    base += P.nchunks;
    exp_elems += (size_t)Ne * Ne + Ne;
    L.n_max = std::max(L.n_max, n);
  }
  L.total_chunks = base;
  size_t off = align_up(base_off);
  L.off_in = off; off = align_up(off + sizeof(BatchInput) * count);
  L.off_prob = off; off = align_up(off + sizeof(BatchProblem) * count);
  L.off_expanded = off; off = align_up(off + sizeof(double2) * exp_elems);
  L.off_partials = off; off = align_up(off + sizeof(double) * 5 * (size_t)L.total_chunks);
  L.off_counter = off; off = align_up(off + sizeof(unsigned));
  L.off_out = off; off = align_up(off + sizeof(double) * 3 * (size_t)count);
  L.bytes = off;
  return L;
}

cudaError_t batch_run(BatchLayout& L, const std::vector<BatchInput>& in, int count, int precision,
                      int warps_pref, void* ws, cudaStream_t st, double* out3) {
  char* w = static_cast<char*>(ws);
  std::vector<BatchInput> in_sorted(count);
  double2* exp_base = reinterpret_cast<double2*>(w + L.off_expanded);
  size_t e_off = 0;
  for (int q = 0; q < count; ++q) {
    in_sorted[q] = in[L.order[q]];
    BatchProblem& P = L.table[q];
    P.A0 = exp_base + e_off;
    P.v = exp_base + e_off + (size_t)P.Ne * P.Ne;
    e_off += (size_t)P.Ne * P.Ne + P.Ne;
  }
  cudaError_t e = cudaMemcpyAsync(w + L.off_in, in_sorted.data(), sizeof(BatchInput) * count,
                                  cudaMemcpyHostToDevice, st);
  if (e != cudaSuccess) return e;
  e = cudaMemcpyAsync(w + L.off_prob, L.table.data(), sizeof(BatchProblem) * count,
                      cudaMemcpyHostToDevice, st);
  if (e != cudaSuccess) return e;
  DeviceInfo dev;
  e = device_info(&dev);
  if (e != cudaSuccess) return e;
  e = ensure_constants();
  if (e != cudaSuccess) return e;
  const int W = batch_warps_for(std::max(L.n_max, 1), precision, dev, warps_pref);
  if (W < 1) return cudaErrorInvalidValue;
  e = launch_batch(reinterpret_cast<const BatchInput*>(w + L.off_in),
                   reinterpret_cast<const BatchProblem*>(w + L.off_prob), count, L.total_chunks,
                   L.n_max, precision, W, reinterpret_cast<unsigned*>(w + L.off_counter),
                   reinterpret_cast<double*>(w + L.off_partials),
                   reinterpret_cast<double*>(w + L.off_out), st);
  if (e != cudaSuccess) return e;
  std::vector<double> res(3 * (size_t)count);
  e = cudaMemcpyAsync(res.data(), w + L.off_out, sizeof(double) * res.size(),
                      cudaMemcpyDeviceToHost, st);
  if (e != cudaSuccess) return e;
  e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) return e;
  for (int q = 0; q < count; ++q)
    for (int j = 0; j < 3; ++j) out3[3 * (size_t)L.order[q] + j] = res[3 * (size_t)q + j];
  return cudaSuccess;
}

}  // namespace gbsh
