// gbsh_lhaf_noalloc: loop hafnian whose scratch memory is a fixed array inside the library,
// for callers that must not allocate device memory (declaration and contract in
// include/gbsh.h).
//
// Some callers cannot call cudaMalloc: code that runs inside another framework's
// memory-managed region (a plugin or hook whose host owns the device memory through its
// own caching allocator and forbids driver allocations), and latency-critical loops where
// the implicit device synchronisation of cudaMalloc/cudaFree is not acceptable. This entry
// point takes its scratch (expanded matrix, chunk partial sums, chunk counters, result)
// from the file-scope array below instead of allocating it, and otherwise runs the same
// kernels with the same launch plan as the other entry points.
#include <cstdint>
#include <mutex>

#include <cuda_runtime.h>

#include "../../include/gbsh.h"
#include "lhaf_kernels.cuh"

namespace {

// Scratch of the no-allocation entry point. Every GPU that loads this library holds these
// GBSH_NOALLOC_SCRATCH_BYTES until the process exits. All calls share it.
static __device__ __align__(256) unsigned char g_noalloc_scratch[GBSH_NOALLOC_SCRATCH_BYTES];

// Device address of g_noalloc_scratch, looked up once per device. In host code the
// array's name is only a host-side stand-in, not a device address, so the address must
// come from cudaGetSymbolAddress with that device current.
std::mutex g_mu;
void* g_scratch_ptr[64] = {};

int fail(cudaError_t e) {
  return e == cudaErrorMemoryAllocation ? GBSH_ENOMEM : GBSH_ECUDA;
}

// The library's plan for size N (the tuning table's launch shape), with the chunk count
// halved until the scratch fits the fixed array: GBSH_OK, or GBSH_ENOMEM when even one chunk
// does not fit.
int fit_plan(int N, gbsh::LhafPlan* plan) {
  gbsh::DeviceInfo info;
  cudaError_t e = gbsh::device_info(&info);
  if (e != cudaSuccess) return fail(e);
  e = gbsh::ensure_constants();
  if (e != cudaSuccess) return fail(e);
  unsigned max_chunks = gbsh::kTargetChunks;
  for (;;) {
    if (!gbsh::make_tuned_plan(N, info, gbsh::kPrecFP64, plan, max_chunks)) return GBSH_EINVAL;
    if (plan->bytes <= (size_t)GBSH_NOALLOC_SCRATCH_BYTES) return GBSH_OK;
    if (plan->nchunks <= 1u) return GBSH_ENOMEM;
    max_chunks = plan->nchunks / 2;
  }
}

}  // namespace

extern "C" {

int gbsh_lhaf_noalloc(const gbsh_c128* dA, int N, int lda, gbsh_c128* d_out, double* d_abs_sum,
                      void* stream) {
  if (!d_out || N < 0 || N > GBSH_MAX_N) return GBSH_EINVAL;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  if (N == 0) {
    // lhaf of the empty matrix is 1, written by a one-thread kernel on the stream (no host
    // memory involved, so the call stays asynchronous)
    cudaError_t e = gbsh::launch_write_unit(reinterpret_cast<double2*>(d_out), d_abs_sum, st);
    if (e != cudaSuccess) return fail(e);
    return GBSH_OK;
  }
  if (!dA || lda < N) return GBSH_EINVAL;

  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return fail(e);
  if (dev < 0 || dev >= 64) return GBSH_EINVAL;
  void* scratch = nullptr;
  {
    // One-time set-up per device, done by the first call on that device (with it current).
    std::lock_guard<std::mutex> lk(g_mu);
    if (!g_scratch_ptr[dev]) {
      void* p = nullptr;
      e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
      if (e != cudaSuccess) return fail(e);
      g_scratch_ptr[dev] = p;
    }
    scratch = g_scratch_ptr[dev];
  }

  gbsh::LhafPlan plan;
  int rc = fit_plan(N, &plan);
  if (rc != GBSH_OK) return rc;

  // The chunk counters are zeroed inside launch_lhaf; every other scratch byte the
  // kernels read is written earlier in the same launch sequence.
  e = gbsh::launch_lhaf(plan, reinterpret_cast<const double2*>(dA), lda, nullptr, nullptr,
                        scratch, st);
  if (e != cudaSuccess) return fail(e);
  const char* res = static_cast<const char*>(scratch) + plan.off_out;
  e = cudaMemcpyAsync(d_out, res, 2 * sizeof(double), cudaMemcpyDeviceToDevice, st);
  if (e != cudaSuccess) return fail(e);
  if (d_abs_sum) {
    e = cudaMemcpyAsync(d_abs_sum, res + 2 * sizeof(double), sizeof(double),
                        cudaMemcpyDeviceToDevice, st);
    if (e != cudaSuccess) return fail(e);
  }
  return GBSH_OK;
}

int gbsh_lhaf_noalloc_plan(int N, int* nchunks) {
  if (N < 1 || N > GBSH_MAX_N) return GBSH_EINVAL;
  gbsh::LhafPlan plan;
  const int rc = fit_plan(N, &plan);
  if (rc == GBSH_OK && nchunks) *nchunks = (int)plan.nchunks;
  return rc;
}

}  // extern "C"
