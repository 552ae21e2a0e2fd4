// C ABI of the loop-hafnian engine (declarations and contracts in include/gbsh.h).
// Host code only: argument checks, device scratch, launches of the kernels in
// lhaf_kernels.cu, and the host<->device copies of the synchronous entry points.
#include <algorithm>
#include <cmath>
#include <cstdint>
#include <cstring>
#include <mutex>
#include <numeric>
#include <vector>

#include <cuda_runtime.h>

#include "../../include/gbsh.h"
#include "batch_host.h"
#include "lhaf_kernels.cuh"
#include "tuning.h"

namespace {

thread_local cudaError_t t_last_cuda = cudaSuccess;

int cuda_fail(cudaError_t e) {
  t_last_cuda = e;
  return e == cudaErrorMemoryAllocation ? GBSH_ENOMEM : GBSH_ECUDA;
}

#define GBSH_CUDA(call)                         \
  do {                                          \
    cudaError_t _e = (call);                    \
    if (_e != cudaSuccess) return cuda_fail(_e); \
  } while (0)

int g_tune_warps = 0;
int g_tune_kcap = 0;
std::mutex g_tune_mu;

// Per-device scratch for the synchronous entry points: grown on demand, kept until exit.
// A call holds the device's lock from its first launch to its final synchronisation, so
// concurrent synchronous calls on one device serialise on the host.
struct Scratch {
  std::mutex mu;
  void* ptr = nullptr;
  size_t bytes = 0;
};
Scratch g_scratch[64];

int scratch_get(Scratch& s, size_t need, void** out) {
  if (s.bytes < need) {
    if (s.ptr) {
      cudaError_t e = cudaFree(s.ptr);
      s.ptr = nullptr;
      s.bytes = 0;
      if (e != cudaSuccess) return cuda_fail(e);
    }
    size_t want = need < (1u << 20) ? (1u << 20) : need;
    cudaError_t e = cudaMalloc(&s.ptr, want);
    if (e != cudaSuccess) {
      s.ptr = nullptr;
      return cuda_fail(e);
    }
    s.bytes = want;
  }
  *out = s.ptr;
  return GBSH_OK;
}

bool is_device_pointer(const void* p) {
  cudaPointerAttributes a;
  cudaError_t e = cudaPointerGetAttributes(&a, p);
  if (e != cudaSuccess) {
    cudaGetLastError();  // clear the sticky-free error of an unknown pointer
    return false;
  }
  return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

// Precisions of the single-evaluation entry points.
bool valid_single_precision(int p) { return p == GBSH_PREC_FP64 || p == GBSH_PREC_TF; }

int plan_for(int N, gbsh::LhafPlan* plan, int prec = GBSH_PREC_FP64) {
  if (!valid_single_precision(prec)) return GBSH_EINVAL;
  gbsh::DeviceInfo dev;
  GBSH_CUDA(gbsh::device_info(&dev));
  GBSH_CUDA(gbsh::ensure_constants());
  int w, k;
  {
    std::lock_guard<std::mutex> lk(g_tune_mu);
    w = g_tune_warps;
    k = g_tune_kcap;
  }
  const int kprec = prec == GBSH_PREC_TF ? gbsh::kPrecTF : gbsh::kPrecFP64;
  // a process-wide override (gbsh_set_lhaf_tuning) replaces the per-size tuning table
  const bool ok = (w != 0 || k != 0)
                      ? gbsh::make_plan(N, dev, w, k, plan, gbsh::kTargetChunks, kprec)
                      : gbsh::make_tuned_plan(N, dev, kprec, plan);
  return ok ? GBSH_OK : GBSH_EINVAL;
}

// Unit roundoff of a precision's per-subset arithmetic (for the error estimate).
double unit_roundoff(int prec) {
  switch (prec) {
    case GBSH_PREC_C32: return std::ldexp(1.0, -24);
    case GBSH_PREC_DD: return std::ldexp(1.0, -100);
    case GBSH_PREC_TF: return std::ldexp(1.0, -70);
    default: return std::ldexp(1.0, -53);
  }
}

size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }

// Runs one loop hafnian whose (already device-resident) matrix is base[idx][idx] with
// diagonal from `diag` (or base), and copies lhaf and sum|p_Z| to the host.
int run_sync(const gbsh::LhafPlan& plan, const double2* base, int ld, const double2* diag,
             const int* idx, void* ws, cudaStream_t st, gbsh_c128* out, double* abs_sum) {
  GBSH_CUDA(gbsh::launch_lhaf(plan, base, ld, diag, idx, ws, st));
  double res[3];
  GBSH_CUDA(cudaMemcpyAsync(res, static_cast<char*>(ws) + plan.off_out, sizeof(res),
                            cudaMemcpyDeviceToHost, st));
  GBSH_CUDA(cudaStreamSynchronize(st));
  out->re = res[0];
  out->im = res[1];
  if (abs_sum) *abs_sum = res[2];
  return GBSH_OK;
}

double err_from(double abs_sum, gbsh_c128 v, int prec = GBSH_PREC_FP64) {
  double mag = std::hypot(v.re, v.im);
  if (mag == 0.0) return INFINITY;
  return unit_roundoff(prec) * abs_sum / mag;
}


// ---------------------------------------------------------------- batched evaluation
using gbsh::BatchLayout;
using gbsh::batch_layout;

int batch_run(BatchLayout& L, const std::vector<gbsh::BatchInput>& in, int count, int precision,
              void* ws, cudaStream_t st, double* out3) {
  cudaError_t e = gbsh::batch_run(L, in, count, precision, 0, ws, st, out3);
  if (e == cudaErrorInvalidValue) return GBSH_EINVAL;
  if (e != cudaSuccess) return cuda_fail(e);
  return GBSH_OK;
}

bool valid_precision(int p) {
  return p == GBSH_PREC_FP64 || p == GBSH_PREC_C32 || p == GBSH_PREC_MIXED || p == GBSH_PREC_DD ||
         p == GBSH_PREC_TF;
}


// Runs the batch in the requested precision. GBSH_PREC_MIXED evaluates the problems with
// N <= GBSH_C32_MAX_N in complex FP32 and the others in FP64, as two launches that share
// the workspace (the first `staged` bytes hold the caller's inputs).
int batch_run_mixed(const int* Ns, const std::vector<gbsh::BatchInput>& in, int count,
                    int precision, size_t staged, Scratch& s, void** ws, cudaStream_t st,
                    double* out3) {
  if (precision != GBSH_PREC_MIXED) {
    BatchLayout L = batch_layout(Ns, count, staged);
    int rc = scratch_get(s, L.bytes, ws);
    if (rc != GBSH_OK) return rc;
    return batch_run(L, in, count, precision, *ws, st, out3);
  }
  for (int pass = 0; pass < 2; ++pass) {
    const int prec = pass == 0 ? GBSH_PREC_C32 : GBSH_PREC_FP64;
    std::vector<int> sel;
    for (int p = 0; p < count; ++p)
      if ((Ns[p] <= GBSH_C32_MAX_N) == (pass == 0)) sel.push_back(p);
    if (sel.empty()) continue;
    std::vector<int> Ns_sel(sel.size());
    std::vector<gbsh::BatchInput> in_sel(sel.size());
    for (size_t q = 0; q < sel.size(); ++q) {
      Ns_sel[q] = Ns[sel[q]];
      in_sel[q] = in[sel[q]];
    }
    BatchLayout L = batch_layout(Ns_sel.data(), (int)sel.size(), staged);
    void* before = *ws;
    int rc = scratch_get(s, L.bytes, ws);
    if (rc != GBSH_OK) return rc;
    if (*ws != before) return GBSH_ENOMEM;  // staged inputs must not move between passes
    std::vector<double> o((size_t)3 * sel.size());
    rc = batch_run(L, in_sel, (int)sel.size(), prec, *ws, st, o.data());
    if (rc != GBSH_OK) return rc;
    for (size_t q = 0; q < sel.size(); ++q)
      for (int j = 0; j < 3; ++j) out3[3 * (size_t)sel[q] + j] = o[3 * q + j];
  }
  return GBSH_OK;
}

}  // namespace

extern "C" {

const char* gbsh_strerror(int code) {
  switch (code) {
    case GBSH_OK: return "ok";
    case GBSH_EINVAL: return "invalid argument";
    case GBSH_ENOMEM: return "out of device memory";
    case GBSH_ECUDA: return cudaGetErrorString(t_last_cuda);
    case GBSH_ETIMEOUT: return "bounded wait timed out";
    case GBSH_PENDING: return "request pending";
    case GBSH_ENOTFOUND: return "unknown request";
    default: return "unknown status";
  }
}

int gbsh_version(void) { return 100; }

int gbsh_set_lhaf_tuning(int warps_per_cta, int kcap) {
  if (warps_per_cta < 0 || warps_per_cta > gbsh::kMaxWarps || kcap < 0) return GBSH_EINVAL;
  std::lock_guard<std::mutex> lk(g_tune_mu);
  g_tune_warps = warps_per_cta;
  g_tune_kcap = kcap;
  return GBSH_OK;
}

int gbsh_lhaf_plan(int N, int* nclass, int* kernels, int* warps, int* kcap, int* nchunks) {
  return gbsh_lhaf_plan_ex(N, GBSH_PREC_FP64, nclass, kernels, warps, kcap, nchunks);
}

int gbsh_lhaf_plan_ex(int N, int precision, int* nclass, int* kernels, int* warps, int* kcap,
                      int* nchunks) {
  if (N < 1 || N > GBSH_MAX_N) return GBSH_EINVAL;
  gbsh::LhafPlan plan;
  int rc = plan_for(N, &plan, precision);
  if (rc != GBSH_OK) return rc;
  if (nclass) *nclass = plan.nclass;
  if (kernels) *kernels = plan.nclass + 3;
  if (warps) *warps = plan.cls[0].warps;
  if (kcap) *kcap = plan.cls[0].k_hi;
  if (nchunks) *nchunks = (int)plan.nchunks;
  return GBSH_OK;
}

size_t gbsh_lhaf_workspace_size(int N) { return gbsh_lhaf_workspace_size_ex(N, GBSH_PREC_FP64); }

size_t gbsh_lhaf_workspace_size_ex(int N, int precision) {
  if (N < 1 || N > GBSH_MAX_N) return 0;
  gbsh::LhafPlan plan;
  if (plan_for(N, &plan, precision) != GBSH_OK) return 0;
  return plan.bytes;
}

int gbsh_lhaf(const gbsh_c128* A, int N, int lda, gbsh_c128* out, double* err_est,
              void* stream) {
  return gbsh_lhaf_ex(A, N, lda, GBSH_PREC_FP64, out, err_est, stream);
}

int gbsh_lhaf_ex(const gbsh_c128* A, int N, int lda, int precision, gbsh_c128* out,
                 double* err_est, void* stream) {
  if (!out || N < 0 || N > GBSH_MAX_N || !valid_single_precision(precision)) return GBSH_EINVAL;
  if (N == 0) {
    out->re = 1.0;
    out->im = 0.0;
    if (err_est) *err_est = 0.0;
    return GBSH_OK;
  }
  if (!A || lda < N) return GBSH_EINVAL;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  gbsh::LhafPlan plan;
  int rc = plan_for(N, &plan, precision);
  if (rc != GBSH_OK) return rc;
  int dev = 0;
  GBSH_CUDA(cudaGetDevice(&dev));
  Scratch& s = g_scratch[dev & 63];
  std::lock_guard<std::mutex> lk(s.mu);
  const bool on_dev = is_device_pointer(A);
  const size_t in_off = align256(plan.bytes);
  const size_t need = on_dev ? plan.bytes : in_off + sizeof(double2) * (size_t)N * N;
  void* ws = nullptr;
  rc = scratch_get(s, need, &ws);
  if (rc != GBSH_OK) return rc;
  const double2* base = reinterpret_cast<const double2*>(A);
  int ld = lda;
  if (!on_dev) {
    double2* dA = reinterpret_cast<double2*>(static_cast<char*>(ws) + in_off);
    GBSH_CUDA(cudaMemcpy2DAsync(dA, sizeof(double2) * N, A, sizeof(double2) * lda,
                                sizeof(double2) * N, N, cudaMemcpyHostToDevice, st));
    base = dA;
    ld = N;
  }
  double asum = 0.0;
  rc = run_sync(plan, base, ld, nullptr, nullptr, ws, st, out, &asum);
  if (rc != GBSH_OK) return rc;
  if (err_est) *err_est = err_from(asum, *out, precision);
  return GBSH_OK;
}

int gbsh_lhaf_async(const gbsh_c128* dA, int N, int lda, gbsh_c128* d_out, double* d_abs_sum,
                    void* workspace, size_t workspace_bytes, void* stream) {
  return gbsh_lhaf_async_ex(dA, N, lda, GBSH_PREC_FP64, d_out, d_abs_sum, workspace,
                            workspace_bytes, stream);
}

int gbsh_lhaf_async_ex(const gbsh_c128* dA, int N, int lda, int precision, gbsh_c128* d_out,
                       double* d_abs_sum, void* workspace, size_t workspace_bytes,
                       void* stream) {
  if (!d_out || N < 0 || N > GBSH_MAX_N || !valid_single_precision(precision)) return GBSH_EINVAL;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  if (N == 0) {  // lhaf = 1, written on the stream by a one-thread kernel
    GBSH_CUDA(gbsh::launch_write_unit(reinterpret_cast<double2*>(d_out), d_abs_sum, st));
    return GBSH_OK;
  }
  if (!dA || lda < N || !workspace) return GBSH_EINVAL;
  if ((reinterpret_cast<uintptr_t>(workspace) & 255u) != 0) return GBSH_EINVAL;
  gbsh::LhafPlan plan;
  int rc = plan_for(N, &plan, precision);
  if (rc != GBSH_OK) return rc;
  if (workspace_bytes < plan.bytes) return GBSH_EINVAL;
  GBSH_CUDA(gbsh::launch_lhaf(plan, reinterpret_cast<const double2*>(dA), lda, nullptr,
                              nullptr, workspace, st));
  const char* res = static_cast<const char*>(workspace) + plan.off_out;
  GBSH_CUDA(cudaMemcpyAsync(d_out, res, 2 * sizeof(double), cudaMemcpyDeviceToDevice, st));
  if (d_abs_sum)
    GBSH_CUDA(cudaMemcpyAsync(d_abs_sum, res + 2 * sizeof(double), sizeof(double),
                              cudaMemcpyDeviceToDevice, st));
  return GBSH_OK;
}

int gbsh_lhaf_range_async(const gbsh_c128* dA, int N, int lda, int precision, uint64_t i_begin,
                          uint64_t i_end, double* d_partial, void* workspace,
                          size_t workspace_bytes, void* stream) {
  if (N < 1 || N > GBSH_MAX_N || !dA || lda < N || !d_partial || !workspace) return GBSH_EINVAL;
  if (!valid_single_precision(precision)) return GBSH_EINVAL;
  if ((reinterpret_cast<uintptr_t>(workspace) & 255u) != 0) return GBSH_EINVAL;
  const int n = (N + (N & 1)) / 2;
  if (i_begin > i_end || i_end > ((uint64_t)1 << n)) return GBSH_EINVAL;
  gbsh::LhafPlan plan;
  int rc = plan_for(N, &plan, precision);
  if (rc != GBSH_OK) return rc;
  if (workspace_bytes < plan.bytes) return GBSH_EINVAL;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  GBSH_CUDA(gbsh::launch_lhaf_range(plan, reinterpret_cast<const double2*>(dA), lda, workspace,
                                    st, i_begin, i_end));
  const char* res = static_cast<const char*>(workspace) + plan.off_out + 3 * sizeof(double);
  GBSH_CUDA(cudaMemcpyAsync(d_partial, res, 5 * sizeof(double), cudaMemcpyDeviceToDevice, st));
  return GBSH_OK;
}

int gbsh_combine_partials(const double* partials, int count, double* out) {
  if (count < 0 || !out || (count > 0 && !partials)) return GBSH_EINVAL;
  double re_hi = 0, re_lo = 0, im_hi = 0, im_lo = 0, as = 0;
  auto two_sum = [](double a, double b, double& s, double& e) {
    s = a + b;
    const double bb = s - a;
    e = (a - (s - bb)) + (b - bb);
  };
  for (int q = 0; q < count; ++q) {  // fixed input order
    const double* p = partials + 5 * (size_t)q;
    double s, e;
    two_sum(re_hi, p[0], s, e); re_hi = s; re_lo += e + p[1];
    two_sum(im_hi, p[2], s, e); im_hi = s; im_lo += e + p[3];
    as += p[4];
  }
  out[0] = re_hi; out[1] = re_lo; out[2] = im_hi; out[3] = im_lo; out[4] = as;
  return GBSH_OK;
}

int gbsh_gbs_prob(const gbsh_c128* B, int M, int ldb, const gbsh_c128* gamma,
                  const int* pattern, double p_vac, double* prob, gbsh_c128* lhaf_out,
                  void* stream) {
  if (!B || !gamma || !pattern || !prob || M < 1 || ldb < M) return GBSH_EINVAL;
  long long N = 0;
  double fact = 1.0;
  for (int i = 0; i < M; ++i) {
    if (pattern[i] < 0) return GBSH_EINVAL;
    N += pattern[i];
    for (int f = 2; f <= pattern[i]; ++f) fact *= (double)f;
  }
  if (N > GBSH_MAX_N) return GBSH_EINVAL;
  gbsh_c128 l{1.0, 0.0};
  if (N > 0) {
    // index list of B_S: mode i repeated s_i times, ascending (Sec. II)
    std::vector<int> idx;
    idx.reserve((size_t)N);
    for (int i = 0; i < M; ++i)
      for (int r = 0; r < pattern[i]; ++r) idx.push_back(i);
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    gbsh::LhafPlan plan;
    int rc = plan_for((int)N, &plan);
    if (rc != GBSH_OK) return rc;
    int dev = 0;
    GBSH_CUDA(cudaGetDevice(&dev));
    Scratch& s = g_scratch[dev & 63];
    std::lock_guard<std::mutex> lk(s.mu);
    const bool on_dev = is_device_pointer(B);
    const size_t idx_off = align256(plan.bytes);
    const size_t b_off = align256(idx_off + sizeof(int) * (size_t)N);
    const size_t g_off = align256(b_off + (on_dev ? 0 : sizeof(double2) * (size_t)M * M));
    const size_t need = align256(g_off + (on_dev ? 0 : sizeof(double2) * (size_t)M));
    void* ws = nullptr;
    rc = scratch_get(s, need, &ws);
    if (rc != GBSH_OK) return rc;
    char* w = static_cast<char*>(ws);
    int* d_idx = reinterpret_cast<int*>(w + idx_off);
    GBSH_CUDA(cudaMemcpyAsync(d_idx, idx.data(), sizeof(int) * idx.size(),
                              cudaMemcpyHostToDevice, st));
    const double2* dB = reinterpret_cast<const double2*>(B);
    const double2* dg = reinterpret_cast<const double2*>(gamma);
    int ld = ldb;
    if (!on_dev) {
      double2* b2 = reinterpret_cast<double2*>(w + b_off);
      double2* g2 = reinterpret_cast<double2*>(w + g_off);
      GBSH_CUDA(cudaMemcpy2DAsync(b2, sizeof(double2) * M, B, sizeof(double2) * ldb,
                                  sizeof(double2) * M, M, cudaMemcpyHostToDevice, st));
      GBSH_CUDA(cudaMemcpyAsync(g2, gamma, sizeof(double2) * M, cudaMemcpyHostToDevice, st));
      dB = b2;
      dg = g2;
      ld = M;
    }
    rc = run_sync(plan, dB, ld, dg, d_idx, ws, st, &l, nullptr);
    if (rc != GBSH_OK) return rc;
  }
  if (lhaf_out) *lhaf_out = l;
  *prob = p_vac * (l.re * l.re + l.im * l.im) / fact;
  return GBSH_OK;
}

int gbsh_subset_terms(const gbsh_c128* dA, int N, int lda, const uint64_t* d_z, int count,
                      gbsh_c128* d_out, void* stream) {
  return gbsh_subset_terms_ex(dA, N, lda, GBSH_PREC_FP64, d_z, count, d_out, stream);
}

int gbsh_subset_terms_ex(const gbsh_c128* dA, int N, int lda, int precision, const uint64_t* d_z,
                         int count, gbsh_c128* d_out, void* stream) {
  if (N < 1 || N > GBSH_MAX_N || !dA || lda < N || count < 0 || (count > 0 && (!d_z || !d_out)))
    return GBSH_EINVAL;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  gbsh::LhafPlan plan;
  int rc = plan_for(N, &plan, precision);
  if (rc != GBSH_OK) return rc;
  int dev = 0;
  GBSH_CUDA(cudaGetDevice(&dev));
  Scratch& s = g_scratch[dev & 63];
  std::lock_guard<std::mutex> lk(s.mu);
  void* ws = nullptr;
  rc = scratch_get(s, plan.bytes, &ws);
  if (rc != GBSH_OK) return rc;
  GBSH_CUDA(gbsh::launch_subset_terms(plan, reinterpret_cast<const double2*>(dA), lda, d_z,
                                      count, reinterpret_cast<double2*>(d_out), ws, st));
  GBSH_CUDA(cudaStreamSynchronize(st));
  return GBSH_OK;
}

int gbsh_visit_counts(int N, unsigned* d_counts, void* stream) {
  if (N < 1 || N > 40 || !d_counts) return GBSH_EINVAL;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  gbsh::LhafPlan plan;
  int rc = plan_for(N, &plan);
  if (rc != GBSH_OK) return rc;
  int dev = 0;
  GBSH_CUDA(cudaGetDevice(&dev));
  Scratch& s = g_scratch[dev & 63];
  std::lock_guard<std::mutex> lk(s.mu);
  void* ws = nullptr;
  rc = scratch_get(s, plan.bytes, &ws);
  if (rc != GBSH_OK) return rc;
  GBSH_CUDA(gbsh::launch_visit_count(plan, d_counts, ws, st));
  GBSH_CUDA(cudaStreamSynchronize(st));
  return GBSH_OK;
}

int gbsh_lhaf_batch(const gbsh_c128* A_packed, const int64_t* offsets, const int* Ns, int count,
                    gbsh_c128* outs, double* abs_sums, int precision, void* stream) {
  if (count < 0 || (count > 0 && (!A_packed || !offsets || !Ns || !outs))) return GBSH_EINVAL;
  if (!valid_precision(precision)) return GBSH_EINVAL;
  if (count == 0) return GBSH_OK;
  int64_t span = 0;
  for (int p = 0; p < count; ++p) {
    if (Ns[p] < 0 || Ns[p] > GBSH_MAX_N || offsets[p] < 0) return GBSH_EINVAL;
    span = std::max<int64_t>(span, offsets[p] + (int64_t)Ns[p] * Ns[p]);
  }
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  int dev = 0;
  GBSH_CUDA(cudaGetDevice(&dev));
  Scratch& s = g_scratch[dev & 63];
  std::lock_guard<std::mutex> lk(s.mu);
  const bool on_dev = is_device_pointer(A_packed);
  const size_t in_bytes = on_dev ? 0 : sizeof(double2) * (size_t)span;
  BatchLayout L = batch_layout(Ns, count, in_bytes);
  void* ws = nullptr;
  int rc = scratch_get(s, L.bytes, &ws);  // the full layout bounds every sub-batch
  if (rc != GBSH_OK) return rc;
  const double2* base = reinterpret_cast<const double2*>(A_packed);
  if (!on_dev) {
    GBSH_CUDA(cudaMemcpyAsync(ws, A_packed, in_bytes, cudaMemcpyHostToDevice, st));
    base = static_cast<const double2*>(ws);
  }
  std::vector<gbsh::BatchInput> in(count);
  for (int p = 0; p < count; ++p) in[p] = gbsh::BatchInput{base + offsets[p], nullptr, nullptr, Ns[p], Ns[p]};
  std::vector<double> out3(3 * (size_t)count);
  rc = batch_run_mixed(Ns, in, count, precision, in_bytes, s, &ws, st, out3.data());
  if (rc != GBSH_OK) return rc;
  for (int p = 0; p < count; ++p) {
    outs[p].re = out3[3 * p];
    outs[p].im = out3[3 * p + 1];
    if (abs_sums) abs_sums[p] = out3[3 * p + 2];
  }
  return GBSH_OK;
}

int gbsh_gbs_prob_batch(const gbsh_c128* B, int M, int ldb, const gbsh_c128* gammas,
                        int64_t gamma_stride, const int* patterns, int count,
                        const double* p_vacs, double* probs, gbsh_c128* lhafs, int precision,
                        void* stream) {
  if (count < 0 || (count > 0 && (!B || !gammas || !patterns || !probs))) return GBSH_EINVAL;
  if (M < 1 || ldb < M || gamma_stride < 0) return GBSH_EINVAL;
  if (!valid_precision(precision)) return GBSH_EINVAL;
  if (count == 0) return GBSH_OK;
  std::vector<int> Ns(count);
  std::vector<int64_t> idx_off(count + 1, 0);
  std::vector<double> fact(count, 1.0);
  for (int p = 0; p < count; ++p) {
    long long N = 0;
    for (int i = 0; i < M; ++i) {
      const int si = patterns[(size_t)p * M + i];
      if (si < 0) return GBSH_EINVAL;
      N += si;
      for (int f = 2; f <= si; ++f) fact[p] *= (double)f;
    }
    if (N > GBSH_MAX_N) return GBSH_EINVAL;
    Ns[p] = (int)N;
    idx_off[p + 1] = idx_off[p] + N;
  }
  std::vector<int> idx((size_t)idx_off[count]);
  for (int p = 0; p < count; ++p) {
    int64_t o = idx_off[p];
    for (int i = 0; i < M; ++i)
      for (int r = 0; r < patterns[(size_t)p * M + i]; ++r) idx[(size_t)o++] = i;
  }
  const int64_t gstride = gamma_stride;
  const int64_t g_elems = gstride == 0 ? M : gstride * (int64_t)(count - 1) + M;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  int dev = 0;
  GBSH_CUDA(cudaGetDevice(&dev));
  Scratch& s = g_scratch[dev & 63];
  std::lock_guard<std::mutex> lk(s.mu);
  const bool on_dev = is_device_pointer(B);
  const size_t idx_bytes = align256(sizeof(int) * std::max<size_t>(idx.size(), 1));
  const size_t b_bytes = on_dev ? 0 : align256(sizeof(double2) * (size_t)M * M);
  const size_t g_bytes = on_dev ? 0 : align256(sizeof(double2) * (size_t)g_elems);
  BatchLayout L = batch_layout(Ns.data(), count, idx_bytes + b_bytes + g_bytes);
  void* ws = nullptr;
  int rc = scratch_get(s, L.bytes, &ws);
  if (rc != GBSH_OK) return rc;
  char* w = static_cast<char*>(ws);
  int* d_idx = reinterpret_cast<int*>(w);
  if (!idx.empty())
    GBSH_CUDA(cudaMemcpyAsync(d_idx, idx.data(), sizeof(int) * idx.size(), cudaMemcpyHostToDevice, st));
  const double2* dB = reinterpret_cast<const double2*>(B);
  const double2* dg = reinterpret_cast<const double2*>(gammas);
  int ld = ldb;
  if (!on_dev) {
    double2* b2 = reinterpret_cast<double2*>(w + idx_bytes);
    double2* g2 = reinterpret_cast<double2*>(w + idx_bytes + b_bytes);
    GBSH_CUDA(cudaMemcpy2DAsync(b2, sizeof(double2) * M, B, sizeof(double2) * ldb,
                                sizeof(double2) * M, M, cudaMemcpyHostToDevice, st));
    GBSH_CUDA(cudaMemcpyAsync(g2, gammas, sizeof(double2) * (size_t)g_elems,
                              cudaMemcpyHostToDevice, st));
    dB = b2;
    dg = g2;
    ld = M;
  }
  std::vector<gbsh::BatchInput> in(count);
  for (int p = 0; p < count; ++p)
    in[p] = gbsh::BatchInput{dB, dg + gstride * p, d_idx + idx_off[p], ld, Ns[p]};
  std::vector<double> out3(3 * (size_t)count);
  rc = batch_run_mixed(Ns.data(), in, count, precision, idx_bytes + b_bytes + g_bytes, s, &ws, st,
                       out3.data());
  if (rc != GBSH_OK) return rc;
  for (int p = 0; p < count; ++p) {
    const double re = out3[3 * p], im = out3[3 * p + 1];
    if (lhafs) { lhafs[p].re = re; lhafs[p].im = im; }
    probs[p] = (p_vacs ? p_vacs[p] : 1.0) * (re * re + im * im) / fact[p];
  }
  return GBSH_OK;
}

int gbsh_set_batch_tuning(int precision, int n_max, int warps_per_cta) {
  if (precision != GBSH_PREC_FP64 && precision != GBSH_PREC_C32 && precision != GBSH_PREC_DD &&
      precision != GBSH_PREC_TF)
    return GBSH_EINVAL;
  if (n_max < 0 || n_max > gbsh::kMaxN / 2 || warps_per_cta < 0 || warps_per_cta > gbsh::kMaxWarps)
    return GBSH_EINVAL;
  gbsh::BatchTuning t = gbsh::batch_tuning(precision, n_max);
  t.warps_large = warps_per_cta;
  gbsh::set_batch_tuning(precision, n_max, t);
  return GBSH_OK;
}

int gbsh_set_batch_tuning_ex(int precision, int n_max, int warps_small, int warps_large) {
  if (precision != GBSH_PREC_FP64 && precision != GBSH_PREC_C32 && precision != GBSH_PREC_DD &&
      precision != GBSH_PREC_TF)
    return GBSH_EINVAL;
  if (n_max < 0 || n_max > gbsh::kMaxN / 2 || warps_small < 0 || warps_small > gbsh::kMaxWarps ||
      warps_large < 0 || warps_large > gbsh::kMaxWarps)
    return GBSH_EINVAL;
  gbsh::set_batch_tuning(precision, n_max, gbsh::BatchTuning{warps_small, warps_large});
  return GBSH_OK;
}

int gbsh_set_lhaf_tuning_ex(int precision, int N, int warps_cap, int ladder, int log2_chunks) {
  if (!valid_single_precision(precision) || N < 1 || N > GBSH_MAX_N) return GBSH_EINVAL;
  if (warps_cap < 0 || warps_cap > gbsh::kMaxWarps || ladder < 0 || ladder > 2 ||
      log2_chunks < 0 || log2_chunks > 18)
    return GBSH_EINVAL;
  const int kprec = precision == GBSH_PREC_TF ? gbsh::kPrecTF : gbsh::kPrecFP64;
  gbsh::set_single_tuning(kprec, N, gbsh::SingleTuning{warps_cap, ladder, log2_chunks});
  return GBSH_OK;
}

int gbsh_get_lhaf_tuning(int precision, int N, int* warps_cap, int* ladder, int* log2_chunks) {
  if (!valid_single_precision(precision) || N < 1 || N > GBSH_MAX_N) return GBSH_EINVAL;
  const int kprec = precision == GBSH_PREC_TF ? gbsh::kPrecTF : gbsh::kPrecFP64;
  const gbsh::SingleTuning t = gbsh::single_tuning(kprec, N);
  if (warps_cap) *warps_cap = t.warps_cap;
  if (ladder) *ladder = t.ladder;
  if (log2_chunks) *log2_chunks = t.log2_chunks;
  return GBSH_OK;
}

int gbsh_get_batch_tuning(int precision, int n_max, int* warps_small, int* warps_large) {
  if (precision < 0 || precision >= gbsh::kNumPrec || precision == GBSH_PREC_MIXED || n_max < 0 ||
      n_max > gbsh::kMaxN / 2)
    return GBSH_EINVAL;
  const gbsh::BatchTuning t = gbsh::batch_tuning(precision, n_max);
  if (warps_small) *warps_small = t.warps_small;
  if (warps_large) *warps_large = t.warps_large;
  return GBSH_OK;
}

int gbsh_builtin_tuning_entries(void) { return gbsh::builtin_tuning_entries(nullptr, nullptr); }

int gbsh_set_batch_graphs(int enable) {
  gbsh::set_batch_graphs(enable != 0);
  return GBSH_OK;
}

int gbsh_batch_graph_stats(long long* captures, long long* replays) {
  gbsh::batch_graph_stats(captures, replays);
  return GBSH_OK;
}

}  // extern "C"
