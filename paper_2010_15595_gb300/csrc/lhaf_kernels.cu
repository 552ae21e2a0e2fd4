// Loop-hafnian kernels for sm_103a (GB300).
//
//   expand_problem_kernel   pattern expansion + filldiag (Sec. II: B_S repeats row/column i
//                           s_i times, Eq. lhaf-pure puts the fill vector on the diagonal),
//                           padding to even size, diagonal split off into the loop weights.
//   lhaf_subsets_kernel     the signed sum over pair subsets (the cited O(N^3 2^{N/2})
//                           subset formula, Sec. II / Sec. IV), one warp per subset, subsets
//                           visited in Gray-code order inside fixed chunks that warps claim
//                           from a counter; one compensated partial per chunk.
//   lhaf_finalize_kernel    fixed-order compensated reduction of the chunk partials.
//
// The result depends only on the chunking (the chunk count of the plan) and the popcount
// classes, not on the warps per CTA or on which warp took which chunk, so a given plan is
// bit-reproducible.
#include <cmath>
#include <mutex>

#include "lhaf_core.cuh"
#include "lhaf_kernels.cuh"
#include "tuning.h"

namespace gbsh {

// ------------------------------------------------------------------ expansion
// A0[r][c] = base[idx[r]][idx[c]] (r != c), v[r] = diag ? diag[idx[r]] : base[idx[r]][idx[r]].
// Rows/columns >= N (odd padding) are zero with loop weight 1.
__global__ void expand_problem_kernel(const double2* __restrict__ base, int ld,
                                      const double2* __restrict__ diag,
                                      const int* __restrict__ idx, int N, int Ne,
                                      double2* __restrict__ A0, double2* __restrict__ v) {
  const int tid = blockIdx.x * blockDim.x + threadIdx.x;
  const int stride = gridDim.x * blockDim.x;
  for (int e = tid; e < Ne * Ne; e += stride) {
    int r = e / Ne, c = e - r * Ne;
    double2 val = make_double2(0.0, 0.0);
    if (r != c && r < N && c < N) {
      int ir = idx ? idx[r] : r, ic = idx ? idx[c] : c;
      val = base[(size_t)ir * ld + ic];
    }
    A0[e] = val;
  }
  for (int r = tid; r < Ne; r += stride) {
    double2 w = make_double2(1.0, 0.0);
    if (r < N) {
      int ir = idx ? idx[r] : r;
      w = diag ? diag[ir] : base[(size_t)ir * ld + ir];
    }
    v[r] = w;
  }
}

// ------------------------------------------------------------------ subset sum
// kVisit = true replaces the per-subset term by a visit count (enumeration check).
// T: complex type of the per-subset arithmetic (double2, or tfc for the triple-float path).
template <class T, bool kVisit>
__global__ void __launch_bounds__(32 * kMaxWarps, 1)
lhaf_subsets_kernel(Problem P, int k_lo, int k_hi, int area_elems, uint64_t chunk_size,
                    uint64_t i_base, uint64_t i_end, unsigned nchunks,
                    unsigned* __restrict__ counter, double* __restrict__ partials,
                    unsigned* __restrict__ visits) {
  extern __shared__ double2 smem_raw[];
  T* smem = reinterpret_cast<T*>(smem_raw);
  const int lane = threadIdx.x & 31;
  const int warp = threadIdx.x >> 5;
  T* area = smem + (size_t)warp * area_elems;
  const int n = P.n;

  for (;;) {
    unsigned ch = 0;
    if (lane == 0) ch = atomicAdd(counter, 1u);
    ch = __shfl_sync(FULL, ch, 0);
    if (ch >= nchunks) break;
    DDAcc acc;
    acc.zero();
    // chunk ch covers the enumeration indices [i0, i1) of the evaluated range
    const uint64_t i0 = i_base + (uint64_t)ch * chunk_size;
    const uint64_t i1 = i0 + chunk_size < i_end ? i0 + chunk_size : i_end;
    for (uint64_t i = i0; i < i1; ++i) {
      const uint64_t z = i ^ (i >> 1);  // Gray-code order of the chunk's indices
      const int k = __popcll(z);
      if (k < k_lo || k > k_hi || k == 0) continue;
      if (kVisit) {
        if (lane == 0) atomicAdd(visits + z, 1u);
        continue;
      }
      Term t = subset_term_full<T>(P, z, k, area, lane);
      if ((n - k) & 1) t = Term{-t.re_hi, -t.re_lo, -t.im_hi, -t.im_lo};
      acc.add(t);
    }
    if (!kVisit && lane == 0) {
      double* o = partials + (size_t)ch * 5;
      o[0] = acc.re_hi; o[1] = acc.re_lo; o[2] = acc.im_hi; o[3] = acc.im_lo; o[4] = acc.abs_sum;
    }
  }
}

// p_Z for a list of subsets (debug / sampled parity). One warp per listed subset.
template <class T>
__global__ void __launch_bounds__(32 * kMaxWarps, 1)
subset_terms_kernel(Problem P, int area_elems, const uint64_t* __restrict__ zs, int count,
                    double2* __restrict__ out) {
  extern __shared__ double2 smem_raw[];
  T* smem = reinterpret_cast<T*>(smem_raw);
  const int lane = threadIdx.x & 31;
  const int warp = threadIdx.x >> 5;
  const int wpb = blockDim.x >> 5;
  T* area = smem + (size_t)warp * area_elems;
  for (int q = blockIdx.x * wpb + warp; q < count; q += gridDim.x * wpb) {
    const uint64_t z = zs[q];
    const int k = __popcll(z);
    double2 pz = make_double2(P.n == 0 ? 1.0 : 0.0, 0.0);
    if (k > 0) pz = subset_term<T>(P, z, k, area, lane);
    if (lane == 0) out[q] = pz;
  }
}

// ------------------------------------------------------------------ finalize
// Two levels, both in a fixed order (results do not depend on scheduling):
//   lhaf_partials_kernel: CTA b sums chunks [b*per, (b+1)*per) of every class into
//     block_out[b][5] (per = ceil(nchunks / gridDim.x));
//   lhaf_finalize_kernel: one CTA sums block_out[0..nblocks) in block order into
//     out[0..1] = lhaf (re, im), out[2] = sum over subsets of |Re p_Z| + |Im p_Z|.
// Each level: thread-strided compensated sums, then a fixed binary tree in shared memory.
__device__ __forceinline__ void add_partial(DDAcc& a, const double* __restrict__ q) {
  double s, e;
  DDAcc::two_sum(a.re_hi, q[0], s, e); a.re_hi = s; a.re_lo += e + q[1];
  DDAcc::two_sum(a.im_hi, q[2], s, e); a.im_hi = s; a.im_lo += e + q[3];
  a.abs_sum += q[4];
}

// Tree over the CTA's threads; the CTA total ends in sh[.][0].
__device__ __forceinline__ void block_tree(DDAcc a, double (*sh)[kFinalizeThreads]) {
  const int t = threadIdx.x;
  sh[0][t] = a.re_hi; sh[1][t] = a.re_lo; sh[2][t] = a.im_hi; sh[3][t] = a.im_lo; sh[4][t] = a.abs_sum;
  __syncthreads();
  for (int w = kFinalizeThreads / 2; w > 0; w >>= 1) {
    if (t < w) {
      double s, e;
      DDAcc::two_sum(sh[0][t], sh[0][t + w], s, e); sh[0][t] = s; sh[1][t] += e + sh[1][t + w];
      DDAcc::two_sum(sh[2][t], sh[2][t + w], s, e); sh[2][t] = s; sh[3][t] += e + sh[3][t + w];
      sh[4][t] += sh[4][t + w];
    }
    __syncthreads();
  }
}

__global__ void __launch_bounds__(kFinalizeThreads)
lhaf_partials_kernel(const double* __restrict__ partials, unsigned nchunks, unsigned stride,
                     int nclass, double* __restrict__ block_out) {
  __shared__ double sh[5][kFinalizeThreads];
  const unsigned per = (nchunks + gridDim.x - 1) / gridDim.x;
  const unsigned c0 = blockIdx.x * per;
  const unsigned c1 = c0 + per < nchunks ? c0 + per : nchunks;
  DDAcc a;
  a.zero();
  for (int cls = 0; cls < nclass; ++cls) {
    const double* p = partials + (size_t)cls * stride * 5;
    for (unsigned ch = c0 + threadIdx.x; ch < c1; ch += kFinalizeThreads) add_partial(a, p + (size_t)ch * 5);
  }
  block_tree(a, sh);
  if (threadIdx.x == 0)
    for (int j = 0; j < 5; ++j) block_out[(size_t)blockIdx.x * 5 + j] = sh[j][0];
}

__global__ void __launch_bounds__(kFinalizeThreads)
lhaf_finalize_kernel(const double* __restrict__ block_out, int nblocks, double* __restrict__ out) {
  __shared__ double sh[5][kFinalizeThreads];
  DDAcc a;
  a.zero();
  for (int b = threadIdx.x; b < nblocks; b += kFinalizeThreads) add_partial(a, block_out + (size_t)b * 5);
  block_tree(a, sh);
  if (threadIdx.x == 0) {
    out[0] = sh[0][0] + sh[1][0];
    out[1] = sh[2][0] + sh[3][0];
    out[2] = sh[4][0];
    // the unrounded compensated sum (re_hi, re_lo, im_hi, im_lo, sum |p|) for range partials
    for (int j = 0; j < 5; ++j) out[3 + j] = sh[j][0];
  }
}

// ================================================================== batched evaluation
// Many loop hafnians of uneven size in one persistent launch. Problem p owns global
// chunks [chunk_base, chunk_base + nchunks); warps claim global chunks from a counter in
// increasing order, and problems are ordered by decreasing size, so the expensive chunks
// go first and the tail is made of small ones (longest-processing-time order). Each
// problem's chunking depends only on its own size, so its result is bit-identical whether
// it runs alone or inside any batch.

__global__ void expand_batch_kernel(const BatchInput* __restrict__ in,
                                    const BatchProblem* __restrict__ prob, int count) {
  const int p = blockIdx.x;
  if (p >= count) return;
  const BatchInput I = in[p];
  const BatchProblem Q = prob[p];
  double2* A0 = const_cast<double2*>(Q.A0);
  double2* v = const_cast<double2*>(Q.v);
  const int N = I.N, Ne = Q.Ne;
  for (int e = threadIdx.x; e < Ne * Ne; e += blockDim.x) {
    int r = e / Ne, c = e - r * Ne;
    double2 val = make_double2(0.0, 0.0);
    if (r != c && r < N && c < N) {
      int ir = I.idx ? I.idx[r] : r, ic = I.idx ? I.idx[c] : c;
      val = I.base[(size_t)ir * I.ld + ic];
    }
    A0[e] = val;
  }
  for (int r = threadIdx.x; r < Ne; r += blockDim.x) {
    double2 w = make_double2(1.0, 0.0);
    if (r < N) {
      int ir = I.idx ? I.idx[r] : r;
      w = I.diag ? I.diag[ir] : I.base[(size_t)ir * I.ld + ir];
    }
    v[r] = w;
  }
}

template <class T>
__global__ void __launch_bounds__(32 * kMaxWarps, 1)
lhaf_batch_kernel(const BatchProblem* __restrict__ prob, int count, unsigned total_chunks,
                  int k_lo, int k_hi, int area_elems, unsigned* __restrict__ counter,
                  double* __restrict__ partials) {
  extern __shared__ double2 smem_raw[];
  T* smem = reinterpret_cast<T*>(smem_raw);
  const int lane = threadIdx.x & 31;
  const int warp = threadIdx.x >> 5;
  T* area = smem + (size_t)warp * area_elems;
  for (;;) {
    unsigned g = 0;
    if (lane == 0) g = atomicAdd(counter, 1u);
    g = __shfl_sync(FULL, g, 0);
    if (g >= total_chunks) break;
    // problem owning chunk g: last p with chunk_base <= g (bases are increasing)
    int lo = 0, hi = count - 1;
    while (lo < hi) {
      int mid = (lo + hi + 1) >> 1;
      if (prob[mid].chunk_base <= g) lo = mid; else hi = mid - 1;
    }
    const BatchProblem Q = prob[lo];
    Problem P;
    P.A0 = Q.A0;
    P.v = Q.v;
    P.Ne = Q.Ne;
    P.n = Q.n;
    DDAcc acc;
    acc.zero();
    const uint64_t i0 = (uint64_t)(g - Q.chunk_base) * Q.chunk_size, i1 = i0 + Q.chunk_size;
    for (uint64_t i = i0; i < i1; ++i) {
      const uint64_t z = i ^ (i >> 1);
      const int k = __popcll(z);
      if (k == 0 || k < k_lo || k > k_hi) continue;
      Term t = subset_term_full<T>(P, z, k, area, lane);
      if ((P.n - k) & 1) t = Term{-t.re_hi, -t.re_lo, -t.im_hi, -t.im_lo};
      acc.add(t);
    }
    if (lane == 0) {
      double* o = partials + (size_t)g * 5;
      o[0] = acc.re_hi; o[1] = acc.re_lo; o[2] = acc.im_hi; o[3] = acc.im_lo; o[4] = acc.abs_sum;
    }
  }
}

// One thread per problem: its chunk partials in increasing chunk order, the class-0 partial
// of a chunk before its class-1 partial (nclass = 1 or 2 popcount classes, partials of class
// c at partials + c * total_chunks * 5). A class that holds no subset of a chunk wrote an
// exact zero there, so a problem's result does not depend on whether the second class ran.
// out[p] = (re, im, sum|p|).
__global__ void lhaf_batch_finalize_kernel(const BatchProblem* __restrict__ prob, int count,
                                           const double* __restrict__ partials,
                                           unsigned total_chunks, int nclass,
                                           double* __restrict__ out) {
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= count) return;
  const BatchProblem Q = prob[p];
  DDAcc a;
  a.zero();
  for (unsigned c = 0; c < Q.nchunks; ++c) {
    for (int cls = 0; cls < nclass; ++cls) {
      const double* q = partials + ((size_t)cls * total_chunks + Q.chunk_base + c) * 5;
      double s, e;
      DDAcc::two_sum(a.re_hi, q[0], s, e); a.re_hi = s; a.re_lo += e + q[1];
      DDAcc::two_sum(a.im_hi, q[2], s, e); a.im_hi = s; a.im_lo += e + q[3];
      a.abs_sum += q[4];
    }
  }
  out[3 * p + 0] = Q.n == 0 ? 1.0 : a.re_hi + a.re_lo;
  out[3 * p + 1] = Q.n == 0 ? 0.0 : a.im_hi + a.im_lo;
  out[3 * p + 2] = Q.n == 0 ? 1.0 : a.abs_sum;
}

// ================================================================== host side

namespace {
std::mutex g_mu;
bool g_const_done[64] = {};
DeviceInfo g_info[64];
bool g_info_done[64] = {};

size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }
}  // namespace

cudaError_t device_info(DeviceInfo* info) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= 64) return cudaErrorInvalidDevice;
  std::lock_guard<std::mutex> lk(g_mu);
  if (!g_info_done[dev]) {
    DeviceInfo d{};
    e = cudaDeviceGetAttribute(&d.sm_count, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess) return e;
    e = cudaDeviceGetAttribute(&d.smem_optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    if (e != cudaSuccess) return e;
    e = cudaFuncSetAttribute(lhaf_subsets_kernel<double2, false>,
                             cudaFuncAttributeMaxDynamicSharedMemorySize, d.smem_optin);
    if (e != cudaSuccess) return e;
    e = cudaFuncSetAttribute(lhaf_subsets_kernel<double2, true>,
                             cudaFuncAttributeMaxDynamicSharedMemorySize, d.smem_optin);
    if (e != cudaSuccess) return e;
    e = cudaFuncSetAttribute(lhaf_subsets_kernel<tfc, false>,
                             cudaFuncAttributeMaxDynamicSharedMemorySize, d.smem_optin);
    if (e != cudaSuccess) return e;
    e = cudaFuncSetAttribute(subset_terms_kernel<double2>,
                             cudaFuncAttributeMaxDynamicSharedMemorySize, d.smem_optin);
    if (e != cudaSuccess) return e;
    e = cudaFuncSetAttribute(subset_terms_kernel<tfc>,
                             cudaFuncAttributeMaxDynamicSharedMemorySize, d.smem_optin);
    if (e != cudaSuccess) return e;
    e = cudaFuncSetAttribute(lhaf_batch_kernel<tfc>,
                             cudaFuncAttributeMaxDynamicSharedMemorySize, d.smem_optin);
    if (e != cudaSuccess) return e;
    e = cudaFuncSetAttribute(lhaf_batch_kernel<double2>,
                             cudaFuncAttributeMaxDynamicSharedMemorySize, d.smem_optin);
    if (e != cudaSuccess) return e;
    e = cudaFuncSetAttribute(lhaf_batch_kernel<float2>,
                             cudaFuncAttributeMaxDynamicSharedMemorySize, d.smem_optin);
    if (e != cudaSuccess) return e;
    e = cudaFuncSetAttribute(lhaf_batch_kernel<ddc>,
                             cudaFuncAttributeMaxDynamicSharedMemorySize, d.smem_optin);
    if (e != cudaSuccess) return e;
    g_info[dev] = d;
    g_info_done[dev] = true;
  }
  *info = g_info[dev];
  return cudaSuccess;
}

cudaError_t ensure_constants() {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  std::lock_guard<std::mutex> lk(g_mu);
  if (!g_const_done[dev]) {
    double inv[64];
    inv[0] = 0.0;
    for (int k = 1; k < 64; ++k) inv[k] = 1.0 / (double)k;
    e = cudaMemcpyToSymbol(c_inv_int, inv, sizeof(inv));
    if (e != cudaSuccess) return e;
    // 1/k as three FP32 words: q = floor(2^100 / k) exactly, then its leading 24 bits, the
    // next 24 bits and the next 24 bits (truncation keeps the words non-overlapping and of
    // one sign; the value is within 2^-90 of 1/k).
    float invt[64][3] = {};
    for (int k = 1; k < 64; ++k) {
      unsigned __int128 q = (((unsigned __int128)1) << 100) / (unsigned)k;
      for (int w = 0; w < 3; ++w) {
        if (q == 0) break;
        int h = 127;
        while (!((q >> h) & 1)) --h;
        const int sh = h >= 23 ? h - 23 : 0;
        const unsigned long long top = (unsigned long long)(q >> sh);
        invt[k][w] = std::ldexp((float)top, sh - 100);
        q -= ((unsigned __int128)top) << sh;
      }
    }
    e = cudaMemcpyToSymbol(c_inv_tf, invt, sizeof(invt));
    if (e != cudaSuccess) return e;
    g_const_done[dev] = true;
  }
  return cudaSuccess;
}

bool make_plan(int N, const DeviceInfo& dev, int warps_main, int kcap_override, LhafPlan* p,
               unsigned max_chunks, int prec, int ladder) {
  if (N < 1 || N > kMaxN) return false;
  if (prec != kPrecFP64 && prec != kPrecTF) return false;
  LhafPlan plan{};
  plan.prec = prec;
  plan.esz = prec_elem_bytes(prec);
  plan.N = N;
  plan.Ne = N + (N & 1);
  plan.n = plan.Ne / 2;
  const int n = plan.n;
  const size_t limit = (size_t)dev.smem_optin;
  const int esz = plan.esz;
  auto area_bytes = [&](int k) { return (size_t)warp_area_elems(k, n, esz) * esz; };
  // largest popcount whose work area fits W warps per CTA (0 if none)
  auto kfit = [&](int W) {
    int kc = 0;
    for (int k = 1; k <= n; ++k)
      if ((size_t)W * area_bytes(k) <= limit) kc = k;
    return kc;
  };
  // default cap: 12 warps per CTA for FP64 (the FP64 pipe is the limit, measured best);
  // 16 for triple-float, whose FP32 instruction stream needs more warps to hide latency
  int W = warps_main > 0 ? warps_main : (prec == kPrecTF ? 16 : 12);
  if (W > kMaxWarps) W = kMaxWarps;
  // Popcount classes: subsets with popcount in (k_prev, k_c] run in one launch with W_c warps
  // per CTA, W_c the largest count of a fixed ladder (capped at W) whose work areas fit.
  // Most subsets (popcount near n/2) have small matrices and run with many warps per SM to
  // hide the FP64 latency; the few large ones run with larger work areas.
  // The fine ladder adds intermediate steps, so that more popcounts run with more warps (at
  // the cost of more class launches and partial sums).
  static const int kCoarse[] = {16, 12, 8, 6, 4, 3, 2, 1};
  static const int kFine[] = {16, 14, 12, 10, 8, 7, 6, 5, 4, 3, 2, 1};
  const int* lad = ladder == kLadderFine ? kFine : kCoarse;
  const int nlad = ladder == kLadderFine ? (int)(sizeof(kFine) / sizeof(kFine[0]))
                                         : (int)(sizeof(kCoarse) / sizeof(kCoarse[0]));
  plan.nclass = 0;
  int k_done = 0;
  for (int wi = 0; wi < nlad && k_done < n; ++wi) {
    const int Wc = lad[wi];
    if (Wc > W) continue;
    int kc = kfit(Wc);
    if (plan.nclass == 0 && kcap_override > 0 && kcap_override < kc) kc = kcap_override;
    if (kc > k_done) {
      if (plan.nclass == kMaxClasses) return false;
      plan.cls[plan.nclass++] = ClassPlan{k_done + 1, kc, Wc, warp_area_elems(kc, n, esz), 0};
      k_done = kc;
    }
  }
  if (k_done < n) return false;
  for (int c = 0; c < plan.nclass; ++c) {
    ClassPlan& cp = plan.cls[c];
    int per_sm = 0;
    size_t smem = (size_t)cp.warps * cp.area_elems * esz;
    cudaError_t oe = prec == kPrecTF
                         ? cudaOccupancyMaxActiveBlocksPerMultiprocessor(
                               &per_sm, lhaf_subsets_kernel<tfc, false>, 32 * cp.warps, smem)
                         : cudaOccupancyMaxActiveBlocksPerMultiprocessor(
                               &per_sm, lhaf_subsets_kernel<double2, false>, 32 * cp.warps, smem);
    if (oe != cudaSuccess || per_sm < 1) per_sm = 1;
    cp.blocks = per_sm * dev.sm_count;
  }
  const uint64_t total = (uint64_t)1 << n;
  unsigned cap = kTargetChunks;  // largest power of two <= max_chunks
  while (cap > 1u && cap > max_chunks) cap >>= 1;
  plan.nchunks = (unsigned)(total < cap ? total : cap);
  plan.chunk_size = total / plan.nchunks;
  size_t off = 0;
  plan.off_A0 = off; off = align256(off + sizeof(double2) * plan.Ne * plan.Ne);
  plan.off_v = off; off = align256(off + sizeof(double2) * plan.Ne);
  plan.off_partials = off; off = align256(off + sizeof(double) * 5 * (size_t)plan.nclass * plan.nchunks);
  plan.off_counters = off; off = align256(off + sizeof(unsigned) * kMaxClasses);
  plan.off_blocks = off; off = align256(off + sizeof(double) * 5 * kReduceBlocks);
  plan.off_out = off; off = align256(off + sizeof(double) * 8);
  plan.bytes = off;
  *p = plan;
  return true;
}

bool make_tuned_plan(int N, const DeviceInfo& dev, int prec, LhafPlan* p, unsigned max_chunks) {
  const SingleTuning t = single_tuning(prec, N);
  unsigned cap = max_chunks;
  if (t.log2_chunks >= 1 && t.log2_chunks <= 18 && (1u << t.log2_chunks) < cap)
    cap = 1u << t.log2_chunks;
  return make_plan(N, dev, t.warps_cap, 0, p, cap, prec, t.ladder);
}

static Problem problem_of(const LhafPlan& plan, void* ws) {
  char* b = static_cast<char*>(ws);
  Problem P;
  P.A0 = reinterpret_cast<const double2*>(b + plan.off_A0);
  P.v = reinterpret_cast<const double2*>(b + plan.off_v);
  P.Ne = plan.Ne;
  P.n = plan.n;
  return P;
}

static cudaError_t launch_expand(const LhafPlan& plan, const double2* base, int ld,
                                 const double2* diag, const int* idx, void* ws,
                                 cudaStream_t stream) {
  char* b = static_cast<char*>(ws);
  const int elems = plan.Ne * plan.Ne;
  const int threads = 256;
  const int blocks = (elems + threads - 1) / threads;
  expand_problem_kernel<<<blocks, threads, 0, stream>>>(
      base, ld, diag, idx, plan.N, plan.Ne, reinterpret_cast<double2*>(b + plan.off_A0),
      reinterpret_cast<double2*>(b + plan.off_v));
  return cudaGetLastError();
}

// Side streams on which the popcount classes after the first run, so that the tail of one
// class launch overlaps the next (each class has its own counter and partial sums). One set
// per device, created on first use and kept for the life of the process.
static cudaError_t side_streams(cudaStream_t** out) {
  static cudaStream_t streams[64][kMaxClasses] = {};
  static bool made[64] = {};
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= 64) return cudaErrorInvalidDevice;
  std::lock_guard<std::mutex> lk(g_mu);
  if (!made[dev]) {
    for (int c = 1; c < kMaxClasses; ++c) {
      e = cudaStreamCreateWithFlags(&streams[dev][c], cudaStreamNonBlocking);
      if (e != cudaSuccess) {
        for (int d = 1; d < c; ++d) cudaStreamDestroy(streams[dev][d]);
        return e;
      }
    }
    made[dev] = true;
  }
  *out = streams[dev];
  return cudaSuccess;
}

// Launches every popcount class. Class 0 runs on `stream`; the others on the side streams,
// forked from and joined back into `stream` with events, so all work of the evaluation is
// ordered after what precedes it on `stream` and before what follows.
template <bool kVisit>
static cudaError_t launch_classes(const LhafPlan& plan, void* ws, unsigned* visits,
                                  cudaStream_t stream, uint64_t i_base, uint64_t i_end,
                                  unsigned nchunks) {
  char* b = static_cast<char*>(ws);
  unsigned* counters = reinterpret_cast<unsigned*>(b + plan.off_counters);
  double* partials = reinterpret_cast<double*>(b + plan.off_partials);
  cudaError_t e = cudaMemsetAsync(counters, 0, sizeof(unsigned) * kMaxClasses, stream);
  if (e != cudaSuccess) return e;
  const Problem P = problem_of(plan, ws);
  cudaStream_t* side = nullptr;
  cudaEvent_t fork = nullptr;
  if (plan.nclass > 1) {
    e = side_streams(&side);
    if (e != cudaSuccess) return e;
    e = cudaEventCreateWithFlags(&fork, cudaEventDisableTiming);
    if (e != cudaSuccess) return e;
    e = cudaEventRecord(fork, stream);
  }
  for (int c = 0; c < plan.nclass && e == cudaSuccess; ++c) {
    const ClassPlan& cp = plan.cls[c];
    cudaStream_t sc = c == 0 ? stream : side[c];
    if (c > 0) e = cudaStreamWaitEvent(sc, fork, 0);
    if (e != cudaSuccess) break;
    const size_t smem = (size_t)cp.warps * cp.area_elems * plan.esz;
    if (!kVisit && plan.prec == kPrecTF)
      lhaf_subsets_kernel<tfc, false><<<cp.blocks, 32 * cp.warps, smem, sc>>>(
          P, cp.k_lo, cp.k_hi, cp.area_elems, plan.chunk_size, i_base, i_end, nchunks,
          counters + c, partials + (size_t)c * plan.nchunks * 5, visits);
    else
      lhaf_subsets_kernel<double2, kVisit><<<cp.blocks, 32 * cp.warps, smem, sc>>>(
          P, cp.k_lo, cp.k_hi, cp.area_elems, plan.chunk_size, i_base, i_end, nchunks,
          counters + c, partials + (size_t)c * plan.nchunks * 5, visits);
    e = cudaGetLastError();
    if (e == cudaSuccess && c > 0) {
      cudaEvent_t join = nullptr;
      e = cudaEventCreateWithFlags(&join, cudaEventDisableTiming);
      if (e == cudaSuccess) e = cudaEventRecord(join, sc);
      if (e == cudaSuccess) e = cudaStreamWaitEvent(stream, join, 0);
      if (join) cudaEventDestroy(join);
    }
  }
  if (fork) cudaEventDestroy(fork);
  return e;
}

// Subsets of the enumeration indices [i_begin, i_end) (z = i ^ (i >> 1)), in chunks of the
// plan's chunk size starting at i_begin, then the two-level fixed-order finalize.
cudaError_t launch_range(const LhafPlan& plan, const double2* base, int ld,
                         const double2* diag, const int* idx, void* ws,
                         cudaStream_t stream, uint64_t i_begin, uint64_t i_end) {
  cudaError_t e = launch_expand(plan, base, ld, diag, idx, ws, stream);
  if (e != cudaSuccess) return e;
  const uint64_t span = i_end > i_begin ? i_end - i_begin : 0;
  const unsigned nchunks = (unsigned)((span + plan.chunk_size - 1) / plan.chunk_size);
  e = launch_classes<false>(plan, ws, nullptr, stream, i_begin, i_end, nchunks);
  if (e != cudaSuccess) return e;
  char* b = static_cast<char*>(ws);
  double* blocks = reinterpret_cast<double*>(b + plan.off_blocks);
  lhaf_partials_kernel<<<kReduceBlocks, kFinalizeThreads, 0, stream>>>(
      reinterpret_cast<const double*>(b + plan.off_partials), nchunks, plan.nchunks, plan.nclass,
      blocks);
  lhaf_finalize_kernel<<<1, kFinalizeThreads, 0, stream>>>(blocks, kReduceBlocks,
                                                           reinterpret_cast<double*>(b + plan.off_out));
  return cudaGetLastError();
}

cudaError_t launch_lhaf(const LhafPlan& plan, const double2* base, int ld, const double2* diag,
                        const int* idx, void* ws, cudaStream_t stream) {
  return launch_range(plan, base, ld, diag, idx, ws, stream, 0, (uint64_t)1 << plan.n);
}

cudaError_t launch_lhaf_range(const LhafPlan& plan, const double2* base, int ld, void* ws,
                              cudaStream_t stream, uint64_t i_begin, uint64_t i_end) {
  return launch_range(plan, base, ld, nullptr, nullptr, ws, stream, i_begin, i_end);
}

cudaError_t launch_subset_terms(const LhafPlan& plan, const double2* base, int ld,
                                const uint64_t* z, int count, double2* out, void* ws,
                                cudaStream_t stream) {
  cudaError_t e = launch_expand(plan, base, ld, nullptr, nullptr, ws, stream);
  if (e != cudaSuccess) return e;
  if (count <= 0) return cudaSuccess;
  // every listed subset may be the full set: size the area for k = n
  const int area = warp_area_elems(plan.n, plan.n, plan.esz);
  DeviceInfo dev;
  e = device_info(&dev);
  if (e != cudaSuccess) return e;
  int W = (int)((size_t)dev.smem_optin / ((size_t)area * plan.esz));
  if (W > 4) W = 4;
  if (W < 1) return cudaErrorInvalidValue;
  int blocks = (count + W - 1) / W;
  if (blocks > 4 * dev.sm_count) blocks = 4 * dev.sm_count;
  const size_t smem = (size_t)W * area * plan.esz;
  if (plan.prec == kPrecTF)
    subset_terms_kernel<tfc><<<blocks, 32 * W, smem, stream>>>(problem_of(plan, ws), area, z, count, out);
  else
    subset_terms_kernel<double2><<<blocks, 32 * W, smem, stream>>>(problem_of(plan, ws), area, z, count, out);
  return cudaGetLastError();
}

__global__ void write_unit_kernel(double2* __restrict__ out, double* __restrict__ abs_sum) {
  out[0] = make_double2(1.0, 0.0);
  if (abs_sum) abs_sum[0] = 0.0;
}

cudaError_t launch_write_unit(double2* out, double* abs_sum, cudaStream_t stream) {
  write_unit_kernel<<<1, 1, 0, stream>>>(out, abs_sum);
  return cudaGetLastError();
}

cudaError_t launch_visit_count(const LhafPlan& plan, unsigned* counts, void* ws,
                               cudaStream_t stream) {
  return launch_classes<true>(plan, ws, counts, stream, 0, (uint64_t)1 << plan.n, plan.nchunks);
}

}  // namespace gbsh

namespace gbsh {

int batch_warps_for(int n_max, int precision, const DeviceInfo& dev, int warps_pref) {
  const int esz = prec_elem_bytes(precision);
  const size_t area = (size_t)warp_area_elems(n_max, n_max, esz) * esz;
  int W = warps_pref > 0 ? warps_pref : 8;
  if (W > kMaxWarps) W = kMaxWarps;
  while (W > 1 && (size_t)W * area > (size_t)dev.smem_optin) --W;
  if ((size_t)W * area > (size_t)dev.smem_optin) return 0;
  return W;
}

// Blocks per SM of the batch kernel for precision `precision`, W warps and `smem` bytes.
static int batch_blocks_per_sm(int precision, int W, size_t smem) {
  int per_sm = 1;
  if (precision == kPrecC32) {
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, lhaf_batch_kernel<float2>, 32 * W, smem);
  } else if (precision == kPrecDD) {
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, lhaf_batch_kernel<ddc>, 32 * W, smem);
  } else if (precision == kPrecTF) {
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, lhaf_batch_kernel<tfc>, 32 * W, smem);
  } else {
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, lhaf_batch_kernel<double2>, 32 * W, smem);
  }
  return per_sm < 1 ? 1 : per_sm;
}

static cudaError_t launch_batch_class(const BatchProblem* d_prob, int count, unsigned total_chunks,
                                      int k_lo, int k_hi, int area, int W, int precision,
                                      const DeviceInfo& dev, unsigned* d_counter,
                                      double* d_partials, cudaStream_t stream) {
  const int esz = prec_elem_bytes(precision);
  const size_t smem = (size_t)W * area * esz;
  unsigned blocks = (unsigned)(batch_blocks_per_sm(precision, W, smem) * dev.sm_count);
  const unsigned need = (total_chunks + W - 1) / W;
  if (blocks > need) blocks = need;
  if (precision == kPrecC32) {
    lhaf_batch_kernel<float2><<<blocks, 32 * W, smem, stream>>>(
        d_prob, count, total_chunks, k_lo, k_hi, area, d_counter, d_partials);
  } else if (precision == kPrecDD) {
    lhaf_batch_kernel<ddc><<<blocks, 32 * W, smem, stream>>>(
        d_prob, count, total_chunks, k_lo, k_hi, area, d_counter, d_partials);
  } else if (precision == kPrecTF) {
    lhaf_batch_kernel<tfc><<<blocks, 32 * W, smem, stream>>>(
        d_prob, count, total_chunks, k_lo, k_hi, area, d_counter, d_partials);
  } else {
    lhaf_batch_kernel<double2><<<blocks, 32 * W, smem, stream>>>(
        d_prob, count, total_chunks, k_lo, k_hi, area, d_counter, d_partials);
  }
  return cudaGetLastError();
}

int batch_classes(int n_max) { return n_max > kBatchSplitK ? 2 : 1; }

cudaError_t launch_batch(const BatchInput* d_in, const BatchProblem* d_prob, int count,
                         unsigned total_chunks, int n_max, int precision, int warps,
                         int warps_small, unsigned* d_counter, double* d_partials, double* d_out,
                         cudaStream_t stream, cudaStream_t side_stream) {
  if (count <= 0) return cudaSuccess;
  DeviceInfo dev;
  cudaError_t e = device_info(&dev);
  if (e != cudaSuccess) return e;
  expand_batch_kernel<<<count, 256, 0, stream>>>(d_in, d_prob, count);
  e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  const int nclass = batch_classes(n_max);
  e = cudaMemsetAsync(d_counter, 0, sizeof(unsigned) * 2, stream);
  if (e != cudaSuccess) return e;
  if (total_chunks > 0) {
    const int esz = prec_elem_bytes(precision);
    const int nm = n_max > 0 ? n_max : 1;
    if (nclass == 1) {
      e = launch_batch_class(d_prob, count, total_chunks, 1, nm, warp_area_elems(nm, nm, esz),
                             warps, precision, dev, d_counter, d_partials, stream);
    } else {
      // Class 0 (popcount <= kBatchSplitK, most subsets): small work areas, many warps.
      const int area0 = warp_area_elems(kBatchSplitK, nm, esz);
      int W0 = warps_small > 0 && warps_small < kMaxWarps ? warps_small : kMaxWarps;
      while (W0 > 1 && (size_t)W0 * area0 * esz > (size_t)dev.smem_optin) --W0;
      // Class 1 (larger popcounts) on a side stream, forked from and joined into `stream`.
      cudaStream_t sc = side_stream;
      if (!sc) {
        cudaStream_t* side = nullptr;
        e = side_streams(&side);
        if (e != cudaSuccess) return e;
        sc = side[1];
      }
      cudaEvent_t fork = nullptr, join = nullptr;
      e = cudaEventCreateWithFlags(&fork, cudaEventDisableTiming);
      if (e == cudaSuccess) e = cudaEventCreateWithFlags(&join, cudaEventDisableTiming);
      if (e == cudaSuccess) e = cudaEventRecord(fork, stream);
      if (e == cudaSuccess)
        e = launch_batch_class(d_prob, count, total_chunks, 1, kBatchSplitK, area0, W0,
                               precision, dev, d_counter, d_partials, stream);
      if (e == cudaSuccess) e = cudaStreamWaitEvent(sc, fork, 0);
      if (e == cudaSuccess)
        e = launch_batch_class(d_prob, count, total_chunks, kBatchSplitK + 1, nm,
                               warp_area_elems(nm, nm, esz), warps, precision, dev,
                               d_counter + 1, d_partials + (size_t)total_chunks * 5, sc);
      if (e == cudaSuccess) e = cudaEventRecord(join, sc);
      if (e == cudaSuccess) e = cudaStreamWaitEvent(stream, join, 0);
      if (fork) cudaEventDestroy(fork);
      if (join) cudaEventDestroy(join);
    }
    if (e != cudaSuccess) return e;
  }
  lhaf_batch_finalize_kernel<<<(count + 127) / 128, 128, 0, stream>>>(
      d_prob, count, d_partials, total_chunks, total_chunks > 0 ? nclass : 0, d_out);
  return cudaGetLastError();
}

}  // namespace gbsh
