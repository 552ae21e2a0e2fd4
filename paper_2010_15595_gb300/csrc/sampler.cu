// Chain-rule GBS sampler with continuous batching (declarations and contracts in
// include/gbsh.h).
//
// The algorithm of Sec. III for a pure state (steps 2-6): draw heterodyne outcomes
// alpha_2..alpha_m once from the Husimi distribution of modes 2..m (Eq. heterodyne); then
// for k = 1..m, compute the conditional probabilities of s_k = 0..d given s_1..s_{k-1} and
// alpha_{k+1..m} with Eq. lhaf-pure, draw s_k, and forget alpha_{k+1}.
//
// Conditional state. For a pure state whose Fock amplitudes are generated by
// exp(x^T B x / 2 + gamma^T x) (the form behind Eq. lhaf-pure), a heterodyne outcome
// alpha_B on modes B (projection onto the coherent state |alpha_B>) sets x_B = conj(alpha_B)
// and leaves modes A in the pure state with kernel B_AA and fill vector
// gamma_A + B_AB conj(alpha_B); this equals the state given by Eqs. condV/condR (checked
// against those equations in the tests). The conditional vacuum
// probability is common to all candidates s_k and cancels in the normalisation of step 5,
// so each step only needs loop hafnians: p(s_k) ~ |lhaf(filldiag(B_S, gamma^(k)_S))|^2 / s_k!.
//
// Serving: a worker thread owns the device state. Each "tick" advances every admitted
// chain by one mode: one kernel forms the fill vectors gamma^(k) of all chains, and one
// batched launch evaluates all (chain, s_k) loop hafnians together. Chains are admitted as
// slots and device memory allow, so requests that arrive while others are on the GPU join
// the next tick (continuous batching). With split evaluation on (tick_subsets), loop
// hafnians above that many subsets run instead as fixed subset ranges spread over ticks
// (like chunked prefill in LLM serving), so one chain's large loop hafnians do not set the
// pace of every other chain; such a chain advances when its last range is done. All
// randomness of a chain is drawn from a counter-based generator keyed by the request seed,
// and a loop hafnian's value does not depend on the batch or ticks it runs in, so a sample
// is the same alone and in any mix.
#include <algorithm>
#include <chrono>
#include <cmath>
#include <condition_variable>
#include <cstdint>
#include <cstring>
#include <deque>
#include <map>
#include <memory>
#include <mutex>
#include <thread>
#include <vector>

#include <cuda_runtime.h>

#include "../../include/gbsh.h"
#include "batch_host.h"
#include "lhaf_kernels.cuh"

namespace {

// ------------------------------------------------------------------ Philox4x32-10
// Counter-based generator of Salmon, Moraes, Dror and Shaw, "Parallel random numbers: as
// easy as 1, 2, 3" (SC'11): 10 rounds of
//   (c0, c1, c2, c3) <- (hi(M1 c2) ^ c1 ^ k0, lo(M1 c2), hi(M0 c0) ^ c3 ^ k1, lo(M0 c0))
// with M0 = 0xD2511F53, M1 = 0xCD9E8D57, the key advanced by (0x9E3779B9, 0xBB67AE85)
// between rounds.
void philox4x32_10(const uint32_t ctr_in[4], const uint32_t key_in[2], uint32_t out[4]) {
  uint32_t c0 = ctr_in[0], c1 = ctr_in[1], c2 = ctr_in[2], c3 = ctr_in[3];
  uint32_t k0 = key_in[0], k1 = key_in[1];
  for (int r = 0; r < 10; ++r) {
    const uint64_t p0 = (uint64_t)0xD2511F53u * c0;
    const uint64_t p1 = (uint64_t)0xCD9E8D57u * c2;
    const uint32_t n0 = (uint32_t)(p1 >> 32) ^ c1 ^ k0;
    const uint32_t n1 = (uint32_t)p1;
    const uint32_t n2 = (uint32_t)(p0 >> 32) ^ c3 ^ k1;
    const uint32_t n3 = (uint32_t)p0;
    c0 = n0; c1 = n1; c2 = n2; c3 = n3;
    k0 += 0x9E3779B9u;
    k1 += 0xBB67AE85u;
  }
  out[0] = c0; out[1] = c1; out[2] = c2; out[3] = c3;
}

// Uniform in [0, 1) from two 32-bit words: the top 53 bits of (hi:lo).
double u53(uint32_t hi, uint32_t lo) {
  const uint64_t x = ((uint64_t)hi << 32) | lo;
  return (double)(x >> 11) * 0x1.0p-53;
}

// Stream layout of one chain: key = request seed; counter = (chain number, stream, index, 0).
// Stream 2 draws the displacement of a mixed state's pure component (step 1).
constexpr uint32_t kStreamNormals = 0, kStreamUniforms = 1, kStreamMixture = 2;

void chain_words(uint64_t seed, uint32_t chain, uint32_t stream, uint32_t index, uint32_t out[4]) {
  const uint32_t key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)};
  const uint32_t ctr[4] = {chain, stream, index, 0u};
  philox4x32_10(ctr, key, out);
}

// `count2` standard normals of one stream by the Box-Muller transform, two per call.
void chain_normals(uint64_t seed, uint32_t chain, int count2, double* z,
                   uint32_t stream = kStreamNormals) {
  const double two_pi = 6.283185307179586476925286766559;
  for (int b = 0; 2 * b < count2; ++b) {
    uint32_t w[4];
    chain_words(seed, chain, stream, (uint32_t)b, w);
    const double u1 = u53(w[0], w[1]), u2 = u53(w[2], w[3]);
    const double r = std::sqrt(-2.0 * std::log(1.0 - u1));
    z[2 * b] = r * std::cos(two_pi * u2);
    if (2 * b + 1 < count2) z[2 * b + 1] = r * std::sin(two_pi * u2);
  }
}

double chain_uniform(uint64_t seed, uint32_t chain, uint32_t k) {
  uint32_t w[4];
  chain_words(seed, chain, kStreamUniforms, k, w);
  return u53(w[0], w[1]);
}

// ------------------------------------------------------------------ fill-vector kernel
// gam[c][i] = gbar_c[i] + sum_{j > k_c} B[i][j] conj(alpha_c[j]) for i <= k_c (one block per
// chain; alpha_c is the chain's heterodyne outcome vector, entry 0 unused; gbar_c is the
// fill vector of the chain's pure state, per slot).
__global__ void sampler_gamma_kernel(const double2* __restrict__ B, int ldb,
                                     const double2* __restrict__ gbar,
                                     const double2* __restrict__ alpha, const int* __restrict__ slot,
                                     const int* __restrict__ kk, int nchains, int M,
                                     double2* __restrict__ gam) {
  const int c = blockIdx.x;
  if (c >= nchains) return;
  const int k = kk[c];
  const double2* a = alpha + (size_t)slot[c] * M;
  const double2* gb = gbar + (size_t)slot[c] * M;
  double2* g = gam + (size_t)slot[c] * M;
  for (int i = threadIdx.x; i <= k; i += blockDim.x) {
    double re = 0.0, im = 0.0;
    for (int j = k + 1; j < M; ++j) {
      const double2 b = B[(size_t)i * ldb + j], x = a[j];  // b * conj(x)
      re = fma(b.x, x.x, fma(b.y, x.y, re));
      im = fma(b.y, x.x, fma(-b.x, x.y, im));
    }
    g[i] = make_double2(gb[i].x + re, gb[i].y + im);
  }
}

using Clock = std::chrono::steady_clock;

double seconds_since(Clock::time_point t0, Clock::time_point t) {
  return std::chrono::duration<double>(t - t0).count();
}

struct Request {
  uint64_t id = 0, seed = 0;
  int n_samples = 0, done = 0;
  bool cancelled = false;
  std::vector<int> samples;  // n_samples x M
  Clock::time_point t_submit, t_start, t_done;
  bool started = false, finished = false;
  int lhafs = 0, ticks = 0, truncated = 0;
};

// A loop hafnian evaluated in fixed subset ranges over several ticks; `acc` is the
// compensated partial (re_hi, re_lo, im_hi, im_lo, sum |p_Z|) of the ranges done so far.
struct SplitCand {
  int s = 0, N = 0;
  uint64_t next = 0, total = 0;
  double acc[5] = {0, 0, 0, 0, 0};
};

struct Chain {
  std::shared_ptr<Request> req;
  uint32_t chain_no = 0;
  int k = 0;          // next mode to sample
  int nphot = 0;      // photons in modes < k
  int slot = -1;
  std::vector<int> s;
  size_t mem = 0;
  // mode k's candidates while they are evaluated (split ones may take several ticks)
  bool open = false;
  bool trunc = false;
  int ncand = 0;
  std::vector<double> val;        // (re, im) of candidate s = 0..ncand-1
  std::vector<SplitCand> split;   // the split candidates, in increasing s
};

// Adds a range's compensated partial to an accumulated one (fixed order: ranges are added in
// increasing index order, so the result does not depend on the ticks they ran in).
void acc_add(double* acc, const double* p) {
  auto two_sum = [](double a, double b, double& sm, double& e) {
    sm = a + b;
    const double bb = sm - a;
    e = (a - (sm - bb)) + (b - bb);
  };
  double sm, e;
  two_sum(acc[0], p[0], sm, e);
  acc[0] = sm;
  acc[1] += e + p[1];
  two_sum(acc[2], p[2], sm, e);
  acc[2] = sm;
  acc[3] += e + p[3];
  acc[4] += p[4];
}

}  // namespace

struct gbsh_sampler {
  gbsh_sampler_cfg cfg{};
  std::vector<double2> B, gbar;
  std::vector<double> het_mean, het_chol;
  std::vector<double> mix_mean, mix_wf;  // mixed states: R-bar (2M), W factor (2M x 2M)
  std::vector<double2> fill_map;         // mixed states: M x 2M, fill vector = fill_map R
  int device = 0;
  // threading
  std::mutex mu;
  std::condition_variable cv_work, cv_done;
  bool stop = false;
  std::thread worker;
  int worker_error = GBSH_OK;
  uint64_t next_id = 1;
  std::map<uint64_t, std::shared_ptr<Request>> requests;
  std::deque<Chain> pending;
  Clock::time_point t0 = Clock::now();
  // device state (worker thread only)
  cudaStream_t st = nullptr;
  double2 *dB = nullptr, *dgbar = nullptr, *dalpha = nullptr, *dgam = nullptr;
  int *dslot = nullptr, *dk = nullptr, *didx = nullptr;
  size_t idx_cap = 0;
  void* ws = nullptr;
  size_t ws_bytes = 0;
  double* dpart = nullptr;  // range partials of one tick (5 doubles each)
  size_t part_cap = 0;
  std::vector<int> free_slots;

  void run();
  int tick(std::vector<Chain>& active);
  int ensure_ws(size_t bytes);
  int ensure_idx(size_t n);
  int ensure_part(size_t n);
  uint64_t split_size() const;
  size_t chain_mem_estimate(int nphot) const;
};

namespace {

int from_cuda(cudaError_t e) {
  return e == cudaSuccess ? GBSH_OK : (e == cudaErrorMemoryAllocation ? GBSH_ENOMEM : GBSH_ECUDA);
}

}  // namespace

size_t gbsh_sampler::chain_mem_estimate(int nphot) const {
  // device bytes of the next tick's candidates of a chain with nphot photons so far
  size_t total = 0;
  for (int s = 0; s <= cfg.cutoff; ++s) {
    const int N = nphot + s;
    if (N > cfg.n_cap) break;
    const int Ne = N + (N & 1), n = Ne / 2;
    const size_t chunks = n > 0 ? ((size_t)1 << n) / gbsh::batch_chunk_size(n) : 0;
    total += sizeof(double2) * ((size_t)Ne * Ne + Ne) + 2 * 40 * chunks + 128 + 4 * (size_t)N;
  }
  return total;
}

int gbsh_sampler::ensure_ws(size_t bytes) {
  if (bytes <= ws_bytes) return GBSH_OK;
  if (ws) cudaFree(ws);
  ws = nullptr;
  ws_bytes = 0;
  size_t want = std::max(bytes, (size_t)1 << 22);
  cudaError_t e = cudaMalloc(&ws, want);
  if (e != cudaSuccess) return from_cuda(e);
  ws_bytes = want;
  return GBSH_OK;
}

int gbsh_sampler::ensure_part(size_t n) {
  if (n <= part_cap) return GBSH_OK;
  if (dpart) cudaFree(dpart);
  dpart = nullptr;
  part_cap = 0;
  const size_t want = std::max(n, (size_t)64);
  cudaError_t e = cudaMalloc(&dpart, sizeof(double) * 5 * want);
  if (e != cudaSuccess) return from_cuda(e);
  part_cap = want;
  return GBSH_OK;
}

// Subset-range length of split evaluation (a power of two >= 64), 0 when disabled.
uint64_t gbsh_sampler::split_size() const {
  if (!cfg.batching || cfg.precision != GBSH_PREC_FP64 || cfg.tick_subsets == 0) return 0;
  uint64_t t = 64;
  while (t * 2 <= (uint64_t)cfg.tick_subsets && t < ((uint64_t)1 << 40)) t *= 2;
  return t;
}

int gbsh_sampler::ensure_idx(size_t n) {
  if (n <= idx_cap) return GBSH_OK;
  if (didx) cudaFree(didx);
  didx = nullptr;
  size_t want = std::max(n, (size_t)4096);
  cudaError_t e = cudaMalloc(&didx, sizeof(int) * want);
  if (e != cudaSuccess) return from_cuda(e);
  idx_cap = want;
  return GBSH_OK;
}

// Advances every chain in `active` whose candidates complete in this tick by one mode (with
// split evaluation off, every chain). Returns a status code.
int gbsh_sampler::tick(std::vector<Chain>& active) {
  const int M = cfg.M, d = cfg.cutoff;
  const int nch = (int)active.size();
  const uint64_t R = split_size();
  // fill vectors gamma^(k) of all chains (a chain whose mode is still open gets the same
  // vector again)
  std::vector<int> slots(nch), ks(nch);
  for (int c = 0; c < nch; ++c) {
    slots[c] = active[c].slot;
    ks[c] = active[c].k;
  }
  cudaError_t e = cudaMemcpyAsync(dslot, slots.data(), sizeof(int) * nch, cudaMemcpyHostToDevice, st);
  if (e != cudaSuccess) return from_cuda(e);
  e = cudaMemcpyAsync(dk, ks.data(), sizeof(int) * nch, cudaMemcpyHostToDevice, st);
  if (e != cudaSuccess) return from_cuda(e);
  sampler_gamma_kernel<<<nch, 128, 0, st>>>(dB, M, dgbar, dalpha, dslot, dk, nch, M, dgam);
  e = cudaGetLastError();
  if (e != cudaSuccess) return from_cuda(e);

  // Open the mode of every chain that has none open: candidates s_k = 0..d with their index
  // lists (mode i repeated s_i times). Candidates with more than R subsets are split; the
  // others go into this tick's batched launch. Index lists of split candidates are listed
  // again every tick while they have ranges left.
  struct Cand { int chain, s, N; size_t idx_off; };
  std::vector<Cand> cands;                   // batched
  std::vector<std::pair<int, int>> splits;   // (chain, split index) with ranges left
  std::vector<size_t> split_idx;             // their index-list offsets
  std::vector<int> idx;
  auto push_list = [&](const Chain& ch, int s) {
    const size_t off = idx.size();
    for (int i = 0; i < ch.k; ++i)
      for (int r = 0; r < ch.s[i]; ++r) idx.push_back(i);
    for (int r = 0; r < s; ++r) idx.push_back(ch.k);
    return off;
  };
  uint64_t batch_subsets = 0;
  for (int c = 0; c < nch; ++c) {
    Chain& ch = active[c];
    if (!ch.open) {
      ch.open = true;
      ch.trunc = false;
      ch.ncand = 0;
      ch.split.clear();
      for (int s = 0; s <= d; ++s) {
        const int N = ch.nphot + s;
        if (N > cfg.n_cap) {
          ch.trunc = true;
          break;
        }
        const int n = (N + (N & 1)) / 2;
        if (R > 0 && ((uint64_t)1 << n) > R) {
          SplitCand sc;
          sc.s = s;
          sc.N = N;
          sc.total = (uint64_t)1 << n;
          ch.split.push_back(sc);
        } else {
          cands.push_back(Cand{c, s, N, push_list(ch, s)});
          batch_subsets += (uint64_t)1 << n;
        }
        ch.ncand += 1;
      }
      ch.val.assign(2 * (size_t)ch.ncand, 0.0);
    }
    for (int j = 0; j < (int)ch.split.size(); ++j)
      if (ch.split[j].next < ch.split[j].total) {
        splits.emplace_back(c, j);
        split_idx.push_back(push_list(ch, ch.split[j].s));
      }
  }
  int rc = ensure_idx(idx.size() + 1);
  if (rc != GBSH_OK) return rc;
  if (!idx.empty()) {
    e = cudaMemcpyAsync(didx, idx.data(), sizeof(int) * idx.size(), cudaMemcpyHostToDevice, st);
    if (e != cudaSuccess) return from_cuda(e);
  }

  const int nc = (int)cands.size();
  std::vector<double> out3(3 * (size_t)nc);
  std::vector<int> Ns(nc);
  std::vector<gbsh::BatchInput> in(nc);
  for (int q = 0; q < nc; ++q) {
    Ns[q] = cands[q].N;
    in[q] = gbsh::BatchInput{dB, dgam + (size_t)active[cands[q].chain].slot * M,
                             didx + cands[q].idx_off, M, cands[q].N};
  }
  if (cfg.batching) {
    if (nc > 0) {
      gbsh::BatchLayout L = gbsh::batch_layout(Ns.data(), nc, 0);
      rc = ensure_ws(L.bytes);
      if (rc != GBSH_OK) return rc;
      e = gbsh::batch_run(L, in, nc, cfg.precision, 0, ws, st, out3.data());
      if (e != cudaSuccess) return from_cuda(e);
    }
  } else {
    // plain path: one single-evaluation launch sequence (expansion of B, the fill vector and
    // the pattern on the device, the popcount-class launches, finalize) and one
    // synchronisation per loop hafnian -- what a caller of gbsh_gbs_prob would do per
    // candidate. The complex-FP32 and double-double variants exist only in the batched
    // kernel, so for them each candidate is a one-problem batch instead.
    gbsh::DeviceInfo dev;
    e = gbsh::device_info(&dev);
    if (e != cudaSuccess) return from_cuda(e);
    e = gbsh::ensure_constants();
    if (e != cudaSuccess) return from_cuda(e);
    for (int q = 0; q < nc; ++q) {
      if (Ns[q] == 0) {
        out3[3 * (size_t)q] = 1.0;
        out3[3 * (size_t)q + 1] = 0.0;
        out3[3 * (size_t)q + 2] = 1.0;
        continue;
      }
      if (cfg.precision != GBSH_PREC_FP64) {
        gbsh::BatchLayout L = gbsh::batch_layout(&Ns[q], 1, 0);
        rc = ensure_ws(L.bytes);
        if (rc != GBSH_OK) return rc;
        std::vector<gbsh::BatchInput> one(1, in[q]);
        e = gbsh::batch_run(L, one, 1, cfg.precision, 0, ws, st, &out3[3 * (size_t)q]);
        if (e != cudaSuccess) return from_cuda(e);
        continue;
      }
      gbsh::LhafPlan plan;
      if (!gbsh::make_tuned_plan(Ns[q], dev, gbsh::kPrecFP64, &plan)) return GBSH_EINVAL;
      rc = ensure_ws(plan.bytes);
      if (rc != GBSH_OK) return rc;
      const gbsh::BatchInput& b = in[q];
      e = gbsh::launch_lhaf(plan, b.base, b.ld, b.diag, b.idx, ws, st);
      if (e == cudaSuccess)
        e = cudaMemcpyAsync(&out3[3 * (size_t)q], static_cast<char*>(ws) + plan.off_out,
                            3 * sizeof(double), cudaMemcpyDeviceToHost, st);
      if (e == cudaSuccess) e = cudaStreamSynchronize(st);
      if (e != cudaSuccess) return from_cuda(e);
    }
  }
  for (int q = 0; q < nc; ++q) {
    Chain& ch = active[cands[q].chain];
    ch.val[2 * (size_t)cands[q].s] = out3[3 * (size_t)q];
    ch.val[2 * (size_t)cands[q].s + 1] = out3[3 * (size_t)q + 1];
  }

  // Split candidates: ranges of R enumeration indices, oldest chains first, at most
  // max(R, batched subsets) subsets in this tick (at least one range) -- unless every active
  // chain is waiting for ranges, in which case nothing would advance sooner for the limit
  // and all ranges run.
  if (!splits.empty()) {
    gbsh::DeviceInfo dev;
    e = gbsh::device_info(&dev);
    if (e != cudaSuccess) return from_cuda(e);
    e = gbsh::ensure_constants();
    if (e != cudaSuccess) return from_cuda(e);
    std::vector<char> waits(nch, 0);
    for (const auto& sp : splits) waits[sp.first] = 1;
    const bool all_wait = std::all_of(waits.begin(), waits.end(), [](char w) { return w != 0; });
    const uint64_t budget = all_wait ? ~(uint64_t)0 : std::max<uint64_t>(R, batch_subsets);
    // choose the ranges first, so the workspace and the partial array are sized before the
    // first launch (neither may be reallocated under queued work)
    struct Ran { int chain, j; size_t q; uint64_t i0, i1; };
    std::vector<Ran> ran;
    std::vector<gbsh::LhafPlan> plans(splits.size());
    size_t ws_need = 0;
    uint64_t used = 0;
    for (size_t q = 0; q < splits.size() && used < budget; ++q) {
      const SplitCand& sc = active[splits[q].first].split[splits[q].second];
      if (!gbsh::make_tuned_plan(sc.N, dev, gbsh::kPrecFP64, &plans[q])) return GBSH_EINVAL;
      ws_need = std::max(ws_need, plans[q].bytes);
      for (uint64_t i0 = sc.next; i0 < sc.total && used < budget;) {
        const uint64_t i1 = std::min(i0 + R, sc.total);
        ran.push_back(Ran{splits[q].first, splits[q].second, q, i0, i1});
        used += i1 - i0;
        i0 = i1;
      }
    }
    rc = ensure_ws(ws_need);
    if (rc == GBSH_OK) rc = ensure_part(ran.size());
    if (rc != GBSH_OK) return rc;
    for (size_t r = 0; r < ran.size(); ++r) {
      const Ran& x = ran[r];
      const gbsh::LhafPlan& plan = plans[x.q];
      e = gbsh::launch_range(plan, dB, M, dgam + (size_t)active[x.chain].slot * M,
                             didx + split_idx[x.q], ws, st, x.i0, x.i1);
      if (e == cudaSuccess)
        e = cudaMemcpyAsync(dpart + 5 * r, static_cast<char*>(ws) + plan.off_out + 3 * sizeof(double),
                            5 * sizeof(double), cudaMemcpyDeviceToDevice, st);
      if (e != cudaSuccess) return from_cuda(e);
      active[x.chain].split[x.j].next = x.i1;
    }
    std::vector<double> parts(5 * ran.size());
    e = cudaMemcpyAsync(parts.data(), dpart, sizeof(double) * parts.size(), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return from_cuda(e);
    for (size_t r = 0; r < ran.size(); ++r) {  // launch order = index order per candidate
      Chain& ch = active[ran[r].chain];
      SplitCand& sc = ch.split[ran[r].j];
      acc_add(sc.acc, &parts[5 * r]);
      if (ran[r].i1 == sc.total) {  // its last range
        ch.val[2 * (size_t)sc.s] = sc.acc[0] + sc.acc[1];
        ch.val[2 * (size_t)sc.s + 1] = sc.acc[2] + sc.acc[3];
      }
    }
  }

  // step 5: every chain whose candidates are all done draws s_k from the normalised
  // weights |lhaf|^2 / s!
  std::vector<double> w((size_t)d + 1);
  for (int c = 0; c < nch; ++c) {
    Chain& ch = active[c];
    bool ready = ch.open;
    for (const SplitCand& sc : ch.split) ready = ready && sc.next == sc.total;
    if (!ready) continue;
    std::fill(w.begin(), w.end(), 0.0);
    double total = 0.0, fact = 1.0;
    for (int s = 0; s < ch.ncand; ++s) {
      if (s > 1) fact *= (double)s;
      const double re = ch.val[2 * (size_t)s], im = ch.val[2 * (size_t)s + 1];
      w[s] = (re * re + im * im) / fact;
      total += w[s];
    }
    const double u = chain_uniform(ch.req->seed, ch.chain_no, (uint32_t)ch.k);
    int sk = 0;
    if (total > 0.0) {
      double cum = 0.0;
      sk = ch.ncand - 1;
      for (int s = 0; s < ch.ncand; ++s) {
        cum += w[s] / total;
        if (cum > u) {
          sk = s;
          break;
        }
      }
    }
    ch.s[ch.k] = sk;
    ch.nphot += sk;
    ch.k += 1;
    ch.req->lhafs += ch.ncand;
    if (ch.trunc) ch.req->truncated += 1;
    ch.open = false;
  }
  return GBSH_OK;
}

void gbsh_sampler::run() {
  int rc = from_cuda(cudaSetDevice(device));
  std::vector<Chain> active;
  size_t mem_in_use = 0;  // estimate for the next tick of the admitted chains
  const int max_active = cfg.batching ? std::max(1, cfg.max_active) : 1;
  const int R = 2 * (cfg.M - 1);
  std::vector<double> z(R), quad(R), zmix, rdisp, hmean_stage;
  std::vector<double2> alpha_stage, gbar_stage;
  while (rc == GBSH_OK) {
    {
      std::unique_lock<std::mutex> lk(mu);
      // admission: by free slots and by the device-memory budget of the next tick
      size_t first_new = active.size();
      while (!pending.empty() && (int)active.size() < max_active) {
        const size_t need = chain_mem_estimate(0);
        if (!active.empty() && mem_in_use + need > cfg.mem_budget) break;
        Chain ch = std::move(pending.front());
        pending.pop_front();
        if (ch.req->cancelled) continue;
        if (!ch.req->started) {
          ch.req->started = true;
          ch.req->t_start = Clock::now();
        }
        ch.slot = free_slots.back();
        free_slots.pop_back();
        ch.mem = need;
        mem_in_use += need;
        active.push_back(std::move(ch));
      }
      if (active.empty()) {
        if (stop) break;
        cv_work.wait_for(lk, std::chrono::milliseconds(20));
        continue;
      }
      lk.unlock();
      // step 2 for the newly admitted chains: heterodyne outcomes of modes 2..M from the
      // Husimi distribution, staged and copied to their device slots
      for (size_t c = first_new; c < active.size(); ++c) {
        Chain& a = active[c];
        const double* hmean = het_mean.data();
        if (cfg.mixed) {
          // step 1: displacement of this sample's pure component, R ~ N(R-bar, W); its fill
          // vector fill_map R and Husimi means R restricted to modes 2..M
          const int R2 = 2 * cfg.M;
          zmix.resize(R2);
          rdisp.resize(R2);
          chain_normals(a.req->seed, a.chain_no, R2, zmix.data(), kStreamMixture);
          for (int r = 0; r < R2; ++r) {
            double acc = mix_mean[r];
            for (int q = 0; q < R2; ++q) acc += mix_wf[(size_t)r * R2 + q] * zmix[q];
            rdisp[r] = acc;
          }
          gbar_stage.assign(cfg.M, make_double2(0.0, 0.0));
          for (int i = 0; i < cfg.M; ++i) {
            double re = 0.0, im = 0.0;
            for (int q = 0; q < R2; ++q) {
              re += fill_map[(size_t)i * R2 + q].x * rdisp[q];
              im += fill_map[(size_t)i * R2 + q].y * rdisp[q];
            }
            gbar_stage[i] = make_double2(re, im);
          }
          hmean_stage.resize(R);
          for (int j = 1; j < cfg.M; ++j) {
            hmean_stage[j - 1] = rdisp[j];
            hmean_stage[(cfg.M - 1) + j - 1] = rdisp[cfg.M + j];
          }
          hmean = hmean_stage.data();
        } else {
          gbar_stage = gbar;
        }
        cudaError_t eg = cudaMemcpyAsync(dgbar + (size_t)a.slot * cfg.M, gbar_stage.data(),
                                         sizeof(double2) * cfg.M, cudaMemcpyHostToDevice, st);
        if (eg != cudaSuccess) {
          rc = from_cuda(eg);
          break;
        }
        chain_normals(a.req->seed, a.chain_no, R, z.data());
        for (int r = 0; r < R; ++r) {
          double acc = hmean[r];
          for (int q = 0; q <= r; ++q) acc += het_chol[(size_t)r * R + q] * z[q];
          quad[r] = acc;
        }
        alpha_stage.assign(cfg.M, make_double2(0.0, 0.0));
        for (int j = 1; j < cfg.M; ++j)  // alpha = (q + i p) / 2   (hbar = 2)
          alpha_stage[j] = make_double2(0.5 * quad[j - 1], 0.5 * quad[(cfg.M - 1) + j - 1]);
        cudaError_t e = cudaMemcpyAsync(dalpha + (size_t)a.slot * cfg.M, alpha_stage.data(),
                                        sizeof(double2) * cfg.M, cudaMemcpyHostToDevice, st);
        if (e != cudaSuccess) {
          rc = from_cuda(e);
          break;
        }
      }
      if (rc != GBSH_OK) break;
    }
    rc = tick(active);
    if (rc != GBSH_OK) break;
    // retire finished chains, refresh the memory estimate of the others
    std::lock_guard<std::mutex> lk(mu);
    std::vector<Chain> keep;
    keep.reserve(active.size());
    std::map<Request*, bool> ticked;
    mem_in_use = 0;
    for (auto& ch : active) {
      if (!ticked[ch.req.get()]) {
        ch.req->ticks += 1;
        ticked[ch.req.get()] = true;
      }
      if (ch.k >= cfg.M || ch.req->cancelled) {
        if (!ch.req->cancelled) {
          int* out = &ch.req->samples[(size_t)ch.chain_no * cfg.M];
          for (int i = 0; i < cfg.M; ++i)  // threshold detectors: click iff s_i > 0
            out[i] = cfg.threshold ? (ch.s[i] > 0 ? 1 : 0) : ch.s[i];
          ch.req->done += 1;
          if (ch.req->done == ch.req->n_samples) {
            ch.req->finished = true;
            ch.req->t_done = Clock::now();
            cv_done.notify_all();
          }
        }
        free_slots.push_back(ch.slot);
      } else {
        ch.mem = chain_mem_estimate(ch.nphot);
        mem_in_use += ch.mem;
        keep.push_back(std::move(ch));
      }
    }
    active.swap(keep);
  }
  std::lock_guard<std::mutex> lk(mu);
  if (rc != GBSH_OK) worker_error = rc;
  cv_done.notify_all();
}

extern "C" {

int gbsh_philox4x32(const uint32_t counter[4], const uint32_t key[2], uint32_t out[4]) {
  if (!counter || !key || !out) return GBSH_EINVAL;
  philox4x32_10(counter, key, out);
  return GBSH_OK;
}

int gbsh_sampler_create(const gbsh_sampler_cfg* cfg, gbsh_sampler** out) {
  if (!cfg || !out) return GBSH_EINVAL;
  const int M = cfg->M;
  if (M < 1 || !cfg->B || cfg->ldb < M || !cfg->gamma || cfg->cutoff < 0 || cfg->cutoff > 16 ||
      cfg->n_cap < 0 || cfg->n_cap > GBSH_MAX_N || cfg->max_active < 1 ||
      (M > 1 && !cfg->het_chol) || (M > 1 && !cfg->mixed && !cfg->het_mean) ||
      (cfg->mixed && (!cfg->mean || !cfg->w_factor || !cfg->fill_map)) ||
      (cfg->precision != GBSH_PREC_FP64 && cfg->precision != GBSH_PREC_C32))
    return GBSH_EINVAL;
  std::unique_ptr<gbsh_sampler> h(new gbsh_sampler());
  h->cfg = *cfg;
  h->device = cfg->device;
  h->B.resize((size_t)M * M);
  for (int i = 0; i < M; ++i)
    for (int j = 0; j < M; ++j) {
      const gbsh_c128 b = cfg->B[(size_t)i * cfg->ldb + j];
      h->B[(size_t)i * M + j] = make_double2(b.re, b.im);
    }
  h->gbar.resize(M);
  for (int i = 0; i < M; ++i) h->gbar[i] = make_double2(cfg->gamma[i].re, cfg->gamma[i].im);
  const int R = 2 * (M - 1);
  h->het_mean.assign(cfg->het_mean ? cfg->het_mean : nullptr,
                     cfg->het_mean ? cfg->het_mean + R : nullptr);
  h->het_chol.assign(cfg->het_chol ? cfg->het_chol : nullptr,
                     cfg->het_chol ? cfg->het_chol + (size_t)R * R : nullptr);
  if (cfg->mixed) {
    const int R2 = 2 * M;
    h->mix_mean.assign(cfg->mean, cfg->mean + R2);
    h->mix_wf.assign(cfg->w_factor, cfg->w_factor + (size_t)R2 * R2);
    h->fill_map.resize((size_t)M * R2);
    for (size_t i = 0; i < (size_t)M * R2; ++i)
      h->fill_map[i] = make_double2(cfg->fill_map[i].re, cfg->fill_map[i].im);
    h->het_mean.assign(R, 0.0);
  }
  h->cfg.B = nullptr;
  h->cfg.gamma = nullptr;
  h->cfg.het_mean = nullptr;
  h->cfg.het_chol = nullptr;
  h->cfg.mean = nullptr;
  h->cfg.w_factor = nullptr;
  h->cfg.fill_map = nullptr;
  const int slots = cfg->batching ? cfg->max_active : 1;
  h->free_slots.resize(slots);
  for (int i = 0; i < slots; ++i) h->free_slots[i] = slots - 1 - i;
  // device state
  int prev = 0;
  cudaError_t e = cudaGetDevice(&prev);
  if (e != cudaSuccess) return from_cuda(e);
  e = cudaSetDevice(h->device);
  if (e != cudaSuccess) return from_cuda(e);
  auto fail = [&](cudaError_t err) {
    cudaSetDevice(prev);
    return from_cuda(err);
  };
  if ((e = cudaStreamCreateWithFlags(&h->st, cudaStreamNonBlocking)) != cudaSuccess) return fail(e);
  if ((e = cudaMalloc(&h->dB, sizeof(double2) * M * M)) != cudaSuccess) return fail(e);
  if ((e = cudaMalloc(&h->dgbar, sizeof(double2) * (size_t)M * slots)) != cudaSuccess) return fail(e);
  if ((e = cudaMalloc(&h->dalpha, sizeof(double2) * (size_t)M * slots)) != cudaSuccess) return fail(e);
  if ((e = cudaMalloc(&h->dgam, sizeof(double2) * (size_t)M * slots)) != cudaSuccess) return fail(e);
  if ((e = cudaMalloc(&h->dslot, sizeof(int) * slots)) != cudaSuccess) return fail(e);
  if ((e = cudaMalloc(&h->dk, sizeof(int) * slots)) != cudaSuccess) return fail(e);
  if ((e = cudaMemcpy(h->dB, h->B.data(), sizeof(double2) * M * M, cudaMemcpyHostToDevice)) != cudaSuccess)
    return fail(e);
  cudaSetDevice(prev);
  gbsh_sampler* raw = h.release();
  raw->worker = std::thread([raw] { raw->run(); });
  *out = raw;
  return GBSH_OK;
}

int gbsh_sampler_submit(gbsh_sampler* h, uint64_t seed, int n_samples, uint64_t* req_id) {
  if (!h || !req_id || n_samples < 1) return GBSH_EINVAL;
  std::lock_guard<std::mutex> lk(h->mu);
  if (h->worker_error != GBSH_OK) return h->worker_error;
  auto r = std::make_shared<Request>();
  r->id = h->next_id++;
  r->seed = seed;
  r->n_samples = n_samples;
  r->samples.assign((size_t)n_samples * h->cfg.M, 0);
  r->t_submit = Clock::now();
  h->requests[r->id] = r;
  for (int c = 0; c < n_samples; ++c) {
    Chain ch;
    ch.req = r;
    ch.chain_no = (uint32_t)c;
    ch.s.assign(h->cfg.M, 0);
    h->pending.push_back(std::move(ch));
  }
  *req_id = r->id;
  h->cv_work.notify_one();
  return GBSH_OK;
}

static int fill_result(gbsh_sampler* h, Request& r, int* samples, gbsh_req_stats* stats) {
  if (samples) std::memcpy(samples, r.samples.data(), sizeof(int) * r.samples.size());
  if (stats) {
    stats->queue_s = seconds_since(r.t_submit, r.t_start);
    stats->run_s = seconds_since(r.t_start, r.t_done);
    stats->latency_s = seconds_since(r.t_submit, r.t_done);
    stats->submit_s = seconds_since(h->t0, r.t_submit);
    stats->lhafs = r.lhafs;
    stats->ticks = r.ticks;
    stats->truncated = r.truncated;
  }
  return GBSH_OK;
}

int gbsh_sampler_poll(gbsh_sampler* h, uint64_t req_id, int* samples, gbsh_req_stats* stats) {
  if (!h) return GBSH_EINVAL;
  std::lock_guard<std::mutex> lk(h->mu);
  auto it = h->requests.find(req_id);
  if (it == h->requests.end()) return GBSH_ENOTFOUND;
  if (!it->second->finished) return h->worker_error != GBSH_OK ? h->worker_error : GBSH_PENDING;
  fill_result(h, *it->second, samples, stats);
  h->requests.erase(it);
  return GBSH_OK;
}

int gbsh_sampler_wait(gbsh_sampler* h, uint64_t req_id, double timeout_s, int* samples,
                      gbsh_req_stats* stats) {
  if (!h || timeout_s < 0) return GBSH_EINVAL;
  std::unique_lock<std::mutex> lk(h->mu);
  auto deadline = Clock::now() + std::chrono::duration_cast<Clock::duration>(
                                     std::chrono::duration<double>(timeout_s));
  for (;;) {
    auto it = h->requests.find(req_id);
    if (it == h->requests.end()) return GBSH_ENOTFOUND;
    if (it->second->finished) {
      fill_result(h, *it->second, samples, stats);
      h->requests.erase(it);
      return GBSH_OK;
    }
    if (h->worker_error != GBSH_OK) return h->worker_error;
    if (h->cv_done.wait_until(lk, deadline) == std::cv_status::timeout) {
      auto it2 = h->requests.find(req_id);
      if (it2 != h->requests.end() && it2->second->finished) continue;
      return GBSH_ETIMEOUT;
    }
  }
}

int gbsh_sampler_cancel(gbsh_sampler* h, uint64_t req_id) {
  if (!h) return GBSH_EINVAL;
  std::lock_guard<std::mutex> lk(h->mu);
  auto it = h->requests.find(req_id);
  if (it == h->requests.end()) return GBSH_ENOTFOUND;
  it->second->cancelled = true;
  h->requests.erase(it);
  return GBSH_OK;
}

int gbsh_sampler_destroy(gbsh_sampler* h) {
  if (!h) return GBSH_EINVAL;
  {
    std::lock_guard<std::mutex> lk(h->mu);
    h->stop = true;
    for (auto& kv : h->requests) kv.second->cancelled = true;
    h->pending.clear();
  }
  h->cv_work.notify_all();
  if (h->worker.joinable()) h->worker.join();
  int prev = 0;
  cudaGetDevice(&prev);
  cudaSetDevice(h->device);
  if (h->st) cudaStreamSynchronize(h->st);
  cudaFree(h->dB);
  cudaFree(h->dgbar);
  cudaFree(h->dalpha);
  cudaFree(h->dgam);
  cudaFree(h->dslot);
  cudaFree(h->dk);
  cudaFree(h->didx);
  cudaFree(h->dpart);
  cudaFree(h->ws);
  if (h->st) cudaStreamDestroy(h->st);
  cudaSetDevice(prev);
  delete h;
  return GBSH_OK;
}

}  // extern "C"
