// Host helpers of the batched evaluation (see batch_host.h).
#include <algorithm>
#include <atomic>
#include <mutex>
#include <numeric>
#include <vector>

#include "batch_host.h"
#include "lhaf_kernels.cuh"
#include "tuning.h"

namespace gbsh {

namespace {
size_t align_up(size_t x) { return (x + 255) & ~(size_t)255; }

// ---- CUDA-graph replay of the device part of a batched evaluation.
// The device work of batch_run (expansion, the popcount-class launches, finalize) depends on
// its inputs only through the workspace contents, which are uploaded before it, and through
// the launch shape: the device addresses its kernels are given (tables, counters, partial
// sums, results; they move with the caller's staged bytes and the batch's size mix), problem
// count, chunk total, n_max, precision and warps per CTA. A shape seen a second time is
// captured once into a graph (on a private
// stream, with a private side stream for the second class) and replayed with
// cudaGraphLaunch from then on; graph and direct launches run the same kernels with the same
// arguments, so results are bit-identical.
struct GraphKey {
  int dev, count, n_max, precision, warps, warps_small;
  unsigned total_chunks;
  const char *in, *prob, *counter, *partials, *out;
  bool operator==(const GraphKey& o) const {
    return dev == o.dev && count == o.count && n_max == o.n_max && precision == o.precision &&
           warps == o.warps && warps_small == o.warps_small && total_chunks == o.total_chunks &&
           in == o.in && prob == o.prob && counter == o.counter && partials == o.partials &&
           out == o.out;
  }
};
struct GraphEntry {
  GraphKey key;
  cudaGraphExec_t exec;
  unsigned long long last_use;
};
constexpr size_t kMaxGraphs = 8;     // instantiated graphs kept (least recently used evicted)
constexpr size_t kMaxSeenKeys = 64;  // shapes seen once (captured on their second use)
std::mutex g_graph_mu;
std::vector<GraphEntry> g_graphs;
std::vector<GraphKey> g_seen;
unsigned long long g_clock = 0;
std::atomic<bool> g_graphs_enabled{true};
std::atomic<long long> g_captures{0}, g_replays{0};
cudaStream_t g_cap_stream[64] = {}, g_cap_side[64] = {};

// If an executable graph for `key` is cached, launches it on `st` while holding the cache
// lock (so that another thread's eviction cannot destroy it between lookup and launch) and
// returns true with the launch status in *e. Otherwise records the first sighting of the
// key, or sets *capture_now on its second one, and returns false.
bool graph_try_launch(const GraphKey& key, cudaStream_t st, bool* capture_now, cudaError_t* e) {
  std::lock_guard<std::mutex> lk(g_graph_mu);
  *capture_now = false;
  for (GraphEntry& g : g_graphs)
    if (g.key == key) {
      g.last_use = ++g_clock;
      *e = cudaGraphLaunch(g.exec, st);
      return true;
    }
  for (const GraphKey& k : g_seen)
    if (k == key) {
      *capture_now = true;
      return false;
    }
  if (g_seen.size() >= kMaxSeenKeys) g_seen.erase(g_seen.begin());
  g_seen.push_back(key);
  return false;
}

// Caches a newly captured graph (evicting the least recently used one; an evicted graph
// still in flight is freed by CUDA when it completes) and launches it under the lock.
cudaError_t graph_store_and_launch(const GraphKey& key, cudaGraphExec_t exec, cudaStream_t st) {
  std::lock_guard<std::mutex> lk(g_graph_mu);
  if (g_graphs.size() >= kMaxGraphs) {
    auto lru = std::min_element(g_graphs.begin(), g_graphs.end(),
                                [](const GraphEntry& a, const GraphEntry& b) {
                                  return a.last_use < b.last_use;
                                });
    cudaGraphExecDestroy(lru->exec);
    g_graphs.erase(lru);
  }
  g_graphs.push_back(GraphEntry{key, exec, ++g_clock});
  return cudaGraphLaunch(exec, st);
}

// Captures launch_batch for `key` into an executable graph (nullptr on any failure: the
// caller then launches directly).
cudaGraphExec_t graph_capture(const GraphKey& key, const BatchLayout& L, char* w, int count,
                              int precision, int W, int W0) {
  if (key.dev < 0 || key.dev >= 64) return nullptr;
  {
    std::lock_guard<std::mutex> lk(g_graph_mu);
    if (!g_cap_stream[key.dev]) {
      cudaStream_t a = nullptr, b = nullptr;
      if (cudaStreamCreateWithFlags(&a, cudaStreamNonBlocking) != cudaSuccess ||
          cudaStreamCreateWithFlags(&b, cudaStreamNonBlocking) != cudaSuccess) {
        if (a) cudaStreamDestroy(a);
        cudaGetLastError();
        return nullptr;
      }
      g_cap_side[key.dev] = b;
      g_cap_stream[key.dev] = a;
    }
  }
  cudaStream_t cs = g_cap_stream[key.dev];
  if (cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal) != cudaSuccess) {
    cudaGetLastError();  // e.g. another thread is capturing on this stream: launch directly
    return nullptr;
  }
  cudaError_t e = launch_batch(reinterpret_cast<const BatchInput*>(w + L.off_in),
                               reinterpret_cast<const BatchProblem*>(w + L.off_prob), count,
                               L.total_chunks, L.n_max, precision, W, W0,
                               reinterpret_cast<unsigned*>(w + L.off_counter),
                               reinterpret_cast<double*>(w + L.off_partials),
                               reinterpret_cast<double*>(w + L.off_out), cs, g_cap_side[key.dev]);
  cudaGraph_t graph = nullptr;
  cudaError_t e2 = cudaStreamEndCapture(cs, &graph);
  if (e != cudaSuccess || e2 != cudaSuccess || !graph) {
    if (graph) cudaGraphDestroy(graph);
    cudaGetLastError();
    return nullptr;
  }
  cudaGraphExec_t exec = nullptr;
  e = cudaGraphInstantiate(&exec, graph, 0);
  cudaGraphDestroy(graph);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return nullptr;
  }
  g_captures.fetch_add(1);
  return exec;
}
}  // namespace

void set_batch_graphs(bool enable) { g_graphs_enabled.store(enable); }
void batch_graph_stats(long long* captures, long long* replays) {
  if (captures) *captures = g_captures.load();
  if (replays) *replays = g_replays.load();
}

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
  L.off_partials = off; off = align_up(off + sizeof(double) * 5 * 2 * (size_t)L.total_chunks);
  L.off_counter = off; off = align_up(off + sizeof(unsigned) * 2);
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
  const BatchTuning bt = batch_tuning(precision, L.n_max);
  const int W = batch_warps_for(std::max(L.n_max, 1), precision, dev,
                                warps_pref > 0 ? warps_pref : bt.warps_large);
  if (W < 1) return cudaErrorInvalidValue;
  const int W0 = bt.warps_small;
  bool launched = false;
  if (g_graphs_enabled.load() && count > 0) {
    int d = 0;
    e = cudaGetDevice(&d);
    if (e != cudaSuccess) return e;
    const GraphKey key{d, count, L.n_max, precision, W, W0, L.total_chunks, w + L.off_in,
                       w + L.off_prob, w + L.off_counter, w + L.off_partials, w + L.off_out};
    bool capture_now = false;
    launched = graph_try_launch(key, st, &capture_now, &e);
    if (!launched && capture_now) {
      cudaGraphExec_t exec = graph_capture(key, L, w, count, precision, W, W0);
      if (exec) {
        e = graph_store_and_launch(key, exec, st);
        launched = true;
      }
    }
    if (launched && e == cudaSuccess) g_replays.fetch_add(1);
  }
  if (!launched) {
    e = launch_batch(reinterpret_cast<const BatchInput*>(w + L.off_in),
                     reinterpret_cast<const BatchProblem*>(w + L.off_prob), count, L.total_chunks,
                     L.n_max, precision, W, W0, reinterpret_cast<unsigned*>(w + L.off_counter),
                     reinterpret_cast<double*>(w + L.off_partials),
                     reinterpret_cast<double*>(w + L.off_out), st);
  }
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
