/*
 * gbsh.h — C ABI of the GB300 loop-hafnian engine for Gaussian boson sampling.
 *
 * The engine evaluates the loop hafnian lhaf(A) of a complex symmetric N x N matrix, the
 * quantity behind every pure-state GBS probability (Eq. lhaf-pure of Sec. II:
 * p(S) = p(vac) |lhaf(filldiag(B_S, gamma_S))|^2 / (s_1! ... s_m!)), by the signed sum over
 * the 2^{N/2} subsets of index pairs of the algorithm the paper cites for loop hafnians
 * (Sec. II, O(N^3 2^{N/2})) and benchmarks in Sec. IV. All arithmetic runs in CUDA kernels
 * for sm_103a; there is no CPU fallback.
 *
 * Conventions shared by every entry point
 *   - Complex numbers are gbsh_c128 {re, im}: the layout of C double _Complex, numpy
 *     complex128 and torch.complex128.
 *   - Matrices are row-major with a leading dimension (elements between rows) >= the
 *     number of columns. Symmetry is assumed, not checked: both triangles are read and
 *     should be equal. The diagonal holds the loop weights.
 *   - N = 0 gives lhaf = 1 (the empty matching). Odd N is allowed: the matrix is padded
 *     internally with one vertex of loop weight 1 and no edges, which leaves the loop
 *     hafnian unchanged. The largest supported N is GBSH_MAX_N.
 *   - `stream` is a cudaStream_t (NULL = the legacy default stream). Work is ordered on it.
 *   - Every function returns a status code (GBSH_OK = 0, never an exception). After
 *     GBSH_ECUDA, gbsh_strerror(code) names the last CUDA error of the calling thread.
 *   - Results are bit-reproducible for a given N on a given GPU model: the subset sum is
 *     split into fixed chunks whose compensated partial sums are combined in a fixed order.
 *   - Functions are re-entrant; calls on different streams may run concurrently. Host
 *     buffers are owned by the caller and only read/written during the call.
 */
#ifndef GBSH_H
#define GBSH_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct {
  double re, im;
} gbsh_c128;

#define GBSH_MAX_N 60

enum {
  GBSH_OK = 0,
  GBSH_EINVAL = 1,    /* bad argument: N out of range, null pointer, bad leading dimension */
  GBSH_ENOMEM = 2,    /* device memory could not be obtained / admission refused */
  GBSH_ECUDA = 3,     /* a CUDA call failed; see gbsh_strerror */
  GBSH_ETIMEOUT = 4,  /* a bounded device or host wait gave up */
  GBSH_PENDING = 5,   /* asynchronous request not finished yet */
  GBSH_ENOTFOUND = 6  /* unknown request id */
};

/* Human-readable text for a status code (for GBSH_ECUDA: the last CUDA error of this
 * thread). The string is static or thread-local; do not free it. */
const char* gbsh_strerror(int code);

/* Library version as MAJOR*10000 + MINOR*100 + PATCH. */
int gbsh_version(void);

/*
 * gbsh_lhaf — loop hafnian of one matrix (Sec. II, loop hafnian after Eq. lhaf; the
 * subset-sum algorithm the paper cites and benchmarks in Sec. IV).
 *   A        N x N matrix, leading dimension lda >= N; host OR device memory (the call
 *            detects which with cudaPointerGetAttributes; host memory is copied in).
 *            May be NULL only when N == 0.
 *   out      host pointer, receives lhaf(A).
 *   err_est  host pointer or NULL; receives an estimate of the relative rounding error:
 *            2^-53 * sum_Z (|Re p_Z| + |Im p_Z|) / |lhaf(A)|, i.e. unit roundoff times the
 *            cancellation ratio of the signed subset sum.
 *   stream   cudaStream_t. The call synchronises this stream before returning.
 * Scratch memory (partial sums) is taken from a per-device cache that the library grows
 * on demand with cudaMalloc and keeps until exit.
 * Errors: GBSH_EINVAL (N < 0, N > GBSH_MAX_N, lda < N, A/out NULL), GBSH_ENOMEM,
 * GBSH_ECUDA.
 */
int gbsh_lhaf(const gbsh_c128* A, int N, int lda, gbsh_c128* out, double* err_est,
              void* stream);

/* Bytes of device workspace gbsh_lhaf_async needs for size N (0 for N outside 1..MAX_N). */
size_t gbsh_lhaf_workspace_size(int N);
/* The same for gbsh_lhaf_async_ex in `precision` (0 for an unsupported precision). */
size_t gbsh_lhaf_workspace_size_ex(int N, int precision);

/*
 * gbsh_lhaf_async — gbsh_lhaf with everything on the device and no synchronisation.
 *   dA          device matrix, leading dimension lda >= N.
 *   d_out       device pointer to one gbsh_c128, receives lhaf(A).
 *   d_abs_sum   device pointer to one double or NULL; receives sum_Z |Re p_Z| + |Im p_Z|.
 *   workspace   device buffer of at least gbsh_lhaf_workspace_size(N) bytes, 256-byte
 *               aligned, owned by the caller; must not be used by another call that may
 *               run at the same time.
 * Streams: the popcount classes after the first run on side streams that the library
 * creates once per device; they are forked from `stream` and joined back into it with
 * events, so the whole evaluation is ordered after the work already queued on `stream` and
 * before the work queued on it afterwards, as if it ran on `stream` alone. Concurrent calls
 * from several threads share the side streams (correct, possibly serialised). The first
 * multi-class evaluation on a device creates them; make it before any stream capture.
 * N == 0 writes 1 to d_out. Errors: GBSH_EINVAL, GBSH_ECUDA (launch errors only; device
 * faults surface at the caller's next synchronisation).
 */
int gbsh_lhaf_async(const gbsh_c128* dA, int N, int lda, gbsh_c128* d_out, double* d_abs_sum,
                    void* workspace, size_t workspace_bytes, void* stream);

/*
 * gbsh_lhaf_ex, gbsh_lhaf_async_ex — gbsh_lhaf and gbsh_lhaf_async with the per-subset
 * arithmetic chosen by `precision`: GBSH_PREC_FP64 (what gbsh_lhaf and gbsh_lhaf_async
 * use) or GBSH_PREC_TF (triple-float, the accurate path; see GBSH_PREC_TF below). Every
 * other argument, the stream semantics and the errors are those of the plain entry points;
 * any other precision is GBSH_EINVAL. err_est uses the precision's unit roundoff (2^-53
 * for FP64, 2^-70 for triple-float). For gbsh_lhaf_async_ex the workspace must hold
 * gbsh_lhaf_workspace_size_ex(N, precision) bytes.
 */
int gbsh_lhaf_ex(const gbsh_c128* A, int N, int lda, int precision, gbsh_c128* out,
                 double* err_est, void* stream);
int gbsh_lhaf_async_ex(const gbsh_c128* dA, int N, int lda, int precision, gbsh_c128* d_out,
                       double* d_abs_sum, void* workspace, size_t workspace_bytes,
                       void* stream);

/* Per-subset arithmetic of the batched entry points. GBSH_PREC_FP64: complex FP64
 * throughout. GBSH_PREC_C32: each subset term in complex FP32 (the characteristic
 * polynomial, traces and exp-polynomial steps), the signed sum over subsets still
 * compensated in FP64; only for sizes where its measured error is acceptable. */
#define GBSH_PREC_FP64 0
#define GBSH_PREC_C32 1
/* GBSH_PREC_MIXED: complex FP32 per subset only for matrices with N <= GBSH_C32_MAX_N, where
 * its measured error against the FP64 path stays within 1e-5 relative (measured on the
 * batched GBS workload: max 5e-7 at N=2, 2.1e-6 at N=4, 2.3e-5 at N=6); FP64 otherwise. */
#define GBSH_PREC_MIXED 2
#define GBSH_C32_MAX_N 4
/* GBSH_PREC_DD: each subset term in double-double arithmetic (~106-bit significand): about
 * 25x the FP64 cost, for results whose FP64 rounding floor (unit roundoff times the
 * cancellation of the signed subset sum) is too coarse; the cross-subset sum is the same
 * compensated FP64 sum. */
#define GBSH_PREC_DD 3
/* GBSH_PREC_TF: each subset term in triple-float arithmetic -- every real number the
 * Hessenberg reduction, La Budde's recursion and the power series handle is the unevaluated
 * sum of three FP32 words (~72-bit significand), and each term reaches the compensated
 * cross-subset sum as an exact double-double. This is the path that meets the relative
 * tolerance the heavy cancellation of the signed subset sum demands at N >= 32 (the
 * accuracy concern of Sec. IV and Fig. 2): FP64 per subset leaves the N = 40 and N = 50
 * configuration matrices about 6e-8 and 1.5e-5 off, triple-float about 1e-13 and 1e-10 in
 * a CPU emulation of the same arithmetic. It runs on the FP32 pipe, which GB300 issues at
 * 64 times its FP64 rate. Accepted by the batched entry points and by the _ex
 * single-evaluation entry points below. Its words are FP32, so entries of the matrix, the
 * Hessenberg form and the polynomial coefficients must stay within about 2^-78 .. 2^127
 * in magnitude for full precision (every workload of the paper does by a wide margin). */
#define GBSH_PREC_TF 4

/*
 * gbsh_lhaf_batch — loop hafnians of `count` matrices of uneven size in one persistent
 * launch (same algorithm as gbsh_lhaf per matrix).
 *   A_packed  matrices, each Ns[p] x Ns[p] row-major (leading dimension Ns[p]) starting at
 *             element offsets[p]; host or device memory (detected; host data is copied in).
 *   offsets, Ns  host arrays of `count` entries; 0 <= Ns[p] <= GBSH_MAX_N.
 *   outs      host array of `count` gbsh_c128 (results in input order).
 *   abs_sums  host array of `count` doubles or NULL: sum_Z |Re p_Z| + |Im p_Z| per matrix.
 *   precision GBSH_PREC_FP64, GBSH_PREC_C32 (every matrix in FP32 per subset, at the
 *             caller's risk: use abs_sums to bound the error), GBSH_PREC_MIXED or
 *             GBSH_PREC_DD.
 * Each matrix's subsets are split into chunks whose size depends only on its own N, so a
 * matrix's result is bit-identical alone (count = 1) and inside any batch. Problems are
 * ordered largest first (longest-processing-time order) for the persistent launch.
 * Synchronises `stream`. Errors: GBSH_EINVAL, GBSH_ENOMEM, GBSH_ECUDA.
 */
int gbsh_lhaf_batch(const gbsh_c128* A_packed, const int64_t* offsets, const int* Ns, int count,
                    gbsh_c128* outs, double* abs_sums, int precision, void* stream);

/*
 * gbsh_gbs_prob_batch — Eq. lhaf-pure for `count` photon patterns of one kernel matrix B
 * (Sec. II): p = p_vac[p] |lhaf(filldiag(B_S, gamma_S))|^2 / prod_i s_i!.
 *   B         M x M (leading dimension ldb), host or device memory.
 *   gammas    fill vectors, same memory kind as B: problem p uses gammas + p*gamma_stride
 *             (gamma_stride = 0: one shared vector).
 *   patterns  host array count x M of photon numbers (row p = pattern of problem p).
 *   p_vacs    host array of `count` vacuum probabilities, or NULL for 1.
 *   probs     host array of `count` probabilities; lhafs: host array or NULL.
 * Synchronises `stream`. Errors: GBSH_EINVAL (bad sizes, negative counts, N > GBSH_MAX_N),
 * GBSH_ENOMEM, GBSH_ECUDA.
 */
int gbsh_gbs_prob_batch(const gbsh_c128* B, int M, int ldb, const gbsh_c128* gammas,
                        int64_t gamma_stride, const int* patterns, int count,
                        const double* p_vacs, double* probs, gbsh_c128* lhafs, int precision,
                        void* stream);

/* Warps per CTA of the large-popcount class of the batched kernel for batches whose largest
 * matrix has n_max pairs (N = 2 n_max), per precision (0 = the tuning table's value); the
 * small-popcount class keeps its setting. Results do not depend on it. GBSH_OK or
 * GBSH_EINVAL (precision GBSH_PREC_MIXED, n_max outside 0..30, warps outside 0..16). */
int gbsh_set_batch_tuning(int precision, int n_max, int warps_per_cta);

/*
 * Launch-shape tuning table. The library's default launch shapes come from a built-in table
 * that the autotuner (autotune.py) measured on a GB300; these calls override or read its
 * entries for this process. A launch shape never changes which subsets are summed:
 *
 * gbsh_set_batch_tuning_ex — batched kernel, batches whose largest matrix has n_max pairs:
 *   warps per CTA of the small-popcount class (popcounts <= 10) and of the large-popcount
 *   class (1..16; 0 in both restores the built-in entry, 0 in one selects the library
 *   default for that class). Results are bit-identical under any setting.
 * gbsh_set_lhaf_tuning_ex — single evaluations (gbsh_lhaf*, gbsh_gbs_prob, the range and
 *   no-allocation entries) of size N in precision GBSH_PREC_FP64 or GBSH_PREC_TF:
 *   warps_cap  most warps per CTA of any popcount class (1..16; 0 = 12 FP64, 16 TF)
 *   ladder     1 coarse {16,12,8,6,4,3,2,1} or 2 fine {16,14,12,10,8,7,6,5,4,3,2,1}: the
 *              warps-per-CTA steps by which popcounts are assigned to classes (0 = coarse)
 *   log2_chunks  enumeration chunks of one evaluation, 2^log2_chunks capped at 2^(N/2)
 *              (1..18; 0 = 18)
 *   All three 0 restores the built-in entry. The ladder and chunk count regroup the
 *   compensated cross-subset sum, so results agree with other settings to its rounding and
 *   are bit-reproducible under any one setting. gbsh_set_lhaf_tuning's process-wide
 *   override, while set, takes precedence over this table. Ranks that split one evaluation
 *   with gbsh_lhaf_range_async must use the same entry.
 * gbsh_get_lhaf_tuning / gbsh_get_batch_tuning — the current entry (0 = library default).
 * gbsh_builtin_tuning_entries — number of measured entries in the built-in table.
 * All return GBSH_OK or GBSH_EINVAL (arguments outside the ranges above); output pointers may
 * be NULL.
 */
int gbsh_set_batch_tuning_ex(int precision, int n_max, int warps_small, int warps_large);
int gbsh_set_lhaf_tuning_ex(int precision, int N, int warps_cap, int ladder, int log2_chunks);
int gbsh_get_lhaf_tuning(int precision, int N, int* warps_cap, int* ladder, int* log2_chunks);
int gbsh_get_batch_tuning(int precision, int n_max, int* warps_small, int* warps_large);
int gbsh_builtin_tuning_entries(void);

/* CUDA-graph replay of the batched evaluations (gbsh_lhaf_batch, gbsh_gbs_prob_batch and the
 * sampler's ticks). The device work of one batched evaluation -- expansion, the persistent
 * popcount-class launches, the finalize -- is captured into a CUDA graph the second time the
 * same launch shape is seen (same device, workspace layout and addresses, problem count,
 * chunk total, largest size, precision and warps per CTA) and replayed with one graph launch
 * from then on; the
 * per-call tables are uploaded before the launch. Results are bit-identical to direct
 * launches. enable = 1 (the default) or 0. Returns GBSH_OK. */
int gbsh_set_batch_graphs(int enable);
/* Process-wide counts of graphs captured and of graph launches by the batched path. */
int gbsh_batch_graph_stats(long long* captures, long long* replays);

/*
 * gbsh_gbs_prob — pure-state GBS probability, Eq. lhaf-pure (Sec. II):
 *   p(S) = p_vac * |lhaf(filldiag(B_S, gamma_S))|^2 / prod_i s_i!
 * where B_S repeats row and column i of B s_i times (modes in ascending order) and
 * gamma_S repeats gamma_i s_i times (Sec. II after Eq. GBS-pure).
 *   B        M x M kernel matrix (A = B (+) B* of the pure state), leading dimension ldb,
 *            host or device memory.
 *   gamma    M fill-vector entries, host or device memory (same kind as B).
 *   pattern  host array of M photon numbers s_i >= 0 (pattern[i] belongs to mode i).
 *   p_vac    vacuum probability of the state (Sec. II).
 *   prob     host pointer, receives p(S).
 *   lhaf_out host pointer or NULL, receives the loop hafnian itself.
 * Errors: GBSH_EINVAL (M < 1, ldb < M, negative s_i, sum s_i > GBSH_MAX_N, NULL pointers),
 * GBSH_ENOMEM, GBSH_ECUDA. Synchronises `stream`.
 */
int gbsh_gbs_prob(const gbsh_c128* B, int M, int ldb, const gbsh_c128* gamma,
                  const int* pattern, double p_vac, double* prob, gbsh_c128* lhaf_out,
                  void* stream);

/*
 * gbsh_lhaf_range_async — the part of the subset sum (Sec. II after Eq. lhaf-pure: the
 * signed sum over the 2^n subsets Z of index pairs) that comes from the subsets
 * z = i XOR (i >> 1) for enumeration indices i in [i_begin, i_end), n = ceil(N/2). Any
 * partition of [0, 2^n) into ranges covers every subset exactly once, so ranges can be
 * evaluated separately -- on different GPUs, in different processes -- and combined with
 * gbsh_combine_partials: the only exchange a split of one loop hafnian needs.
 *   dA, N, lda, precision, workspace, stream: as for gbsh_lhaf_async_ex (the workspace must
 *               hold gbsh_lhaf_workspace_size_ex(N, precision) bytes).
 *   d_partial   device array of 5 doubles, receives the range's compensated partial
 *               (re_hi, re_lo, im_hi, im_lo, sum |Re p_Z| + |Im p_Z|): the sum over the
 *               range is (re_hi + re_lo) + i (im_hi + im_lo).
 * The range is cut into chunks of the size gbsh_lhaf uses for N, starting at i_begin.
 * No synchronisation. Errors: GBSH_EINVAL (sizes, i_begin > i_end, i_end > 2^n, null
 * pointers, unsupported precision), GBSH_ECUDA.
 */
int gbsh_lhaf_range_async(const gbsh_c128* dA, int N, int lda, int precision, uint64_t i_begin,
                          uint64_t i_end, double* d_partial, void* workspace,
                          size_t workspace_bytes, void* stream);

/*
 * gbsh_combine_partials — host-side sum of `count` range partials (host array, count x 5
 * doubles as written by gbsh_lhaf_range_async) into out[5], compensated (TwoSum on the high
 * words, low words added), in the given order. Host code only: no device, no allocation.
 */
int gbsh_combine_partials(const double* partials, int count, double* out);

/*
 * gbsh_subset_terms — diagnostic: the individual subset terms p_Z (before the sign
 * (-1)^{n-|Z|}) of the subset sum for the listed subsets z of the pairs (j, j+n) of A
 * padded to even size Ne = N + (N odd), n = Ne/2; bit j of z <=> pair j in Z.
 *   dA   device N x N matrix (lda >= N); d_z device array of `count` subsets (< 2^n);
 *   d_out device array of `count` gbsh_c128. Synchronises `stream`.
 */
int gbsh_subset_terms(const gbsh_c128* dA, int N, int lda, const uint64_t* d_z, int count,
                      gbsh_c128* d_out, void* stream);
/* The same with the per-subset arithmetic of `precision` (GBSH_PREC_FP64 or GBSH_PREC_TF);
 * triple-float terms are rounded to the nearest complex double on output. */
int gbsh_subset_terms_ex(const gbsh_c128* dA, int N, int lda, int precision, const uint64_t* d_z,
                         int count, gbsh_c128* d_out, void* stream);

/*
 * gbsh_visit_counts — diagnostic: runs the subset enumeration of gbsh_lhaf for size N
 * (N <= 40) and adds 1 to d_counts[z] for every subset z it evaluates (z = 0 is skipped,
 * its term is zero). d_counts: device array of 2^n unsigned ints, zeroed by the caller.
 * A correct enumeration leaves every entry but [0] equal to 1. Synchronises `stream`.
 */
int gbsh_visit_counts(int N, unsigned* d_counts, void* stream);

/*
 * gbsh_set_lhaf_tuning — process-wide launch-shape override of the subset kernel for
 * subsequent single evaluations of every size and precision: a cap on warps per CTA (1..16)
 * and a cap on the popcount handled by the first (many-warp) class (0 = largest that fits in
 * shared memory); subsets above it run in further launches with fewer warps and larger work
 * areas. While either value is nonzero it replaces the tuning table (gbsh_set_lhaf_tuning_ex)
 * with the coarse ladder and 2^18 chunks; (0, 0) returns to the table. The warps cap does not
 * change results; the popcount cap regroups the cross-subset sum (agreement to its rounding).
 */
int gbsh_set_lhaf_tuning(int warps_per_cta, int kcap);

/*
 * gbsh_lhaf_plan — launch plan that gbsh_lhaf / gbsh_lhaf_async use for size N on the
 * current device, under the current tuning. Any output pointer may be NULL.
 *   nclass     number of subset-kernel launches (popcount classes, 1..12)
 *   kernels    CUDA kernels launched per evaluation (expansion + classes + two-level finalize)
 *   warps      warps per CTA of the first class
 *   kcap       largest popcount of the first class
 *   nchunks    number of fixed subset chunks (with the popcount classes, it fixes the
 *              reduction order)
 * Errors: GBSH_EINVAL for N outside 1..GBSH_MAX_N, GBSH_ECUDA without a device.
 */
int gbsh_lhaf_plan(int N, int* nclass, int* kernels, int* warps, int* kcap, int* nchunks);
/* The same for the plan of `precision` (GBSH_PREC_FP64 or GBSH_PREC_TF). */
int gbsh_lhaf_plan_ex(int N, int precision, int* nclass, int* kernels, int* warps, int* kcap,
                      int* nchunks);

/* ---------------------------------------------------------------- chain-rule sampler
 * The sampling algorithm of Sec. III (steps 2-6) for a pure Gaussian state, served with
 * continuous batching. State: kernel matrix B and fill vector gamma of Eq. lhaf-pure, and
 * the Husimi (heterodyne) distribution of modes 2..M (Eq. heterodyne): mean and lower
 * Cholesky factor of V_Q restricted to those modes, in quadrature order
 * (q_2..q_M, p_2..p_M), hbar = 2 (alpha = (q + i p) / 2).
 * Each request draws n_samples independent samples; each sample's randomness comes from
 * Philox4x32-10 keyed by the request seed (counter = (sample index, stream, index, 0)),
 * so results do not depend on what else is being served.
 * Step k conditions on alpha_{k+1..M} through the fill vector gamma_A + B_AB conj(alpha_B)
 * (equal to Eqs. condV/condR for pure states) and draws s_k from
 * |lhaf(filldiag(B_S, gamma_S))|^2 / s_k! over s_k = 0..cutoff. A candidate whose loop
 * hafnian would exceed n_cap photons is dropped (probability 0) and counted in `truncated`.
 */
typedef struct gbsh_sampler gbsh_sampler;

typedef struct {
  int M;                    /* modes */
  const gbsh_c128* B;       /* M x M host, leading dimension ldb (copied at create) */
  int ldb;
  const gbsh_c128* gamma;   /* M host fill vector of the full state (copied) */
  const double* het_mean;   /* 2(M-1) host: Husimi means of (q_2..q_M, p_2..p_M) */
  const double* het_chol;   /* 2(M-1) x 2(M-1) host, row-major lower Cholesky factor of V_Q */
  int cutoff;               /* Fock cutoff d per mode (0..16) */
  int n_cap;                /* largest loop hafnian size evaluated (<= GBSH_MAX_N) */
  int max_active;           /* samples in flight (device slots); 1 with batching = 0 */
  size_t mem_budget;        /* device bytes admitted samples may use (admission control) */
  int batching;             /* 1: continuous batching, one launch per tick for all samples;
                               0: plain path, one single-evaluation launch sequence and one
                                  synchronisation per loop hafnian (a one-problem batch for
                                  GBSH_PREC_C32), one sample at a time */
  int precision;            /* GBSH_PREC_FP64 or GBSH_PREC_C32 */
  int device;               /* CUDA device the sampler's worker thread uses */
  int threshold;            /* 1: report threshold-detector clicks (s_i > 0 -> 1), the
                               post-processing of the end of Sec. III; 0: photon numbers */
  /* Mixed states (step 1 of Sec. III, Eqs. split/decomp/mnpdf): with mixed = 1, B and
   * het_chol describe the pure part T of the Williamson split V = T + W, and every sample
   * first draws its displacement R = mean + w_factor xi (xi standard normal), which sets
   * its fill vector gamma = fill_map R and its Husimi means (R restricted to modes 2..M).
   * gamma and het_mean are then ignored. */
  int mixed;
  const double* mean;           /* 2M host: quadrature means R-bar */
  const double* w_factor;       /* 2M x 2M host row-major: W = w_factor w_factor^T */
  const gbsh_c128* fill_map;    /* M x 2M host row-major complex */
  /* Split evaluation (batching = 1, GBSH_PREC_FP64): 0 evaluates every loop hafnian of a
   * tick in the tick's batched launch. T > 0 (rounded down to a power of two, at least
   * 64) evaluates a loop hafnian with more than T pair subsets in fixed ranges of T
   * enumeration indices, spread over ticks: each tick runs at most max(T, the subsets of
   * its batched launch) subsets of such ranges, oldest chains first (all of them when every
   * active chain is waiting for ranges), and a chain draws its next photon number once all
   * its candidates are done. This bounds the time of a tick,
   * so chains with small loop hafnians are not held up by ones with large ones. The
   * ranges depend only on the size and T, so samples stay the same alone and in any mix. */
  size_t tick_subsets;
} gbsh_sampler_cfg;

typedef struct {
  double submit_s;   /* submission time since sampler creation */
  double queue_s;    /* submission to first admission */
  double run_s;      /* first admission to completion */
  double latency_s;  /* submission to completion */
  int lhafs;         /* loop hafnians evaluated for this request */
  int ticks;         /* serving ticks the request took part in */
  int truncated;     /* steps where a candidate exceeded n_cap */
} gbsh_req_stats;

/* Creates a sampler and starts its worker thread. Errors: GBSH_EINVAL, GBSH_ENOMEM,
 * GBSH_ECUDA. */
int gbsh_sampler_create(const gbsh_sampler_cfg* cfg, gbsh_sampler** out);
/* Queues a request for n_samples samples; returns its id. Thread-safe. */
int gbsh_sampler_submit(gbsh_sampler* h, uint64_t seed, int n_samples, uint64_t* req_id);
/* GBSH_PENDING until done; then copies n_samples x M photon numbers into `samples` (host,
 * may be NULL) and the stats, and forgets the request. GBSH_ENOTFOUND for unknown ids. */
int gbsh_sampler_poll(gbsh_sampler* h, uint64_t req_id, int* samples, gbsh_req_stats* stats);
/* Like poll, but waits at most timeout_s seconds (GBSH_ETIMEOUT after that). */
int gbsh_sampler_wait(gbsh_sampler* h, uint64_t req_id, double timeout_s, int* samples,
                      gbsh_req_stats* stats);
/* Drops a request (its chains retire at the next tick). */
int gbsh_sampler_cancel(gbsh_sampler* h, uint64_t req_id);
/* Stops the worker (cancelling outstanding requests) and frees the device state. */
int gbsh_sampler_destroy(gbsh_sampler* h);
/* Philox4x32-10 (Salmon et al., SC'11) of the sampler, exposed for verification. */
int gbsh_philox4x32(const uint32_t counter[4], const uint32_t key[2], uint32_t out[4]);

/*
 * gbsh_lhaf_noalloc — gbsh_lhaf_async for callers that cannot allocate device memory.
 * The paper has no counterpart; this is an engineering entry point.
 *
 * Who needs it: code that must not call cudaMalloc/cudaFree -- for example a plugin or
 * hook running inside another framework whose caching allocator owns the device memory
 * and forbids driver allocations, or a latency-critical loop that cannot afford the
 * implicit device synchronisation of an allocation. The caller still passes the input and
 * output buffers; the scratch (expanded matrix, chunk partial sums, chunk counters) comes
 * from a fixed array compiled into this library, GBSH_NOALLOC_SCRATCH_BYTES bytes, which
 * every GPU that loads the library holds until the process exits. No cudaMalloc, cudaFree
 * or allocating library routine is called.
 *   dA          device matrix, leading dimension lda >= N (device memory only).
 *   d_out       device pointer to one gbsh_c128, receives lhaf(A).
 *   d_abs_sum   device pointer to one double or NULL; receives sum_Z |Re p_Z| + |Im p_Z|.
 *   stream      cudaStream_t; no synchronisation.
 * Set-up: the first call on a device looks up the device address of the fixed array
 * (cudaGetSymbolAddress, with that device current) and caches it; make that first call
 * before any stream capture.
 * Sharing: all calls share the one array, which keeps the last call's contents (the call
 * clears what must start at zero). Calls whose GPU work may overlap -- on different
 * streams, or from different threads without ordering -- race on it; serialise them.
 * The launch plan is the tuning table's entry for N (gbsh_set_lhaf_tuning's process-wide
 * override does not apply), except
 * that for large N the number of subset chunks is halved until the chunk partial sums fit
 * the array; the result then agrees with gbsh_lhaf's to rounding, not bit for bit.
 * Errors: GBSH_EINVAL (N < 0, N > GBSH_MAX_N, lda < N, NULL pointers); GBSH_ENOMEM if an
 * evaluation would need more than GBSH_NOALLOC_SCRATCH_BYTES of scratch; GBSH_ECUDA.
 */
#define GBSH_NOALLOC_SCRATCH_BYTES (8u << 20)
int gbsh_lhaf_noalloc(const gbsh_c128* dA, int N, int lda, gbsh_c128* d_out, double* d_abs_sum,
                      void* stream);
/* Diagnostic: the number of subset chunks gbsh_lhaf_noalloc would use for size N on the
 * current device (the default plan's count, or fewer where that plan's scratch would not
 * fit the fixed array), or GBSH_ENOMEM when no chunking fits. Runs no kernel and touches
 * no device memory. Errors: GBSH_EINVAL for N outside 1..GBSH_MAX_N, GBSH_ECUDA. */
int gbsh_lhaf_noalloc_plan(int N, int* nchunks);

#ifdef __cplusplus
}
#endif

#endif /* GBSH_H */
