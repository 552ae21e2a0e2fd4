// Types shared by the host launch code and the device kernels of the loop-hafnian engine.
#pragma once

#include <cuda_runtime.h>

namespace gbsh {

constexpr int kMaxN = 60;  // n = N/2 <= 30 so that the n+2 series coefficients fit a warp

// One loop-hafnian problem as the kernels see it: the padded even-size matrix with zero
// diagonal (row-major, leading dimension Ne) and its loop weights.
struct Problem {
  const double2* A0;   // Ne x Ne, zero diagonal
  const double2* v;    // Ne loop weights
  int Ne;              // even size (N or N+1)
  int n;               // Ne / 2
};

// One problem of a batched evaluation, after expansion (device table entry).
struct BatchProblem {
  const double2* A0;        // Ne x Ne, zero diagonal (in the batch workspace)
  const double2* v;         // Ne loop weights
  int Ne, n;
  unsigned chunk_base;      // first global chunk of this problem
  unsigned nchunks;         // chunks of this problem (2^n / chunk_size)
  unsigned long long chunk_size;
};

// Where a batched problem's matrix comes from: A[r][c] = base[idx[r]][idx[c]] (r != c),
// A[r][r] = diag ? diag[idx[r]] : base[idx[r]][idx[r]]; idx == nullptr means identity.
struct BatchInput {
  const double2* base;
  const double2* diag;
  const int* idx;
  int ld;
  int N;
};

// Per-subset arithmetic of an evaluation: complex FP64, or complex FP32 per subset with
// the cross-subset sum still compensated in FP64.
constexpr int kPrecFP64 = 0;
constexpr int kPrecC32 = 1;
constexpr int kPrecDD = 3;  // double-double per subset (value 2 is the API's mixed mode)
constexpr int kPrecTF = 4;  // triple-float per subset (three FP32 words, ~72-bit significand)
constexpr int kNumPrec = 5;

// Bytes of one complex element of the per-subset arithmetic of a precision.
__host__ __device__ inline int prec_elem_bytes(int precision) {
  return precision == kPrecC32 ? 8 : (precision == kPrecDD ? 32 : (precision == kPrecTF ? 24 : 16));
}

// Chunk size of a batched problem with n pairs: a function of n alone (so a problem's
// result does not depend on its batch), one subset up to n = 10 and 2^(n-10) above, i.e. at
// most 1024 chunks per problem. A small batch (a serving tick with a few candidates) then
// spreads each problem over many warps instead of running 64 subsets one after another in
// one warp; a large batch has chunks enough either way.
__host__ __device__ inline unsigned long long batch_chunk_size(int n) {
  return n > 10 ? (1ull << (n - 10)) : 1ull;
}

// La Budde accumulators P_0..P_t are stored packed: P_u has degree <= u and is kept up to
// degree D, i.e. min(u, D) + 1 coefficients. Offset of P_t in that packed array.
__host__ __device__ __forceinline__ int poly_offset(int t, int D) {
  return t <= D + 1 ? t * (t + 1) / 2 : (D + 1) * (D + 2) / 2 + (t - D - 1) * (D + 1);
}

// Shared-memory footprint, in elements of `elem_bytes` bytes (16 for the complex FP64
// path, 8 for the complex FP32 variant), of one warp's work area for subsets with
// m = 2k <= 2*kmax and series degree D = n+1: the bordered matrix (S x S, S = m+1 is odd
// so the row stride is conflict-free for column access), the packed accumulators
// P_0..P_S and the subset's index list of S ints.
__host__ __device__ inline int warp_area_elems(int kmax, int n, int elem_bytes = 16) {
  int S = 2 * kmax + 1;
  int ldh = S | 1;
  int D = n + 1;
  int idx_units = (S * 4 + elem_bytes - 1) / elem_bytes;  // S ints, rounded up to elements
  return S * ldh + poly_offset(S + 1, D) + idx_units;
}

}  // namespace gbsh
