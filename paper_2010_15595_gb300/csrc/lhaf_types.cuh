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

// La Budde accumulators P_0..P_t are stored packed: P_u has degree <= u and is kept up to
// degree D, i.e. min(u, D) + 1 coefficients. Offset of P_t in that packed array.
__host__ __device__ __forceinline__ int poly_offset(int t, int D) {
  return t <= D + 1 ? t * (t + 1) / 2 : (D + 1) * (D + 2) / 2 + (t - D - 1) * (D + 1);
}

// Shared-memory footprint (in double2 units) of one warp's work area for subsets with
// m = 2k <= 2*kmax and series degree D = n+1: the bordered matrix (S x S, S = m+1 is odd
// so the row stride is conflict-free for column access), the packed accumulators
// P_0..P_S and the subset's index list.
__host__ __device__ inline int warp_area_elems(int kmax, int n) {
  int S = 2 * kmax + 1;
  int ldh = S | 1;
  int D = n + 1;
  int idx_units = (S + 3) / 4;  // S ints packed into 16-byte units
  return S * ldh + poly_offset(S + 1, D) + idx_units;
}

}  // namespace gbsh
