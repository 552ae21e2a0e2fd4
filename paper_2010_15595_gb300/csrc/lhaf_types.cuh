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

// Shared-memory footprint (in double2 units) of one warp's work area for subsets with
// m = 2k <= 2*kmax and series degree D = n+1.
__host__ __device__ inline int warp_area_elems(int kmax, int n) {
  int S = 2 * kmax + 1;
  int ldh = S | 1;
  int D = n + 1;
  int idx_units = (S + 3) / 4;  // S ints packed into 16-byte units
  return S * ldh + (S + 1) * (D + 1) + idx_units;
}

}  // namespace gbsh
