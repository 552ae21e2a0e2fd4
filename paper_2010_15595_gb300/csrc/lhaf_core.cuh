// Per-subset term of the loop-hafnian subset formula, computed by one warp.
//
// The loop hafnian of an N x N complex symmetric matrix A (N = 2n after padding) is
//     lhaf(A) = sum over subsets Z of the n index pairs (j, j+n) of (-1)^{n-|Z|} p_Z,
//     p_Z     = [lambda^n] det(I - lambda M_Z)^{-1/2} exp( 1/2 sum_j l_j lambda^j ),
// with M_Z = X_Z A0_Z (A0 = A without its diagonal, X_Z swapping the two halves of the
// subset's rows) and loop terms l_j = v_Z^T M_Z^{j-1} X_Z v_Z (v = diag A). This is the
// O(N^3 2^{N/2}) algorithm the paper cites for loop hafnians (Sec. II after
// Eq. lhaf-pure) and benchmarks in Sec. IV; the paper evaluates its characteristic
// polynomial by La Budde's method after a Hessenberg reduction (Sec. IV).
//
// GB300 design: FP64 is the scarce unit (about two FP64 FMA lanes per SM per clock), so
// every step is arranged to keep the 32 lanes of each FP64 warp instruction busy and to
// avoid FP64 work that the formula does not need:
//   1. Build the bordered (m+1) x (m+1) matrix K' = [[0, v^T], [X v, M]] in shared memory.
//      Since det(I - lambda K') = det(I - lambda M) (1 - lambda^2 v^T (I - lambda M)^{-1} X v),
//      the loop terms follow from the ratio of two characteristic polynomials and need no
//      Krylov matrix-vector products.
//   2. Reduce K' to upper Hessenberg form by stabilised elementary similarity
//      transformations (Gaussian elimination with row pivoting), leaving index 0 fixed,
//      so that the trailing m x m block stays similar to M. Half the flops of Householder.
//      Each step also applies a diagonal similarity that makes the subdiagonal entry a
//      power of two, so that La Budde's subdiagonal products are exact exponent shifts
//      (no FP64 work). The column update of each step is spread over all 32 lanes.
//   3. La Budde's recursion over the trailing principal submatrices, in "push" form (each
//      finished polynomial is scattered into all later ones at once, lanes spread over
//      (target, coefficient) pairs), truncated at degree n+1. It yields det(I - lambda M)
//      and det(I - lambda K').
//   4. Power-series steps with one lane per coefficient: the ratio gives l_j, Newton's
//      identities give the power traces tr(M^j), and the exp-polynomial recursion gives
//      p_Z = [lambda^n] exp(sum_j c_j lambda^j), c_j = tr(M^j)/(2j) + l_j/2.
#pragma once

#include <cstdint>
#include <type_traits>
#include <cuda_runtime.h>

#include "lhaf_tf.cuh"
#include "lhaf_types.cuh"

namespace gbsh {

constexpr unsigned FULL = 0xffffffffu;

// ---------------------------------------------------------------- complex helpers
__device__ __forceinline__ double2 cadd(double2 a, double2 b) { return make_double2(a.x + b.x, a.y + b.y); }
__device__ __forceinline__ double2 csub(double2 a, double2 b) { return make_double2(a.x - b.x, a.y - b.y); }
__device__ __forceinline__ double2 cmul(double2 a, double2 b) {
  return make_double2(fma(a.x, b.x, -a.y * b.y), fma(a.x, b.y, a.y * b.x));
}
// acc + a*b  (4 FMA)
__device__ __forceinline__ double2 cfma(double2 acc, double2 a, double2 b) {
  return make_double2(fma(a.x, b.x, fma(-a.y, b.y, acc.x)), fma(a.x, b.y, fma(a.y, b.x, acc.y)));
}
// acc - a*b  (4 FMA)
__device__ __forceinline__ double2 cfms(double2 acc, double2 a, double2 b) {
  return make_double2(fma(-a.x, b.x, fma(a.y, b.y, acc.x)), fma(-a.x, b.y, fma(-a.y, b.x, acc.y)));
}
__device__ __forceinline__ double2 cscale(double2 a, double s) { return make_double2(a.x * s, a.y * s); }
// 1/a for complex a = conj(a) / |a|^2. The real reciprocal of d = |a|^2 starts from the
// hardware approximation (rcp.approx.ftz.f64) and is refined by two Newton-Raphson steps
// r <- r + r (1 - d r), each of which roughly doubles the number of correct bits; the
// result is accurate to a few ulps (not correctly rounded), ample for a pivot reciprocal,
// and costs 8 FP64 instructions instead of a full IEEE division. It is applied to pivots
// normalised to magnitude [1, 2 sqrt 2), so |a|^2 cannot underflow or overflow.
__device__ __forceinline__ double2 crecip(double2 a) {
  const double d = fma(a.x, a.x, a.y * a.y);
  double r;
  asm("rcp.approx.ftz.f64 %0, %1;" : "=d"(r) : "d"(d));
  double e = fma(-d, r, 1.0);
  r = fma(r, e, r);
  e = fma(-d, r, 1.0);
  r = fma(r, e, r);
  return make_double2(a.x * r, -a.y * r);
}
// x * 2^s, exact unless the result is subnormal. Integer instructions on the exponent field
// when x and the result are normal (no FP64 issue); zero stays zero; subnormal inputs and
// results outside the normal range go through ldexp.
__device__ __forceinline__ double pow2_scale(double x, int s) {
  const int hi = __double2hiint(x), lo = __double2loint(x);
  const int ef = (hi >> 20) & 0x7ff;
  if (ef != 0 && ef != 2047 && ef + s >= 1 && ef + s <= 2046)
    return __hiloint2double((int)((unsigned)hi + ((unsigned)s << 20)), lo);
  if (ef == 0 && ((hi & 0x000fffff) | lo) == 0) return x;  // +-0
  return ldexp(x, s);
}
// Unbiased binary exponent of the larger component's magnitude (|a| in [2^E, 2^(E+1)*sqrt 2)).
__device__ __forceinline__ int pow2_exponent(double2 a) {
  const int ex = (__double2hiint(a.x) >> 20) & 0x7ff;
  const int ey = (__double2hiint(a.y) >> 20) & 0x7ff;
  const int eb = ex > ey ? ex : ey;
  return (eb == 0 ? 1 : eb) - 1023;  // subnormals: scale as the smallest normal exponent
}
__device__ __forceinline__ double2 shfl_c(double2 v, int src) {
  return make_double2(__shfl_sync(FULL, v.x, src), __shfl_sync(FULL, v.y, src));
}
__device__ __forceinline__ double2 shfl_up_c(double2 v, unsigned d) {
  return make_double2(__shfl_up_sync(FULL, v.x, d), __shfl_up_sync(FULL, v.y, d));
}
__device__ __forceinline__ double2 shfl_down_c(double2 v, unsigned d) {
  return make_double2(__shfl_down_sync(FULL, v.x, d), __shfl_down_sync(FULL, v.y, d));
}
// Magnitude key for pivoting: the larger of |re|, |im| compared through the high word of
// the IEEE-754 encoding (sign cleared). Integer-only, so pivot search costs no FP64 issue.
__device__ __forceinline__ unsigned mag_key(double2 a) {
  unsigned hx = (unsigned)__double2hiint(a.x) & 0x7fffffffu;
  unsigned hy = (unsigned)__double2hiint(a.y) & 0x7fffffffu;
  return hx > hy ? hx : hy;
}

// ---- complex FP32 versions (per-subset arithmetic of the reduced-precision variant)
__device__ __forceinline__ float2 cadd(float2 a, float2 b) { return make_float2(a.x + b.x, a.y + b.y); }
__device__ __forceinline__ float2 cmul(float2 a, float2 b) {
  return make_float2(fmaf(a.x, b.x, -a.y * b.y), fmaf(a.x, b.y, a.y * b.x));
}
__device__ __forceinline__ float2 cfma(float2 acc, float2 a, float2 b) {
  return make_float2(fmaf(a.x, b.x, fmaf(-a.y, b.y, acc.x)), fmaf(a.x, b.y, fmaf(a.y, b.x, acc.y)));
}
__device__ __forceinline__ float2 cfms(float2 acc, float2 a, float2 b) {
  return make_float2(fmaf(-a.x, b.x, fmaf(a.y, b.y, acc.x)), fmaf(-a.x, b.y, fmaf(-a.y, b.x, acc.y)));
}
__device__ __forceinline__ float2 cscale(float2 a, float s) { return make_float2(a.x * s, a.y * s); }
__device__ __forceinline__ float2 crecip(float2 a) {
  const float inv = 1.0f / fmaf(a.x, a.x, a.y * a.y);
  return make_float2(a.x * inv, -a.y * inv);
}
__device__ __forceinline__ int pow2_exponent(float2 a) {
  int e = 0;
  frexpf(fmaxf(fabsf(a.x), fabsf(a.y)), &e);
  return e - 1;
}
__device__ __forceinline__ float2 shfl_c(float2 v, int src) {
  return make_float2(__shfl_sync(FULL, v.x, src), __shfl_sync(FULL, v.y, src));
}
__device__ __forceinline__ float2 shfl_up_c(float2 v, unsigned d) {
  return make_float2(__shfl_up_sync(FULL, v.x, d), __shfl_up_sync(FULL, v.y, d));
}
__device__ __forceinline__ float2 shfl_down_c(float2 v, unsigned d) {
  return make_float2(__shfl_down_sync(FULL, v.x, d), __shfl_down_sync(FULL, v.y, d));
}
__device__ __forceinline__ unsigned mag_key(float2 a) {
  unsigned hx = __float_as_uint(a.x) & 0x7fffffffu;
  unsigned hy = __float_as_uint(a.y) & 0x7fffffffu;
  return hx > hy ? hx : hy;
}


// ---- double-double (unevaluated sum hi + lo, ~106-bit significand) for the extended-
// precision variant. Error-free transformations: TwoSum (Knuth), FMA-based TwoProduct;
// addition and multiplication in the style of Dekker's double-length arithmetic with a
// final renormalisation; reciprocal by one Newton step from the double reciprocal.
struct dd {
  double hi, lo;
  dd() = default;
  __device__ __forceinline__ explicit dd(double h) : hi(h), lo(0.0) {}
  __device__ __forceinline__ dd(double h, double l) : hi(h), lo(l) {}
};
__device__ __forceinline__ dd dd_make(double a) { return dd{a, 0.0}; }
__device__ __forceinline__ void two_sum_d(double a, double b, double& s, double& e) {
  s = a + b;
  const double bb = s - a;
  e = (a - (s - bb)) + (b - bb);
}
__device__ __forceinline__ void quick_two_sum_d(double a, double b, double& s, double& e) {
  s = a + b;
  e = b - (s - a);
}
__device__ __forceinline__ dd operator+(dd x, dd y) {
  double s, e, t, f;
  two_sum_d(x.hi, y.hi, s, e);
  two_sum_d(x.lo, y.lo, t, f);
  e += t;
  quick_two_sum_d(s, e, s, e);
  e += f;
  quick_two_sum_d(s, e, s, e);
  return dd{s, e};
}
__device__ __forceinline__ dd operator-(dd x) { return dd{-x.hi, -x.lo}; }
__device__ __forceinline__ dd operator-(dd x, dd y) { return x + (-y); }
__device__ __forceinline__ dd operator*(dd x, dd y) {
  const double p = x.hi * y.hi;
  double e = fma(x.hi, y.hi, -p);
  e = fma(x.hi, y.lo, e);
  e = fma(x.lo, y.hi, e);
  double s, t;
  quick_two_sum_d(p, e, s, t);
  return dd{s, t};
}
// a*b + c in each real type of the per-subset arithmetic
__device__ __forceinline__ double rfma(double a, double b, double c) { return ::fma(a, b, c); }
__device__ __forceinline__ float rfma(float a, float b, float c) { return fmaf(a, b, c); }
__device__ __forceinline__ dd rfma(dd a, dd b, dd c) { return a * b + c; }
__device__ __forceinline__ dd dd_recip(dd x) {
  const double r0 = 1.0 / x.hi;
  const dd r = dd_make(r0);
  const dd e = dd_make(1.0) - x * r;  // 1 - x r0
  return r + r * e;
}

struct ddc {
  dd x, y;
};
__device__ __forceinline__ ddc cadd(ddc a, ddc b) { return ddc{a.x + b.x, a.y + b.y}; }
__device__ __forceinline__ ddc cmul(ddc a, ddc b) {
  return ddc{a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x};
}
__device__ __forceinline__ ddc cfma(ddc acc, ddc a, ddc b) {
  return ddc{acc.x + (a.x * b.x - a.y * b.y), acc.y + (a.x * b.y + a.y * b.x)};
}
__device__ __forceinline__ ddc cfms(ddc acc, ddc a, ddc b) {
  return ddc{acc.x - (a.x * b.x - a.y * b.y), acc.y - (a.x * b.y + a.y * b.x)};
}
__device__ __forceinline__ ddc cscale(ddc a, dd s) { return ddc{a.x * s, a.y * s}; }
__device__ __forceinline__ ddc crecip(ddc a) {
  const dd r = dd_recip(a.x * a.x + a.y * a.y);
  return ddc{a.x * r, -(a.y * r)};
}
__device__ __forceinline__ int pow2_exponent(ddc a) { return pow2_exponent(make_double2(a.x.hi, a.y.hi)); }
__device__ __forceinline__ dd shfl_d(dd v, int src) {
  return dd{__shfl_sync(FULL, v.hi, src), __shfl_sync(FULL, v.lo, src)};
}
__device__ __forceinline__ ddc shfl_c(ddc v, int src) { return ddc{shfl_d(v.x, src), shfl_d(v.y, src)}; }
__device__ __forceinline__ ddc shfl_up_c(ddc v, unsigned d) {
  return ddc{dd{__shfl_up_sync(FULL, v.x.hi, d), __shfl_up_sync(FULL, v.x.lo, d)},
             dd{__shfl_up_sync(FULL, v.y.hi, d), __shfl_up_sync(FULL, v.y.lo, d)}};
}
__device__ __forceinline__ ddc shfl_down_c(ddc v, unsigned d) {
  return ddc{dd{__shfl_down_sync(FULL, v.x.hi, d), __shfl_down_sync(FULL, v.x.lo, d)},
             dd{__shfl_down_sync(FULL, v.y.hi, d), __shfl_down_sync(FULL, v.y.lo, d)}};
}
__device__ __forceinline__ unsigned mag_key(ddc a) { return mag_key(make_double2(a.x.hi, a.y.hi)); }

// A subset term handed to the accumulator: value hi + lo per component (lo = 0 unless the
// per-subset arithmetic is double-double, whose low parts must not be rounded away).
struct Term {
  double re_hi, re_lo, im_hi, im_lo;
};

// Scalar-type traits: T is the per-subset complex type (double2, float2 or ddc).
template <class T> struct Cx;
template <> struct Cx<double2> {
  using R = double;
  __device__ __forceinline__ static double2 make(double a, double b) { return make_double2(a, b); }
  __device__ __forceinline__ static double2 from(double2 v) { return v; }
  __device__ __forceinline__ static double2 to_d(double2 v) { return v; }
  __device__ __forceinline__ static Term to_term(double2 v) { return Term{v.x, 0.0, v.y, 0.0}; }
  __device__ __forceinline__ static double2 scale2(double2 v, int s) {
    return make_double2(pow2_scale(v.x, s), pow2_scale(v.y, s));
  }
};
template <> struct Cx<ddc> {
  using R = dd;
  __device__ __forceinline__ static ddc make(dd a, dd b) { return ddc{a, b}; }
  __device__ __forceinline__ static ddc from(double2 v) { return ddc{dd_make(v.x), dd_make(v.y)}; }
  __device__ __forceinline__ static double2 to_d(ddc v) {
    return make_double2(v.x.hi + v.x.lo, v.y.hi + v.y.lo);
  }
  __device__ __forceinline__ static Term to_term(ddc v) { return Term{v.x.hi, v.x.lo, v.y.hi, v.y.lo}; }
  __device__ __forceinline__ static ddc scale2(ddc v, int s) {
    return ddc{dd{ldexp(v.x.hi, s), ldexp(v.x.lo, s)}, dd{ldexp(v.y.hi, s), ldexp(v.y.lo, s)}};
  }
};
template <> struct Cx<float2> {
  using R = float;
  __device__ __forceinline__ static float2 make(float a, float b) { return make_float2(a, b); }
  __device__ __forceinline__ static float2 from(double2 v) {
    return make_float2((float)v.x, (float)v.y);
  }
  __device__ __forceinline__ static double2 to_d(float2 v) { return make_double2(v.x, v.y); }
  __device__ __forceinline__ static Term to_term(float2 v) { return Term{v.x, 0.0, v.y, 0.0}; }
  __device__ __forceinline__ static float2 scale2(float2 v, int s) {
    return make_float2(ldexpf(v.x, s), ldexpf(v.y, s));
  }
};

template <> struct Cx<tfc> {
  using R = tf3;
  __device__ __forceinline__ static tfc make(tf3 a, tf3 b) { return tfc{a, b}; }
  __device__ __forceinline__ static tfc from(double2 v) { return tfc{tf3(v.x), tf3(v.y)}; }
  __device__ __forceinline__ static double2 to_d(tfc v) {
    double h, l;
    tf_to_dd(v.x, h, l);
    double h2, l2;
    tf_to_dd(v.y, h2, l2);
    return make_double2(h + l, h2 + l2);
  }
  __device__ __forceinline__ static Term to_term(tfc v) {
    Term t;
    tf_to_dd(v.x, t.re_hi, t.re_lo);
    tf_to_dd(v.y, t.im_hi, t.im_lo);
    return t;
  }
  __device__ __forceinline__ static tfc scale2(tfc v, int s) { return tfc_scale2(v, s); }
};
__device__ __forceinline__ tf3 rfma(tf3 a, tf3 b, tf3 c) { return tf_fma(a, b, c); }

// 1/k for k = 0..63 (entry 0 unused), filled by the host with correctly rounded values.
// Defined here because this header is included by exactly one translation unit.
__constant__ double c_inv_int[64];
// 1/k as three FP32 words (a + b + c within 2^-90 of 1/k), filled by the host from an
// exact integer division.
__constant__ float c_inv_tf[64][3];

// 1/k in the real type R of the per-subset arithmetic (exact to that type's precision).
template <class R> __device__ __forceinline__ R inv_int(int k);
template <> __device__ __forceinline__ double inv_int<double>(int k) { return c_inv_int[k]; }
template <> __device__ __forceinline__ float inv_int<float>(int k) { return (float)c_inv_int[k]; }
template <> __device__ __forceinline__ dd inv_int<dd>(int k) { return dd_recip(dd((double)k)); }
template <> __device__ __forceinline__ tf3 inv_int<tf3>(int k) {
  return tf3(c_inv_tf[k][0], c_inv_tf[k][1], c_inv_tf[k][2]);
}

// for (i = begin; i < end; i += step) f(i), kept rolled on the triple-float path, where
// code size is what limits speed: the 16 warps of an SM run different phases of the
// per-subset code at once, and the profile showed them waiting for instructions more than
// for anything else. Every loop of the per-subset code goes through it. The other
// arithmetic types get the plain loop.
template <class T, class F>
__device__ __forceinline__ void for_rolled(int begin, int end, int step, F&& f) {
  if constexpr (std::is_same<T, tfc>::value) {
#pragma unroll 1
    for (int i = begin; i < end; i += step) f(i);
  } else {
    for (int i = begin; i < end; i += step) f(i);
  }
}

// floor(e / d) for 0 <= e < 4096 and 1 <= d <= 64, given inv_d = the FP32 reciprocal of d
// rounded to nearest: (e + 1/2) inv_d is within (e + 1/2)/d * 2^-23 < 5e-4 of (e + 1/2)/d,
// whose distance to the nearest integer is at least 1/(2d) >= 1/128, so truncation is exact.
// Three instructions where an integer division takes about twenty.
__device__ __forceinline__ int div_small(int e, float inv_d) {
  return __float2int_rz(__fmul_rn(__int2float_rn(e) + 0.5f, inv_d));
}

// Compensated (two-sum) accumulator for the signed subset sum.
struct DDAcc {
  double re_hi, re_lo, im_hi, im_lo, abs_sum;
  __device__ __forceinline__ void zero() { re_hi = re_lo = im_hi = im_lo = abs_sum = 0.0; }
  __device__ __forceinline__ static void two_sum(double a, double b, double& s, double& e) {
    s = a + b;
    double bb = s - a;
    e = (a - (s - bb)) + (b - bb);
  }
  __device__ __forceinline__ void add(double2 x) {
    double s, e;
    two_sum(re_hi, x.x, s, e); re_hi = s; re_lo += e;
    two_sum(im_hi, x.y, s, e); im_hi = s; im_lo += e;
    abs_sum += fabs(x.x) + fabs(x.y);
  }
  __device__ __forceinline__ void add(const Term& t) {
    double s, e;
    two_sum(re_hi, t.re_hi, s, e); re_hi = s; re_lo += e + t.re_lo;
    two_sum(im_hi, t.im_hi, s, e); im_hi = s; im_lo += e + t.im_lo;
    abs_sum += fabs(t.re_hi) + fabs(t.im_hi);
  }
};

// Column c+1 of elimination step c of the Hessenberg reduction:
//     H[r][c+1] <- f_r H[r][c+1] + sum_{i=c+2}^{S-1} H[r][i] H[i][c]   for every row r,
// with f_r = piv except f_{c+1} = 1 (piv: the factor of the diagonal similarity of step c).
// The S x Rr products are split evenly over the 32 lanes in row-major order, q per lane, so
// one lane's range covers the tail of one row, possibly a whole row, and the head of another
// (S <= 64 bounds it to three rows). Each lane runs one accumulator chain and parks the
// partial of each row it finishes; the lane holding the first element of a row (its owner)
// adds, in lane order, the head partials of the lanes that start inside that row, so the
// rounding order is fixed. For short rows the plain one-lane-per-row loop issues fewer FP64
// instructions and is used instead; the choice depends on (S, Rr) only, so it is uniform
// across the warp.
template <class T>
__device__ __forceinline__ void column_update(T* __restrict__ H, int ldh, int S, int c, int Rr,
                                              const T piv, const T one, int lane) {
  using R = typename Cx<T>::R;
  const T zero = Cx<T>::make(R(0), R(0));
  const int passes = (S + 31) >> 5;
  const int tot = S * Rr;
  const int q = (tot + 31) >> 5;
  const int G = Rr > 1 ? (Rr - 2 + q) / q : 0;  // lanes that can start inside one row
  const bool seg = Rr > 0 && (4 * q + 2 * G + 4 * passes) < passes * (4 * Rr + 4);
  if (!seg) {
    for_rolled<T>(lane, S, 32, [&](int r) {
      T acc = zero;
      for_rolled<T>(c + 2, S, 1, [&](int i) { acc = cfma(acc, H[r * ldh + i], H[i * ldh + c]); });
      H[r * ldh + c + 1] = cfma(acc, r == c + 1 ? one : piv, H[r * ldh + c + 1]);
    });
    return;
  }
  const int e0 = lane * q;
  const bool has = e0 < tot;
  const int e1 = has ? min(e0 + q, tot) : e0;
  const int ra = has ? e0 / Rr : 0;  // first row touched
  const int o = has ? e0 - ra * Rr : 0;
  // running partial `acc` of the current row; finished rows move to h0, h1
  T acc = zero, h0 = zero, h1 = zero;
  int nfl = 0;
  int i = o;
  const int cnt = e1 - e0;
  const T* xr = H + ra * ldh + c + 2;
  for_rolled<T>(0, q, 1, [&](int t) {
    if (t < cnt) {
      acc = cfma(acc, xr[i], H[(c + 2 + i) * ldh + c]);
      if (++i == Rr) {
        i = 0;
        xr += ldh;
        if (nfl == 0) h0 = acc; else h1 = acc;
        ++nfl;
        acc = zero;
      }
    }
  });
  const T a0 = nfl >= 1 ? h0 : acc;
  const T a1 = nfl >= 2 ? h1 : (nfl == 1 ? acc : zero);
  const T a2 = nfl >= 2 ? acc : zero;
  const int rz = has ? (e1 - 1) / Rr : -1;  // last row touched
  const int zs = rz - ra;
  T tail = zs == 0 ? a0 : (zs == 1 ? a1 : a2);
  const int ra_key = has ? ra : -1;
  for_rolled<T>(1, G + 1, 1, [&](int j) {
    const T nb = shfl_down_c(a0, (unsigned)j);
    const int rj = __shfl_down_sync(FULL, ra_key, (unsigned)j);
    if (has && lane + j < 32 && rj == rz) tail = cadd(tail, nb);
  });
  // rows owned: ra when the lane starts it, then the following rows that start in range
  const int own1 = (o == 0) ? ra : ra + 1;
  for_rolled<T>(0, passes, 1, [&](int w) {
    const int r = own1 + w;
    if (has && r <= rz) {
      const int sl = r - ra;
      const T v = (r == rz) ? tail : (sl == 0 ? a0 : (sl == 1 ? a1 : a2));
      H[r * ldh + c + 1] = cfma(v, r == c + 1 ? one : piv, H[r * ldh + c + 1]);
    }
  });
}

// ------------------------------------------------------------------------------------
// p_Z for subset z (bit j <=> pair (j, j+n) in Z) with k = popcount(z) >= 1.
// `area` is this warp's shared work area (warp_area_elems(k, n) elements of T at least).
// T is the per-subset complex type: double2 (FP64 path) or float2 (reduced-precision
// variant, whose terms are still accumulated in compensated FP64 by the caller), ddc
// (double-double) or tfc (triple-float, the accurate path: see lhaf_tf.cuh).
// All 32 lanes must call it; every lane returns the same value.
// ------------------------------------------------------------------------------------
template <class T>
__device__ __noinline__ Term subset_term_full(const Problem& P, uint64_t z, int k,
                                              T* __restrict__ area, int lane) {
  using R = typename Cx<T>::R;
  const int n = P.n;
  const int m = 2 * k;
  const int S = m + 1;
  const int ldh = S | 1;
  const int D = n + 1;
  T* H = area;                                    // S x ldh
  T* Pl = area + S * ldh;                         // packed polynomial accumulators P_0..P_S
  int* idx = reinterpret_cast<int*>(Pl + poly_offset(S + 1, D));

  // ---- 1. index list of the subset: idx[a] = a-th pair in Z, idx[k+a] = that pair + n
  {
    unsigned bits = (unsigned)z;  // n <= 30
    bool in = (lane < n) && ((bits >> lane) & 1u);
    unsigned bal = __ballot_sync(FULL, in);
    if (in) {
      int pos = __popc(bal & ((1u << lane) - 1u));
      idx[pos] = lane;
      idx[k + pos] = lane + n;
    }
  }
  __syncwarp();

  // ---- 1b. K' = [[0, v^T], [X v, X A0_Z]]; row r>=1 of the M block is row (r-1+k) mod m
  for_rolled<T>(lane, S * S, 32, [&](int e) {
    int r = e / S, c = e - r * S;
    double2 val;
    if (r == 0) {
      val = (c == 0) ? make_double2(0.0, 0.0) : __ldg(P.v + idx[c - 1]);
    } else {
      int rr = r - 1 + k;
      rr = rr >= m ? rr - m : rr;
      int rs = idx[rr];
      val = (c == 0) ? __ldg(P.v + rs) : __ldg(P.A0 + (size_t)rs * P.Ne + idx[c - 1]);
    }
    H[r * ldh + c] = Cx<T>::from(val);
  });
  // polynomial accumulators: P_0 = 1, P_t = 0
  for_rolled<T>(lane, poly_offset(S + 1, D), 32,
                [&](int e) { Pl[e] = Cx<T>::make(e == 0 ? R(1) : R(0), R(0)); });
  __syncwarp();

  // ---- 2. Hessenberg reduction by stabilised elementary similarities (index 0 fixed
  //         automatically: column c only mixes rows/columns >= c+1), with subdiagonal
  //         entries normalised to powers of two. At step c, after the row interchange, the
  //         pivot pi = 2^E b with |b| in [1, 2 sqrt 2); the diagonal similarity that divides
  //         row c+1 and multiplies column c+1 by b turns the pivot into 2^E, so the
  //         multipliers are H[r][c] 2^-E (exact, integer instructions) and the only FP64
  //         reciprocal is 1/b, which is well conditioned. The working matrix keeps its
  //         natural scale; La Budde's subdiagonal products become powers of two, applied
  //         afterwards without FP64 arithmetic. A column with nothing to eliminate (all
  //         candidates zero) keeps a zero subdiagonal, recorded in `zmask`.
  int* kexp = idx;  // the index list is no longer needed: exponent E of each subdiagonal
  uint64_t zmask = 0;
  for (int c = 0; c + 1 < S; ++c) {
    const int Rr = S - c - 2;  // rows below the pivot row
    // pivot: largest magnitude in column c among rows c+1..S-1
    unsigned best = 0u;
    int brow = c + 1;
    for_rolled<T>(c + 1 + lane, S, 32, [&](int r) {
      unsigned mk = mag_key(H[r * ldh + c]);
      if (mk > best) { best = mk; brow = r; }
    });
    unsigned mx = __reduce_max_sync(FULL, best);
    if constexpr (std::is_same<T, tfc>::value) {
      // A column whose candidates are all below 2^-kZeroBits of the column's largest entry
      // is rounding residue of an exact cancellation (repeated rows and columns of a
      // pattern with repeated modes produce these): pivoting on the residue applies
      // multipliers that are ratios of rounding noise, which costs about 20 of the
      // format's 72 bits on such subsets. It is treated as zero instead -- a perturbation of
      // the column at 2^-kZeroBits of its scale, below the precision the subset sum needs.
      // Keys compare FP32 bit patterns, so 2^-64 is 64 << 23 in the key.
      constexpr unsigned kZeroBits = 64u;
      unsigned cm = 0u;
      for_rolled<T>(lane, c + 1, 32, [&](int r) {
        const unsigned k2 = mag_key(H[r * ldh + c]);
        cm = k2 > cm ? k2 : cm;
      });
      cm = __reduce_max_sync(FULL, cm);
      cm = cm > mx ? cm : mx;
      if (cm >= (kZeroBits << 23) && mx < cm - (kZeroBits << 23)) mx = 0u;
    }
    if (mx == 0u) {  // zero subdiagonal: nothing to eliminate or scale
      zmask |= 1ull << c;
      if (lane == 0) kexp[c] = 0;
      continue;
    }
    unsigned cand = __ballot_sync(FULL, best == mx);
    int p = __shfl_sync(FULL, brow, __ffs(cand) - 1);
    if (p != c + 1) {
      for_rolled<T>(c + lane, S, 32, [&](int j) {  // swap rows p and c+1 (columns >= c)
        T a = H[p * ldh + j], b = H[(c + 1) * ldh + j];
        H[p * ldh + j] = b;
        H[(c + 1) * ldh + j] = a;
      });
      __syncwarp();
      for_rolled<T>(lane, S, 32, [&](int r) {  // swap columns p and c+1
        T a = H[r * ldh + p], b = H[r * ldh + c + 1];
        H[r * ldh + p] = b;
        H[r * ldh + c + 1] = a;
      });
      __syncwarp();
    }
    const T piv = H[(c + 1) * ldh + c];
    const int E = pow2_exponent(piv);
    const T bp = Cx<T>::scale2(piv, -E);  // pivot / 2^E
    const T one = Cx<T>::make(R(1), R(0));
    if (lane == 0) kexp[c] = E;
    __syncwarp();  // every lane holds the pivot before its slot is reused below
    if (Rr > 0) {
      // scaled pivot row u_j = H[c+1][j] / b, j >= c+1. u_{c+1} is only an operand of the
      // elimination (the diagonal entry itself is unchanged by the similarity) and is
      // parked in the subdiagonal slot H[c+1][c], which is never read again.
      const T rinv = crecip(bp);
      for_rolled<T>(c + 1 + lane, S, 32, [&](int j) {
        const T u = cmul(H[(c + 1) * ldh + j], rinv);
        H[(c + 1) * ldh + (j == c + 1 ? c : j)] = u;
      });
      // multipliers H[r][c] / 2^E, kept in column c below the subdiagonal
      for_rolled<T>(c + 2 + lane, S, 32,
                    [&](int r) { H[r * ldh + c] = Cx<T>::scale2(H[r * ldh + c], -E); });
      __syncwarp();
      // rows r >= c+2:  H[r][j] -= m_r u_j,  j >= c+1
      {
        const int C = Rr + 1;
        const float inv_c = __frcp_rn((float)C);
        for_rolled<T>(lane, Rr * C, 32, [&](int e) {
          int rr = div_small(e, inv_c), jj = e - rr * C;
          int r = c + 2 + rr, j = c + 1 + jj;
          const T u = H[(c + 1) * ldh + (jj == 0 ? c : j)];
          H[r * ldh + j] = cfms(H[r * ldh + j], H[r * ldh + c], u);
        });
      }
      __syncwarp();
    }
    // column c+1 <- f_r H[r][c+1] + sum_{i >= c+2} H[r][i] m_i   (f_r = b, 1 at r = c+1)
    column_update<T>(H, ldh, S, c, Rr, bp, one, lane);
    __syncwarp();
  }
  // Subdiagonal l is 2^{E_l} (or zero, see zmask). La Budde needs H[a][b] times the product
  // of the subdiagonals between rows a and b, i.e. H[a][b] 2^{K_b - K_a} with K the prefix
  // sums of E: an exact rescaling of the strict upper triangle, integer-only when in range.
  if (lane == 0) {
    int acc = 0;
    for (int l = 0; l < S; ++l) {
      const int t = (l < S - 1) ? kexp[l] : 0;
      kexp[l] = acc;
      acc += t;
    }
  }
  __syncwarp();
  // Triple-float words have the FP32 exponent range (and lose their low words below about
  // 2^-78), so the triple-float path may evaluate the polynomials in mu = lambda / 2^sig,
  // i.e. of 2^sig H, an exact rescaling. La Budde's factors C(a,b) and diagonal entries
  // grow by at most 2^g per degree (g = max over factors of ceil(e / (b-a+1)), 2^e bounding
  // |C(a,b)|; integer instructions on the exponents only). Over the <= 31 degrees kept, a
  // growth within 2^-3 .. 2^3 per degree leaves every coefficient inside the safe window,
  // so sig is 0 for such matrices and only pulls g back to that band otherwise (e.g. the
  // all-ones matrices, g ~ 8 at N = 56). The power series are rescaled separately below,
  // from the coefficients' own sizes.
  int sig = 0;
  if constexpr (std::is_same<T, tfc>::value) {
    int g = -(1 << 20);
    for_rolled<T>(lane, S * S, 32, [&](int e) {
      const int a = e / S, bb = e - a * S;
      if (a > bb || mag_key(H[a * ldh + bb]) == 0u) return;
      const int len = bb - a + 1;
      if (a < bb && ((zmask >> a) & ((1ull << (bb - a)) - 1ull)) != 0ull) return;
      const int eb = pow2_exponent(H[a * ldh + bb]) + 2 + (a < bb ? kexp[bb] - kexp[a] : 0);
      const int q = eb >= 0 ? (eb + len - 1) / len : -((-eb) / len);
      g = q > g ? q : g;
    });
    g = __reduce_max_sync(FULL, g);
    sig = g == -(1 << 20) ? 0 : (g > 3 ? 3 - g : (g < -3 ? -3 - g : 0));
  }
  for_rolled<T>(lane, S * S, 32, [&](int e) {
    const int a = e / S, bb = e - a * S;
    if (a < bb) H[a * ldh + bb] = Cx<T>::scale2(H[a * ldh + bb], kexp[bb] - kexp[a] + sig * (bb - a + 1));
    else if (a == bb && sig != 0) H[a * ldh + a] = Cx<T>::scale2(H[a * ldh + a], sig);
  });
  __syncwarp();

  // ---- 3. La Budde over trailing blocks. With the subdiagonal products folded into the
  //   upper triangle (H[a][b] now holds C(a,b) = H[a][b] prod_{l=a}^{b-1} H[l+1][l]), the
  //   characteristic polynomials P_t = det(I - lambda H[S-t.., S-t..]) satisfy, for a = S-t,
  //   P_t = P_{t-1} + Dl_t,  Dl_t = -lambda H[a][a] P_{t-1}
  //                                 - sum_{b=a+1}^{S-1} C(a,b) lambda^{b-a+1} P_{S-1-b},
  //   where a term is dropped when a zero subdiagonal lies between rows a and b.
  //   Push form: once P_s is final it is scattered into every Dl_t, t > s (lanes spread
  //   over (target, coefficient) pairs), after which P_{s+1} = P_s + Dl_{s+1} is final.
  for (int s = 0; s < S; ++s) {
    const T* Ps = Pl + poly_offset(s, D);
    const int degs = s < D ? s : D;  // P_s has degree <= s
    const int bcol = S - 1 - s;
    {
      const int nt = S - s;                            // targets t = s+1 .. S
      const int ne = (degs < D - 1 ? degs : D - 1) + 1;
      const float inv_ne = __frcp_rn((float)ne);
      for_rolled<T>(lane, nt * ne, 32, [&](int f) {
        const int ti = div_small(f, inv_ne), e = f - ti * ne;
        const int t = s + 1 + ti;
        const int d = e + 1 + ti;
        const int a = S - t;
        const bool live = (d <= D) && ((zmask >> a) & ((1ull << ti) - 1ull)) == 0ull;
        if (live) {
          T* Pt = Pl + poly_offset(t, D);
          Pt[d] = cfms(Pt[d], H[a * ldh + bcol], Ps[e]);
        }
      });
    }
    __syncwarp();
    {
      T* Pn = Pl + poly_offset(s + 1, D);
      const int dmax = (s + 1) < D ? (s + 1) : D;
      if (lane <= dmax && lane <= degs) Pn[lane] = cadd(Pn[lane], Ps[lane]);
    }
    __syncwarp();
  }

  // ---- 4. series steps, lane d holds coefficient d (d <= D <= 31)
  const T zero = Cx<T>::make(R(0), R(0));
  // P_{S-1} and P_S have degree >= D here only if S-1 >= D; lanes above their degree read 0
  const int degM = (S - 1) < D ? (S - 1) : D, degK = S < D ? S : D;
  T qM = (lane <= degM) ? Pl[poly_offset(S - 1, D) + lane] : zero;
  T qK = (lane <= degK) ? Pl[poly_offset(S, D) + lane] : zero;
  if constexpr (std::is_same<T, tfc>::value) {
    // Series rescaling (triple-float path): the traces and exp-polynomial values grow like
    // rho^j with rho the spectral radius (all-ones matrices: 2^120 and more at N = 46), so
    // the series runs on q(2^sig2 mu) with sig2 from the bound rho <= 2 max_d |q_d|^{1/d}
    // (Fujiwara), which puts every root within 2 of the origin. Exact scaling by 2^{sig2 d}.
    int g2 = -(1 << 20);
    if (lane >= 1 && lane <= D) {
      const int ek = mag_key(qK) ? pow2_exponent(qK) + 2 : -(1 << 20);
      const int em = mag_key(qM) ? pow2_exponent(qM) + 2 : -(1 << 20);
      const int e = ek > em ? ek : em;
      if (e > -(1 << 20)) g2 = e >= 0 ? (e + lane - 1) / lane : -((-e) / lane);
    }
    g2 = __reduce_max_sync(FULL, g2);
    const int sig2 = g2 == -(1 << 20) ? 0 : -g2;
    if (sig2 != 0) {
      qM = Cx<T>::scale2(qM, sig2 * lane);
      qK = Cx<T>::scale2(qK, sig2 * lane);
      sig += sig2;
    }
  }
  // (a) r = qK / qM   (qM_0 = 1), coefficients 0..D
  // (b) power traces t_j = tr(M^j):  t_j = -j q_j - sum_{i=1}^{j-1} q_i t_{j-i}, j = 1..n
  // Both are recursions over s in which coefficient s, once final, updates every higher
  // one. When the D+1 + n coefficients fit the warp (n <= 15) they share one loop: lanes
  // 0..D hold r, lanes D+1..D+n hold t_1..t_n, and one multiply-add per step serves both
  // (the same operations on the same operands as two separate loops).
  T r, tr;
  if (D + 1 + n <= 32) {
    const bool inB = lane > D;
    const int j = inB ? lane - D : lane;
    const T qj = shfl_c(qM, j <= D ? j : 0);
    T v = inB ? cscale(qj, -(R)j) : qK;
    for_rolled<T>(0, D, 1, [&](int s) {
      const T vs = shfl_c(v, inB ? D + s : s);
      const T qs = shfl_c(qM, j > s ? j - s : 0);
      const bool act = inB ? (s >= 1 && s < n && j > s) : (j > s);
      if (act) v = cfms(v, qs, vs);
    });
    r = v;
    tr = shfl_c(v, D + lane <= 31 ? D + lane : 31);  // t_lane on lanes 1..n
  } else {
    r = qK;
    for_rolled<T>(0, D, 1, [&](int s) {
      T rs = shfl_c(r, s);
      T qs = shfl_up_c(qM, s);
      if (lane > s) r = cfms(r, qs, rs);
    });
    tr = cscale(qM, -(R)lane);
    for_rolled<T>(1, n, 1, [&](int s) {
      T ts = shfl_c(tr, s);
      T qs = shfl_up_c(qM, s);
      if (lane > s) tr = cfms(tr, qs, ts);
    });
  }
  // loop terms l_j = -r_{j+1} (for sig != 0: r of the rescaled matrices, whose loop terms
  // carry one factor 2^sig more than the traces of the same degree)
  T lj = shfl_down_c(r, 1);
  lj = Cx<T>::make(-lj.x, -lj.y);
  if (sig != 0) lj = Cx<T>::scale2(lj, -sig);
  // (c) j c_j = (t_j + j l_j) / 2
  const T icj = Cx<T>::make(R(0.5) * rfma((R)lane, lj.x, tr.x), R(0.5) * rfma((R)lane, lj.y, tr.y));
  // (d) exp-polynomial: j p_j = sum_{i=1}^{j} i c_i p_{j-i}, p_0 = 1
  T acc = zero;
  for_rolled<T>(0, n, 1, [&](int s) {
    T ps;
    if (s == 0) {
      ps = Cx<T>::make(R(1), R(0));
    } else {
      ps = cscale(shfl_c(acc, s), inv_int<R>(s));
    }
    T ics = shfl_up_c(icj, s);
    if (lane > s) acc = cfma(acc, ics, ps);
  });
  T pn = cscale(shfl_c(acc, n), inv_int<R>(n));
  __syncwarp();
  Term out = Cx<T>::to_term(pn);
  if (sig != 0) {  // [mu^n] = 2^{sig n} [lambda^n]: undo exactly in FP64
    const int s2 = -sig * n;
    out = Term{ldexp(out.re_hi, s2), ldexp(out.re_lo, s2), ldexp(out.im_hi, s2), ldexp(out.im_lo, s2)};
  }
  return out;
}

// p_Z rounded to complex double.
template <class T>
__device__ __forceinline__ double2 subset_term(const Problem& P, uint64_t z, int k,
                                               T* __restrict__ area, int lane) {
  const Term t = subset_term_full<T>(P, z, k, area, lane);
  return make_double2(t.re_hi + t.re_lo, t.im_hi + t.im_lo);
}

}  // namespace gbsh
