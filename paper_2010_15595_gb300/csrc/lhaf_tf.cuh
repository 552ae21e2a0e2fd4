// Triple-float arithmetic: a real number held as the unevaluated sum of three FP32 words,
// a + b + c with |b| <= ulp(a) and |c| <= ulp(b) after renormalisation, which carries
// about 72 significand bits.
//
// Why it exists on GB300: the per-subset terms p_Z of the loop-hafnian subset sum are tiny
// next to the characteristic-polynomial coefficients they are assembled from, and the
// signed sum over 2^{N/2} subsets cancels by ten or more decimal orders at N >= 40 (Sec. IV
// treats this accuracy problem with long double and La Budde's method). Complex FP64 per
// subset leaves the N = 40 and N = 50 loop hafnians 1e-8 to 1e-5 off; about 70 significand
// bits in every step (Hessenberg reduction, La Budde's recursion, the power series) bring
// them below 1e-10. GB300 issues FP32 at 64 times its FP64 rate, so three FP32 words cost
// about what one FP64 word costs, where FP64 double-double would cost some 15 times more.
//
// Building blocks (error-free transformations, written with the _rn intrinsics so that the
// compiler neither contracts nor reassociates them):
//   TwoSum      s + e = x + y exactly (Knuth, TAOCP vol. 2, 4.2.2)
//   TwoProduct  p + e = x * y exactly, e = fma(x, y, -p) (exact with a fused multiply-add)
// The multiply-accumulate keeps the exact leading product and the exact products of the
// leading word with the second words, rounds only the third-level terms (weight 2^-48
// relative to the operands), sums every second-level term with TwoSum, and renormalises the
// three levels with a chain of TwoSums.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

namespace gbsh {

struct tf3 {
  float a, b, c;
  tf3() = default;
  __device__ __forceinline__ tf3(float x, float y, float z) : a(x), b(y), c(z) {}
  __device__ __forceinline__ explicit tf3(float x) : a(x), b(0.f), c(0.f) {}
  __device__ __forceinline__ explicit tf3(int i) : a((float)i), b(0.f), c(0.f) {}
  // exact for every finite double inside the FP32 exponent range (53 <= 72 bits)
  __device__ __forceinline__ explicit tf3(double d) {
    a = __double2float_rn(d);
    const double r = d - (double)a;
    b = __double2float_rn(r);
    c = __double2float_rn(r - (double)b);
  }
};

__device__ __forceinline__ void tf_two_sum(float x, float y, float& s, float& e) {
  s = __fadd_rn(x, y);
  const float z = __fsub_rn(s, x);
  e = __fadd_rn(__fsub_rn(x, __fsub_rn(s, z)), __fsub_rn(y, z));
}
__device__ __forceinline__ void tf_two_prod(float x, float y, float& p, float& e) {
  p = __fmul_rn(x, y);
  e = __fmaf_rn(x, y, -p);
}
// (s0, s1, s2) with |s1|, |s2| small next to |s0| but possibly overlapping it -> normalised
__device__ __forceinline__ tf3 tf_renorm(float s0, float s1, float s2) {
  float u, w, z0, v, z1, z2;
  tf_two_sum(s1, s2, u, w);
  tf_two_sum(s0, u, z0, v);
  tf_two_sum(v, w, z1, z2);
  return tf3(z0, z1, z2);
}

__device__ __forceinline__ tf3 operator-(tf3 x) { return tf3(-x.a, -x.b, -x.c); }

__device__ __forceinline__ tf3 operator+(tf3 x, tf3 y) {
  float s0, e0, s1, e1, t1, f1;
  tf_two_sum(x.a, y.a, s0, e0);
  tf_two_sum(x.b, y.b, s1, e1);
  tf_two_sum(s1, e0, t1, f1);
  const float t2 = __fadd_rn(__fadd_rn(__fadd_rn(x.c, y.c), e1), f1);
  return tf_renorm(s0, t1, t2);
}
__device__ __forceinline__ tf3 operator-(tf3 x, tf3 y) { return x + (-y); }

// Second- and third-level parts of the product x*y: x*y = p0 + (sum of the four level-1
// words in l[]) + t, exactly up to the rounding of t (weight ~2^-72 of |x y|).
struct TfProd {
  float p0, q0, p1, p2, t;
};
__device__ __forceinline__ TfProd tf_prod_parts(tf3 x, tf3 y) {
  TfProd r;
  float q1, q2;
  tf_two_prod(x.a, y.a, r.p0, r.q0);
  tf_two_prod(x.a, y.b, r.p1, q1);
  tf_two_prod(x.b, y.a, r.p2, q2);
  r.t = __fmaf_rn(x.a, y.c, __fmaf_rn(x.b, y.b, __fmaf_rn(x.c, y.a, __fadd_rn(q1, q2))));
  return r;
}

// acc + x*y
__device__ __forceinline__ tf3 tf_fma(tf3 x, tf3 y, tf3 acc) {
  const TfProd P = tf_prod_parts(x, y);
  float s0, r0, u1, v1, u2, v2, u3, v3, s1, v4;
  tf_two_sum(acc.a, P.p0, s0, r0);
  tf_two_sum(acc.b, P.q0, u1, v1);
  tf_two_sum(P.p1, P.p2, u2, v2);
  tf_two_sum(u1, u2, u3, v3);
  tf_two_sum(u3, r0, s1, v4);
  const float s2 = __fadd_rn(__fadd_rn(__fadd_rn(acc.c, P.t), __fadd_rn(v1, v2)), __fadd_rn(v3, v4));
  return tf_renorm(s0, s1, s2);
}
__device__ __forceinline__ tf3 operator*(tf3 x, tf3 y) {
  const TfProd P = tf_prod_parts(x, y);
  float s1, e1, s1b, e2;
  tf_two_sum(P.q0, P.p1, s1, e1);
  tf_two_sum(s1, P.p2, s1b, e2);
  const float s2 = __fadd_rn(P.t, __fadd_rn(e1, e2));
  return tf_renorm(P.p0, s1b, s2);
}

// acc + x1*y1 + x2*y2 in one pass (one renormalisation): the complex multiply-accumulate
// per component.
__device__ __forceinline__ tf3 tf_dot2(tf3 x1, tf3 y1, tf3 x2, tf3 y2, tf3 acc) {
  const TfProd P = tf_prod_parts(x1, y1);
  const TfProd Q = tf_prod_parts(x2, y2);
  float s0, r1, r2;
  tf_two_sum(acc.a, P.p0, s0, r1);
  tf_two_sum(s0, Q.p0, s0, r2);
  // level 1: acc.b, P.q0, Q.q0, P.p1, P.p2, Q.p1, Q.p2, r1, r2 (a fixed TwoSum tree)
  float a1, e1, a2, e2, a3, e3, a4, e4, b1, f1, b2, f2, c1, g1, s1, g2;
  tf_two_sum(acc.b, P.q0, a1, e1);
  tf_two_sum(Q.q0, r1, a2, e2);
  tf_two_sum(P.p1, P.p2, a3, e3);
  tf_two_sum(Q.p1, Q.p2, a4, e4);
  tf_two_sum(a1, a2, b1, f1);
  tf_two_sum(a3, a4, b2, f2);
  tf_two_sum(b1, b2, c1, g1);
  tf_two_sum(c1, r2, s1, g2);
  // level 2
  float s2 = __fadd_rn(__fadd_rn(acc.c, P.t), Q.t);
  s2 = __fadd_rn(s2, __fadd_rn(__fadd_rn(e1, e2), __fadd_rn(e3, e4)));
  s2 = __fadd_rn(s2, __fadd_rn(__fadd_rn(f1, f2), __fadd_rn(g1, g2)));
  return tf_renorm(s0, s1, s2);
}

// x * 2^s, exact while every word stays normal. The power of two is built from its bits
// (two factors when |s| exceeds one factor's range).
__device__ __forceinline__ float pow2f(int e) { return __int_as_float((127 + e) << 23); }
__device__ __forceinline__ tf3 tf_scale2(tf3 x, int s) {
  if (s >= -126 && s <= 127) {
    const float f = pow2f(s);
    return tf3(__fmul_rn(x.a, f), __fmul_rn(x.b, f), __fmul_rn(x.c, f));
  }
  const int s1 = s < 0 ? -126 : 127;
  const float f1 = pow2f(s1), f2 = pow2f(s - s1 < -126 ? -126 : (s - s1 > 127 ? 127 : s - s1));
  return tf3(__fmul_rn(__fmul_rn(x.a, f1), f2), __fmul_rn(__fmul_rn(x.b, f1), f2),
             __fmul_rn(__fmul_rn(x.c, f1), f2));
}

// out-of-line copies for the once-per-step code (pivot reciprocal): small footprint
__device__ __noinline__ tf3 tf_fma_ool(tf3 x, tf3 y, tf3 acc) { return tf_fma(x, y, acc); }
__device__ __noinline__ tf3 tf_mul_ool(tf3 x, tf3 y) { return x * y; }
// 1/x by Newton's iteration r <- r + r (1 - x r) from the FP32 reciprocal of the leading
// word; each step doubles the correct bits (24 -> 48 -> 96, limited by the format).
__device__ __forceinline__ tf3 tf_recip(tf3 x) {
  tf3 r(__frcp_rn(x.a));
  const tf3 one(1.0f);
  const tf3 mx = -x;
#pragma unroll 1
  for (int it = 0; it < 2; ++it) {
    const tf3 e = tf_fma_ool(mx, r, one);
    r = tf_fma_ool(r, e, r);
  }
  return r;
}

// The value as a normalised double-double hi + lo (hi the nearest double). The words may
// be far apart (an integer 2^97 + 3 is held as a = 2^97, b = 3), so a + b is not exact in
// one double: both additions are TwoSums in FP64 and their errors are kept in lo. A few
// FP64 instructions per subset term.
__device__ __forceinline__ void tf_two_sum_d(double x, double y, double& s, double& e) {
  s = __dadd_rn(x, y);
  const double z = __dsub_rn(s, x);
  e = __dadd_rn(__dsub_rn(x, __dsub_rn(s, z)), __dsub_rn(y, z));
}
__device__ __forceinline__ void tf_to_dd(tf3 x, double& hi, double& lo) {
  double s, e1, h, e2;
  tf_two_sum_d((double)x.a, (double)x.b, s, e1);
  tf_two_sum_d(s, (double)x.c, h, e2);
  const double l = __dadd_rn(e1, e2);
  hi = __dadd_rn(h, l);
  lo = __dsub_rn(l, __dsub_rn(hi, h));
}

// -------------------------------------------------------------------------- complex
struct alignas(8) tfc {  // 8-byte aligned: shared-memory words move in 64-bit pairs
  tf3 x, y;
};

// The complex operations are tens to hundreds of FP32 instructions each and appear at many
// places of the per-subset code; compiled out of line, one copy serves every call site, so
// the instruction footprint of the per-subset code stays small (warps that run different
// phases of it share the instruction cache). Inlined multiply-accumulates were 1.4x slower
// at N = 40; with the add, the real scaling and the power-of-two scaling out of line as
// well, and every loop of the per-subset code kept rolled (for_rolled), the per-subset
// function shrank from 70 KB to 43 KB of code and N = 40 ran 9 % faster.
__device__ __noinline__ tfc cadd(tfc p, tfc q) { return tfc{p.x + q.x, p.y + q.y}; }
// acc - p*q
__device__ __noinline__ tfc cfms(tfc acc, tfc p, tfc q) {
  return tfc{tf_dot2(-p.x, q.x, p.y, q.y, acc.x), tf_dot2(-p.x, q.y, -p.y, q.x, acc.y)};
}
// acc + p*q, through the same out-of-line code
__device__ __forceinline__ tfc cfma(tfc acc, tfc p, tfc q) { return cfms(acc, tfc{-p.x, -p.y}, q); }
__device__ __forceinline__ tfc cmul(tfc p, tfc q) {
  const tf3 z(0.0f);
  return cfma(tfc{z, z}, p, q);
}
__device__ __noinline__ tfc cscale(tfc p, tf3 s) { return tfc{p.x * s, p.y * s}; }
// The pivot reciprocal 1/p = conj(p) / |p|^2, out of line, with a small footprint: |p|^2
// through the shared multiply-add, the Newton steps and the final products through single
// out-of-line copies (the same operations on the same operands as an inline form, so
// bit-identical to it). It runs once per elimination step, and its code displaces the hot
// loops' in the instruction cache: 3 KB instead of 7.4 KB inline made GB300's N = 32 5 % and
// N = 40 2.4 % faster (N = 50 1.2 % slower).
__device__ __noinline__ tfc crecip(tfc p) {
  const tf3 z(0.0f);
  const tf3 d = -cfms(tfc{z, z}, p, tfc{p.x, -p.y}).x;  // p conj(p) = |p|^2
  const tf3 r = tf_recip(d);
  return tfc{tf_mul_ool(p.x, r), -tf_mul_ool(p.y, r)};
}
// exact power-of-two scaling of both parts, out of line like the operations above
__device__ __noinline__ tfc tfc_scale2(tfc v, int s) { return tfc{tf_scale2(v.x, s), tf_scale2(v.y, s)}; }
__device__ __forceinline__ int pow2_exponent(tfc p) {
  const unsigned ex = (__float_as_uint(p.x.a) >> 23) & 0xffu;
  const unsigned ey = (__float_as_uint(p.y.a) >> 23) & 0xffu;
  const int eb = (int)(ex > ey ? ex : ey);
  return (eb == 0 ? 1 : eb) - 127;
}
__device__ __forceinline__ unsigned mag_key(tfc p) {
  const unsigned hx = __float_as_uint(p.x.a) & 0x7fffffffu;
  const unsigned hy = __float_as_uint(p.y.a) & 0x7fffffffu;
  return hx > hy ? hx : hy;
}
__device__ __forceinline__ tf3 shfl_t(tf3 v, int src) {
  return tf3(__shfl_sync(0xffffffffu, v.a, src), __shfl_sync(0xffffffffu, v.b, src),
             __shfl_sync(0xffffffffu, v.c, src));
}
__device__ __forceinline__ tfc shfl_c(tfc v, int src) { return tfc{shfl_t(v.x, src), shfl_t(v.y, src)}; }
__device__ __forceinline__ tf3 shfl_up_t(tf3 v, unsigned d) {
  return tf3(__shfl_up_sync(0xffffffffu, v.a, d), __shfl_up_sync(0xffffffffu, v.b, d),
             __shfl_up_sync(0xffffffffu, v.c, d));
}
__device__ __forceinline__ tfc shfl_up_c(tfc v, unsigned d) { return tfc{shfl_up_t(v.x, d), shfl_up_t(v.y, d)}; }
__device__ __forceinline__ tf3 shfl_down_t(tf3 v, unsigned d) {
  return tf3(__shfl_down_sync(0xffffffffu, v.a, d), __shfl_down_sync(0xffffffffu, v.b, d),
             __shfl_down_sync(0xffffffffu, v.c, d));
}
__device__ __forceinline__ tfc shfl_down_c(tfc v, unsigned d) {
  return tfc{shfl_down_t(v.x, d), shfl_down_t(v.y, d)};
}

}  // namespace gbsh
