// dw.cuh -- double-word arithmetic on the FP32 units: a value is the
// unevaluated sum h + l of two FP32 numbers (about 48 significant bits), the
// storage and arithmetic type of precision LBM_DF64.
//
// The building blocks are the classical error-free transformations:
//  two_sum  (Knuth): s = fl(a + b) and e with s + e = a + b exactly, 6 ops;
//  fast_two_sum (Dekker): the same in 3 ops when |a| >= |b|;
//  two_prod: p = fl(a b), e = fma(a, b, -p), p + e = a b exactly, 2 ops;
// combined as in the double-word algorithms of Joldes, Muller and Popescu
// (ACM TOMS 44, 2017) -- DWPlusDW, DWTimesDW, DWTimesFP -- with one
// difference: intermediate results are left unnormalised (the low word
// collects the exact rounding error of the high word plus the low-order
// terms, without the final fast_two_sum) and are normalised once, before
// they are stored. Every result then carries an absolute error of order
// u^2 (|x| + |y|) with u = 2^-24, the double-word counterpart of FP64's
// u_64 |x + y|.
//
// Two forms:
//  dw        scalar, always normalised, with the operators +, -, *, unary -,
//            comparisons, recip and conversions to and from double: the
//            type R of the generic step templates (boundary ghosts, initial
//            state, moments, audits), where speed does not matter;
//  DW<V>     the fast form used by the interior update, lanes V = float or
//            float2 (two nodes per thread in paired f32x2 instructions),
//            unnormalised between operations.
// Every FP32 operation is an explicitly rounded intrinsic (__fadd_rn,
// __fmul_rn, __fmaf_rn and their f32x2 forms): the compiler may not contract
// or reorder them, which the error-free transformations rely on.
#pragma once

#include <cuda_runtime.h>

#include <cmath>

namespace d2v16 {

// ---------------------------------------------------------------------------
// Lane operations (float and float2)
// ---------------------------------------------------------------------------
#ifdef __CUDACC__
__device__ __forceinline__ float ladd(float a, float b) { return __fadd_rn(a, b); }
__device__ __forceinline__ float lsub(float a, float b) { return __fsub_rn(a, b); }
__device__ __forceinline__ float lmul(float a, float b) { return __fmul_rn(a, b); }
__device__ __forceinline__ float lfma(float a, float b, float c) { return __fmaf_rn(a, b, c); }
__device__ __forceinline__ float lneg(float a) { return -a; }
__device__ __forceinline__ float2 ladd(float2 a, float2 b) { return __fadd2_rn(a, b); }
// a - b as fma(b, -1, a): one instruction, exact product, one rounding.
__device__ __forceinline__ float2 lsub(float2 a, float2 b) {
  return __ffma2_rn(b, make_float2(-1.f, -1.f), a);
}
__device__ __forceinline__ float2 lmul(float2 a, float2 b) { return __fmul2_rn(a, b); }
__device__ __forceinline__ float2 lfma(float2 a, float2 b, float2 c) { return __ffma2_rn(a, b, c); }
__device__ __forceinline__ float2 lneg(float2 a) { return make_float2(-a.x, -a.y); }

template <typename V> __device__ __forceinline__ V bcast_lane(float c);
template <> __device__ __forceinline__ float bcast_lane<float>(float c) { return c; }
template <> __device__ __forceinline__ float2 bcast_lane<float2>(float c) { return make_float2(c, c); }

__device__ __forceinline__ float rcp_lane(float x) {
  float r;
  asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
  return r;
}
__device__ __forceinline__ float2 rcp_lane(float2 x) { return make_float2(rcp_lane(x.x), rcp_lane(x.y)); }

// s + e = a + b exactly (Knuth's TwoSum).
template <typename V>
__device__ __forceinline__ void two_sum(V a, V b, V& s, V& e) {
  s = ladd(a, b);
  const V bb = lsub(s, a);
  e = ladd(lsub(a, lsub(s, bb)), lsub(b, bb));
}
// s + e = a + b exactly when |a| >= |b| (Dekker's Fast2Sum).
template <typename V>
__device__ __forceinline__ void fast_two_sum(V a, V b, V& s, V& e) {
  s = ladd(a, b);
  e = lsub(b, lsub(s, a));
}
#endif  // __CUDACC__

// ---------------------------------------------------------------------------
// dw: scalar, normalised double-word value (generic templates)
// ---------------------------------------------------------------------------
struct dw {
  float h, l;
  dw() = default;
  __host__ __device__ constexpr dw(float hi, float lo) : h(hi), l(lo) {}
  // Nearest double-word split of a double: h = fl32(x), l = fl32(x - h).
  __host__ __device__ constexpr dw(double x) : h((float)x), l((float)(x - (double)(float)x)) {}
  __host__ __device__ explicit operator double() const { return (double)h + (double)l; }
};

#ifdef __CUDACC__
// Normalised pair from s + e (two_sum: valid whatever the magnitudes, as
// after a cancelling sum); dw_norm_prod for a product, where |s| >= |e|.
__device__ __forceinline__ dw dw_norm(float s, float e) {
  float h, l;
  two_sum(s, e, h, l);
  return dw(h, l);
}
__device__ __forceinline__ dw dw_norm_prod(float s, float e) {
  float h, l;
  fast_two_sum(s, e, h, l);
  return dw(h, l);
}
__device__ __forceinline__ dw operator+(dw x, dw y) {
  float s, e;
  two_sum(x.h, y.h, s, e);
  return dw_norm(s, ladd(ladd(x.l, y.l), e));
}
__device__ __forceinline__ dw operator-(dw x) { return dw(-x.h, -x.l); }
__device__ __forceinline__ dw operator-(dw x, dw y) { return x + (-y); }
__device__ __forceinline__ dw operator*(dw x, dw y) {
  const float p = lmul(x.h, y.h);
  float e = lfma(x.h, y.h, -p);
  e = lfma(x.l, y.l, e);
  e = lfma(x.h, y.l, e);
  e = lfma(x.l, y.h, e);
  return dw_norm_prod(p, e);
}
__device__ __forceinline__ dw& operator+=(dw& x, dw y) { return x = x + y; }
__device__ __forceinline__ bool operator>(dw x, dw y) { return x.h > y.h || (x.h == y.h && x.l > y.l); }
__device__ __forceinline__ bool operator<(dw x, dw y) { return y > x; }
__device__ __forceinline__ bool operator<=(dw x, dw y) { return x.h < y.h || (x.h == y.h && x.l <= y.l); }
__device__ __forceinline__ bool isfinite(dw x) { return ::isfinite(x.h) && ::isfinite(x.l); }
// 1 / x: hardware approximation r, the residual d = 1 - x r in double-word
// accuracy (r x.h exact by two_prod; 1 - p exact by Sterbenz), then
// r (1 + d + d^2) (Newton's iteration carried to second order).
__device__ __forceinline__ dw recip(dw x) {
  const float r = rcp_lane(x.h);
  const float p = lmul(x.h, r);
  const float pe = lfma(x.h, r, -p);
  float d = lsub(lsub(1.0f, p), pe);
  d = lfma(-x.l, r, d);
  return dw_norm_prod(r, lmul(r, lfma(d, d, d)));
}
#endif  // __CUDACC__

// ---------------------------------------------------------------------------
// DW<V>: the fast, unnormalised form (lanes V = float or float2)
// ---------------------------------------------------------------------------
template <typename V>
struct DW {
  V h, l;
};

#ifdef __CUDACC__
// Broadcast of a scalar constant to the lanes.
template <typename V>
__device__ __forceinline__ DW<V> dwc(dw k) { return {bcast_lane<V>(k.h), bcast_lane<V>(k.l)}; }

// x + y: two_sum of the high words, the low words and its error summed.
template <typename V>
__device__ __forceinline__ DW<V> dadd(DW<V> x, DW<V> y) {
  V s, e;
  two_sum(x.h, y.h, s, e);
  return {s, ladd(ladd(x.l, y.l), e)};
}
// x - y.
template <typename V>
__device__ __forceinline__ DW<V> dsub(DW<V> x, DW<V> y) {
  const V s = lsub(x.h, y.h);
  const V bb = lsub(s, x.h);
  const V e = lsub(lsub(x.h, lsub(s, bb)), ladd(y.h, bb));
  return {s, ladd(lsub(x.l, y.l), e)};
}
// x y: the exact product of the high words (two_prod) plus the three
// cross and low products.
template <typename V>
__device__ __forceinline__ DW<V> dmul(DW<V> x, DW<V> y) {
  const V p = lmul(x.h, y.h);
  V e = lfma(x.h, y.h, lneg(p));
  e = lfma(x.l, y.l, e);
  e = lfma(x.h, y.l, e);
  e = lfma(x.l, y.h, e);
  return {p, e};
}
// x k for a constant k = k.h + k.l + k3 given to three words: a constant held
// in two words is off by up to 2^-48 of itself, the same error at every node
// and step, and such a bias accumulates linearly over a run (measured on the
// Mach-2.9 reflection, where populations reach 50 rho: 1.7e-12 per step); the
// third word takes it to 2^-72. k3 = 0 for constants exact in two words.
template <typename V>
__device__ __forceinline__ DW<V> dmulk(DW<V> x, dw k, float k3 = 0.0f) {
  const V kh = bcast_lane<V>(k.h), kl = bcast_lane<V>(k.l);
  const V p = lmul(x.h, kh);
  V e = lfma(x.h, kh, lneg(p));
  e = lfma(x.l, kl, e);
  e = lfma(x.h, bcast_lane<V>(k3), e);
  e = lfma(x.h, kl, e);
  e = lfma(x.l, kh, e);
  return {p, e};
}

// Third word of a double's three-word split: x - h - l rounded to FP32
// (h, l the double-word split of x).
__host__ __device__ constexpr float third_word(double x) {
  return (float)((x - (double)(float)x) - (double)(float)(x - (double)(float)x));
}
// x c for an FP32 constant c (exact c: the lattice's coefficients).
template <typename V>
__device__ __forceinline__ DW<V> dmulf(DW<V> x, float c) {
  if (c == 1.0f) return x;
  const V cv = bcast_lane<V>(c);
  const V p = lmul(x.h, cv);
  return {p, lfma(x.l, cv, lfma(x.h, cv, lneg(p)))};
}
// x 2^k (exact).
template <typename V>
__device__ __forceinline__ DW<V> dscale(DW<V> x, float pow2) {
  const V c = bcast_lane<V>(pow2);
  return {lmul(x.h, c), lmul(x.l, c)};
}
// 1 / x (see recip(dw)).
template <typename V>
__device__ __forceinline__ DW<V> drecip(DW<V> x) {
  const V r = rcp_lane(x.h);
  const V p = lmul(x.h, r);
  const V pe = lfma(x.h, r, lneg(p));
  V d = lsub(lsub(bcast_lane<V>(1.0f), p), pe);
  d = lfma(lneg(x.l), r, d);
  return {r, lmul(r, lfma(d, d, d))};
}
// Normalised form (h = fl32(h + l)); two_sum, since a cancelling sum can
// leave |l| > |h|.
template <typename V>
__device__ __forceinline__ DW<V> dnorm(DW<V> x) {
  V s, e;
  two_sum(x.h, x.l, s, e);
  return {s, e};
}
#endif  // __CUDACC__

}  // namespace d2v16
