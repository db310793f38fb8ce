// Double-float ("FP32x2") arithmetic: a value is the unevaluated sum hi + lo of
// two FP32 numbers (|lo| <= ulp(hi)/2), a 48-bit significand carried by the
// FP32 units.  GB300 runs FP32 at 64x its FP64 rate, so transforms in this
// format reach FP64-class rounding (unit roundoff ~2^-48) at FP32-unit speed.
//
// Building blocks are the classical error-free transformations (Knuth's
// TwoSum, Dekker's Fast2Sum, the FMA-based exact product); every operation
// uses the _rn intrinsics, which the compiler never contracts or reorders.
#pragma once

#include <cuda_runtime.h>

namespace fcsph {

struct ff {
  float h, l;
  __host__ __device__ ff() : h(0.f), l(0.f) {}
  // plain conversions, so that constant arguments fold at compile time
  __host__ __device__ ff(double d) : h((float)d), l((float)(d - (double)(float)d)) {}
  // exact for |i| < 2^24 (wavenumber indices), without a trip through FP64
  __host__ __device__ ff(int i) : h((float)i), l(0.f) {}
  __host__ __device__ explicit operator double() const { return (double)h + (double)l; }
  __host__ __device__ explicit operator float() const { return h + l; }
};

__device__ __forceinline__ ff ff_make(float h, float l) {
  ff r;
  r.h = h;
  r.l = l;
  return r;
}

// s + e = a + b exactly (no assumption on |a| vs |b|)
__device__ __forceinline__ void two_sum(float a, float b, float& s, float& e) {
  s = __fadd_rn(a, b);
  const float bb = __fsub_rn(s, a);
  e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
}

// s + e = a + b exactly when |a| >= |b|
__device__ __forceinline__ void fast_two_sum(float a, float b, float& s, float& e) {
  s = __fadd_rn(a, b);
  e = __fsub_rn(b, __fsub_rn(s, a));
}

__device__ __forceinline__ ff operator+(ff a, ff b) {
  float s, e;
  two_sum(a.h, b.h, s, e);
  e = __fadd_rn(e, __fadd_rn(a.l, b.l));
  float h, l;
  fast_two_sum(s, e, h, l);
  return ff_make(h, l);
}

__device__ __forceinline__ ff operator-(ff a) { return ff_make(-a.h, -a.l); }

// a + b without the closing renormalisation: hi = fl(a.h + b.h), lo = its
// exact error plus a.l + b.l, so |lo| may exceed ulp(hi)/2 by a few ulps.
// Used for the sums inside one butterfly, whose results are renormalised
// (ff_norm) before they are stored; 8 FP32 instructions instead of 11.
__device__ __forceinline__ ff ff_add_nr(ff a, ff b) {
  float s, e;
  two_sum(a.h, b.h, s, e);
  return ff_make(s, __fadd_rn(e, __fadd_rn(a.l, b.l)));
}
__device__ __forceinline__ ff ff_norm(ff a) {
  float h, l;
  fast_two_sum(a.h, a.l, h, l);
  return ff_make(h, l);
}
__device__ __forceinline__ ff operator-(ff a, ff b) { return a + (-b); }

__device__ __forceinline__ ff operator*(ff a, ff b) {
  const float p = __fmul_rn(a.h, b.h);
  float e = __fmaf_rn(a.h, b.h, -p);  // exact low part of a.h * b.h
  e = __fmaf_rn(a.h, b.l, e);
  e = __fmaf_rn(a.l, b.h, e);
  float h, l;
  fast_two_sum(p, e, h, l);
  return ff_make(h, l);
}

__device__ __forceinline__ ff& operator+=(ff& a, ff b) {
  a = a + b;
  return a;
}

// a / b: FP32 quotient, one correction from the double-float remainder.
__device__ __forceinline__ ff operator/(ff a, ff b) {
  const float q1 = __fdiv_rn(a.h, b.h);
  const ff r = a - b * ff_make(q1, 0.f);
  const float q2 = __fdiv_rn(r.h, b.h);
  float h, l;
  fast_two_sum(q1, q2, h, l);
  return ff_make(h, l);
}

// acc + a * c with one renormalisation: the exact product's high word and
// its error (3 FMAs) join acc through TwoSum; 15 FP32 instructions instead of
// the 18 of a separate multiply and add.
__device__ __forceinline__ ff ff_fma(ff acc, ff a, ff c) {
  const float p = __fmul_rn(a.h, c.h);
  float e = __fmaf_rn(a.h, c.h, -p);
  e = __fmaf_rn(a.h, c.l, e);
  e = __fmaf_rn(a.l, c.h, e);
  float s, t;
  two_sum(acc.h, p, s, t);
  t = __fadd_rn(t, __fadd_rn(acc.l, e));
  float h, l;
  fast_two_sum(s, t, h, l);
  return ff_make(h, l);
}

// a * b + c * d: both exact products' high words through one TwoSum, their
// error terms added once; 19 FP32 instructions instead of 25.
__device__ __forceinline__ ff ff_dot2(ff a, ff b, ff c, ff d) {
  const float p1 = __fmul_rn(a.h, b.h);
  float e1 = __fmaf_rn(a.h, b.h, -p1);
  e1 = __fmaf_rn(a.h, b.l, e1);
  e1 = __fmaf_rn(a.l, b.h, e1);
  const float p2 = __fmul_rn(c.h, d.h);
  float e2 = __fmaf_rn(c.h, d.h, -p2);
  e2 = __fmaf_rn(c.h, d.l, e2);
  e2 = __fmaf_rn(c.l, d.h, e2);
  float s, t;
  two_sum(p1, p2, s, t);
  t = __fadd_rn(t, __fadd_rn(e1, e2));
  float h, l;
  fast_two_sum(s, t, h, l);
  return ff_make(h, l);
}

// acc + a * c and a * b + c * d as above without the closing
// renormalisation, for chains that end in a butterfly output (renormalised
// when stored): 12 and 16 FP32 instructions.
__device__ __forceinline__ ff ff_fma_nr(ff acc, ff a, ff c) {
  const float p = __fmul_rn(a.h, c.h);
  float e = __fmaf_rn(a.h, c.h, -p);
  e = __fmaf_rn(a.h, c.l, e);
  e = __fmaf_rn(a.l, c.h, e);
  float s, t;
  two_sum(acc.h, p, s, t);
  return ff_make(s, __fadd_rn(t, __fadd_rn(acc.l, e)));
}
__device__ __forceinline__ ff ff_dot2_nr(ff a, ff b, ff c, ff d) {
  const float p1 = __fmul_rn(a.h, b.h);
  float e1 = __fmaf_rn(a.h, b.h, -p1);
  e1 = __fmaf_rn(a.h, b.l, e1);
  e1 = __fmaf_rn(a.l, b.h, e1);
  const float p2 = __fmul_rn(c.h, d.h);
  float e2 = __fmaf_rn(c.h, d.h, -p2);
  e2 = __fmaf_rn(c.h, d.l, e2);
  e2 = __fmaf_rn(c.l, d.h, e2);
  float s, t;
  two_sum(p1, p2, s, t);
  return ff_make(s, __fadd_rn(t, __fadd_rn(e1, e2)));
}

// integer stored in a pool entry (exact in the high word below 2^24)
__device__ __forceinline__ int pool_index(float x) { return (int)x; }
__device__ __forceinline__ int pool_index(double x) { return (int)x; }
__device__ __forceinline__ int pool_index(ff x) { return (int)x.h; }

struct ff2 {
  ff x, y;
};

// Butterfly-internal complex sums without renormalisation, and the
// renormalisation applied when a butterfly's outputs are stored.
__device__ __forceinline__ ff2 cadd_nr(ff2 a, ff2 b) {
  ff2 r;
  r.x = ff_add_nr(a.x, b.x);
  r.y = ff_add_nr(a.y, b.y);
  return r;
}
__device__ __forceinline__ ff2 csub_nr(ff2 a, ff2 b) {
  ff2 r;
  r.x = ff_add_nr(a.x, -b.x);
  r.y = ff_add_nr(a.y, -b.y);
  return r;
}
__device__ __forceinline__ ff2 cnorm(ff2 a) {
  ff2 r;
  r.x = ff_norm(a.x);
  r.y = ff_norm(a.y);
  return r;
}

// Complex products of FP32-pair values (overloads of the generic ones).
__device__ __forceinline__ ff2 cmul(ff2 a, ff2 b) {
  ff2 r;
  r.x = ff_dot2(a.x, b.x, -a.y, b.y);
  r.y = ff_dot2(a.x, b.y, a.y, b.x);
  return r;
}
__device__ __forceinline__ ff2 cmulc(ff2 a, ff2 b) {  // a * conj(b)
  ff2 r;
  r.x = ff_dot2(a.x, b.x, a.y, b.y);
  r.y = ff_dot2(a.y, b.x, -a.x, b.y);
  return r;
}

__device__ __forceinline__ ff2 cmul_nr(ff2 a, ff2 b) {
  ff2 r;
  r.x = ff_dot2_nr(a.x, b.x, -a.y, b.y);
  r.y = ff_dot2_nr(a.x, b.y, a.y, b.x);
  return r;
}

// acc + a * c in every compute type (a contracted FMA for float and double);
// madd_nr leaves an FP32-pair result unrenormalised (butterfly-internal).
__device__ __forceinline__ ff madd(ff acc, ff a, ff c) { return ff_fma(acc, a, c); }
__device__ __forceinline__ ff madd_nr(ff acc, ff a, ff c) { return ff_fma_nr(acc, a, c); }
__device__ __forceinline__ float madd_nr(float acc, float a, float c) { return acc + a * c; }
__device__ __forceinline__ double madd_nr(double acc, double a, double c) { return acc + a * c; }
__device__ __forceinline__ float madd(float acc, float a, float c) { return acc + a * c; }
__device__ __forceinline__ double madd(double acc, double a, double c) { return acc + a * c; }

}  // namespace fcsph
