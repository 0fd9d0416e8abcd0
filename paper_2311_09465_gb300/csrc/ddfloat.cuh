// Double-float ("float-float") arithmetic: a value is the unevaluated sum
// hi + lo of two FP32 numbers with |lo| <= ulp(hi)/2, about 48 significant
// bits.  Built from error-free transformations:
//   TwoSum (Knuth, TAOCP vol. 2, 4.2.2): s + e = a + b exactly;
//   FastTwoSum (Dekker 1971): the same when |a| >= |b|;
//   TwoProd with a fused multiply-add: p + e = a * b exactly.
// sqrt and the reciprocal take one Newton correction from the FP32 value.
// Sums carry an absolute error of about 2^-46 of the largest operand, which
// is what the FP64 tau refinement needs; the exponent range is FP32's, so the
// caller scales its data to magnitudes near 1 first.
#pragma once

namespace ts {

struct dd {
  float hi, lo;
};

__device__ __forceinline__ dd dd_make(float h) { return {h, 0.f}; }

__device__ __forceinline__ dd dd_from_double(double x) {
  const float h = (float)x;
  return {h, (float)(x - (double)h)};
}

__device__ __forceinline__ double dd_to_double(dd a) { return (double)a.hi + (double)a.lo; }

__device__ __forceinline__ void two_sum(float a, float b, float& s, float& e) {
  s = a + b;
  const float bb = s - a;
  e = (a - (s - bb)) + (b - bb);
}

__device__ __forceinline__ void fast_two_sum(float a, float b, float& s, float& e) {
  s = a + b;
  e = b - (s - a);
}

__device__ __forceinline__ dd dd_neg(dd a) { return {-a.hi, -a.lo}; }

__device__ __forceinline__ dd dd_add(dd a, dd b) {
  float s, e;
  two_sum(a.hi, b.hi, s, e);
  e += a.lo + b.lo;
  dd r;
  fast_two_sum(s, e, r.hi, r.lo);
  return r;
}

__device__ __forceinline__ dd dd_add_f(dd a, float b) {
  float s, e;
  two_sum(a.hi, b, s, e);
  e += a.lo;
  dd r;
  fast_two_sum(s, e, r.hi, r.lo);
  return r;
}

// a * b + c
__device__ __forceinline__ dd dd_fma(dd a, dd b, dd c) {
  const float p = a.hi * b.hi;
  float e = fmaf(a.hi, b.hi, -p);
  e = fmaf(a.hi, b.lo, e);
  e = fmaf(a.lo, b.hi, e);
  float s, t;
  two_sum(p, c.hi, s, t);
  t += e + c.lo;
  dd r;
  fast_two_sum(s, t, r.hi, r.lo);
  return r;
}

// a * b + c for FP32 a, b (the product is exact as p + e)
__device__ __forceinline__ dd dd_fma_ff(float a, float b, dd c) {
  const float p = a * b;
  const float e = fmaf(a, b, -p);
  float s, t;
  two_sum(p, c.hi, s, t);
  t += e + c.lo;
  dd r;
  fast_two_sum(s, t, r.hi, r.lo);
  return r;
}

// a * b + c for an FP32 a
__device__ __forceinline__ dd dd_fma_fd(float a, dd b, dd c) {
  const float p = a * b.hi;
  float e = fmaf(a, b.hi, -p);
  e = fmaf(a, b.lo, e);
  float s, t;
  two_sum(p, c.hi, s, t);
  t += e + c.lo;
  dd r;
  fast_two_sum(s, t, r.hi, r.lo);
  return r;
}

__device__ __forceinline__ dd dd_mul(dd a, dd b) {
  const float p = a.hi * b.hi;
  float e = fmaf(a.hi, b.hi, -p);
  e = fmaf(a.hi, b.lo, e);
  e = fmaf(a.lo, b.hi, e);
  dd r;
  fast_two_sum(p, e, r.hi, r.lo);
  return r;
}

__device__ __forceinline__ dd dd_scale(dd a, float pow2) { return {a.hi * pow2, a.lo * pow2}; }

// sqrt(a) for a > 0: s0 = sqrt(hi), then s0 + (a - s0^2) / (2 s0)
__device__ __forceinline__ dd dd_sqrt(dd a) {
  const float s0 = sqrtf(a.hi);
  const float p = s0 * s0;
  const float e = fmaf(s0, s0, -p);
  const float rem = ((a.hi - p) - e) + a.lo;
  dd r;
  fast_two_sum(s0, rem / (2.f * s0), r.hi, r.lo);
  return r;
}

// 1 / a: y0 = 1/hi, then y0 + y0 (1 - a y0)
__device__ __forceinline__ dd dd_rcp(dd a) {
  const float y0 = 1.f / a.hi;
  const float p = a.hi * y0;
  const float e = fmaf(a.hi, y0, -p);
  const float rem = ((1.f - p) - e) - a.lo * y0;
  dd r;
  fast_two_sum(y0, y0 * rem, r.hi, r.lo);
  return r;
}

// A double-float value type with arithmetic operators, so that kernels
// templated on their arithmetic type can run in double-float: storage stays
// FP64 (converted on load and store), every operation runs on the FP32 pipe.
struct ddv {
  dd v;
  __host__ __device__ ddv() : v{0.f, 0.f} {}
  __host__ __device__ ddv(double x) {
    const float h = (float)x;
    v = {h, (float)(x - (double)h)};
  }
  __host__ __device__ ddv(float x) : v{x, 0.f} {}
  __host__ __device__ ddv(int x) : v{(float)x, 0.f} {}   // exact for |x| < 2^24
  __device__ ddv(dd x) : v(x) {}
  __host__ __device__ explicit operator double() const { return (double)v.hi + (double)v.lo; }
};
__device__ __forceinline__ ddv operator+(ddv a, ddv b) { return ddv(dd_add(a.v, b.v)); }
__device__ __forceinline__ ddv operator-(ddv a) { return ddv(dd_neg(a.v)); }
__device__ __forceinline__ ddv operator-(ddv a, ddv b) { return ddv(dd_add(a.v, dd_neg(b.v))); }
__device__ __forceinline__ ddv operator*(ddv a, ddv b) { return ddv(dd_mul(a.v, b.v)); }
__device__ __forceinline__ ddv operator/(ddv a, ddv b) { return ddv(dd_mul(a.v, dd_rcp(b.v))); }
__device__ __forceinline__ ddv& operator+=(ddv& a, ddv b) { a.v = dd_add(a.v, b.v); return a; }
__device__ __forceinline__ bool operator!=(ddv a, ddv b) { return a.v.hi != b.v.hi || a.v.lo != b.v.lo; }

}  // namespace ts
