// Double-float ("float-float") arithmetic for the FP64 spectral passes.
//
// A value is the unevaluated sum hi + lo of two floats with |lo| <= ulp(hi)/2,
// about 48 significant bits.  The operations are built from two error-free
// transformations on floats - Knuth's two-sum (s + e = a + b exactly) and
// the two-product through a fused multiply-add (p + e = a b exactly) - as in
// Dekker's double-length arithmetic (T. J. Dekker, "A floating-point technique
// for extending the available precision", Numer. Math. 18, 1971).  Every
// float operation goes through the __f*_rn intrinsics, which the compiler
// neither contracts into fused multiply-adds nor reassociates, so the
// transformations stay exact.
//
// Why: GB300 runs FP64 at 1/64 of its FP32 rate, so a radix-2 butterfly in
// double-float (about ten times the instructions of the FP64 one) still runs
// several times faster than in FP64.  The addition is the "sloppy" form: its
// error is bounded by about 2^-47 (|a| + |b|), a normwise bound, which is what
// the error analysis of an FFT (a sum of such butterflies) needs.  The
// exponent range is float's: a field whose values all lie below about 1e-30
// (where lo becomes subnormal) or above about 1e38 in magnitude loses its
// precision or overflows; the fields of the method are of order one.
#pragma once

#include "wt_dev.cuh"

namespace wt {

struct ff {
  float hi, lo;
  ff() = default;
  __device__ __forceinline__ constexpr ff(float h, float l) : hi(h), lo(l) {}
  __device__ __forceinline__ explicit ff(int v) : hi((float)v), lo(0.f) {}   // exact for |v| < 2^24
};
struct ff2 {
  ff x, y;
};
template <> struct C2<ff> { using type = ff2; };

__device__ __forceinline__ ff ff_fast_two_sum(float a, float b) {   // |a| >= |b| (or a = 0)
  const float s = __fadd_rn(a, b);
  return ff(s, __fsub_rn(b, __fsub_rn(s, a)));
}
__device__ __forceinline__ ff ff_two_sum(float a, float b) {
  const float s = __fadd_rn(a, b);
  const float bb = __fsub_rn(s, a);
  return ff(s, __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb)));
}
__device__ __forceinline__ ff operator+(ff a, ff b) {
  const ff s = ff_two_sum(a.hi, b.hi);
  return ff_fast_two_sum(s.hi, __fadd_rn(s.lo, __fadd_rn(a.lo, b.lo)));
}
__device__ __forceinline__ ff operator-(ff a) { return ff(-a.hi, -a.lo); }
__device__ __forceinline__ ff operator-(ff a, ff b) { return a + (-b); }
__device__ __forceinline__ ff operator*(ff a, ff b) {
  const float p = __fmul_rn(a.hi, b.hi);
  float e = __fmaf_rn(a.hi, b.hi, -p);                 // exact low part of hi*hi
  e = __fmaf_rn(a.hi, b.lo, e);
  e = __fmaf_rn(a.lo, b.hi, e);
  return ff_fast_two_sum(p, e);
}

template <> __device__ __forceinline__ ff2 mk<ff>(ff re, ff im) {
  ff2 r;
  r.x = re;
  r.y = im;
  return r;
}

// Conversions between the storage type T and the arithmetic type A (the
// identity for float and double, double <-> double-float for the FP64
// passes that run in double-float).
template <typename A, typename T> __device__ __forceinline__ A to_arith(T v);
template <> __device__ __forceinline__ float to_arith<float, float>(float v) { return v; }
template <> __device__ __forceinline__ double to_arith<double, double>(double v) { return v; }
template <> __device__ __forceinline__ ff to_arith<ff, double>(double v) {
  const float h = __double2float_rn(v);
  return ff(h, __double2float_rn(v - (double)h));
}
template <typename T, typename A> __device__ __forceinline__ T from_arith(A v);
template <> __device__ __forceinline__ float from_arith<float, float>(float v) { return v; }
template <> __device__ __forceinline__ double from_arith<double, double>(double v) { return v; }
template <> __device__ __forceinline__ double from_arith<double, ff>(ff v) {
  return (double)v.hi + (double)v.lo;
}

// Constants in the arithmetic type.
template <typename A> __device__ __forceinline__ A a_zero();
template <> __device__ __forceinline__ float a_zero<float>() { return 0.f; }
template <> __device__ __forceinline__ double a_zero<double>() { return 0.0; }
template <> __device__ __forceinline__ ff a_zero<ff>() { return ff(0.f, 0.f); }
template <typename A> __device__ __forceinline__ A a_half();
template <> __device__ __forceinline__ float a_half<float>() { return 0.5f; }
template <> __device__ __forceinline__ double a_half<double>() { return 0.5; }
template <> __device__ __forceinline__ ff a_half<ff>() { return ff(0.5f, 0.f); }
template <typename A> __device__ __forceinline__ A a_int(int v);             // exact for |v| < 2^24
template <> __device__ __forceinline__ float a_int<float>(int v) { return (float)v; }
template <> __device__ __forceinline__ double a_int<double>(int v) { return (double)v; }
template <> __device__ __forceinline__ ff a_int<ff>(int v) { return ff(v); }

__device__ __forceinline__ ff shfl_xor_a(ff v, int m) {
  return ff(__shfl_xor_sync(0xffffffffu, v.hi, m), __shfl_xor_sync(0xffffffffu, v.lo, m));
}
__device__ __forceinline__ float shfl_xor_a(float v, int m) { return __shfl_xor_sync(0xffffffffu, v, m); }

}  // namespace wt
