// dg_dfloat.cuh -- "double-float": a value held as the unevaluated sum hi + lo of two FP32 numbers
// (|lo| <= ulp(hi)/2), giving about 48 significand bits from FP32 arithmetic only.
//
// GB300 issues FP32 FMAs at 62x the rate of FP64 FMAs, so an FP64-accurate operator evaluated with
// these pairs runs on the FP32 pipes.  The arithmetic is built from the classical error-free
// transformations: Knuth's TwoSum, Dekker's Fast2Sum and the FMA-based TwoProduct (the product's
// rounding error is fma(a, b, -a*b) exactly).  Each operation returns a normalised pair; the
// relative error of add, mul and fma is a small multiple of 2^-48 (away from cancellation, where the
// error is relative to the operands' magnitude instead).  The exponent range is FP32's, which the
// operator's values (O(1e-8) .. O(1e8)) stay well inside.
#pragma once

#include <cuda_runtime.h>

namespace dgk {

// keep the built-in float / double fma visible next to the pair overload below
using ::fma;

struct dfl {
  float hi, lo;
  __host__ __device__ dfl() : hi(0.f), lo(0.f) {}
  __host__ __device__ dfl(int v) : hi((float)v), lo(0.f) {}
  __host__ __device__ dfl(float h, float l) : hi(h), lo(l) {}
  // split a double into its nearest FP32 and the FP32 of the remainder (exact to ~2^-48 relative)
  __host__ __device__ explicit dfl(double v) {
    hi = (float)v;
    lo = (float)(v - (double)hi);
  }
  __host__ __device__ explicit operator double() const { return (double)hi + (double)lo; }
};

__device__ __forceinline__ void two_sum(float a, float b, float& s, float& e) {
  s = __fadd_rn(a, b);
  const float bb = __fsub_rn(s, a);
  e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
}

// requires |a| >= |b| (or a == 0)
__device__ __forceinline__ void fast_two_sum(float a, float b, float& s, float& e) {
  s = __fadd_rn(a, b);
  e = __fsub_rn(b, __fsub_rn(s, a));
}

__device__ __forceinline__ dfl operator+(dfl a, dfl b) {
  float s, e;
  two_sum(a.hi, b.hi, s, e);
  e = __fadd_rn(e, __fadd_rn(a.lo, b.lo));
  dfl r;
  fast_two_sum(s, e, r.hi, r.lo);
  return r;
}

__device__ __forceinline__ dfl operator-(dfl a) { return dfl(-a.hi, -a.lo); }
__device__ __forceinline__ dfl operator-(dfl a, dfl b) { return a + (-b); }

__device__ __forceinline__ dfl operator*(dfl a, dfl b) {
  const float p = __fmul_rn(a.hi, b.hi);
  float e = __fmaf_rn(a.hi, b.hi, -p);
  e = __fmaf_rn(a.hi, b.lo, e);
  e = __fmaf_rn(a.lo, b.hi, e);
  dfl r;
  fast_two_sum(p, e, r.hi, r.lo);
  return r;
}

// a * b + c with one final normalisation
__device__ __forceinline__ dfl fma(dfl a, dfl b, dfl c) {
  const float p = __fmul_rn(a.hi, b.hi);
  float e = __fmaf_rn(a.hi, b.hi, -p);
  e = __fmaf_rn(a.hi, b.lo, e);
  e = __fmaf_rn(a.lo, b.hi, e);
  float s, t;
  two_sum(p, c.hi, s, t);
  t = __fadd_rn(t, __fadd_rn(c.lo, e));
  dfl r;
  fast_two_sum(s, t, r.hi, r.lo);
  return r;
}

__device__ __forceinline__ dfl& operator+=(dfl& a, dfl b) {
  a = a + b;
  return a;
}
__device__ __forceinline__ dfl& operator*=(dfl& a, dfl b) {
  a = a * b;
  return a;
}

// sign tests compare the leading part (hi carries the sign of the pair)
__device__ __forceinline__ bool operator>=(dfl a, dfl b) { return a.hi > b.hi || (a.hi == b.hi && a.lo >= b.lo); }
__device__ __forceinline__ bool operator>(dfl a, dfl b) { return a.hi > b.hi || (a.hi == b.hi && a.lo > b.lo); }

}  // namespace dgk
