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

// Dot-product accumulator: sum_i a_i b_i with one normalisation at the end.  The leading sum s is
// advanced with TwoSum (exact: s_new + err = s + p_hi), and every rounding error and low-order product
// part goes into t, so each term costs 12 FP32 operations instead of a full pair fma (15).
struct dacc {
  float s, t;
};

__device__ __forceinline__ dacc dot_begin(dfl a, dfl b) {
  const float p = __fmul_rn(a.hi, b.hi);
  float e = __fmaf_rn(a.hi, b.hi, -p);
  e = __fmaf_rn(a.hi, b.lo, e);
  e = __fmaf_rn(a.lo, b.hi, e);
  return dacc{p, e};
}

__device__ __forceinline__ void dot_add(dacc& c, dfl a, dfl b) {
  const float p = __fmul_rn(a.hi, b.hi);
  float e = __fmaf_rn(a.hi, b.hi, -p);
  e = __fmaf_rn(a.hi, b.lo, e);
  e = __fmaf_rn(a.lo, b.hi, e);
  float s, err;
  two_sum(c.s, p, s, err);
  c.s = s;
  c.t = __fadd_rn(c.t, __fadd_rn(err, e));
}

__device__ __forceinline__ dfl dot_end(const dacc& c) {
  dfl r;
  fast_two_sum(c.s, c.t, r.hi, r.lo);
  return r;
}

// FP64 <-> pair conversions with integer operations.  On GB300 the F2F conversions between FP32 and
// FP64 run on the (slow) FP64 pipe; splitting the bit pattern keeps the vector loads and stores off it.
// v = hi + lo with hi = v truncated to 24 significant bits (exact) and lo = the remaining <= 29 bits
// rounded to FP32 (relative error <= 2^-47 of v).  Values outside the normal FP32 exponent range of
// the remainder take the conversion instructions instead.
__device__ __forceinline__ dfl dfl_from_double(double v) {
  const unsigned long long b = (unsigned long long)__double_as_longlong(v);
  const int e = (int)((b >> 52) & 0x7FF);
  const int fe = e - 1023 + 127;          // FP32 exponent of hi
  const int le = e - 1075 + 127;          // FP32 exponent of 2^(e - 1075), the weight of the remainder's bit 0
  if (fe <= 0 || fe >= 255 || le <= 0) {  // zero, tiny or huge: exact-enough conversion path
    const float h = __double2float_rn(v);
    return dfl(h, __double2float_rn(v - (double)h));
  }
  const unsigned sign = (unsigned)(b >> 63) << 31;
  const unsigned hb = sign | ((unsigned)fe << 23) | (unsigned)((b >> 29) & 0x7FFFFF);
  const unsigned rem = (unsigned)(b & ((1ull << 29) - 1));
  const float scale = __uint_as_float((unsigned)le << 23);
  // rem as FP32 without a conversion instruction: its top 23 bits through the 2^23 bias trick (exact),
  // then one fma adds the low 6 bits with a single rounding (= round-to-nearest of rem)
  const float top = __fsub_rn(__uint_as_float(0x4B000000u | (rem >> 6)), 8388608.0f);
  const float low = __fsub_rn(__uint_as_float(0x4B000000u | (rem & 63u)), 8388608.0f);
  const float remf = __fmaf_rn(top, 64.0f, low);
  const float lo = __uint_as_float(__float_as_uint(__fmul_rn(remf, scale)) | sign);
  return dfl(__uint_as_float(hb), lo);
}

// FP32 -> FP64 widening by placing the bits (normal or zero inputs; denormal FP32 values flush to 0)
__device__ __forceinline__ double widen(float f) {
  const unsigned u = __float_as_uint(f);
  const unsigned ex = (u >> 23) & 0xFF;
  if (ex == 0) return 0.0;
  if (ex == 255) return (double)f;  // Inf / NaN keep their meaning
  const unsigned long long sign = (unsigned long long)(u >> 31) << 63;
  const unsigned long long ee = (unsigned long long)(ex - 127 + 1023) << 52;
  const unsigned long long mm = (unsigned long long)(u & 0x7FFFFF) << 29;
  return __longlong_as_double((long long)(sign | ee | mm));
}

// hi + lo rounded once to FP64 (one FP64 add)
__device__ __forceinline__ double dfl_to_double(dfl a) { return widen(a.hi) + widen(a.lo); }

// sign tests compare the leading part (hi carries the sign of the pair)
__device__ __forceinline__ bool operator>=(dfl a, dfl b) { return a.hi > b.hi || (a.hi == b.hi && a.lo >= b.lo); }
__device__ __forceinline__ bool operator>(dfl a, dfl b) { return a.hi > b.hi || (a.hi == b.hi && a.lo > b.lo); }

}  // namespace dgk
