// Float-float arithmetic: a real is the unevaluated sum hi + lo of two FP32 numbers with
// |lo| <= ulp(hi) / 2 (about 48 significant bits, FP32 exponent range).
//
// Built from the error-free transformations TwoSum (Knuth) and the FMA form of Dekker's
// TwoProduct; the add is the short double-double add of Hida, Li and Bailey (QD library,
// 2001) carried over to FP32 pairs: absolute error about 3 u^2 (|a| + |b|), u = 2^-24; the
// product drops lo*lo: relative error about 4 u^2.  Every step is written with the _rn
// intrinsics so that the compiler cannot contract or reassociate it.
//
// On GB300 FP32 instructions issue at 64 times the FP64 rate, so a transform in this
// arithmetic runs several times faster than in FP64 and is still far more accurate than
// a residual check at 1e-6 needs (the FFT of the operator adds O(u^2 log L) relative error).
#pragma once

#include <cuda_runtime.h>

namespace ls {

struct ff {
  float hi, lo;
  ff() = default;
  __host__ __device__ constexpr ff(float h, float l) : hi(h), lo(l) {}
  __host__ __device__ constexpr ff(int v) : hi((float)v), lo(0.f) {}
};

struct __align__(16) ffc {
  ff x, y;
};

#ifdef __CUDA_ARCH__
#define LS_FADD(a, b) __fadd_rn(a, b)
#define LS_FSUB(a, b) __fsub_rn(a, b)
#define LS_FMUL(a, b) __fmul_rn(a, b)
#define LS_FFMA(a, b, c) __fmaf_rn(a, b, c)
#else
#define LS_FADD(a, b) ((a) + (b))
#define LS_FSUB(a, b) ((a) - (b))
#define LS_FMUL(a, b) ((a) * (b))
#define LS_FFMA(a, b, c) std::fma(a, b, c)
#endif

// s + e == a + b exactly
__host__ __device__ __forceinline__ ff ff_two_sum(float a, float b) {
  const float s = LS_FADD(a, b);
  const float bb = LS_FSUB(s, a);
  const float e = LS_FADD(LS_FSUB(a, LS_FSUB(s, bb)), LS_FSUB(b, bb));
  return ff(s, e);
}
// s + e == a + b exactly when |a| >= |b| (or a == 0)
__host__ __device__ __forceinline__ ff ff_fast_two_sum(float a, float b) {
  const float s = LS_FADD(a, b);
  const float e = LS_FSUB(b, LS_FSUB(s, a));
  return ff(s, e);
}

__host__ __device__ __forceinline__ ff operator+(ff a, ff b) {
  const ff s = ff_two_sum(a.hi, b.hi);
  const float t = LS_FADD(s.lo, LS_FADD(a.lo, b.lo));
  return ff_fast_two_sum(s.hi, t);
}
__host__ __device__ __forceinline__ ff operator-(ff a) { return ff(-a.hi, -a.lo); }
__host__ __device__ __forceinline__ ff operator-(ff a, ff b) { return a + (-b); }
__host__ __device__ __forceinline__ ff operator*(ff a, ff b) {
  const float p = LS_FMUL(a.hi, b.hi);
  float e = LS_FFMA(a.hi, b.hi, -p);
  e = LS_FFMA(a.hi, b.lo, e);
  e = LS_FFMA(a.lo, b.hi, e);
  return ff_fast_two_sum(p, e);
}
// s is +1 or -1 where the FFT uses it (the transform sign)
__host__ __device__ __forceinline__ ff operator*(int s, ff a) { return s >= 0 ? a : -a; }
__host__ __device__ __forceinline__ ff& operator+=(ff& a, ff b) { return a = a + b; }
__host__ __device__ __forceinline__ ff& operator-=(ff& a, ff b) { return a = a - b; }
__host__ __device__ __forceinline__ ff& operator*=(ff& a, ff b) { return a = a * b; }

#undef LS_FADD
#undef LS_FSUB
#undef LS_FMUL
#undef LS_FFMA

__host__ __device__ __forceinline__ ff ff_from(double v) {
  const float h = (float)v;
  return ff(h, (float)(v - (double)h));
}
__host__ __device__ __forceinline__ double ff_to(ff a) { return (double)a.hi + (double)a.lo; }
__host__ __device__ __forceinline__ ffc ffc_from(double2 v) {
  ffc r;
  r.x = ff_from(v.x);
  r.y = ff_from(v.y);
  return r;
}
__host__ __device__ __forceinline__ double2 ffc_to(ffc v) { return make_double2(ff_to(v.x), ff_to(v.y)); }

// Renormalisation deferred: an add keeps the exact TwoSum of the leading parts and adds the
// trailing parts without the final fast-TwoSum (8 FP32 operations instead of 11), a product
// keeps the FMA TwoProduct and the cross terms without it (4 instead of 7; 3 for an FP32
// factor).  The pair then is an exact unevaluated sum whose trailing part may exceed half an
// ulp of the leading one; a chain of k such operations adds about k u^2 of its operands'
// magnitudes in error before the final lz_norm.
__device__ __forceinline__ ff lz_add(ff a, ff b) {
  const ff s = ff_two_sum(a.hi, b.hi);
  return ff(s.hi, __fadd_rn(s.lo, __fadd_rn(a.lo, b.lo)));
}
__device__ __forceinline__ ff lz_neg(ff a) { return ff(-a.hi, -a.lo); }
__device__ __forceinline__ ff lz_mul(ff a, ff b) {
  const float p = __fmul_rn(a.hi, b.hi);
  float e = __fmaf_rn(a.hi, b.hi, -p);
  e = __fmaf_rn(a.hi, b.lo, e);
  e = __fmaf_rn(a.lo, b.hi, e);
  return ff(p, e);
}
__device__ __forceinline__ ff lz_mul_f(ff a, float b) {
  const float p = __fmul_rn(a.hi, b);
  return ff(p, __fmaf_rn(a.lo, b, __fmaf_rn(a.hi, b, -p)));
}
__device__ __forceinline__ ff lz_norm(ff a) { return ff_fast_two_sum(a.hi, a.lo); }

// Conversions between FP64 and FP32 pairs on the integer and FP32 pipes.  GB300 runs FP64
// instructions (conversions to and from FP64 among them) at a small fraction of its FP32
// rate, so a streaming kernel that converts every element through FP64 is bound by them.
// Both are written from the IEEE 754 binary32 / binary64 layouts (1 sign, 8 / 11 exponent
// and 23 / 52 fraction bits, exponent biases 127 / 1023).

// the exact FP64 value of an FP32 number: normal numbers by moving the fields, zeros, FP32
// subnormals, infinities and NaNs by the FP64 conversion
__device__ __forceinline__ double f64_of(float f) {
  const unsigned b = __float_as_uint(f);
  const unsigned e = (b >> 23) & 0xffu;
  if (e - 1u < 254u) {
    const unsigned long long sign = (unsigned long long)(b >> 31) << 63;
    const unsigned long long exp = (unsigned long long)(e + (1023u - 127u)) << 52;
    const unsigned long long frac = (unsigned long long)(b & 0x7fffffu) << 29;
    return __longlong_as_double((long long)(sign | exp | frac));
  }
  if ((b & 0x7fffffffu) == 0u) return __longlong_as_double((long long)((unsigned long long)(b >> 31) << 63));
  return (double)f;
}
// hi + lo of a float-float as FP64: one FP64 add (exact when the pair is normalized)
__device__ __forceinline__ double ff_to_f64(ff a) { return f64_of(a.hi) + f64_of(a.lo); }
__device__ __forceinline__ double2 ffc_to_f64(ffc v) { return make_double2(ff_to_f64(v.x), ff_to_f64(v.y)); }

// an FP64 number as a float-float: hi = its leading 24 significant bits (truncated), lo =
// the next 23 bits (truncated), so |x - (hi + lo)| < 2^-46 |x|; lo is built as an exact
// FP32 integer (the magic-number form) scaled by a power of two.  Outside
// 2^-74 <= |x| < 2^128 (where lo or hi would leave the FP32 normal range) and for
// infinities and NaNs the FP64 conversion is used; zeros stay zeros.  |lo| may reach
// ulp(hi) rather than ulp(hi) / 2: the operations above take such pairs as they are.
__device__ __forceinline__ ff ff_of_f64(double x) {
  const unsigned long long b = (unsigned long long)__double_as_longlong(x);
  const unsigned e = (unsigned)(b >> 52) & 0x7ffu;
  const unsigned sign = (unsigned)(b >> 63) << 31;
  if (e == 0u) return ff(__uint_as_float(sign), 0.f);
  if (e - 949u < 1150u - 949u + 1u) {
    const unsigned hi = sign | ((e - (1023u - 127u)) << 23) | (unsigned)((b >> 29) & 0x7fffffu);
    const unsigned r = (unsigned)(b >> 6) & 0x7fffffu;  // fraction bits 28..6
    // r as an FP32 integer: 2^23 + r has the exponent field of 2^23 and fraction r
    const float rf = __fsub_rn(__uint_as_float(0x4b000000u | r), 8388608.0f);
    // lo = r * 2^(E - 46), E = e - 1023 the unbiased exponent of x
    const float scale = __uint_as_float((e - (1023u + 46u - 127u)) << 23);
    return ff(__uint_as_float(hi), __uint_as_float(__float_as_uint(__fmul_rn(rf, scale)) | sign));
  }
  return ff_from(x);
}
__device__ __forceinline__ ffc ffc_of_f64(double2 v) {
  ffc r;
  r.x = ff_of_f64(v.x);
  r.y = ff_of_f64(v.y);
  return r;
}

}  // namespace ls
