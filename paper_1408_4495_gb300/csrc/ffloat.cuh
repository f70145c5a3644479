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

}  // namespace ls
