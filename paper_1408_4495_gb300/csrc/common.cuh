// Shared device/host helpers of libls: complex arithmetic on float2/double2, error plumbing.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <cmath>
#include <cstdio>
#include <string>

namespace ls {

template <typename R> struct CxOf;
template <> struct CxOf<float> { using T = float2; };
template <> struct CxOf<double> { using T = double2; };
template <typename R> using cx = typename CxOf<R>::T;

template <typename C> struct RealOf;
template <> struct RealOf<float2> { using T = float; };
template <> struct RealOf<double2> { using T = double; };

__host__ __device__ __forceinline__ float2 cmake(float x, float y) { return make_float2(x, y); }
__host__ __device__ __forceinline__ double2 cmake(double x, double y) { return make_double2(x, y); }
template <typename C> __host__ __device__ __forceinline__ C czero() { C z; z.x = 0; z.y = 0; return z; }

template <typename C> __host__ __device__ __forceinline__ C cadd(C a, C b) { a.x += b.x; a.y += b.y; return a; }
template <typename C> __host__ __device__ __forceinline__ C csub(C a, C b) { a.x -= b.x; a.y -= b.y; return a; }
template <typename C> __host__ __device__ __forceinline__ C cmul(C a, C b) {
  C r; r.x = a.x * b.x - a.y * b.y; r.y = a.x * b.y + a.y * b.x; return r;
}
// a * conj(b)
template <typename C> __host__ __device__ __forceinline__ C cmulc(C a, C b) {
  C r; r.x = a.x * b.x + a.y * b.y; r.y = a.y * b.x - a.x * b.y; return r;
}
// conj(a) * b
template <typename C> __host__ __device__ __forceinline__ C cconjmul(C a, C b) {
  C r; r.x = a.x * b.x + a.y * b.y; r.y = a.x * b.y - a.y * b.x; return r;
}
template <typename C> __host__ __device__ __forceinline__ C cconj(C a) { a.y = -a.y; return a; }
template <typename C, typename R> __host__ __device__ __forceinline__ C cscale(C a, R s) { a.x *= s; a.y *= s; return a; }
template <typename C> __host__ __device__ __forceinline__ typename RealOf<C>::T cabs2(C a) { return a.x * a.x + a.y * a.y; }
// a / b
template <typename C> __host__ __device__ __forceinline__ C cdiv(C a, C b) {
  typename RealOf<C>::T den = b.x * b.x + b.y * b.y;
  C r; r.x = (a.x * b.x + a.y * b.y) / den; r.y = (a.y * b.x - a.x * b.y) / den; return r;
}
__host__ __device__ __forceinline__ float rfma(float a, float b, float c) { return fmaf(a, b, c); }
__host__ __device__ __forceinline__ double rfma(double a, double b, double c) { return fma(a, b, c); }
// multiply-subtract acc - a*b and multiply-add acc + a*b: each component is two chained
// FMAs into the accumulator (four instructions per complex product instead of six)
template <typename C> __host__ __device__ __forceinline__ C cfms(C acc, C a, C b) {
  acc.x = rfma(-a.x, b.x, acc.x); acc.x = rfma(a.y, b.y, acc.x);
  acc.y = rfma(-a.x, b.y, acc.y); acc.y = rfma(-a.y, b.x, acc.y);
  return acc;
}
template <typename C> __host__ __device__ __forceinline__ C cfma(C acc, C a, C b) {
  acc.x = rfma(a.x, b.x, acc.x); acc.x = rfma(-a.y, b.y, acc.x);
  acc.y = rfma(a.x, b.y, acc.y); acc.y = rfma(a.y, b.x, acc.y);
  return acc;
}

template <typename Cto, typename Cfrom> __host__ __device__ __forceinline__ Cto ccast(Cfrom a) {
  Cto r; r.x = (typename RealOf<Cto>::T)a.x; r.y = (typename RealOf<Cto>::T)a.y; return r;
}

// Status codes mirror ls_status in include/ls.h.
enum Status { OK = 0, EINVAL_ = 1, ENOMEM_ = 2, ECUDA_ = 3, ENOCONV_ = 4, ESTATE_ = 5, ETIMEOUT_ = 6, EBUFFER_ = 7 };

struct Error {
  int code;
  std::string msg;
};

}  // namespace ls

// Evaluates a CUDA call; on failure returns an ls::Error-compatible status through the
// enclosing function's error sink `err` (a std::string*) and returns LS_ECUDA.
#define LS_CUDA(call)                                                                      \
  do {                                                                                     \
    cudaError_t e_ = (call);                                                               \
    if (e_ != cudaSuccess) {                                                               \
      char b_[512];                                                                        \
      snprintf(b_, sizeof b_, "%s failed: %s (%s:%d)", #call, cudaGetErrorString(e_),      \
               __FILE__, __LINE__);                                                        \
      throw ls::Error{ls::ECUDA_, b_};                                                     \
    }                                                                                      \
  } while (0)

#define LS_CHECK_LAUNCH() LS_CUDA(cudaGetLastError())

#define LS_FAIL(code, ...)                                                                 \
  do {                                                                                     \
    char b_[512];                                                                          \
    snprintf(b_, sizeof b_, __VA_ARGS__);                                                  \
    throw ls::Error{(code), b_};                                                           \
  } while (0)
