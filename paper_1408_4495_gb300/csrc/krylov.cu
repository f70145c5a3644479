// FP64 Krylov kernels of the GMRES iteration (Sec. 3.3), batched over right-hand sides:
// classical Gram-Schmidt with one reorthogonalisation (CGS2) against the Arnoldi basis,
// norms, scaling, the solution update u += Z y and the residual g - A u.  Every vector is
// laid out [nrhs][N] (complex128); reductions are two-stage with a fixed summation order,
// so results do not depend on scheduling.
#include <type_traits>

#include "common.cuh"
#include "ffloat.cuh"
#include "krylov.h"
#include "prof.h"

namespace ls {

constexpr int KT = 256;

template <typename T> __device__ __forceinline__ double2 to64(T v) { return make_double2((double)v.x, (double)v.y); }

__device__ __forceinline__ double2 block_sum(double2 v, double2* sh) {
  for (int o = 16; o > 0; o >>= 1) {
    v.x += __shfl_down_sync(0xffffffffu, v.x, o);
    v.y += __shfl_down_sync(0xffffffffu, v.y, o);
  }
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  if (lane == 0) sh[wid] = v;
  __syncthreads();
  double2 r = make_double2(0, 0);
  if (threadIdx.x == 0)
    for (int i = 0; i < (int)(blockDim.x >> 5); ++i) { r.x += sh[i].x; r.y += sh[i].y; }
  __syncthreads();
  return r;
}

// partial[(rhs * nv + j) * nblk + blk] = sum over the block's chunk of conj(V_j) w
template <typename Cw>
__global__ void __launch_bounds__(KT) k_dots(const double2* const* __restrict__ V, int nv, const Cw* __restrict__ w,
                                             long N, double2* __restrict__ partial, int nblk) {
  __shared__ double2 sh[KT / 32];
  const int rhs = blockIdx.y, blk = blockIdx.x;
  const long chunk = (N + nblk - 1) / nblk;
  const long i0 = blk * chunk, i1 = min(N, i0 + chunk);
  const Cw* wr = w + (size_t)rhs * N;
  for (int j = 0; j < nv; ++j) {
    const double2* vr = V[j] + (size_t)rhs * N;
    double2 acc = make_double2(0, 0);
    for (long i = i0 + threadIdx.x; i < i1; i += KT) acc = cfma(acc, cconj(vr[i]), to64(wr[i]));
    const double2 s = block_sum(acc, sh);
    if (threadIdx.x == 0) partial[((size_t)rhs * nv + j) * nblk + blk] = s;
  }
}

struct ffc;
__device__ void store_ff_pair(void* outf, size_t i, double2 v);

// out[rhs * ostride + j] = sum_blk partial  (ordered), optionally accumulated into out; with
// outf, also the result as FP32 pairs at the same index
__global__ void k_reduce(const double2* __restrict__ partial, int nv, int nrhs, int nblk, double2* out, int ostride,
                         int accumulate, void* outf = nullptr) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= nv * nrhs) return;
  const int rhs = t / nv, j = t % nv;
  double2 s = make_double2(0, 0);
  const double2* p = partial + ((size_t)rhs * nv + j) * nblk;
  for (int b = 0; b < nblk; ++b) { s.x += p[b].x; s.y += p[b].y; }
  double2* o = out + (size_t)rhs * ostride + j;
  if (accumulate) { o->x += s.x; o->y += s.y; }
  else *o = s;
  if (outf) store_ff_pair(outf, (size_t)rhs * ostride + j, *o);
}

// wout = win - sum_j V_j h[rhs][j]
template <typename Cw>
__global__ void k_sub_proj(const double2* const* __restrict__ V, int nv, const Cw* __restrict__ win, double2* wout,
                           const double2* __restrict__ h, int hstride, long N, int nrhs) {
  const long tot = N * nrhs;
  for (long idx = blockIdx.x * (long)blockDim.x + threadIdx.x; idx < tot; idx += (long)gridDim.x * blockDim.x) {
    const long rhs = idx / N;
    double2 acc = to64(win[idx]);
    const double2* hr = h + rhs * hstride;
    for (int j = 0; j < nv; ++j) acc = cfms(acc, V[j][idx], hr[j]);
    wout[idx] = acc;
  }
}

// partial[rhs * nblk + blk] = sum |w|^2 over the chunk (as the .x of a double2)
template <typename Cw>
__global__ void __launch_bounds__(KT) k_norm2(const Cw* __restrict__ w, long N, double2* partial, int nblk) {
  __shared__ double2 sh[KT / 32];
  const int rhs = blockIdx.y, blk = blockIdx.x;
  const long chunk = (N + nblk - 1) / nblk;
  const long i0 = blk * chunk, i1 = min(N, i0 + chunk);
  const Cw* wr = w + (size_t)rhs * N;
  double2 acc = make_double2(0, 0);
  for (long i = i0 + threadIdx.x; i < i1; i += KT) {
    const double2 v = to64(wr[i]);
    acc.x += v.x * v.x + v.y * v.y;
  }
  const double2 s = block_sum(acc, sh);
  if (threadIdx.x == 0) partial[(size_t)rhs * nblk + blk] = s;
}

// out[rhs] = w[rhs] * scale[rhs]  (scale 0 clears)
__global__ void k_scale(const double2* __restrict__ w, double2* out, const double* __restrict__ scale, long N, int nrhs) {
  const long tot = N * nrhs;
  for (long idx = blockIdx.x * (long)blockDim.x + threadIdx.x; idx < tot; idx += (long)gridDim.x * blockDim.x) {
    const double s = scale[idx / N];
    double2 v = w[idx];
    v.x *= s;
    v.y *= s;
    out[idx] = v;
  }
}

// u[rhs] += sum_j Z_j[rhs] y[rhs][j]
template <typename Cz>
__global__ void k_update_u(const Cz* const* __restrict__ Z, int nz, const double2* __restrict__ y, int ystride,
                           double2* u, long N, int nrhs) {
  const long tot = N * nrhs;
  for (long idx = blockIdx.x * (long)blockDim.x + threadIdx.x; idx < tot; idx += (long)gridDim.x * blockDim.x) {
    const long rhs = idx / N;
    double2 acc = u[idx];
    const double2* yr = y + rhs * ystride;
    for (int j = 0; j < nz; ++j) acc = cfma(acc, to64(Z[j][idx]), yr[j]);
    u[idx] = acc;
  }
}

// r = g - Au
__global__ void k_residual(const double2* __restrict__ g, const double2* __restrict__ Au, double2* r, long tot) {
  for (long idx = blockIdx.x * (long)blockDim.x + threadIdx.x; idx < tot; idx += (long)gridDim.x * blockDim.x)
    r[idx] = csub(g[idx], Au[idx]);
}

template <typename Cin, typename Cout>
__global__ void k_cast(const Cin* __restrict__ in, Cout* __restrict__ out, long tot) {
  for (long idx = blockIdx.x * (long)blockDim.x + threadIdx.x; idx < tot; idx += (long)gridDim.x * blockDim.x)
    out[idx] = ccast<Cout>(in[idx]);
}

static unsigned grid_for(long tot) {
  long b = (tot + 255) / 256;
  if (b > 152L * 32) b = 152L * 32;
  return (unsigned)(b < 1 ? 1 : b);
}

int dots_blocks(long N) {
  long b = (N + 4095) / 4096;
  if (b > 64) b = 64;
  return (int)(b < 1 ? 1 : b);
}

template <typename Cw>
void dots(const double2* const* V, int nv, const Cw* w, long N, int nrhs, double2* partial, double2* out, int ostride,
          bool accumulate, cudaStream_t st) {
  const int nblk = dots_blocks(N);
  LS_LAUNCH("kr_dots", st, k_dots<Cw><<<dim3(nblk, nrhs), KT, 0, st>>>(V, nv, w, N, partial, nblk));
  LS_LAUNCH("kr_reduce", st,
            k_reduce<<<(nv * nrhs + 127) / 128, 128, 0, st>>>(partial, nv, nrhs, nblk, out, ostride, accumulate ? 1 : 0));
}

template <typename Cw>
void sub_proj(const double2* const* V, int nv, const Cw* win, double2* wout, const double2* h, int hstride, long N,
              int nrhs, cudaStream_t st) {
  LS_LAUNCH("kr_sub_proj", st, k_sub_proj<Cw><<<grid_for(N * nrhs), 256, 0, st>>>(V, nv, win, wout, h, hstride, N, nrhs));
}

template <typename Cw>
void norms2(const Cw* w, long N, int nrhs, double2* partial, double2* out, int ostride, cudaStream_t st) {
  const int nblk = dots_blocks(N);
  LS_LAUNCH("kr_norm2", st, k_norm2<Cw><<<dim3(nblk, nrhs), KT, 0, st>>>(w, N, partial, nblk));
  LS_LAUNCH("kr_reduce", st, k_reduce<<<(nrhs + 127) / 128, 128, 0, st>>>(partial, 1, nrhs, nblk, out, ostride, 0));
}

void scale(const double2* w, double2* out, const double* s, long N, int nrhs, cudaStream_t st) {
  LS_LAUNCH("kr_scale", st, k_scale<<<grid_for(N * nrhs), 256, 0, st>>>(w, out, s, N, nrhs));
}

template <typename Cz>
void update_u(const Cz* const* Z, int nz, const double2* y, int ystride, double2* u, long N, int nrhs, cudaStream_t st) {
  LS_LAUNCH("kr_update_u", st, k_update_u<Cz><<<grid_for(N * nrhs), 256, 0, st>>>(Z, nz, y, ystride, u, N, nrhs));
}

void residual(const double2* g, const double2* Au, double2* r, long tot, cudaStream_t st) {
  LS_LAUNCH("kr_residual", st, k_residual<<<grid_for(tot), 256, 0, st>>>(g, Au, r, tot));
}

template <typename Cin, typename Cout> void cast(const Cin* in, Cout* out, long tot, cudaStream_t st) {
  LS_LAUNCH("kr_cast", st, k_cast<Cin, Cout><<<grid_for(tot), 256, 0, st>>>(in, out, tot));
}

template void dots<float2>(const double2* const*, int, const float2*, long, int, double2*, double2*, int, bool, cudaStream_t);
template void dots<double2>(const double2* const*, int, const double2*, long, int, double2*, double2*, int, bool, cudaStream_t);
template void sub_proj<float2>(const double2* const*, int, const float2*, double2*, const double2*, int, long, int, cudaStream_t);
template void sub_proj<double2>(const double2* const*, int, const double2*, double2*, const double2*, int, long, int, cudaStream_t);
template void norms2<double2>(const double2*, long, int, double2*, double2*, int, cudaStream_t);
template void norms2<float2>(const float2*, long, int, double2*, double2*, int, cudaStream_t);
template void update_u<float2>(const float2* const*, int, const double2*, int, double2*, long, int, cudaStream_t);
template void update_u<double2>(const double2* const*, int, const double2*, int, double2*, long, int, cudaStream_t);
template void cast<double2, float2>(const double2*, float2*, long, cudaStream_t);
template void cast<float2, double2>(const float2*, double2*, long, cudaStream_t);

// ---- right-hand-side subsets (the ones still iterating)
template <typename T, bool SCATTER>
__global__ void k_rhs_move(const T* __restrict__ src, T* __restrict__ dst, const int* __restrict__ idx, int n, long N) {
  const long tot = (long)n * N;
  for (long e = blockIdx.x * (long)blockDim.x + threadIdx.x; e < tot; e += (long)gridDim.x * blockDim.x) {
    const long i = e / N, k = e - i * N;
    const long j = idx[i];
    if (SCATTER) dst[j * N + k] = src[e];
    else dst[e] = src[j * N + k];
  }
}

template <typename T> void rhs_gather(const T* src, T* dst, const int* idx, int n, long N, cudaStream_t st) {
  if (n <= 0) return;
  LS_LAUNCH("kr_move", st, k_rhs_move<T, false><<<1024, 256, 0, st>>>(src, dst, idx, n, N));
}
template <typename T> void rhs_scatter(const T* src, T* dst, const int* idx, int n, long N, cudaStream_t st) {
  if (n <= 0) return;
  LS_LAUNCH("kr_move", st, k_rhs_move<T, true><<<1024, 256, 0, st>>>(src, dst, idx, n, N));
}
template void rhs_gather<double2>(const double2*, double2*, const int*, int, long, cudaStream_t);
template void rhs_gather<float2>(const float2*, float2*, const int*, int, long, cudaStream_t);
template void rhs_scatter<double2>(const double2*, double2*, const int*, int, long, cudaStream_t);
template void rhs_scatter<float2>(const float2*, float2*, const int*, int, long, cudaStream_t);

// ---- mixed path: the Arnoldi basis and the projected vector are stored as FP32 complex
// (float2: the precision of the FP32 preconditioner and operator that produce them), and
// every dot product, projection, norm and scaling runs in float-float arithmetic on the FP32
// pipes (GB300 issues FP32 at 64 times its FP64 rate).  Partial sums leave the blocks as
// FP64 for the ordered cross-block reduction.

__device__ __forceinline__ ffc ffc_of(float2 v) {
  ffc r;
  r.x = ff(v.x, 0.f);
  r.y = ff(v.y, 0.f);
  return r;
}
__device__ __forceinline__ ffc ffc_of(double2 v) { return ffc_of_f64(v); }

// the exact product of two FP32 numbers as a float-float (FMA TwoProduct)
__device__ __forceinline__ ff ff_prod(float a, float b) {
  const float p = __fmul_rn(a, b);
  return ff(p, __fmaf_rn(a, b, -p));
}
// a * b for a float-float a and an FP32 b (relative error about 2 u^2)
__device__ __forceinline__ ff ff_mul_f(ff a, float b) {
  const float p = __fmul_rn(a.hi, b);
  float e = __fmaf_rn(a.hi, b, -p);
  e = __fmaf_rn(a.lo, b, e);
  const float s = __fadd_rn(p, e);
  return ff(s, __fsub_rn(e, __fsub_rn(s, p)));
}
__device__ __forceinline__ float2 rnd(ffc v) { return make_float2(v.x.hi, v.y.hi); }
__device__ __forceinline__ ff ff_shfl_down(ff v, int o) {
  return ff(__shfl_down_sync(0xffffffffu, v.hi, o), __shfl_down_sync(0xffffffffu, v.lo, o));
}

// sum of v over the CTA in FP64 (thread 0); float-float adds within warps
__device__ __forceinline__ double2 block_sum_ff(ffc v, double2* sh) {
  for (int o = 16; o > 0; o >>= 1) {
    v.x = v.x + ff_shfl_down(v.x, o);
    v.y = v.y + ff_shfl_down(v.y, o);
  }
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  if (lane == 0) sh[wid] = make_double2(ff_to(v.x), ff_to(v.y));
  __syncthreads();
  double2 r = make_double2(0, 0);
  if (threadIdx.x == 0)
    for (int i = 0; i < (int)(blockDim.x >> 5); ++i) { r.x += sh[i].x; r.y += sh[i].y; }
  __syncthreads();
  return r;
}

__device__ void store_ff_pair(void* outf, size_t i, double2 v) {
  const ffc f = ffc_from(v);
  *reinterpret_cast<float4*>(reinterpret_cast<ffc*>(outf) + i) = make_float4(f.x.hi, f.x.lo, f.y.hi, f.y.lo);
}

constexpr int JB = 4;   // basis vectors per pass over w
constexpr int RUN = 4;  // elements per thread summed in FP32 before a float-float add

// partial[(rhs * nv + j) * nblk + blk] = sum over the block's chunk of conj(V_j) w, JB
// vectors per pass over the chunk.  Each thread sums the products of RUN of its elements
// with FP32 FMAs (error at most about RUN u times the sum of their magnitudes, u = 2^-24)
// and adds the run into a float-float accumulator, so that the error of a coefficient
// stays near RUN u |V_j| |w| however long the vectors are.  Such an error only leaves a
// component of that size along V_j in the projected vector, which CGS2's second pass
// removes; the Arnoldi relation holds with the coefficients as computed, because the
// projection itself (k_sub_proj_f) runs in float-float.
__global__ void __launch_bounds__(KT) k_dots_f(const float2* const* __restrict__ V, int nv, const float2* __restrict__ w,
                                               long N, double2* __restrict__ partial, int nblk) {
  __shared__ double2 sh[KT / 32];
  const int rhs = blockIdx.y, blk = blockIdx.x;
  const long chunk = (N + nblk - 1) / nblk;
  const long i0 = blk * chunk, i1 = min(N, i0 + chunk);
  const size_t base = (size_t)rhs * N;
  for (int jg = 0; jg < nv; jg += JB) {
    const int nj = min(JB, nv - jg);
    ffc acc[JB];
    const float2* vp[JB];  // the vectors' base pointers, loaded once (not per element)
#pragma unroll
    for (int q = 0; q < JB; ++q) {
      acc[q].x = acc[q].y = ff(0);
      vp[q] = q < nj ? V[jg + q] + base : w + base;
    }
    for (long i = i0 + threadIdx.x; i < i1; i += (long)KT * RUN) {
      float2 sr[JB];
#pragma unroll
      for (int q = 0; q < JB; ++q) sr[q] = make_float2(0.f, 0.f);
      // every load of the run issued before the arithmetic
      float2 b[RUN], a[RUN][JB];
#pragma unroll
      for (int u = 0; u < RUN; ++u) {
        const long e = i + (long)u * KT;
        const bool in = e < i1;
        b[u] = in ? w[base + e] : make_float2(0.f, 0.f);
#pragma unroll
        for (int q = 0; q < JB; ++q) a[u][q] = in && q < nj ? vp[q][e] : make_float2(0.f, 0.f);
      }
#pragma unroll
      for (int u = 0; u < RUN; ++u)
#pragma unroll
        for (int q = 0; q < JB; ++q) {
          sr[q].x = __fmaf_rn(a[u][q].x, b[u].x, __fmaf_rn(a[u][q].y, b[u].y, sr[q].x));
          sr[q].y = __fmaf_rn(a[u][q].x, b[u].y, __fmaf_rn(-a[u][q].y, b[u].x, sr[q].y));
        }
#pragma unroll
      for (int q = 0; q < JB; ++q)
        if (q < nj) {
          acc[q].x = acc[q].x + ff(sr[q].x, 0.f);
          acc[q].y = acc[q].y + ff(sr[q].y, 0.f);
        }
    }
#pragma unroll
    for (int q = 0; q < JB; ++q)
      if (q < nj) {
        const double2 s = block_sum_ff(acc[q], sh);
        if (threadIdx.x == 0) partial[((size_t)rhs * nv + jg + q) * nblk + blk] = s;
      }
  }
}

// wout = win - sum_j V_j h[rhs][j] (h as FP32 pairs), rounded to FP32; with NORM, also the
// partial sums of |wout|^2 (as stored) in the layout of k_dots_f.  The sum runs in
// float-float with deferred renormalisation (one lz_norm per element before the rounding),
// RUN elements per thread at a time so that their loads are in flight together; the
// coefficients sit in shared memory (up to SP_MAXV of them, else they are read from global
// memory).  |wout|^2 sums FP32 runs of RUN squares (positive terms: relative error about
// RUN u) into float-float.  win may equal wout.
constexpr int SP_MAXV = 64;
template <bool NORM>
__global__ void __launch_bounds__(KT) k_sub_proj_f(const float2* const* __restrict__ V, int nv, const float2* win,
                                                   float2* wout, const ffc* __restrict__ hf, int hstride, long N,
                                                   double2* __restrict__ partial, int nblk) {
  __shared__ double2 sh[KT / 32];
  __shared__ ffc hs[SP_MAXV];
  __shared__ const float2* vps[SP_MAXV];
  const int rhs = blockIdx.y, blk = blockIdx.x;
  const long chunk = (N + nblk - 1) / nblk;
  const long i0 = blk * chunk, i1 = min(N, i0 + chunk);
  const size_t base = (size_t)rhs * N;
  const ffc* hr = hf + (size_t)rhs * hstride;
  const bool staged = nv <= SP_MAXV;
  if (staged)
    for (int j = threadIdx.x; j < nv; j += KT) {
      hs[j] = hr[j];
      vps[j] = V[j];
    }
  __syncthreads();
  const ffc* hc = staged ? hs : hr;
  ffc nacc;
  nacc.x = nacc.y = ff(0);
  for (long i = i0 + threadIdx.x; i < i1; i += (long)KT * RUN) {
    ffc acc[RUN];
#pragma unroll
    for (int u = 0; u < RUN; ++u) {
      const long e = i + (long)u * KT;
      acc[u] = ffc_of(e < i1 ? win[base + e] : make_float2(0.f, 0.f));
    }
    // two basis vectors per step: their 2 RUN loads are issued before the arithmetic
    for (int j = 0; j < nv; j += 2) {
      const bool two = j + 1 < nv;
      const float2* vj = (staged ? vps[j] : V[j]) + base;
      const float2* vk = two ? (staged ? vps[j + 1] : V[j + 1]) + base : vj;
      float2 a[RUN], b[RUN];
#pragma unroll
      for (int u = 0; u < RUN; ++u) {
        const long e = i + (long)u * KT;
        a[u] = e < i1 ? vj[e] : make_float2(0.f, 0.f);
        b[u] = e < i1 && two ? vk[e] : make_float2(0.f, 0.f);
      }
      const ffc h = hc[j];
      const ffc g = two ? hc[j + 1] : h;
#pragma unroll
      for (int u = 0; u < RUN; ++u) {
        acc[u].x = lz_add(acc[u].x, lz_neg(lz_add(lz_mul_f(h.x, a[u].x), lz_neg(lz_mul_f(h.y, a[u].y)))));
        acc[u].y = lz_add(acc[u].y, lz_neg(lz_add(lz_mul_f(h.y, a[u].x), lz_mul_f(h.x, a[u].y))));
        if (two) {
          acc[u].x = lz_add(acc[u].x, lz_neg(lz_add(lz_mul_f(g.x, b[u].x), lz_neg(lz_mul_f(g.y, b[u].y)))));
          acc[u].y = lz_add(acc[u].y, lz_neg(lz_add(lz_mul_f(g.y, b[u].x), lz_mul_f(g.x, b[u].y))));
        }
      }
    }
    float nr = 0.f;
#pragma unroll
    for (int u = 0; u < RUN; ++u) {
      const long e = i + (long)u * KT;
      if (e < i1) {
        const float2 o = make_float2(lz_norm(acc[u].x).hi, lz_norm(acc[u].y).hi);
        wout[base + e] = o;
        if (NORM) nr = __fmaf_rn(o.x, o.x, __fmaf_rn(o.y, o.y, nr));
      }
    }
    if (NORM) nacc.x = nacc.x + ff(nr, 0.f);
  }
  if (NORM) {
    const double2 s = block_sum_ff(nacc, sh);
    if (threadIdx.x == 0) partial[(size_t)rhs * nblk + blk] = s;
  }
}

// out[rhs] = in[rhs] * scale[rhs] rounded to FP32; in FP64 (the residual) or FP32
template <typename Cin>
__global__ void k_scale_f(const Cin* __restrict__ in, float2* out, const double* __restrict__ scale, long N) {
  const int rhs = blockIdx.y;
  const ff s = ff_of_f64(scale[rhs]);
  const size_t base = (size_t)rhs * N;
  for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < N; i += (long)gridDim.x * blockDim.x) {
    ffc v = ffc_of(in[base + i]);
    v.x = v.x * s;
    v.y = v.y * s;
    out[base + i] = rnd(v);
  }
}

// u[rhs] += sum_j Z_j[rhs] y[rhs][j] for FP32 Z (mixed path): the sum in float-float on the
// FP32 pipes, the coefficients converted once per CTA, and two FP64 adds per component into
// u (the FP64 form of k_update_u spends four FP64 FMAs per basis vector and component, at
// GB300's small FP64 rate).  At most UPD_MAXZ vectors per launch.
constexpr int UPD_MAXZ = 64;
__global__ void __launch_bounds__(256) k_update_u_f(const float2* const* __restrict__ Z, int nz,
                                                   const double2* __restrict__ y, int ystride, double2* u, long N) {
  __shared__ ffc hy[UPD_MAXZ];
  __shared__ const float2* zps[UPD_MAXZ];
  const int rhs = blockIdx.y;
  const double2* yr = y + (size_t)rhs * ystride;
  for (int j = threadIdx.x; j < nz; j += blockDim.x) {
    hy[j] = ffc_of_f64(yr[j]);
    zps[j] = Z[j];
  }
  __syncthreads();
  const size_t base = (size_t)rhs * N;
  const long stride = (long)gridDim.x * blockDim.x;
  // UR elements per thread at a time, two basis vectors per step: their loads (and those of
  // u) issued before the arithmetic
  constexpr int UR = 2;
  for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < N; i += stride * UR) {
    ffc acc[UR];
    double2 uv[UR];
#pragma unroll
    for (int r = 0; r < UR; ++r) {
      acc[r].x = acc[r].y = ff(0);
      const long e = i + r * stride;
      uv[r] = e < N ? u[base + e] : make_double2(0.0, 0.0);
    }
    for (int j = 0; j < nz; j += 2) {
      const bool two = j + 1 < nz;
      float2 za[UR], zb[UR];
#pragma unroll
      for (int r = 0; r < UR; ++r) {
        const long e = i + r * stride;
        za[r] = e < N ? zps[j][base + e] : make_float2(0.f, 0.f);
        zb[r] = e < N && two ? zps[j + 1][base + e] : make_float2(0.f, 0.f);
      }
      const ffc h = hy[j], q = two ? hy[j + 1] : hy[j];
#pragma unroll
      for (int r = 0; r < UR; ++r) {
        acc[r].x = acc[r].x + (ff_mul_f(h.x, za[r].x) - ff_mul_f(h.y, za[r].y));
        acc[r].y = acc[r].y + (ff_mul_f(h.y, za[r].x) + ff_mul_f(h.x, za[r].y));
        if (two) {
          acc[r].x = acc[r].x + (ff_mul_f(q.x, zb[r].x) - ff_mul_f(q.y, zb[r].y));
          acc[r].y = acc[r].y + (ff_mul_f(q.y, zb[r].x) + ff_mul_f(q.x, zb[r].y));
        }
      }
    }
#pragma unroll
    for (int r = 0; r < UR; ++r) {
      const long e = i + r * stride;
      if (e < N) u[base + e] = make_double2(uv[r].x + ff_to_f64(acc[r].x), uv[r].y + ff_to_f64(acc[r].y));
    }
  }
}

static dim3 grid_rows(long N, int nrhs) {
  long b = (N + 255) / 256;
  const long cap = (152L * 16 + nrhs - 1) / nrhs;
  if (b > cap) b = cap;
  return dim3((unsigned)(b < 1 ? 1 : b), nrhs);
}

void dots_f(const float2* const* V, int nv, const float2* w, long N, int nrhs, double2* partial, double2* out,
            ffc* outf, int ostride, cudaStream_t st) {
  const int nblk = dots_blocks(N);
  LS_LAUNCH("kr_dots", st, k_dots_f<<<dim3(nblk, nrhs), KT, 0, st>>>(V, nv, w, N, partial, nblk));
  LS_LAUNCH("kr_reduce", st,
            k_reduce<<<(nv * nrhs + 127) / 128, 128, 0, st>>>(partial, nv, nrhs, nblk, out, ostride, 0, outf));
}

void sub_proj_f(const float2* const* V, int nv, const float2* win, float2* wout, const ffc* hf, int hstride, long N,
                int nrhs, double2* partial, double2* norm_out, int ostride, cudaStream_t st) {
  const int nblk = dots_blocks(N);
  if (norm_out) {
    LS_LAUNCH("kr_sub_proj", st,
              k_sub_proj_f<true><<<dim3(nblk, nrhs), KT, 0, st>>>(V, nv, win, wout, hf, hstride, N, partial, nblk));
    LS_LAUNCH("kr_reduce", st,
              k_reduce<<<(nrhs + 127) / 128, 128, 0, st>>>(partial, 1, nrhs, nblk, norm_out, ostride, 0));
  } else {
    LS_LAUNCH("kr_sub_proj", st,
              k_sub_proj_f<false><<<dim3(nblk, nrhs), KT, 0, st>>>(V, nv, win, wout, hf, hstride, N, partial, nblk));
  }
}

void update_u_f(const float2* const* Z, int nz, const double2* y, int ystride, double2* u, long N, int nrhs,
                cudaStream_t st) {
  for (int j0 = 0; j0 < nz; j0 += UPD_MAXZ)
    LS_LAUNCH("kr_update_u", st,
              k_update_u_f<<<grid_rows(N, nrhs), 256, 0, st>>>(Z + j0, std::min(UPD_MAXZ, nz - j0), y + j0, ystride,
                                                               u, N));
}

template <typename Cin> void scale_f(const Cin* in, float2* out, const double* s, long N, int nrhs, cudaStream_t st) {
  LS_LAUNCH("kr_scale", st, k_scale_f<Cin><<<grid_rows(N, nrhs), 256, 0, st>>>(in, out, s, N));
}

template void scale_f<double2>(const double2*, float2*, const double*, long, int, cudaStream_t);
template void scale_f<float2>(const float2*, float2*, const double*, long, int, cudaStream_t);

}  // namespace ls
