// FP64 Krylov kernels (krylov.cu); vectors are [nrhs][N] complex.
#pragma once

#include <cuda_runtime.h>

namespace ls {

struct ffc;

int dots_blocks(long N);
// out[rhs * ostride + j] (+)= sum_i conj(V_j[rhs][i]) w[rhs][i], j < nv; partial: nrhs*nv*dots_blocks(N)
template <typename Cw>
void dots(const double2* const* V, int nv, const Cw* w, long N, int nrhs, double2* partial, double2* out, int ostride,
          bool accumulate, cudaStream_t st);
// wout = win - sum_j V_j h[rhs * hstride + j]
template <typename Cw>
void sub_proj(const double2* const* V, int nv, const Cw* win, double2* wout, const double2* h, int hstride, long N,
              int nrhs, cudaStream_t st);
// out[rhs * ostride].x = |w[rhs]|^2
template <typename Cw>
void norms2(const Cw* w, long N, int nrhs, double2* partial, double2* out, int ostride, cudaStream_t st);
void scale(const double2* w, double2* out, const double* s, long N, int nrhs, cudaStream_t st);
template <typename Cz>
void update_u(const Cz* const* Z, int nz, const double2* y, int ystride, double2* u, long N, int nrhs, cudaStream_t st);
void residual(const double2* g, const double2* Au, double2* r, long tot, cudaStream_t st);
template <typename Cin, typename Cout> void cast(const Cin* in, Cout* out, long tot, cudaStream_t st);
// Mixed path: V and the projected vector stored as FP32 complex, arithmetic in float-float.
// dots_f also writes the coefficients as FP32 pairs (outf, same indexing as out), which
// sub_proj_f reads; sub_proj_f with norm_out != NULL also writes |wout|^2 to
// norm_out[rhs * ostride].x.  win may equal wout.
void dots_f(const float2* const* V, int nv, const float2* w, long N, int nrhs, double2* partial, double2* out,
            ffc* outf, int ostride, cudaStream_t st);
void sub_proj_f(const float2* const* V, int nv, const float2* win, float2* wout, const ffc* hf, int hstride, long N,
                int nrhs, double2* partial, double2* norm_out, int ostride, cudaStream_t st);
template <typename Cin> void scale_f(const Cin* in, float2* out, const double* s, long N, int nrhs, cudaStream_t st);
// u += sum_j Z_j y_j with FP32 Z, the sum in float-float
void update_u_f(const float2* const* Z, int nz, const double2* y, int ystride, double2* u, long N, int nrhs,
                cudaStream_t st);
// dst[i] = src[idx[i]] (gather) or dst[idx[i]] = src[i] (scatter) for i < n right-hand
// sides of N entries each; idx on the device
template <typename T> void rhs_gather(const T* src, T* dst, const int* idx, int n, long N, cudaStream_t st);
template <typename T> void rhs_scatter(const T* src, T* dst, const int* idx, int n, long N, cudaStream_t st);

}  // namespace ls
