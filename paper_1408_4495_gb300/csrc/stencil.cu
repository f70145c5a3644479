// Stencil apply r = [A; B] v of the preconditioner (Sec. 2.2, eq. PC; Sec. 3.1): every grid
// point i uses the 3^d-point stencil alpha of its class (interior, face, edge, corner),
//   r_i = sum_{t in mu(i)} alpha_cls(i)(t) v_{i+t}.
// One thread per output point; consecutive threads take consecutive points of a grid line
// so that the loads of v and the stores of r are coalesced, and the 3^d neighbours of
// adjacent points are shared in L1.  The coefficient table (3^d classes x 3^d offsets)
// is staged in shared memory.  General domains (Sec. 4) give every point its own stencil
// (PT: row i of an N x 3^d table, read from global memory).
#include "common.cuh"
#include "ffloat.cuh"
#include "kernels.h"
#include "prof.h"

namespace ls {

// one input entry in the output arithmetic (float-float input: its leading FP32 part)
template <typename Cout, typename Cin> __device__ __forceinline__ Cout ld_in(const Cin* p) { return ccast<Cout>(__ldg(p)); }
template <> __device__ __forceinline__ float2 ld_in<float2, ffc>(const ffc* p) {
  const float4 v = __ldg(reinterpret_cast<const float4*>(p));
  return make_float2(v.x, v.z);
}

template <typename Cin, typename Cout, int D, bool PT>
__global__ void __launch_bounds__(256) k_stencil(int n, int nrhs, const Cin* __restrict__ v, Cout* __restrict__ r,
                                                 long rs_i, long rs_r, const Cout* __restrict__ alpha) {
  constexpr int P3 = D == 2 ? 9 : 27;
  __shared__ Cout sa[PT ? 1 : P3 * P3];
  if constexpr (!PT) {
    for (int i = threadIdx.x; i < P3 * P3; i += blockDim.x) sa[i] = alpha[i];
    __syncthreads();
  }
  const long N = D == 2 ? (long)n * n : (long)n * n * n;
  const long total = N * nrhs;
  for (long idx = blockIdx.x * (long)blockDim.x + threadIdx.x; idx < total; idx += (long)gridDim.x * blockDim.x) {
    const long rhs = idx / N, i = idx - rhs * N;
    int c[3];
    long q = i;
    for (int a = D - 1; a >= 0; --a) {
      c[a] = (int)(q % n);
      q /= n;
    }
    int cls = 0;
    for (int a = 0; a < D; ++a) cls = cls * 3 + (c[a] == 0 ? 0 : (c[a] == n - 1 ? 2 : 1));
    const Cin* vr = v + rhs * N;
    Cout acc = czero<Cout>();
    const Cout* al = PT ? alpha + i * P3 : sa + cls * P3;
    if constexpr (D == 2) {
#pragma unroll
      for (int t0 = -1; t0 <= 1; ++t0)
#pragma unroll
        for (int t1 = -1; t1 <= 1; ++t1) {
          const int a0 = c[0] + t0, a1 = c[1] + t1;
          if (a0 >= 0 && a0 < n && a1 >= 0 && a1 < n) {
            const Cout x = ld_in<Cout>(&vr[(long)a0 * n + a1]);
            acc = cfma(acc, al[(t0 + 1) * 3 + (t1 + 1)], x);
          }
        }
    } else {
#pragma unroll
      for (int t0 = -1; t0 <= 1; ++t0)
#pragma unroll
        for (int t1 = -1; t1 <= 1; ++t1)
#pragma unroll
          for (int t2 = -1; t2 <= 1; ++t2) {
            const int a0 = c[0] + t0, a1 = c[1] + t1, a2 = c[2] + t2;
            if (a0 >= 0 && a0 < n && a1 >= 0 && a1 < n && a2 >= 0 && a2 < n) {
              const Cout x = ld_in<Cout>(&vr[((long)a0 * n + a1) * n + a2]);
              acc = cfma(acc, al[((t0 + 1) * 3 + (t1 + 1)) * 3 + (t2 + 1)], x);
            }
          }
    }
    r[i * rs_i + rhs * rs_r] = acc;
  }
}

template <typename Cin, typename Cout>
void stencil_apply(int d, int n, int nrhs, const Cin* v, Cout* r, long rs_i, long rs_r, const void* alpha,
                   cudaStream_t st) {
  const long N = d == 2 ? (long)n * n : (long)n * n * n;
  const long total = N * nrhs;
  long blocks = (total + 255) / 256;
  if (blocks > 152L * 64) blocks = 152L * 64;
  if (blocks == 0) return;
  const char* cls = sizeof(Cout) == 8 ? "stencil_c64" : "stencil_c128";
  if (d == 2)
    LS_LAUNCH(cls, st, k_stencil<Cin, Cout, 2, false><<<(unsigned)blocks, 256, 0, st>>>(n, nrhs, v, r, rs_i, rs_r, (const Cout*)alpha));
  else
    LS_LAUNCH(cls, st, k_stencil<Cin, Cout, 3, false><<<(unsigned)blocks, 256, 0, st>>>(n, nrhs, v, r, rs_i, rs_r, (const Cout*)alpha));
}

template <typename Cin, typename Cout>
void stencil_apply_pt(int d, int n, int nrhs, const Cin* v, Cout* r, long rs_i, long rs_r, const void* alpha_pt,
                      cudaStream_t st) {
  const long N = d == 2 ? (long)n * n : (long)n * n * n;
  const long total = N * nrhs;
  long blocks = (total + 255) / 256;
  if (blocks > 152L * 64) blocks = 152L * 64;
  if (blocks == 0) return;
  const char* cls = sizeof(Cout) == 8 ? "stencil_pt_c64" : "stencil_pt_c128";
  if (d == 2)
    LS_LAUNCH(cls, st, k_stencil<Cin, Cout, 2, true><<<(unsigned)blocks, 256, 0, st>>>(n, nrhs, v, r, rs_i, rs_r, (const Cout*)alpha_pt));
  else
    LS_LAUNCH(cls, st, k_stencil<Cin, Cout, 3, true><<<(unsigned)blocks, 256, 0, st>>>(n, nrhs, v, r, rs_i, rs_r, (const Cout*)alpha_pt));
}

template void stencil_apply<float2, float2>(int, int, int, const float2*, float2*, long, long, const void*, cudaStream_t);
template void stencil_apply<ffc, float2>(int, int, int, const ffc*, float2*, long, long, const void*, cudaStream_t);
template void stencil_apply<double2, float2>(int, int, int, const double2*, float2*, long, long, const void*, cudaStream_t);
template void stencil_apply<double2, double2>(int, int, int, const double2*, double2*, long, long, const void*, cudaStream_t);
template void stencil_apply_pt<float2, float2>(int, int, int, const float2*, float2*, long, long, const void*, cudaStream_t);
template void stencil_apply_pt<ffc, float2>(int, int, int, const ffc*, float2*, long, long, const void*, cudaStream_t);
template void stencil_apply_pt<double2, float2>(int, int, int, const double2*, float2*, long, long, const void*, cudaStream_t);
template void stencil_apply_pt<double2, double2>(int, int, int, const double2*, double2*, long, long, const void*, cudaStream_t);

}  // namespace ls
