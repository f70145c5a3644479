// Stencil apply r = [A; B] v of the preconditioner (Sec. 2.2, eq. PC; Sec. 3.1): every grid
// point i uses the 3^d-point stencil alpha of its class (interior, face, edge, corner),
//   r_i = sum_{t in mu(i)} alpha_cls(i)(t) v_{i+t}.
// Consecutive threads take consecutive points of a grid line so that the loads of v and the
// stores of r are coalesced, and the 3^d neighbours of adjacent points are shared in L1.  The coefficient table (3^d classes x 3^d offsets)
// is staged in shared memory.  General domains (Sec. 4) give every point its own stencil
// (PT: row i of an N x 3^d table, read from global memory).
#include <type_traits>

#include "common.cuh"
#include "ffloat.cuh"
#include "kernels.h"
#include "prof.h"

namespace ls {

// one input entry in the output arithmetic
template <typename Cout, typename Cin> __device__ __forceinline__ Cout ld_in(const Cin* p) { return ccast<Cout>(__ldg(p)); }

// A CTA takes whole grid lines (the last axis): lpb = max(1, 256 / n) lines of n points, the
// threads of a line stepping through its points, so that no per-point index division is
// needed; the line's coordinates on the other axes come from one division per line.
template <typename Cin, typename Cout, int D, bool PT>
__global__ void __launch_bounds__(256) k_stencil(int n, int nrhs, const Cin* __restrict__ v, Cout* __restrict__ r,
                                                 long rs_i, long rs_r, const Cout* __restrict__ alpha) {
  constexpr int P3 = D == 2 ? 9 : 27;
  __shared__ Cout sa[PT ? 1 : P3 * P3];
  if constexpr (!PT) {
    for (int i = threadIdx.x; i < P3 * P3; i += blockDim.x) sa[i] = alpha[i];
    __syncthreads();
  }
  const int width = n < (int)blockDim.x ? n : (int)blockDim.x;  // threads per line
  const int lpb = (int)blockDim.x / width;                       // lines per CTA
  const int sub = threadIdx.x / width, lane = threadIdx.x - sub * width;
  if (sub >= lpb) return;
  const long lines = (D == 2 ? (long)n : (long)n * n);  // lines per right-hand side
  const long N = lines * n;
  for (long line = (long)blockIdx.x * lpb + sub; line < lines * nrhs; line += (long)gridDim.x * lpb) {
    const long rhs = line / lines, l = line - rhs * lines;
    const int c0 = D == 2 ? (int)l : (int)(l / n);
    const int c1 = D == 2 ? 0 : (int)(l - (long)c0 * n);
    const int k0 = c0 == 0 ? 0 : (c0 == n - 1 ? 2 : 1);
    const int k1 = c1 == 0 ? 0 : (c1 == n - 1 ? 2 : 1);
    const Cin* vr = v + rhs * N;
    for (int c2 = lane; c2 < n; c2 += width) {
      const int k2 = c2 == 0 ? 0 : (c2 == n - 1 ? 2 : 1);
      const long i = l * n + c2;
      Cout acc = czero<Cout>();
      if constexpr (D == 2) {
        const Cout* al = PT ? alpha + i * P3 : sa + (k0 * 3 + k2) * P3;
#pragma unroll
        for (int t0 = -1; t0 <= 1; ++t0)
#pragma unroll
          for (int t1 = -1; t1 <= 1; ++t1) {
            const int a0 = c0 + t0, a1 = c2 + t1;
            if (a0 >= 0 && a0 < n && a1 >= 0 && a1 < n) {
              const Cout x = ld_in<Cout>(&vr[(long)a0 * n + a1]);
              acc = cfma(acc, al[(t0 + 1) * 3 + (t1 + 1)], x);
            }
          }
      } else {
        const Cout* al = PT ? alpha + i * P3 : sa + ((k0 * 3 + k1) * 3 + k2) * P3;
#pragma unroll
        for (int t0 = -1; t0 <= 1; ++t0)
#pragma unroll
          for (int t1 = -1; t1 <= 1; ++t1)
#pragma unroll
            for (int t2 = -1; t2 <= 1; ++t2) {
              const int a0 = c0 + t0, a1 = c1 + t1, a2 = c2 + t2;
              if (a0 >= 0 && a0 < n && a1 >= 0 && a1 < n && a2 >= 0 && a2 < n) {
                const Cout x = ld_in<Cout>(&vr[((long)a0 * n + a1) * n + a2]);
                acc = cfma(acc, al[((t0 + 1) * 3 + (t1 + 1)) * 3 + (t2 + 1)], x);
              }
            }
      }
      r[i * rs_i + rhs * rs_r] = acc;
    }
  }
}

// 2D FP32 stencil r = [A; B] v (RESID false) and preconditioner residual r2 (RESID true,
// k_pre_resid's sums) with a rolling window along axis 0: a thread takes one grid column c
// of one right-hand side over a run of R rows and reads the entries c - 1, c, c + 1 of each
// row once for the three output rows that use them (three loads per point and array
// instead of nine).  The 9-point sums keep k_stencil's and k_pre_resid's order; entries
// outside the grid read as zero.
template <bool RESID>
__device__ __forceinline__ void roll_row(const float2* __restrict__ vr, const float2* __restrict__ zr,
                                         const float* __restrict__ w2m, int n, int a0, int c, float2* d, float2* e) {
#pragma unroll
  for (int t = 0; t < 3; ++t) {
    d[t] = make_float2(0.f, 0.f);
    e[t] = make_float2(0.f, 0.f);
  }
  if (a0 < 0 || a0 >= n) return;
#pragma unroll
  for (int t = 0; t < 3; ++t) {
    const int a2 = c + t - 1;
    if (a2 < 0 || a2 >= n) continue;
    const long j = (long)a0 * n + a2;
    if constexpr (RESID) {
      const float2 zv = __ldg(&zr[j]);
      d[t] = csub(__ldg(&vr[j]), zv);
      const float w = __ldg(&w2m[j]);
      e[t] = make_float2(w * zv.x, w * zv.y);
    } else {
      d[t] = __ldg(&vr[j]);
    }
  }
}

template <bool RESID>
__global__ void __launch_bounds__(256, 3) k_stencil2_roll(int n, int nrhs, int R, int nseg, const float2* __restrict__ v,
                                                       const float2* __restrict__ z, float2* __restrict__ out,
                                                       const float2* __restrict__ alpha,
                                                       const double2* __restrict__ cint, const float* __restrict__ w2m) {
  __shared__ float2 sa[81];
  __shared__ float2 sc[9];
  for (int i = threadIdx.x; i < 81; i += blockDim.x) sa[i] = alpha[i];
  if constexpr (RESID) {
    for (int i = threadIdx.x; i < 9; i += blockDim.x) sc[i] = make_float2((float)cint[i].x, (float)cint[i].y);
  }
  __syncthreads();
  const long per = (long)nseg * n;  // threads per right-hand side
  const long g = (long)blockIdx.x * blockDim.x + threadIdx.x;
  if (g >= per * nrhs) return;
  const long rhs = g / per;
  const int rem = (int)(g - rhs * per), seg = rem / n, c = rem - seg * n;
  const int r0 = seg * R, r1 = r0 + R < n ? r0 + R : n;
  const int k2 = c == 0 ? 0 : (c == n - 1 ? 2 : 1);
  const long N = (long)n * n;
  const float2* vr = v + rhs * N;
  const float2* zr = RESID ? z + rhs * N : nullptr;
  float2* o = out + rhs * N;
  float2 D[3][3], E[3][3];  // rows a0 - 1, a0, a0 + 1; columns c - 1, c, c + 1
  roll_row<RESID>(vr, zr, w2m, n, r0 - 1, c, D[0], E[0]);
  roll_row<RESID>(vr, zr, w2m, n, r0, c, D[1], E[1]);
#pragma unroll 2
  for (int a0 = r0; a0 < r1; ++a0) {
    roll_row<RESID>(vr, zr, w2m, n, a0 + 1, c, D[2], E[2]);
    const int k0 = a0 == 0 ? 0 : (a0 == n - 1 ? 2 : 1);
    const float2* al = sa + (k0 * 3 + k2) * 9;
    float2 acc = make_float2(0.f, 0.f);
#pragma unroll
    for (int t = 0; t < 9; ++t) {
      acc = cfma(acc, al[t], D[t / 3][t % 3]);
      if constexpr (RESID) acc = cfms(acc, sc[t], E[t / 3][t % 3]);
    }
    o[(long)a0 * n + c] = acc;
#pragma unroll
    for (int t = 0; t < 3; ++t) {
      D[0][t] = D[1][t];
      D[1][t] = D[2][t];
      E[0][t] = E[1][t];
      E[1][t] = E[2][t];
    }
  }
}

// rows per thread of k_stencil2_roll: runs of up to 32 rows, shorter while the grid would
// give fewer than about 2048 threads per SM
static int roll_rows(int n, int nrhs) {
  int R = 32;
  while (R > 1 && (long)nrhs * n * ((n + R - 1) / R) < 152L * 2048) R /= 2;
  return R;
}

static void launch_roll(bool resid, int n, int nrhs, const float2* v, const float2* z, float2* out, const float2* alpha,
                        const double2* cint, const float* w2m, cudaStream_t st) {
  const int R = roll_rows(n, nrhs), nseg = (n + R - 1) / R;
  const long threads = (long)nrhs * nseg * n;
  if (threads == 0) return;
  const unsigned blocks = (unsigned)((threads + 255) / 256);
  if (resid)
    LS_LAUNCH("stencil_c64", st, k_stencil2_roll<true><<<blocks, 256, 0, st>>>(n, nrhs, R, nseg, v, z, out, alpha, cint, w2m));
  else
    LS_LAUNCH("stencil_c64", st, k_stencil2_roll<false><<<blocks, 256, 0, st>>>(n, nrhs, R, nseg, v, z, out, alpha, cint, w2m));
}

// The same sums written straight into the solve's item layout T[group][N][RC] (right-hand
// side j of group g at T[(g N + i) RC + j], sides past nrhs zero), so that the solve needs no
// transposition pass: a CTA takes CW = 256 / RC columns of the RC right-hand sides of one
// group over a run of R rows (warps read whole 128-byte runs of a row of one right-hand
// side), and each output row goes through a shared-memory tile (double-buffered: one
// barrier per row) to contiguous CW x RC stores.
template <bool RESID, int RC>
__global__ void __launch_bounds__(256, 3) k_stencil2_items(int n, int nrhs, int R, int ctiles,
                                                           const float2* __restrict__ v, const float2* __restrict__ z,
                                                           float2* __restrict__ T, const float2* __restrict__ alpha,
                                                           const double2* __restrict__ cint,
                                                           const float* __restrict__ w2m) {
  constexpr int CW = 256 / RC;
  __shared__ float2 sa[81];
  __shared__ float2 sc[9];
  __shared__ float2 tile[2][CW * (RC + 1)];
  for (int i = threadIdx.x; i < 81; i += blockDim.x) sa[i] = alpha[i];
  if constexpr (RESID) {
    for (int i = threadIdx.x; i < 9; i += blockDim.x) sc[i] = make_float2((float)cint[i].x, (float)cint[i].y);
  }
  __syncthreads();
  const int ct = (int)(blockIdx.x % ctiles), seg = (int)(blockIdx.x / ctiles), g = (int)blockIdx.y;
  const int j = threadIdx.x / CW, cl = threadIdx.x - j * CW;
  const int c = ct * CW + cl, rhs = g * RC + j;
  const bool act = c < n && rhs < nrhs;
  const int r0 = seg * R, r1 = r0 + R < n ? r0 + R : n;
  const int k2 = c == 0 ? 0 : (c == n - 1 ? 2 : 1);
  const long N = (long)n * n;
  const float2* vr = v + (long)(act ? rhs : 0) * N;
  const float2* zr = RESID ? z + (long)(act ? rhs : 0) * N : nullptr;
  // the writer's entry of the tile: column oc, right-hand side oj
  const int oc = threadIdx.x / RC, oj = threadIdx.x - oc * RC;
  float2* Tg = T + (size_t)g * N * RC;
  float2 D[3][3], E[3][3];
  for (int t = 0; t < 9; ++t) D[t / 3][t % 3] = E[t / 3][t % 3] = make_float2(0.f, 0.f);
  if (act) {
    roll_row<RESID>(vr, zr, w2m, n, r0 - 1, c, D[0], E[0]);
    roll_row<RESID>(vr, zr, w2m, n, r0, c, D[1], E[1]);
  }
  for (int a0 = r0; a0 < r1; ++a0) {
    float2 acc = make_float2(0.f, 0.f);
    if (act) {
      roll_row<RESID>(vr, zr, w2m, n, a0 + 1, c, D[2], E[2]);
      const int k0 = a0 == 0 ? 0 : (a0 == n - 1 ? 2 : 1);
      const float2* al = sa + (k0 * 3 + k2) * 9;
#pragma unroll
      for (int t = 0; t < 9; ++t) {
        acc = cfma(acc, al[t], D[t / 3][t % 3]);
        if constexpr (RESID) acc = cfms(acc, sc[t], E[t / 3][t % 3]);
      }
#pragma unroll
      for (int t = 0; t < 3; ++t) {
        D[0][t] = D[1][t];
        D[1][t] = D[2][t];
        E[0][t] = E[1][t];
        E[1][t] = E[2][t];
      }
    }
    float2* tb = tile[(a0 - r0) & 1];
    tb[cl * (RC + 1) + j] = acc;
    __syncthreads();
    if (ct * CW + oc < n) Tg[((long)a0 * n + ct * CW + oc) * RC + oj] = tb[oc * (RC + 1) + oj];
  }
}

static void launch_items(bool resid, int n, int nrhs, int rc, const float2* v, const float2* z, float2* T,
                         const float2* alpha, const double2* cint, const float* w2m, cudaStream_t st) {
  const int cw = 256 / rc, ctiles = (n + cw - 1) / cw, ng = (nrhs + rc - 1) / rc;
  int R = 32;  // runs of up to 32 rows, shorter while the grid would give fewer than ~2048 threads per SM
  while (R > 1 && (long)ng * ctiles * ((n + R - 1) / R) * 256 < 152L * 2048) R /= 2;
  const long tiles = (long)ctiles * ((n + R - 1) / R);
  if (tiles == 0 || ng == 0) return;
  const dim3 grid((unsigned)tiles, (unsigned)ng);
#define LS_ITEMS(RS, RCC)                                                                                   \
  LS_LAUNCH("stencil_c64", st,                                                                            \
            k_stencil2_items<RS, RCC><<<grid, 256, 0, st>>>(n, nrhs, R, ctiles, v, z, T, alpha, cint, w2m))
  if (rc == 16) {
    if (resid) LS_ITEMS(true, 16);
    else LS_ITEMS(false, 16);
  } else if (rc == 4) {
    if (resid) LS_ITEMS(true, 4);
    else LS_ITEMS(false, 4);
  } else {
    LS_FAIL(EINVAL_, "stencil items: group width %d (4 or 16)", rc);
  }
#undef LS_ITEMS
}

void stencil_items_2d(int n, int nrhs, int rc, const float2* v, const float2* z, float2* T, const float2* alpha32,
                      const double2* cint64, const float* w2m32, cudaStream_t st) {
  launch_items(z != nullptr, n, nrhs, rc, v, z, T, alpha32, cint64, w2m32, st);
}

static unsigned stencil_blocks(int d, int n, int nrhs) {
  const long lines = (d == 2 ? (long)n : (long)n * n) * nrhs;
  const int lpb = n < 256 ? 256 / n : 1;
  long blocks = (lines + lpb - 1) / lpb;
  if (blocks > 152L * 64) blocks = 152L * 64;
  return (unsigned)blocks;
}

template <typename Cin, typename Cout>
void stencil_apply(int d, int n, int nrhs, const Cin* v, Cout* r, long rs_i, long rs_r, const void* alpha,
                   cudaStream_t st) {
  if constexpr (std::is_same<Cin, float2>::value && std::is_same<Cout, float2>::value) {
    if (d == 2 && rs_i == 1 && rs_r == (long)n * n) {
      launch_roll(false, n, nrhs, v, nullptr, r, (const float2*)alpha, nullptr, nullptr, st);
      return;
    }
  }
  const unsigned blocks = stencil_blocks(d, n, nrhs);
  if (blocks == 0) return;
  const char* cls = sizeof(Cout) == 8 ? "stencil_c64" : "stencil_c128";
  if (d == 2)
    LS_LAUNCH(cls, st, k_stencil<Cin, Cout, 2, false><<<blocks, 256, 0, st>>>(n, nrhs, v, r, rs_i, rs_r, (const Cout*)alpha));
  else
    LS_LAUNCH(cls, st, k_stencil<Cin, Cout, 3, false><<<blocks, 256, 0, st>>>(n, nrhs, v, r, rs_i, rs_r, (const Cout*)alpha));
}

template <typename Cin, typename Cout>
void stencil_apply_pt(int d, int n, int nrhs, const Cin* v, Cout* r, long rs_i, long rs_r, const void* alpha_pt,
                      cudaStream_t st) {
  const unsigned blocks = stencil_blocks(d, n, nrhs);
  if (blocks == 0) return;
  const char* cls = sizeof(Cout) == 8 ? "stencil_pt_c64" : "stencil_pt_c128";
  if (d == 2)
    LS_LAUNCH(cls, st, k_stencil<Cin, Cout, 2, true><<<blocks, 256, 0, st>>>(n, nrhs, v, r, rs_i, rs_r, (const Cout*)alpha_pt));
  else
    LS_LAUNCH(cls, st, k_stencil<Cin, Cout, 3, true><<<blocks, 256, 0, st>>>(n, nrhs, v, r, rs_i, rs_r, (const Cout*)alpha_pt));
}

// Residual of a preconditioner application, r2 = [A;B] v - M z with
// M(i, i+t) = alpha_cls(i)(t) + c(t) omega^2 m_{i+t} (eq. PC; the c term vanishes on the
// boundary rows because m is zero on the b+1 outermost layers):
//   r2_i = sum_t alpha_cls(i)(t) (v - z)_{i+t} - sum_t c(t) (omega^2 m z)_{i+t}.
// FP32; same line-wise thread layout as k_stencil.
template <int D>
__global__ void __launch_bounds__(256) k_pre_resid(int n, int nrhs, const float2* __restrict__ v,
                                                   const float2* __restrict__ z, float2* __restrict__ r2,
                                                   const float2* __restrict__ alpha, const double2* __restrict__ cint,
                                                   const float* __restrict__ w2m) {
  constexpr int P3 = D == 2 ? 9 : 27;
  __shared__ float2 sa[P3 * P3];
  __shared__ float2 sc[P3];
  for (int i = threadIdx.x; i < P3 * P3; i += blockDim.x) sa[i] = alpha[i];
  for (int i = threadIdx.x; i < P3; i += blockDim.x) sc[i] = make_float2((float)cint[i].x, (float)cint[i].y);
  __syncthreads();
  const int width = n < (int)blockDim.x ? n : (int)blockDim.x;
  const int lpb = (int)blockDim.x / width;
  const int sub = threadIdx.x / width, lane = threadIdx.x - sub * width;
  if (sub >= lpb) return;
  const long lines = (D == 2 ? (long)n : (long)n * n);
  const long N = lines * n;
  for (long line = (long)blockIdx.x * lpb + sub; line < lines * nrhs; line += (long)gridDim.x * lpb) {
    const long rhs = line / lines, l = line - rhs * lines;
    const int c0 = D == 2 ? (int)l : (int)(l / n);
    const int c1 = D == 2 ? 0 : (int)(l - (long)c0 * n);
    const int k0 = c0 == 0 ? 0 : (c0 == n - 1 ? 2 : 1);
    const int k1 = c1 == 0 ? 0 : (c1 == n - 1 ? 2 : 1);
    const float2* vr = v + rhs * N;
    const float2* zr = z + rhs * N;
    for (int c2 = lane; c2 < n; c2 += width) {
      const int k2 = c2 == 0 ? 0 : (c2 == n - 1 ? 2 : 1);
      const long i = l * n + c2;
      float2 acc = make_float2(0.f, 0.f);
      const int cls = D == 2 ? k0 * 3 + k2 : (k0 * 3 + k1) * 3 + k2;
      const float2* al = sa + cls * P3;
#pragma unroll
      for (int t = 0; t < P3; ++t) {
        const int t0 = D == 2 ? t / 3 - 1 : t / 9 - 1;
        const int t1 = D == 2 ? 0 : (t / 3) % 3 - 1;
        const int t2 = t % 3 - 1;
        const int a0 = c0 + t0, a1 = c1 + t1, a2 = c2 + t2;
        if (a0 < 0 || a0 >= n || a2 < 0 || a2 >= n || (D == 3 && (a1 < 0 || a1 >= n))) continue;
        const long j = D == 2 ? (long)a0 * n + a2 : ((long)a0 * n + a1) * n + a2;
        const float2 zv = __ldg(&zr[j]);
        const float2 d = csub(__ldg(&vr[j]), zv);
        acc = cfma(acc, al[t], d);
        const float w = __ldg(&w2m[j]);
        acc = cfms(acc, sc[t], make_float2(w * zv.x, w * zv.y));
      }
      r2[rhs * N + i] = acc;
    }
  }
}

void pre_resid(int d, int n, int nrhs, const float2* v, const float2* z, float2* r2, const float2* alpha32,
               const double2* cint64, const float* w2m32, cudaStream_t st) {
  if (d == 2) {
    launch_roll(true, n, nrhs, v, z, r2, alpha32, cint64, w2m32, st);
    return;
  }
  const unsigned blocks = stencil_blocks(d, n, nrhs);
  if (blocks == 0) return;
  LS_LAUNCH("stencil_c64", st, k_pre_resid<3><<<blocks, 256, 0, st>>>(n, nrhs, v, z, r2, alpha32, cint64, w2m32));
}


template void stencil_apply<float2, float2>(int, int, int, const float2*, float2*, long, long, const void*, cudaStream_t);
template void stencil_apply<double2, float2>(int, int, int, const double2*, float2*, long, long, const void*, cudaStream_t);
template void stencil_apply<double2, double2>(int, int, int, const double2*, double2*, long, long, const void*, cudaStream_t);
template void stencil_apply_pt<float2, float2>(int, int, int, const float2*, float2*, long, long, const void*, cudaStream_t);
template void stencil_apply_pt<double2, float2>(int, int, int, const double2*, float2*, long, long, const void*, cudaStream_t);
template void stencil_apply_pt<double2, double2>(int, int, int, const double2*, double2*, long, long, const void*, cudaStream_t);

}  // namespace ls
