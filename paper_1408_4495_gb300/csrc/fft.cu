// FFT operator apply of the discrete Lippmann-Schwinger operator (Sec. 2.1, eqs. lsd/lso;
// Sec. 1: the convolution structure allows the FFT).
//
//   y = u + K (omega^2 m . u),  (K v)_i = sum_j k_{i-j} v_j,  i, j in [0, n)^d
//
// is computed as a cyclic convolution on the zero-padded grid of L = 2n points per axis
// with the Fourier symbol  s_hat = DFT(kpad) / L^d  of the circulant embedding of k.
// Each axis is transformed by one pass that keeps whole lines in shared memory and runs a
// radix-8 (then 4 or 2) Stockham autosort FFT on them (Stockham formulation as in
// Govindaraju et al., SC'08).  The pad, the omega^2 m scaling, the symbol multiply, the
// crop and the "+u" are fused into the passes, so the only HBM traffic is one read and one
// write of the intermediate per pass.
//
//   2D:  P1 rows(axis 1) fwd  [scale by omega^2 m, pad n -> L]
//        P2 cols(axis 0) fwd, * s_hat, inv, crop -> n     (in place)
//        P3 rows(axis 1) inv, crop -> n, + u
//   3D:  P1 axis 2 fwd [scale, pad] -> P2 axis 1 fwd [pad] -> P3 axis 0 fwd * s_hat inv
//        -> P4 axis 1 inv [crop] -> P5 axis 2 inv [crop, + u]
#include <atomic>
#include <algorithm>
#include <cmath>
#include <type_traits>

#include "common.cuh"
#include "ffloat.cuh"
#include "kernels.h"
#include "prof.h"

namespace ls {

template <> struct RealOf<ffc> { using T = ff; };

// read-only cached load of one complex entry
template <typename C> __device__ __forceinline__ C ldg_c(const C* p) { return __ldg(p); }
template <> __device__ __forceinline__ ffc ldg_c<ffc>(const ffc* p) {
  const float4 v = __ldg(reinterpret_cast<const float4*>(p));
  ffc r;
  r.x = ff(v.x, v.y);
  r.y = ff(v.z, v.w);
  return r;
}

// kernel-class names of the three arithmetics
template <typename C> constexpr const char* arith_tag();
template <> constexpr const char* arith_tag<float2>() { return "c64"; }
template <> constexpr const char* arith_tag<double2>() { return "c128"; }
template <> constexpr const char* arith_tag<ffc>() { return "cff"; }

// Padded shared-memory index: one spare slot every 8 complex entries keeps the strided
// Stockham writes (stride R = 8 in the first pass) free of bank conflicts.
__device__ __forceinline__ int pidx(int i) { return i + (i >> 3); }
template <int L> struct Lay { static constexpr int LS = L + L / 8 + 1; };

template <int SIGN, typename C> __device__ __forceinline__ C rot_i(C a) {
  C r;
  if (SIGN > 0) { r.x = -a.y; r.y = a.x; } else { r.x = a.y; r.y = -a.x; }
  return r;
}

// In-register R-point DFT, out[q] = sum_r v[r] exp(SIGN 2 pi i r q / R).
template <int R, int SIGN, typename C> __device__ __forceinline__ void dft(C* v);
template <> __device__ __forceinline__ void dft<2, -1, float2>(float2* v) { float2 a = v[0]; v[0] = cadd(a, v[1]); v[1] = csub(a, v[1]); }
template <> __device__ __forceinline__ void dft<2, 1, float2>(float2* v) { float2 a = v[0]; v[0] = cadd(a, v[1]); v[1] = csub(a, v[1]); }
template <> __device__ __forceinline__ void dft<2, -1, double2>(double2* v) { double2 a = v[0]; v[0] = cadd(a, v[1]); v[1] = csub(a, v[1]); }
template <> __device__ __forceinline__ void dft<2, 1, double2>(double2* v) { double2 a = v[0]; v[0] = cadd(a, v[1]); v[1] = csub(a, v[1]); }
template <> __device__ __forceinline__ void dft<2, -1, ffc>(ffc* v) { ffc a = v[0]; v[0] = cadd(a, v[1]); v[1] = csub(a, v[1]); }
template <> __device__ __forceinline__ void dft<2, 1, ffc>(ffc* v) { ffc a = v[0]; v[0] = cadd(a, v[1]); v[1] = csub(a, v[1]); }

template <int SIGN, typename C> __device__ __forceinline__ void dft4(C& a0, C& a1, C& a2, C& a3) {
  C t0 = cadd(a0, a2), t1 = csub(a0, a2), t2 = cadd(a1, a3), t3 = rot_i<SIGN>(csub(a1, a3));
  a0 = cadd(t0, t2);
  a2 = csub(t0, t2);
  a1 = cadd(t1, t3);
  a3 = csub(t1, t3);
}

template <int SIGN, typename C> __device__ __forceinline__ void dft4v(C* v) { dft4<SIGN>(v[0], v[1], v[2], v[3]); }

template <typename Rl> __device__ __forceinline__ Rl cos_pi4() { return (Rl)0.70710678118654752440; }
// cos(pi/4) as an FP32 pair: 0.70710677 + 1.21016175e-8
template <> __device__ __forceinline__ ff cos_pi4<ff>() { return ff(0.70710677f, 1.21016175e-8f); }

template <int SIGN, typename C> __device__ __forceinline__ void dft8v(C* v) {
  using Rl = typename RealOf<C>::T;
  const Rl c = cos_pi4<Rl>();
  C e0 = v[0], e1 = v[2], e2 = v[4], e3 = v[6];
  C o0 = v[1], o1 = v[3], o2 = v[5], o3 = v[7];
  dft4<SIGN>(e0, e1, e2, e3);
  dft4<SIGN>(o0, o1, o2, o3);
  // o_q *= W8^q, W8 = exp(SIGN 2 pi i / 8)
  C t;
  t.x = c * (o1.x - SIGN * o1.y); t.y = c * (SIGN * o1.x + o1.y); o1 = t;
  o2 = rot_i<SIGN>(o2);
  t.x = c * (-o3.x - SIGN * o3.y); t.y = c * (SIGN * o3.x - o3.y); o3 = t;
  v[0] = cadd(e0, o0); v[4] = csub(e0, o0);
  v[1] = cadd(e1, o1); v[5] = csub(e1, o1);
  v[2] = cadd(e2, o2); v[6] = csub(e2, o2);
  v[3] = cadd(e3, o3); v[7] = csub(e3, o3);
}

template <int R, int SIGN, typename C> __device__ __forceinline__ void dftR(C* v) {
  if constexpr (R == 8) dft8v<SIGN>(v);
  else if constexpr (R == 4) dft4v<SIGN>(v);
  else dft<2, SIGN, C>(v);
}

// One radix-R Stockham pass over NLINES lines of length L held in shared memory.
// Pass input: sub-transforms of length NS; output: sub-transforms of length NS * R.
// Butterfly j of a line reads entries j + r L/R, multiplies by w^{r k} with
// w = exp(SIGN 2 pi i / (NS R)), k = j mod NS, and writes (j / NS) NS R + k + r NS.
template <typename C, int L, int R, int NS, int SIGN, int NLINES, int NT>
__device__ __forceinline__ void fft_pass(C* s, const C* __restrict__ tw) {
  constexpr int LS = Lay<L>::LS;
  constexpr int BPL = L / R;
  constexpr int BF = NLINES * BPL;
  constexpr int PER = (BF + NT - 1) / NT;
  C v[PER][R];
#pragma unroll
  for (int q = 0; q < PER; ++q) {
    const int b = threadIdx.x + q * NT;
    if (BF % NT == 0 || b < BF) {
      const int line = b / BPL, j = b - line * BPL;
      const C* sl = s + line * LS;
#pragma unroll
      for (int r = 0; r < R; ++r) v[q][r] = sl[pidx(j + r * BPL)];
      if constexpr (NS > 1) {
        const int k = j & (NS - 1);
#pragma unroll
        for (int r = 1; r < R; ++r) {
          C w = ldg_c(&tw[r * k * (L / (NS * R))]);
          if (SIGN > 0) w.y = -w.y;
          v[q][r] = cmul(v[q][r], w);
        }
      }
      dftR<R, SIGN>(v[q]);
    }
  }
  __syncthreads();
#pragma unroll
  for (int q = 0; q < PER; ++q) {
    const int b = threadIdx.x + q * NT;
    if (BF % NT == 0 || b < BF) {
      const int line = b / BPL, j = b - line * BPL;
      C* sl = s + line * LS;
      const int k = j & (NS - 1);
      const int base = (j / NS) * NS * R + k;
#pragma unroll
      for (int r = 0; r < R; ++r) sl[pidx(base + r * NS)] = v[q][r];
    }
  }
  __syncthreads();
}

template <typename C, int L, int NS, int SIGN, int NLINES, int NT>
__device__ __forceinline__ void fft_lines(C* s, const C* __restrict__ tw) {
  if constexpr (NS < L) {
    constexpr int REM = L / NS;
    constexpr int R = REM >= 8 ? 8 : REM;
    fft_pass<C, L, R, NS, SIGN, NLINES, NT>(s, tw);
    fft_lines<C, L, NS * R, SIGN, NLINES, NT>(s, tw);
  }
}

// ------------------------------------------------------------------------------------
// Launch shapes
// ------------------------------------------------------------------------------------
template <int L> struct RowShape {
  static constexpr int NT = (L / 8 > 256) ? L / 8 : 256;
  static constexpr int NL = NT * 8 / L;
};
// TC adjacent lines per CTA (about 64 KB of shared memory); FP32 lines of 512 and more
// take 8 lines and 2 butterflies per thread, so that two CTAs fit an SM's registers
template <typename C, int L> struct ColShape {
  static constexpr int raw = 65536 / (L * (int)sizeof(C));
  static constexpr bool f32_long = sizeof(C) == 8 && L >= 512;
  static constexpr int TC = f32_long ? 8 : (raw < 2 ? 2 : (raw > 16 ? 16 : raw));
  static constexpr int t = f32_long ? TC * L / 16 : TC * L / 8;
  static constexpr int NT = t > 512 ? 512 : (t < 64 ? 64 : t);
};

// ------------------------------------------------------------------------------------
// Row pass: lines contiguous in memory.
// ------------------------------------------------------------------------------------
template <typename C, int L, int SIGN>
__global__ void __launch_bounds__(RowShape<L>::NT) k_row_pass(RowPassArgs a) {
  constexpr int NT = RowShape<L>::NT, NL = RowShape<L>::NL, LS = Lay<L>::LS;
  using Rl = typename RealOf<C>::T;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  C* s = reinterpret_cast<C*>(smem_raw);
  const C* __restrict__ tw = reinterpret_cast<const C*>(a.tw);
  const long line0 = (long)blockIdx.x * NL;
  const int n_in = a.n_in;

  // load n_in entries of NL lines (coalesced), apply the prologue
  if (a.plane_dirs == nullptr) {
    // LB independent loads in flight per thread before the first shared-memory store
    constexpr int LB = 4;
    const int tot = NL * n_in;
    const C* __restrict__ in = reinterpret_cast<const C*>(a.in);
    const Rl* __restrict__ pw = reinterpret_cast<const Rl*>(a.pw);
    for (int base = threadIdx.x; base < tot; base += NT * LB) {
      C v[LB];
      Rl wv[LB];
#pragma unroll
      for (int u = 0; u < LB; ++u) {
        const int idx = base + u * NT;
        v[u] = czero<C>();
        wv[u] = (Rl)1;
        if (idx < tot) {
          const int li = idx / n_in, e = idx - li * n_in;
          const long line = line0 + li;
          if (line < a.lines) {
            if constexpr (std::is_same<C, ffc>::value) {
              v[u] = a.in64 ? ffc_from(reinterpret_cast<const double2*>(a.in)[line * a.in_ls + e])
                            : in[line * a.in_ls + e];
            } else {
              v[u] = in[line * a.in_ls + e];
            }
            if (pw != nullptr) wv[u] = pw[(line % a.pw_lines) * n_in + e];
          }
        }
      }
#pragma unroll
      for (int u = 0; u < LB; ++u) {
        const int idx = base + u * NT;
        if (idx < tot) {
          const int li = idx / n_in, e = idx - li * n_in;
          C x = v[u];
          x.x *= wv[u];
          x.y *= wv[u];
          s[li * LS + pidx(e)] = x;
        }
      }
    }
  } else
  for (int idx = threadIdx.x; idx < NL * n_in; idx += NT) {
    const int li = idx / n_in, e = idx - li * n_in;
    const long line = line0 + li;
    C v = czero<C>();
    if (line < a.lines) {
      if (a.plane_dirs != nullptr) {
        if constexpr (std::is_same<C, double2>::value || std::is_same<C, ffc>::value) {
          // v = -omega^2 m(x) exp(i omega x . dir) (right-hand side, eq. ls), in FP64
          const long q = line % a.pw_lines;      // row within the grid
          const long rhs = line / a.pw_lines;
          const double* dir = a.plane_dirs + rhs * a.d;
          double ph = (double)(e + 1) * dir[a.d - 1];
          long qq = q;
          for (int ax = a.d - 2; ax >= 0; --ax) {
            const long ia = qq % a.n;
            qq /= a.n;
            ph += (double)(ia + 1) * dir[ax];
          }
          ph *= a.omega * a.h;
          double sn, cs;
          sincos(ph, &sn, &cs);
          const double w = a.pw64[q * n_in + e];
          if constexpr (std::is_same<C, ffc>::value) v = ffc_from(make_double2(-w * cs, -w * sn));
          else v = make_double2(-w * cs, -w * sn);
        }
      } else {
        v = reinterpret_cast<const C*>(a.in)[line * a.in_ls + e];
        if (a.pw != nullptr) {
          const Rl w = reinterpret_cast<const Rl*>(a.pw)[(line % a.pw_lines) * n_in + e];
          v.x *= w;
          v.y *= w;
        }
      }
    }
    s[li * LS + pidx(e)] = v;
  }
  if (n_in < L) {
    const int padn = L - n_in;
    for (int idx = threadIdx.x; idx < NL * padn; idx += NT) {
      const int li = idx / padn, e = n_in + (idx - li * padn);
      s[li * LS + pidx(e)] = czero<C>();
    }
  }
  __syncthreads();
  fft_lines<C, L, 1, SIGN, NL, NT>(s, tw);
  const int n_out = a.n_out;
  C* out = reinterpret_cast<C*>(a.out);
  const C* addv = reinterpret_cast<const C*>(a.addv);
  for (int idx = threadIdx.x; idx < NL * n_out; idx += NT) {
    const int li = idx / n_out, e = idx - li * n_out;
    const long line = line0 + li;
    if (line < a.lines) {
      C v = s[li * LS + pidx(e)];
      if constexpr (std::is_same<C, ffc>::value) {
        if (a.out64) {
          // FP64 epilogue: y = v + addv, or y = subv - (v + addv)
          double2 o = ffc_to(v);
          if (a.addv != nullptr) o = cadd(o, reinterpret_cast<const double2*>(a.addv)[line * a.add_ls + e]);
          if (a.subv != nullptr) o = csub(reinterpret_cast<const double2*>(a.subv)[line * a.add_ls + e], o);
          reinterpret_cast<double2*>(a.out)[line * a.out_ls + e] = o;
          continue;
        }
      }
      if (addv != nullptr) v = cadd(v, addv[line * a.add_ls + e]);
      out[line * a.out_ls + e] = v;
    }
  }
}

// ------------------------------------------------------------------------------------
// Column pass: lines strided (element stride es), TC adjacent lines per CTA.
// MODE 0: forward; 1: inverse; 2: forward, multiply by the symbol, inverse.
// ------------------------------------------------------------------------------------
template <typename C, int L, int MODE>
__global__ void __launch_bounds__(ColShape<C, L>::NT) k_col_pass(ColPassArgs a) {
  constexpr int NT = ColShape<C, L>::NT, TC = ColShape<C, L>::TC, LS = Lay<L>::LS;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  C* s = reinterpret_cast<C*>(smem_raw);
  const C* __restrict__ tw = reinterpret_cast<const C*>(a.tw);
  const long tiles = (a.inner + TC - 1) / TC;
  const long o = blockIdx.x / tiles;
  const long c0 = (blockIdx.x - o * tiles) * TC;
  const C* in = reinterpret_cast<const C*>(a.in) + o * a.in_os + c0;
  const int n_in = a.n_in;
  {
    // LB independent loads in flight per thread before the first shared-memory store
    constexpr int LB = 4;
    const int tot = n_in * TC;
    for (int base = threadIdx.x; base < tot; base += NT * LB) {
      C v[LB];
#pragma unroll
      for (int u = 0; u < LB; ++u) {
        const int idx = base + u * NT;
        v[u] = czero<C>();
        if (idx < tot) {
          const int e = idx / TC, c = idx - e * TC;
          if (c0 + c < a.inner) v[u] = in[(long)e * a.in_es + c];
        }
      }
#pragma unroll
      for (int u = 0; u < LB; ++u) {
        const int idx = base + u * NT;
        if (idx < tot) {
          const int e = idx / TC, c = idx - e * TC;
          s[c * LS + pidx(e)] = v[u];
        }
      }
    }
  }
  if (n_in < L) {
    const int padn = L - n_in;
    for (int idx = threadIdx.x; idx < padn * TC; idx += NT) {
      const int e = n_in + idx / TC, c = idx % TC;
      s[c * LS + pidx(e)] = czero<C>();
    }
  }
  __syncthreads();
  if constexpr (MODE == 0) {
    fft_lines<C, L, 1, -1, TC, NT>(s, tw);
  } else if constexpr (MODE == 1) {
    fft_lines<C, L, 1, 1, TC, NT>(s, tw);
  } else {
    fft_lines<C, L, 1, -1, TC, NT>(s, tw);
    const C* __restrict__ sym = reinterpret_cast<const C*>(a.sym);
    const int n1 = a.n + 1;
    // symbol values of SB entries loaded together, then applied
    constexpr int SB = 8;
    for (int base = threadIdx.x; base < L * TC; base += NT * SB) {
      C sv[SB];
#pragma unroll
      for (int u = 0; u < SB; ++u) {
        const int idx = base + u * NT;
        const int e = idx / TC, c = idx - e * TC;
        const long cc = c0 + c;
        sv[u] = czero<C>();
        if (idx < L * TC && cc < a.inner) {
          const int q0 = e <= L - e ? e : L - e;
          long si;
          if (a.d == 2) {
            const int k1 = (int)cc;
            si = (long)q0 * n1 + (k1 <= L - k1 ? k1 : L - k1);
          } else {
            const int k1 = (int)(cc / L), k2 = (int)(cc - (long)k1 * L);
            si = ((long)q0 * n1 + (k1 <= L - k1 ? k1 : L - k1)) * n1 + (k2 <= L - k2 ? k2 : L - k2);
          }
          sv[u] = ldg_c(&sym[si]);
        }
      }
#pragma unroll
      for (int u = 0; u < SB; ++u) {
        const int idx = base + u * NT;
        const int e = idx / TC, c = idx - e * TC;
        if (idx < L * TC && c0 + c < a.inner) {
          C& v = s[c * LS + pidx(e)];
          v = cmul(v, sv[u]);
        }
      }
    }
    __syncthreads();
    fft_lines<C, L, 1, 1, TC, NT>(s, tw);
  }
  C* out = reinterpret_cast<C*>(a.out) + o * a.out_os + c0;
  const int n_out = a.n_out;
  for (int idx = threadIdx.x; idx < n_out * TC; idx += NT) {
    const int e = idx / TC, c = idx - e * TC;
    if (c0 + c < a.inner) out[(long)e * a.out_es + c] = s[c * LS + pidx(e)];
  }
}

// ------------------------------------------------------------------------------------
// Host dispatch
// ------------------------------------------------------------------------------------
template <typename C, int L, int SIGN> static void launch_row_L(const RowPassArgs& a, cudaStream_t st) {
  constexpr int NT = RowShape<L>::NT, NL = RowShape<L>::NL;
  const size_t smem = (size_t)NL * Lay<L>::LS * sizeof(C);
  static std::atomic<bool> attr{false};  // set once per process; repeats are harmless
  if (!attr.load(std::memory_order_acquire)) {
    LS_CUDA(cudaFuncSetAttribute(k_row_pass<C, L, SIGN>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    attr.store(true, std::memory_order_release);
  }
  const long blocks = (a.lines + NL - 1) / NL;
  if (blocks == 0) return;
  static const std::string cls = std::string(SIGN < 0 ? "fft_row_fwd_" : "fft_row_inv_") + arith_tag<C>();
  LS_LAUNCH(cls.c_str(), st, k_row_pass<C, L, SIGN><<<(unsigned)blocks, NT, smem, st>>>(a));
}

template <typename C, int L, int MODE> static void launch_col_L(const ColPassArgs& a, cudaStream_t st) {
  constexpr int NT = ColShape<C, L>::NT, TC = ColShape<C, L>::TC;
  const size_t smem = (size_t)TC * Lay<L>::LS * sizeof(C);
  static std::atomic<bool> attr{false};  // set once per process; repeats are harmless
  if (!attr.load(std::memory_order_acquire)) {
    LS_CUDA(cudaFuncSetAttribute(k_col_pass<C, L, MODE>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    attr.store(true, std::memory_order_release);
  }
  const long tiles = (a.inner + TC - 1) / TC;
  const long blocks = tiles * a.outer;
  if (blocks == 0) return;
  static const std::string cls =
      std::string(MODE == 0 ? "fft_col_fwd_" : MODE == 1 ? "fft_col_inv_" : "fft_col_sym_") + arith_tag<C>();
  LS_LAUNCH(cls.c_str(), st, k_col_pass<C, L, MODE><<<(unsigned)blocks, NT, smem, st>>>(a));
}

#define LS_FOR_L(X) X(16) X(32) X(64) X(128) X(256) X(512) X(1024) X(2048) X(4096)

template <typename C> void row_pass(int L, int sign, const RowPassArgs& a, cudaStream_t st) {
  switch (L) {
#define CASE(LL)                                                     \
  case LL:                                                           \
    if (sign < 0) launch_row_L<C, LL, -1>(a, st);                    \
    else launch_row_L<C, LL, 1>(a, st);                              \
    return;
    LS_FOR_L(CASE)
#undef CASE
  }
  LS_FAIL(EINVAL_, "unsupported FFT length %d", L);
}

template <typename C> void col_pass(int L, int mode, const ColPassArgs& a, cudaStream_t st) {
  switch (L) {
#define CASE(LL)                                                     \
  case LL:                                                           \
    if (mode == 0) launch_col_L<C, LL, 0>(a, st);                    \
    else if (mode == 1) launch_col_L<C, LL, 1>(a, st);               \
    else launch_col_L<C, LL, 2>(a, st);                              \
    return;
    LS_FOR_L(CASE)
#undef CASE
  }
  LS_FAIL(EINVAL_, "unsupported FFT length %d", L);
}

template void row_pass<float2>(int, int, const RowPassArgs&, cudaStream_t);
template void row_pass<double2>(int, int, const RowPassArgs&, cudaStream_t);
template void col_pass<float2>(int, int, const ColPassArgs&, cudaStream_t);
template void col_pass<double2>(int, int, const ColPassArgs&, cudaStream_t);
template void row_pass<ffc>(int, int, const RowPassArgs&, cudaStream_t);
template void col_pass<ffc>(int, int, const ColPassArgs&, cudaStream_t);

// ------------------------------------------------------------------------------------
// Operator-level sequences
// ------------------------------------------------------------------------------------

// y = (I + K omega^2 m) u  (add_u = true)  or  y = K (omega^2 m u)  (add_u = false),
// or the right-hand side g = K(-omega^2 m u_I) when plane_dirs != null (FP64 or float-float).
// C is the arithmetic of the passes; with in64 / out64 the first pass reads and the last
// pass writes FP64 (u, y, sub are then double2), and sub != null gives y = sub - (...).
template <typename C>
static void conv_run(const ConvPlan& p, int nrhs, const void* u, void* y, const double* plane_dirs, bool add_u,
                     const void* sub, int in64, int out64, const void* tw, const void* sym, const void* w2m,
                     void* scratch1, void* scratch2, cudaStream_t st) {
  const int n = p.n, L = 2 * n, d = p.d;
  const long rows = (d == 2) ? (long)n : (long)n * n;  // lines of one grid along the last axis
  C* T1 = reinterpret_cast<C*>(scratch1);
  RowPassArgs r{};
  r.in = u; r.out = T1; r.lines = (long)nrhs * rows; r.n_in = n; r.n_out = L;
  r.in_ls = n; r.out_ls = L; r.pw = w2m; r.pw_lines = rows; r.tw = tw;
  r.plane_dirs = plane_dirs; r.d = d; r.n = n; r.omega = p.omega; r.h = p.h; r.in64 = in64;
  r.pw64 = p.w2m64;
  row_pass<C>(L, -1, r, st);
  if (d == 2) {
    ColPassArgs c{};
    c.in = T1; c.out = T1; c.outer = nrhs; c.inner = L;
    c.in_os = (long)n * L; c.in_es = L; c.out_os = (long)n * L; c.out_es = L;
    c.n_in = n; c.n_out = n; c.sym = sym; c.n = n; c.d = 2; c.tw = tw;
    col_pass<C>(L, 2, c, st);
  } else {
    C* T2 = reinterpret_cast<C*>(scratch2);
    ColPassArgs c{};
    c.tw = tw; c.n = n; c.d = 3; c.sym = sym;
    // axis 1 forward, pad n -> L
    c.in = T1; c.out = T2; c.outer = (long)nrhs * n; c.inner = L;
    c.in_os = (long)n * L; c.in_es = L; c.out_os = (long)L * L; c.out_es = L; c.n_in = n; c.n_out = L;
    col_pass<C>(L, 0, c, st);
    // axis 0: forward (pad), symbol, inverse, crop
    c.in = T2; c.out = T2; c.outer = nrhs; c.inner = (long)L * L;
    c.in_os = (long)n * L * L; c.in_es = (long)L * L; c.out_os = c.in_os; c.out_es = c.in_es; c.n_in = n; c.n_out = n;
    col_pass<C>(L, 2, c, st);
    // axis 1 inverse, crop L -> n
    c.in = T2; c.out = T1; c.outer = (long)nrhs * n; c.inner = L;
    c.in_os = (long)L * L; c.in_es = L; c.out_os = (long)n * L; c.out_es = L; c.n_in = L; c.n_out = n;
    col_pass<C>(L, 1, c, st);
  }
  RowPassArgs q{};
  q.in = T1; q.out = y; q.lines = (long)nrhs * rows; q.n_in = L; q.n_out = n;
  q.in_ls = L; q.out_ls = n; q.tw = tw; q.addv = add_u ? u : nullptr; q.add_ls = n;
  q.subv = sub; q.out64 = out64;
  row_pass<C>(L, 1, q, st);
}

template <typename C>
void conv_apply(const ConvPlan& p, int nrhs, const C* u, C* y, const double* plane_dirs, bool add_u,
                void* scratch1, void* scratch2, cudaStream_t st) {
  const bool f32 = std::is_same<C, float2>::value;
  conv_run<C>(p, nrhs, u, y, plane_dirs, add_u, nullptr, 0, 0, f32 ? (const void*)p.tw32 : (const void*)p.tw64,
              f32 ? (const void*)p.sym32 : (const void*)p.sym64, f32 ? (const void*)p.w2m32 : (const void*)p.w2m64,
              scratch1, scratch2, st);
}

void conv_apply_ff(const ConvPlan& p, int nrhs, const double2* u, double2* y, const double2* sub, void* scratch1,
                   void* scratch2, cudaStream_t st) {
  if (!p.twff || !p.symff || !p.w2mff) LS_FAIL(ESTATE_, "float-float operator tables missing");
  conv_run<ffc>(p, nrhs, u, y, nullptr, true, sub, 1, 1, p.twff, p.symff, p.w2mff, scratch1, scratch2, st);
}

void conv_rhs_ff(const ConvPlan& p, int nrhs, const double* plane_dirs, double2* g, void* scratch1, void* scratch2,
                 cudaStream_t st) {
  if (!p.twff || !p.symff) LS_FAIL(ESTATE_, "float-float operator tables missing");
  conv_run<ffc>(p, nrhs, nullptr, g, plane_dirs, false, nullptr, 0, 1, p.twff, p.symff, p.w2mff, scratch1, scratch2,
                st);
}

template void conv_apply<float2>(const ConvPlan&, int, const float2*, float2*, const double*, bool, void*, void*, cudaStream_t);
template void conv_apply<double2>(const ConvPlan&, int, const double2*, double2*, const double*, bool, void*, void*, cudaStream_t);

size_t conv_scratch1_elems(int d, int n, int nrhs) {
  const size_t L = 2 * (size_t)n;
  return d == 2 ? (size_t)nrhs * n * L : (size_t)nrhs * n * n * L;
}
size_t conv_scratch2_elems(int d, int n, int nrhs) {
  const size_t L = 2 * (size_t)n;
  return d == 2 ? 0 : (size_t)nrhs * n * L * L;
}

// ------------------------------------------------------------------------------------
// Sec. 2.1: Nystrom table and the symbol of its circulant embedding (FP64 on the device)
// ------------------------------------------------------------------------------------

// k_t for t in [0, n]^d (the table is even in every component).  2D: G = (i/4) H0(omega r),
// 3D: G = exp(i omega r) / (4 pi r); k_t = G(h|t|) h^d; k_0 = integral of G over the disk /
// ball of area / volume h^d (closed form, see the oracle docstring for the derivation).
// omega = 0 in 3D is the Laplace kernel of Sec. 5: G = 1 / (4 pi r), k_0 = a^2 / 2.
__global__ void k_kernel_quadrant(double2* ktq, int d, int n, double omega, double h) {
  const long n1 = n + 1;
  const long total = d == 2 ? n1 * n1 : n1 * n1 * n1;
  for (long idx = blockIdx.x * (long)blockDim.x + threadIdx.x; idx < total; idx += (long)gridDim.x * blockDim.x) {
    long q = idx;
    double r2 = 0;
    for (int a = 0; a < d; ++a) {
      const long t = q % n1;
      q /= n1;
      r2 += (double)(t * t);
    }
    double2 k;
    if (d == 2) {
      const double hd = h * h;
      if (r2 == 0) {
        const double a = h / sqrt(M_PI);
        const double z = omega * a;
        // (i pi a / (2 omega)) (J1 + i Y1) - 1/omega^2
        const double f = M_PI * a / (2.0 * omega);
        k.x = -f * y1(z) - 1.0 / (omega * omega);
        k.y = f * j1(z);
      } else {
        const double z = omega * h * sqrt(r2);
        // (i/4)(J0 + i Y0) h^2
        k.x = -0.25 * y0(z) * hd;
        k.y = 0.25 * j0(z) * hd;
      }
    } else {
      const double hd = h * h * h;
      if (omega == 0.0) {
        const double a = h * cbrt(3.0 / (4.0 * M_PI));
        k.x = r2 == 0 ? 0.5 * a * a : hd / (4.0 * M_PI * h * sqrt(r2));
        k.y = 0.0;
      } else if (r2 == 0) {
        const double a = h * cbrt(3.0 / (4.0 * M_PI));
        double sn, cs;
        sincos(omega * a, &sn, &cs);
        // e^{i w a} (1/w^2 - i a / w) - 1/w^2
        const double p = 1.0 / (omega * omega), qv = -a / omega;
        k.x = cs * p - sn * qv - p;
        k.y = sn * p + cs * qv;
      } else {
        const double r = h * sqrt(r2);
        double sn, cs;
        sincos(omega * r, &sn, &cs);
        const double f = hd / (4.0 * M_PI * r);
        k.x = cs * f;
        k.y = sn * f;
      }
    }
    ktq[idx] = k;
  }
}

// kpad[k] = k_{t(k)} with t = k for k < n, k - L for k > n, and 0 where any k_a == n.
__global__ void k_kernel_pad(const double2* ktq, double2* kpad, int d, int n) {
  const long L = 2 * n, n1 = n + 1;
  const long total = d == 2 ? L * L : L * L * L;
  for (long idx = blockIdx.x * (long)blockDim.x + threadIdx.x; idx < total; idx += (long)gridDim.x * blockDim.x) {
    long q = idx, src = 0, mul = 1;
    bool zero = false;
    for (int a = 0; a < d; ++a) {
      const long k = q % L;
      q /= L;
      if (k == n) zero = true;
      const long t = k < n ? k : L - k;
      src += t * mul;
      mul *= n1;
    }
    kpad[idx] = zero ? make_double2(0, 0) : ktq[src];
  }
}

// sym[q] = spectrum[q] / L^d on the quadrant q in [0, n]^d; FP64 and FP32 copies.
__global__ void k_symbol_quadrant(const double2* spec, double2* sym64, float2* sym32, int d, int n) {
  const long L = 2 * n, n1 = n + 1;
  const long total = d == 2 ? n1 * n1 : n1 * n1 * n1;
  const double scale = d == 2 ? 1.0 / (double)(L * L) : 1.0 / (double)(L * L * L);
  for (long idx = blockIdx.x * (long)blockDim.x + threadIdx.x; idx < total; idx += (long)gridDim.x * blockDim.x) {
    long q = idx, dst = 0, mul = 1;
    for (int a = 0; a < d; ++a) {
      const long k = q % n1;
      q /= n1;
      dst += k * mul;
      mul *= L;
    }
    double2 v = spec[dst];
    v.x *= scale;
    v.y *= scale;
    sym64[idx] = v;
    sym32[idx] = make_float2((float)v.x, (float)v.y);
  }
}

// float-float copies of FP64 tables (two floats per real)
__global__ void k_to_ff(const double* __restrict__ src, float2* __restrict__ dst, long count) {
  for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < count; i += (long)gridDim.x * blockDim.x) {
    const ff v = ff_from(src[i]);
    dst[i] = make_float2(v.hi, v.lo);
  }
}

void to_ff(const double* src, void* dst, long count, cudaStream_t st) {
  if (count <= 0) return;
  LS_LAUNCH("to_ff", st, k_to_ff<<<512, 256, 0, st>>>(src, reinterpret_cast<float2*>(dst), count));
}

// Sec. 5 right-hand side g = K f for delta sources: f_j = q_r / h^d at the source point p_r
// (unit mass on the cell), so g_r(i) = q_r k_{i - p_r} / h^d, read from the quadrant table
// at |i - p_r| (componentwise).  One thread per output entry, r outermost.
__global__ void k_point_source(double2* g, const int* __restrict__ pts, const double2* __restrict__ q,
                               const double2* __restrict__ ktq, int d, int n, int nrhs, double inv_hd) {
  const long N = d == 2 ? (long)n * n : (long)n * n * n, n1 = n + 1;
  const long total = N * nrhs;
  for (long e = blockIdx.x * (long)blockDim.x + threadIdx.x; e < total; e += (long)gridDim.x * blockDim.x) {
    const int r = (int)(e / N);
    long i = e - (long)r * N, src = 0, mul = 1;
    for (int a = d - 1; a >= 0; --a) {  // C order: the last index is the fastest
      const long ia = i % n;
      i /= n;
      const long t = ia - pts[(size_t)r * d + a];
      src += (t < 0 ? -t : t) * mul;
      mul *= n1;
    }
    const double2 k = ktq[src], s = q ? q[r] : make_double2(1.0, 0.0);
    g[e] = make_double2((k.x * s.x - k.y * s.y) * inv_hd, (k.x * s.y + k.y * s.x) * inv_hd);
  }
}

void point_source(int d, int n, int nrhs, const int* pts, const double2* q, const double2* ktq, double h, double2* g,
                  cudaStream_t st) {
  const double hd = d == 2 ? h * h : h * h * h;
  LS_LAUNCH("point_source", st, k_point_source<<<1024, 256, 0, st>>>(g, pts, q, ktq, d, n, nrhs, 1.0 / hd));
}

void build_kernel_table(int d, int n, double omega, double h, double2* ktq, cudaStream_t st) {
  LS_LAUNCH("kernel_table", st, k_kernel_quadrant<<<1024, 256, 0, st>>>(ktq, d, n, omega, h));
}

void build_symbol(const ConvPlan& p, const double2* ktq, double2* sym64, float2* sym32, double2* work,
                  cudaStream_t st) {
  const int d = p.d, n = p.n, L = 2 * n;
  LS_LAUNCH("kernel_pad", st, k_kernel_pad<<<1024, 256, 0, st>>>(ktq, work, d, n));
  const long lines = d == 2 ? (long)L : (long)L * L;
  RowPassArgs r{};
  r.in = work; r.out = work; r.lines = lines; r.n_in = L; r.n_out = L; r.in_ls = L; r.out_ls = L; r.tw = p.tw64;
  row_pass<double2>(L, -1, r, st);
  ColPassArgs c{};
  c.tw = p.tw64; c.n_in = L; c.n_out = L; c.in = work; c.out = work;
  if (d == 2) {
    c.outer = 1; c.inner = L; c.in_os = 0; c.out_os = 0; c.in_es = L; c.out_es = L;
    col_pass<double2>(L, 0, c, st);
  } else {
    c.outer = L; c.inner = L; c.in_os = (long)L * L; c.out_os = c.in_os; c.in_es = L; c.out_es = L;
    col_pass<double2>(L, 0, c, st);
    c.outer = 1; c.inner = (long)L * L; c.in_os = 0; c.out_os = 0; c.in_es = (long)L * L; c.out_es = c.in_es;
    col_pass<double2>(L, 0, c, st);
  }
  LS_LAUNCH("symbol", st, k_symbol_quadrant<<<1024, 256, 0, st>>>(work, sym64, sym32, d, n));
}

}  // namespace ls
