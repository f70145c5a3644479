// Kernels and launchers of the FFT passes (the radix-8/4/2 Stockham line transforms in shared
// memory, with the pad, omega^2 m scale, symbol multiply, crop and "+u" fused in).  The
// operator-level sequence that chains them is in fft.cu; each arithmetic (FP32, FP64,
// float-float) instantiates the passes in its own translation units (fft_pass_*.cu) so that
// they compile in parallel.
#pragma once

#include <atomic>
#include <algorithm>
#include <cmath>
#include <type_traits>

#include "common.cuh"
#include "ffloat.cuh"
#include "fft_plan.h"
#include "kernels.h"
#include "prof.h"

namespace ls {

template <> struct RealOf<ffc> { using T = ff; };

// Float-float arithmetic inside the passes: the deferred-renormalisation forms of
// ffloat.cuh (lz_add, lz_mul, lz_norm); every value is renormalised when a pass stores it to
// shared memory, so within one radix pass the trailing part stays below about 2^-21 of the
// leading one and the dropped lo * lo term below 2^-42 relative.
__device__ __forceinline__ ffc cadd(ffc a, ffc b) {
  ffc r;
  r.x = lz_add(a.x, b.x);
  r.y = lz_add(a.y, b.y);
  return r;
}
__device__ __forceinline__ ffc csub(ffc a, ffc b) {
  ffc r;
  r.x = lz_add(a.x, lz_neg(b.x));
  r.y = lz_add(a.y, lz_neg(b.y));
  return r;
}
__device__ __forceinline__ ffc cmul(ffc a, ffc b) {
  ffc r;
  r.x = lz_add(lz_mul(a.x, b.x), lz_neg(lz_mul(a.y, b.y)));
  r.y = lz_add(lz_mul(a.x, b.y), lz_mul(a.y, b.x));
  return r;
}
// real helpers of the butterflies: plain arithmetic, deferred float-float for ff
template <typename Rl> __device__ __forceinline__ Rl r_mul(Rl a, Rl b) { return a * b; }
template <> __device__ __forceinline__ ff r_mul<ff>(ff a, ff b) { return lz_mul(a, b); }
template <typename Rl> __device__ __forceinline__ Rl r_add(Rl a, Rl b) { return a + b; }
template <> __device__ __forceinline__ ff r_add<ff>(ff a, ff b) { return lz_add(a, b); }
template <typename Rl> __device__ __forceinline__ Rl r_sub(Rl a, Rl b) { return a - b; }
template <> __device__ __forceinline__ ff r_sub<ff>(ff a, ff b) { return lz_add(a, lz_neg(b)); }
template <typename Rl> __device__ __forceinline__ Rl r_neg(Rl a) { return -a; }
template <> __device__ __forceinline__ ff r_neg<ff>(ff a) { return lz_neg(a); }
template <typename C> __device__ __forceinline__ C c_norm(C v) { return v; }
template <> __device__ __forceinline__ ffc c_norm<ffc>(ffc v) {
  v.x = lz_norm(v.x);
  v.y = lz_norm(v.y);
  return v;
}

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

// Shared-memory layout of the LINES lines of a CTA: line-major without padding; inside
// each 128-byte row of E entries (E = 16 FP32 complex or 8 16-byte entries) the entry
// position is XORed with a function h of the row index and the line (a bank swizzle).  A
// warp's accesses then fall on distinct banks in every pass (modelled per half-warp for
// 8-byte and per quarter-warp for 16-byte entries, the units in which shared memory serves
// them):
//   - loads of consecutive entries, and stores at Stockham strides NS >= E, stay inside
//     whole rows, which the XOR permutes;
//   - the stride-R stores of the first pass (NS = 1) spread over R rows: h's low bits
//     follow the row index, so they land on distinct positions;
//   - the NS = 8 stores (8-byte entries) take two rows R / 2 or 4 apart for the two halves
//     of a half-warp: h's bit 3 carries the parity of the row's low three bits, so the
//     halves differ in it;
//   - h depends on the row's low three bits only, so entries 8 E apart (multiples of whole
//     8-row blocks) share it: a thread's R accesses at such strides take one swizzle and
//     constant offsets, which keeps the address arithmetic (and registers) of the long
//     passes at the level of a plain layout;
//   - column fill, symbol multiply and drain touch E / LINES entries of each line at once:
//     the line term shifts the lines E / LINES positions apart.
// Padding one entry in every 8 instead keeps the first pass's strided stores apart but
// makes every run of 16 consecutive 8-byte entries wrap onto its own banks (67 % extra
// shared-memory wavefronts in the FP32 column pass of L = 2048, measured with ncu).
template <typename C, int L, int LINES> struct SLay {
  static constexpr int E = 128 / (int)sizeof(C);
  static constexpr int KC = E / LINES > 1 ? E / LINES : 1;
  static constexpr int SIZE = LINES * L;  // entries
  static_assert(L % E == 0, "line length must be a multiple of the swizzle row");
  __host__ __device__ static constexpr bool shift_free(int stride) { return stride % (8 * E) == 0; }
  // entries 4 E apart (an odd multiple): their rows' low three bits differ by 4, which flips
  // bit 2 of the swizzle and the parity bit: h alternates between h0 and h0 ^ HALF_FLIP
  __host__ __device__ static constexpr bool half_shift(int stride) {
    return stride % (4 * E) == 0 && stride % (8 * E) != 0;
  }
  static constexpr int HALF_FLIP = E == 16 ? 12 : 4;
  // entries i0 + r, r < 8, of one line with i0 a multiple of 8 share a row and its swizzle:
  // their offsets are rb + (q ^ r)
  __device__ static __forceinline__ void group8(int line, int i0, int& rb, int& q) {
    const int row = (i0 / E) & 7;
    int h = row ^ (line * KC);
    if constexpr (E == 16) h ^= ((row ^ (row >> 1) ^ (row >> 2)) & 1) << 3;
    rb = line * L + (i0 & ~(E - 1));
    q = (i0 ^ h) & (E - 1);
  }
  __device__ static __forceinline__ int off(int line, int i) {
    const int row = (i / E) & 7;
    int h = row ^ (line * KC);
    if constexpr (E == 16) h ^= ((row ^ (row >> 1) ^ (row >> 2)) & 1) << 3;
    return line * L + (i & ~(E - 1)) + ((i ^ h) & (E - 1));
  }
};

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
  if (SIGN > 0) {
    t.x = r_mul(c, r_sub(o1.x, o1.y)); t.y = r_mul(c, r_add(o1.x, o1.y)); o1 = t;
  } else {
    t.x = r_mul(c, r_add(o1.x, o1.y)); t.y = r_mul(c, r_sub(o1.y, o1.x)); o1 = t;
  }
  o2 = rot_i<SIGN>(o2);
  if (SIGN > 0) {
    t.x = r_neg(r_mul(c, r_add(o3.x, o3.y))); t.y = r_mul(c, r_sub(o3.x, o3.y)); o3 = t;
  } else {
    t.x = r_mul(c, r_sub(o3.y, o3.x)); t.y = r_neg(r_mul(c, r_add(o3.x, o3.y))); o3 = t;
  }
  v[0] = cadd(e0, o0); v[4] = csub(e0, o0);
  v[1] = cadd(e1, o1); v[5] = csub(e1, o1);
  v[2] = cadd(e2, o2); v[6] = csub(e2, o2);
  v[3] = cadd(e3, o3); v[7] = csub(e3, o3);
}

template <typename Rl> __device__ __forceinline__ Rl sin_pi3() { return (Rl)0.86602540378443864676; }
// sin(pi/3) = sqrt(3)/2 as an FP32 pair: 0.8660254 + 1.5543625e-8
template <> __device__ __forceinline__ ff sin_pi3<ff>() { return ff(0.8660254f, 1.5543625e-8f); }
template <typename Rl> __device__ __forceinline__ Rl one_half() { return (Rl)0.5; }
template <> __device__ __forceinline__ ff one_half<ff>() { return ff(0.5f, 0.f); }

// 3-point DFT with w = exp(SIGN 2 pi i / 3) = -1/2 + SIGN i sqrt(3)/2:
// X0 = a + (b + c), X1 = a - (b + c)/2 + SIGN i sqrt(3)/2 (b - c), X2 = the same with - for +
template <int SIGN, typename C> __device__ __forceinline__ void dft3v(C* v) {
  using Rl = typename RealOf<C>::T;
  const Rl s3 = sin_pi3<Rl>(), half = one_half<Rl>();
  const C a = v[0], t = cadd(v[1], v[2]);
  C m, d = csub(v[1], v[2]);
  m.x = r_sub(a.x, r_mul(half, t.x));
  m.y = r_sub(a.y, r_mul(half, t.y));
  d.x = r_mul(s3, d.x);
  d.y = r_mul(s3, d.y);
  const C r = rot_i<SIGN>(d);
  v[0] = cadd(a, t);
  v[1] = cadd(m, r);
  v[2] = csub(m, r);
}

template <int R, int SIGN, typename C> __device__ __forceinline__ void dftR(C* v) {
  if constexpr (R == 8) dft8v<SIGN>(v);
  else if constexpr (R == 4) dft4v<SIGN>(v);
  else if constexpr (R == 3) dft3v<SIGN>(v);
  else dft<2, SIGN, C>(v);
}

// Pruned butterflies for the zero-padded transforms: every forward transform of the
// operator reads n = L / 2 entries (the rest is zero padding) and every inverse one keeps
// n = L / 2 outputs (the crop).
// 4-point DFT of (a0, a1, 0, 0): X0 = a0 + a1, X1 = a0 + rot(a1), X2 = a0 - a1, X3 = a0 - rot(a1)
template <int SIGN, typename C> __device__ __forceinline__ void dft4_lo(C& a0, C& a1, C& a2, C& a3) {
  const C b = a1, r = rot_i<SIGN>(a1);
  a1 = cadd(a0, r);
  a2 = csub(a0, b);
  a3 = csub(a0, r);
  a0 = cadd(a0, b);
}
// 8-point DFT of (v0, v1, v2, v3, 0, 0, 0, 0) (the first pass of a padded transform)
template <int SIGN, typename C> __device__ __forceinline__ void dft8v_lo(C* v) {
  using Rl = typename RealOf<C>::T;
  const Rl c = cos_pi4<Rl>();
  C e0 = v[0], e1 = v[2], e2, e3;
  C o0 = v[1], o1 = v[3], o2, o3;
  dft4_lo<SIGN>(e0, e1, e2, e3);
  dft4_lo<SIGN>(o0, o1, o2, o3);
  C t;
  if (SIGN > 0) {
    t.x = r_mul(c, r_sub(o1.x, o1.y)); t.y = r_mul(c, r_add(o1.x, o1.y)); o1 = t;
  } else {
    t.x = r_mul(c, r_add(o1.x, o1.y)); t.y = r_mul(c, r_sub(o1.y, o1.x)); o1 = t;
  }
  o2 = rot_i<SIGN>(o2);
  if (SIGN > 0) {
    t.x = r_neg(r_mul(c, r_add(o3.x, o3.y))); t.y = r_mul(c, r_sub(o3.x, o3.y)); o3 = t;
  } else {
    t.x = r_mul(c, r_sub(o3.y, o3.x)); t.y = r_neg(r_mul(c, r_add(o3.x, o3.y))); o3 = t;
  }
  v[0] = cadd(e0, o0); v[4] = csub(e0, o0);
  v[1] = cadd(e1, o1); v[5] = csub(e1, o1);
  v[2] = cadd(e2, o2); v[6] = csub(e2, o2);
  v[3] = cadd(e3, o3); v[7] = csub(e3, o3);
}
// outputs 0 .. R/2 - 1 only (the last pass of a cropped transform; R even)
template <int R, int SIGN, typename C> __device__ __forceinline__ void dftR_hi_cut(C* v) {
  if constexpr (R == 8) {
    using Rl = typename RealOf<C>::T;
    const Rl c = cos_pi4<Rl>();
    C e0 = v[0], e1 = v[2], e2 = v[4], e3 = v[6];
    C o0 = v[1], o1 = v[3], o2 = v[5], o3 = v[7];
    dft4<SIGN>(e0, e1, e2, e3);
    dft4<SIGN>(o0, o1, o2, o3);
    C t;
    if (SIGN > 0) {
      t.x = r_mul(c, r_sub(o1.x, o1.y)); t.y = r_mul(c, r_add(o1.x, o1.y)); o1 = t;
    } else {
      t.x = r_mul(c, r_add(o1.x, o1.y)); t.y = r_mul(c, r_sub(o1.y, o1.x)); o1 = t;
    }
    o2 = rot_i<SIGN>(o2);
    if (SIGN > 0) {
      t.x = r_neg(r_mul(c, r_add(o3.x, o3.y))); t.y = r_mul(c, r_sub(o3.x, o3.y)); o3 = t;
    } else {
      t.x = r_mul(c, r_sub(o3.y, o3.x)); t.y = r_neg(r_mul(c, r_add(o3.x, o3.y))); o3 = t;
    }
    v[0] = cadd(e0, o0);
    v[1] = cadd(e1, o1);
    v[2] = cadd(e2, o2);
    v[3] = cadd(e3, o3);
  } else if constexpr (R == 4) {
    const C t0 = cadd(v[0], v[2]), t1 = csub(v[0], v[2]), t2 = cadd(v[1], v[3]);
    const C t3 = rot_i<SIGN>(csub(v[1], v[3]));
    v[0] = cadd(t0, t2);
    v[1] = cadd(t1, t3);
  } else {
    static_assert(R == 2, "cropped last pass: even radix");
    v[0] = cadd(v[0], v[1]);
  }
}

// Global-memory ends of a column tile (the column pass's first pass reads its inputs
// straight from global memory, the last pass stores to global memory): entry e of line l is
// in[e * es_in + l] / out[e * es_out + l], lines l < nlines of the tile valid.
template <typename C> struct ColIO {
  const C* in;
  C* out;
  long es_in, es_out;
  int n_in, n_out;  // entries read (the rest zero) / stored
  int nlines;
  bool vec_in, vec_out;  // the tile's lines of one entry as 16-byte vectors (all lines valid, aligned)
  const C* sym;          // symbol quadrant, (n + 1)^d
  long c0, inner;        // first line of the tile within the outer index, lines per outer index
  int n1, d;
};

// Pass geometry: butterfly b = threadIdx.x + q NT of the CTA works on line b / BPL,
// butterfly j = b mod BPL.  When NT divides BPL a thread holds every line of each of its
// butterflies j (q = line * (BPL / NT) + jj).
template <int L, int R, int NLINES, int NT> struct PassGeo {
  static constexpr int BPL = L / R;
  static constexpr int BF = NLINES * BPL;
  static constexpr int PER = (BF + NT - 1) / NT;
  static constexpr bool ALL_LINES = BPL % NT == 0;
  static constexpr int M = ALL_LINES ? BPL / NT : 1;
};

// symbol value of entry e of the column tile's line (2D: the entry is the axis-0 frequency
// and the line the axis-1 one; 3D: the line packs axes 1 and 2)
template <typename C, int L> __device__ __forceinline__ C col_symbol(const ColIO<C>& io, int line, int e) {
  const long cc = io.c0 + line;
  const int q0 = e <= L - e ? e : L - e;
  long si;
  if (io.d == 2) {
    const int k1 = (int)cc;
    si = (long)q0 * io.n1 + (k1 <= L - k1 ? k1 : L - k1);
  } else {
    const int k1 = (int)(cc / L), k2 = (int)(cc - (long)k1 * L);
    si = ((long)q0 * io.n1 + (k1 <= L - k1 ? k1 : L - k1)) * io.n1 + (k2 <= L - k2 ? k2 : L - k2);
  }
  return ldg_c(&io.sym[si]);
}

// One radix-R Stockham pass over NLINES lines of length L held in shared memory.
// Pass input: sub-transforms of length NS; output: sub-transforms of length NS * R.
// Butterfly j of a line reads entries j + r L/R, multiplies by w^{r k} with
// w = exp(SIGN 2 pi i / (NS R)), k = j mod NS, and writes (j / NS) NS R + k + r NS.
// PRUNE 1: the first pass of a zero-padded transform (entries L/2.. are zero: inputs
// r >= R/2 are neither read nor used); PRUNE 2: the last pass of a cropped transform
// (outputs L/2.. are not needed: r >= R/2 neither computed nor stored).
// EP (column tiles, io): 1 the first pass reads global memory instead of shared memory;
// 3 the last pass stores to global memory instead of shared memory.
template <typename C, int L, int R, int NS, int SIGN, int NLINES, int NT, int PRUNE = 0, int EP = 0>
__device__ __forceinline__ void fft_pass(C* s, const C* __restrict__ tw, const ColIO<C>* io = nullptr) {
  using SL = SLay<C, L, NLINES>;
  using G = PassGeo<L, R, NLINES, NT>;
  constexpr int BPL = G::BPL, BF = G::BF, PER = G::PER;
  static_assert(PRUNE != 1 || (NS == 1 && R == 8), "padded first pass: radix 8");
  static_assert(PRUNE != 2 || (NS * R == L && R % 2 == 0), "cropped last pass: even radix");
  static_assert(EP != 1 || NS == 1, "global input: first pass");
  static_assert(EP == 0 || EP == 1 || EP == 3, "pass ends: shared memory, global input, global output");
  static_assert(EP != 3 || NS * R == L, "global output: last pass");
  constexpr int RIN = PRUNE == 1 ? R / 2 : R, ROUT = PRUNE == 2 ? R / 2 : R;
  constexpr int VW = (int)(NLINES * sizeof(C) / sizeof(float4));  // 16-byte vectors per entry
  constexpr bool VEC = G::ALL_LINES && NLINES * sizeof(C) % sizeof(float4) == 0 && VW > 0;
  C v[PER][R];
  if constexpr (EP == 1) {
    // every load issued before the first butterfly
    bool vec = false;
    if constexpr (VEC) {
      if (io->vec_in) {
        vec = true;
#pragma unroll
        for (int jj = 0; jj < G::M; ++jj) {
          const int j = threadIdx.x + jj * NT;
#pragma unroll
          for (int r = 0; r < RIN; ++r) {
            const int e = j + r * BPL;
            float4 w[VW];
            const float4* src = reinterpret_cast<const float4*>(io->in + (long)e * io->es_in);
#pragma unroll
            for (int u = 0; u < VW; ++u) w[u] = e < io->n_in ? __ldg(src + u) : make_float4(0.f, 0.f, 0.f, 0.f);
            C c[NLINES];
            memcpy(c, w, sizeof(c));
#pragma unroll
            for (int line = 0; line < NLINES; ++line) v[line * G::M + jj][r] = c[line];
          }
        }
      }
    }
    if (!vec) {
#pragma unroll
      for (int q = 0; q < PER; ++q) {
        const int b = threadIdx.x + q * NT;
        if (BF % NT == 0 || b < BF) {
          const int line = b / BPL, j = b - line * BPL;
#pragma unroll
          for (int r = 0; r < RIN; ++r) {
            const int e = j + r * BPL;
            v[q][r] = (line < io->nlines && e < io->n_in) ? ldg_c(io->in + (long)e * io->es_in + line) : czero<C>();
          }
        }
      }
    }
#pragma unroll
    for (int q = 0; q < PER; ++q) {
      if constexpr (PRUNE == 1) dft8v_lo<SIGN>(v[q]);
      else dftR<R, SIGN>(v[q]);
    }
  } else {
#pragma unroll
    for (int q = 0; q < PER; ++q) {
      const int b = threadIdx.x + q * NT;
      if (BF % NT == 0 || b < BF) {
        const int line = b / BPL, j = b - line * BPL;
        if constexpr (SL::shift_free(BPL)) {
          const int o = SL::off(line, j);
#pragma unroll
          for (int r = 0; r < RIN; ++r) v[q][r] = s[o + r * BPL];
        } else {
#pragma unroll
          for (int r = 0; r < RIN; ++r) v[q][r] = s[SL::off(line, j + r * BPL)];
        }
        if constexpr (NS > 1) {
          const int k = j % NS;
          if constexpr (std::is_same<C, float2>::value) {
            float2 w[R];
            // FP32: the butterfly's factors w^{r k} are one contiguous run of the per-pass
            // table (fft_plan.h), two per 16-byte load
            const float2* twk = tw + tw_pass_offset(L, NS) + k * R;
            if constexpr (R % 2 == 0) {
              const float4* t4 = reinterpret_cast<const float4*>(twk);
#pragma unroll
              for (int u = 0; u < R / 2; ++u) {
                const float4 t = __ldg(t4 + u);
                w[2 * u] = make_float2(t.x, t.y);
                w[2 * u + 1] = make_float2(t.z, t.w);
              }
            } else {
#pragma unroll
              for (int r = 1; r < R; ++r) w[r] = __ldg(twk + r);
            }
#pragma unroll
            for (int r = 1; r < R; ++r) {
              if (SIGN > 0) w[r].y = -w[r].y;
              v[q][r] = cmul(v[q][r], w[r]);
            }
          } else {
            // FP64 and float-float (16-byte entries): the L-entry table exp(-2 pi i m / L),
            // whose entries r k L / (NS R) of neighbouring butterflies are close together;
            // each factor applied as it arrives (fewer live registers)
#pragma unroll
            for (int r = 1; r < R; ++r) {
              C w = ldg_c(&tw[r * k * (L / (NS * R))]);
              if (SIGN > 0) w.y = -w.y;
              v[q][r] = cmul(v[q][r], w);
            }
          }
        }
        if constexpr (PRUNE == 1) dft8v_lo<SIGN>(v[q]);
        else if constexpr (PRUNE == 2) dftR_hi_cut<R, SIGN>(v[q]);
        else dftR<R, SIGN>(v[q]);
      }
    }
  }
  if constexpr (EP == 3) {
    // last pass: outputs j + r NS of each line straight to global memory
    bool vec = false;
    if constexpr (VEC) {
      if (io->vec_out) {
        vec = true;
#pragma unroll
        for (int jj = 0; jj < G::M; ++jj) {
          const int j = threadIdx.x + jj * NT;
#pragma unroll
          for (int r = 0; r < ROUT; ++r) {
            const int e = j + r * NS;
            if (e < io->n_out) {
              C c[NLINES];
#pragma unroll
              for (int line = 0; line < NLINES; ++line) c[line] = c_norm(v[line * G::M + jj][r]);
              float4 w[VW];
              memcpy(w, c, sizeof(c));
              float4* dst = reinterpret_cast<float4*>(io->out + (long)e * io->es_out);
#pragma unroll
              for (int u = 0; u < VW; ++u) dst[u] = w[u];
            }
          }
        }
      }
    }
    if (!vec) {
#pragma unroll
      for (int q = 0; q < PER; ++q) {
        const int b = threadIdx.x + q * NT;
        if (BF % NT == 0 || b < BF) {
          const int line = b / BPL, j = b - line * BPL;
          if (line < io->nlines) {
#pragma unroll
            for (int r = 0; r < ROUT; ++r) {
              const int e = j + r * NS;
              if (e < io->n_out) io->out[(long)e * io->es_out + line] = c_norm(v[q][r]);
            }
          }
        }
      }
    }
    return;
  }
  if constexpr (EP != 1) __syncthreads();  // (a first pass from global memory read no shared memory)
#pragma unroll
  for (int q = 0; q < PER; ++q) {
    const int b = threadIdx.x + q * NT;
    if (BF % NT == 0 || b < BF) {
      const int line = b / BPL, j = b - line * BPL;
      const int k = j % NS;
      const int base = (j / NS) * NS * R + k;
      if constexpr (SL::shift_free(NS)) {
        const int o = SL::off(line, base);
#pragma unroll
        for (int r = 0; r < ROUT; ++r) s[o + r * NS] = c_norm(v[q][r]);
      } else if constexpr (NS == 1 && R <= 8) {
        // the first pass writes R consecutive entries from a multiple of R
        int rb, qq;
        SL::group8(line, base, rb, qq);
#pragma unroll
        for (int r = 0; r < ROUT; ++r) s[rb + (qq ^ r)] = c_norm(v[q][r]);
      } else if constexpr (SL::half_shift(NS)) {
        const int o0 = SL::off(line, base), p0 = o0 & (SL::E - 1), rb = o0 - p0;
#pragma unroll
        for (int r = 0; r < ROUT; ++r) s[rb + r * NS + (p0 ^ ((r & 1) ? SL::HALF_FLIP : 0))] = c_norm(v[q][r]);
      } else {
#pragma unroll
        for (int r = 0; r < ROUT; ++r) s[SL::off(line, base + r * NS)] = c_norm(v[q][r]);
      }
    }
  }
  __syncthreads();
}

// Radices 8, then 4 or 2 for the rest of the power of two, then 3 for L = 3 * 2^k.
// HIN: the upper half of every line is zero padding (the first pass reads the lower half);
// HOUT: only the lower half of the result is needed (the last pass stores only it, when its
// radix is even).  EPF / EPL: the first / last pass's global-memory end (fft_pass's EP).
template <typename C, int L, int NS, int SIGN, int NLINES, int NT, bool HIN = false, bool HOUT = false, int EPF = 0,
          int EPL = 0>
__device__ __forceinline__ void fft_lines(C* s, const C* __restrict__ tw, const ColIO<C>* io = nullptr) {
  if constexpr (NS < L) {
    constexpr int R = pass_radix(L, NS);
    static_assert((L / NS) % R == 0, "FFT length must be 2^k or 3 * 2^k");
    constexpr int PRUNE = (HIN && NS == 1 && R == 8) ? 1 : ((HOUT && NS * R == L && R % 2 == 0) ? 2 : 0);
    constexpr bool first = NS == 1, last = NS * R == L;
    static_assert(!(first && last && EPF != 0 && EPL != 0), "one pass cannot take both ends");
    constexpr int EP = first && EPF != 0 ? EPF : (last ? EPL : 0);
    fft_pass<C, L, R, NS, SIGN, NLINES, NT, PRUNE, EP>(s, tw, io);
    fft_lines<C, L, NS * R, SIGN, NLINES, NT, false, HOUT, 0, EPL>(s, tw, io);
  }
}

// ------------------------------------------------------------------------------------
// Launch shapes
// ------------------------------------------------------------------------------------
template <int L> struct RowShape {
  static constexpr int NT = (L / 8 > 256) ? L / 8 : 256;
  static constexpr int NL = NT * 8 / L;
};
// TC adjacent lines per CTA (about 64 KB of shared memory).  FP32 lines of 1024 and more:
// 4 lines (32-byte runs of each row), L / 8 threads with 4 butterflies each and two CTAs
// per SM, so that one CTA's global loads and stores overlap the other's passes (measured on
// 2D n = 1024, L = 2048: 8 % faster than 8 lines and one 512-thread CTA per SM, which
// leaves the SM idle while a CTA loads; 1024 threads of 2 butterflies each is 16 % slower).
// FP32 lines of 512: 8 lines, 256 threads.  Float-float lines of 2048: 2 lines, 512
// threads, two CTAs per SM (64 registers suffice; lines of 4096 need more).
template <typename C, int L> struct ColShape {
  static constexpr int raw = 65536 / (L * (int)sizeof(C));
  static constexpr bool f32_long = sizeof(C) == 8 && L >= 512;
  static constexpr int TC = f32_long ? (L >= 1024 ? 4 : 8) : (raw < 2 ? 2 : (raw > 16 ? 16 : raw));
  static constexpr int t = f32_long ? TC * L / (L >= 1024 ? 32 : 16) : TC * L / 8;
  static constexpr int NT = t > 512 ? 512 : (t < 64 ? 64 : t);
  // resident CTAs per SM the register allocation must allow
  static constexpr int MINB =
      f32_long && L >= 1024 && NT < 512 ? 512 / NT : (std::is_same<C, ffc>::value && L <= 2048 && NT == 512 ? 2 : 1);
};

// ------------------------------------------------------------------------------------
// Row pass: lines contiguous in memory.
// ------------------------------------------------------------------------------------
// PR: the operator's half-length form (forward: n_in = L/2, the padding not stored; inverse:
// n_out = L/2, the cropped half not computed)
template <typename C, int L, int SIGN, bool PR>
__global__ void __launch_bounds__(RowShape<L>::NT) k_row_pass(RowPassArgs a) {
  constexpr int NT = RowShape<L>::NT, NL = RowShape<L>::NL;
  using SL = SLay<C, L, NL>;
  using Rl = typename RealOf<C>::T;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  C* s = reinterpret_cast<C*>(smem_raw);
  const C* __restrict__ tw = reinterpret_cast<const C*>(a.tw);
  const long line0 = (long)blockIdx.x * NL;
  // the half-length forms' lengths are compile-time constants (index divisions by constants)
  const int n_in = (PR && SIGN < 0) ? L / 2 : a.n_in;

  // load n_in entries of NL lines (coalesced), apply the prologue
  if (a.plane_dirs == nullptr) {
    // LB independent loads in flight per thread before the first shared-memory store
    constexpr int LB = 4;
    const int tot = NL * n_in;
    const C* __restrict__ in = reinterpret_cast<const C*>(a.in);
    const Rl* __restrict__ pw = reinterpret_cast<const Rl*>(a.pw);
    // row of the weights of each of the CTA's lines (one division per line, not per entry)
    __shared__ int pwrow[NL];
    if (pw != nullptr && threadIdx.x < NL) pwrow[threadIdx.x] = (int)((line0 + threadIdx.x) % a.pw_lines);
    __syncthreads();
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
              v[u] = a.in64 ? ffc_of_f64(reinterpret_cast<const double2*>(a.in)[line * a.in_ls + e])
                            : in[line * a.in_ls + e];
            } else {
              v[u] = in[line * a.in_ls + e];
            }
            if (pw != nullptr) wv[u] = pw[(long)pwrow[li] * n_in + e];
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
          s[SL::off(li, e)] = x;
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
          if constexpr (std::is_same<C, ffc>::value) {
            if (a.phase != nullptr) {
              // float-float: the product of the per-axis phase factors
              const ffc* ph = reinterpret_cast<const ffc*>(a.phase) + rhs * a.d * a.n;
              ffc x = ph[(long)(a.d - 1) * a.n + e];
              long qq = q;
              for (int ax = a.d - 2; ax >= 0; --ax) {
                const long ia = qq % a.n;
                qq /= a.n;
                x = c_norm(cmul(x, ph[(long)ax * a.n + ia]));
              }
              const ff w = lz_neg(ff_of_f64(a.pw64[q * n_in + e]));
              x.x = lz_norm(lz_mul(w, x.x));
              x.y = lz_norm(lz_mul(w, x.y));
              s[SL::off(li, e)] = x;
              continue;
            }
          }
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
    s[SL::off(li, e)] = v;
  }
  if (!(PR && SIGN < 0) && n_in < L) {
    const int padn = L - n_in;
    for (int idx = threadIdx.x; idx < NL * padn; idx += NT) {
      const int li = idx / padn, e = n_in + (idx - li * padn);
      s[SL::off(li, e)] = czero<C>();
    }
  }
  __syncthreads();
  fft_lines<C, L, 1, SIGN, NL, NT, (PR && SIGN < 0), (PR && SIGN > 0)>(s, tw);
  const int n_out = (PR && SIGN > 0) ? L / 2 : a.n_out;
  C* out = reinterpret_cast<C*>(a.out);
  const C* addv = reinterpret_cast<const C*>(a.addv);
  for (int idx = threadIdx.x; idx < NL * n_out; idx += NT) {
    const int li = idx / n_out, e = idx - li * n_out;
    const long line = line0 + li;
    if (line < a.lines) {
      C v = s[SL::off(li, e)];
      if constexpr (std::is_same<C, ffc>::value) {
        if (a.out64) {
          // FP64 epilogue: y = v + addv, or y = subv - (v + addv)
          double2 o = ffc_to_f64(v);
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
// PR: the operator's half-length form (MODE 0 and 2: n_in = L/2, the padding not stored;
// MODE 1 and 2: n_out = L/2, the cropped half not computed)
template <typename C, int L, int MODE, bool PR>
__global__ void __launch_bounds__(ColShape<C, L>::NT, ColShape<C, L>::MINB) k_col_pass(ColPassArgs a) {
  constexpr int NT = ColShape<C, L>::NT, TC = ColShape<C, L>::TC;
  using SL = SLay<C, L, TC>;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  C* s = reinterpret_cast<C*>(smem_raw);
  const C* __restrict__ tw = reinterpret_cast<const C*>(a.tw);
  const long tiles = (a.inner + TC - 1) / TC;
  const long o = blockIdx.x / tiles;
  const long c0 = (blockIdx.x - o * tiles) * TC;
  ColIO<C> io;
  io.in = reinterpret_cast<const C*>(a.in) + o * a.in_os + c0;
  io.out = reinterpret_cast<C*>(a.out) + o * a.out_os + c0;
  io.es_in = a.in_es;
  io.es_out = a.out_es;
  io.n_in = (PR && MODE != 1) ? L / 2 : a.n_in;
  io.n_out = (PR && MODE != 0) ? L / 2 : a.n_out;
  io.nlines = a.inner - c0 < TC ? (int)(a.inner - c0) : TC;
  io.vec_in = io.nlines == TC && (reinterpret_cast<uintptr_t>(io.in) & 15) == 0 && (a.in_es * sizeof(C)) % 16 == 0;
  io.vec_out = io.nlines == TC && (reinterpret_cast<uintptr_t>(io.out) & 15) == 0 && (a.out_es * sizeof(C)) % 16 == 0;
  io.sym = reinterpret_cast<const C*>(a.sym);
  io.c0 = c0;
  io.inner = a.inner;
  io.n1 = a.n + 1;
  io.d = a.d;
  // The first pass loads the tile straight from global memory and the last one stores it
  // there when a thread's accesses stay coalesced: it holds every line of its butterflies
  // (16-byte vectors across the lines), or one entry of all lines fits a 32-byte sector.
  // Otherwise consecutive threads fill and drain consecutive lines through shared memory
  // (tiles of many short lines).
  constexpr bool SECTOR = TC * sizeof(C) <= 32;
  constexpr int EPF = (PassGeo<L, 8, TC, NT>::ALL_LINES || SECTOR) ? 1 : 0;
  constexpr int EPL = (PassGeo<L, last_radix(L), TC, NT>::ALL_LINES || SECTOR) ? 3 : 0;
  static_assert(L % 8 == 0, "column passes: the first radix is 8");
  if constexpr (EPF == 0) {
    // LB independent loads in flight per thread before the first shared-memory store
    constexpr int LB = 4;
    const int tot = io.n_in * TC;
    for (int base = threadIdx.x; base < tot; base += NT * LB) {
      C v[LB];
#pragma unroll
      for (int u = 0; u < LB; ++u) {
        const int idx = base + u * NT;
        v[u] = czero<C>();
        if (idx < tot) {
          const int e = idx / TC, c = idx - e * TC;
          if (c < io.nlines) v[u] = io.in[(long)e * a.in_es + c];
        }
      }
#pragma unroll
      for (int u = 0; u < LB; ++u) {
        const int idx = base + u * NT;
        if (idx < tot) {
          const int e = idx / TC, c = idx - e * TC;
          s[SL::off(c, e)] = v[u];
        }
      }
    }
    if (!(PR && MODE != 1) && io.n_in < L) {
      const int padn = L - io.n_in;
      for (int idx = threadIdx.x; idx < padn * TC; idx += NT) {
        const int e = io.n_in + idx / TC, c = idx % TC;
        s[SL::off(c, e)] = czero<C>();
      }
    }
    __syncthreads();
  }
  if constexpr (MODE == 0) {
    fft_lines<C, L, 1, -1, TC, NT, PR, false, EPF, EPL>(s, tw, &io);
  } else if constexpr (MODE == 1) {
    fft_lines<C, L, 1, 1, TC, NT, false, PR, EPF, EPL>(s, tw, &io);
  } else {
    fft_lines<C, L, 1, -1, TC, NT, PR, false, EPF, 0>(s, tw, &io);
    // symbol values of SB entries loaded together, then applied
    constexpr int SB = 8;
    for (int base = threadIdx.x; base < L * TC; base += NT * SB) {
      C sv[SB];
#pragma unroll
      for (int u = 0; u < SB; ++u) {
        const int idx = base + u * NT;
        const int e = idx / TC, c = idx - e * TC;
        sv[u] = czero<C>();
        if (idx < L * TC && c < io.nlines) sv[u] = col_symbol<C, L>(io, c, e);
      }
#pragma unroll
      for (int u = 0; u < SB; ++u) {
        const int idx = base + u * NT;
        const int e = idx / TC, c = idx - e * TC;
        if (idx < L * TC && c < io.nlines) {
          C& v = s[SL::off(c, e)];
          v = cmul(v, sv[u]);
        }
      }
    }
    __syncthreads();
    fft_lines<C, L, 1, 1, TC, NT, false, PR, 0, EPL>(s, tw, &io);
  }
  if constexpr (EPL == 0) {
    for (int idx = threadIdx.x; idx < io.n_out * TC; idx += NT) {
      const int e = idx / TC, c = idx - e * TC;
      if (c < io.nlines) io.out[(long)e * a.out_es + c] = s[SL::off(c, e)];
    }
  }
}

// ------------------------------------------------------------------------------------
// Host dispatch
// ------------------------------------------------------------------------------------
// the half-length form when the lengths are the operator's (L/2 in or out); the full form
// (the symbol's transforms, FP64 only) otherwise
template <typename C, int L, int SIGN, bool PR> void launch_row_LP(const RowPassArgs& a, cudaStream_t st) {
  constexpr int NT = RowShape<L>::NT, NL = RowShape<L>::NL;
  const size_t smem = (size_t)SLay<C, L, NL>::SIZE * sizeof(C);
  static std::atomic<bool> attr{false};  // set once per process; repeats are harmless
  if (!attr.load(std::memory_order_acquire)) {
    LS_CUDA(cudaFuncSetAttribute(k_row_pass<C, L, SIGN, PR>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    attr.store(true, std::memory_order_release);
  }
  const long blocks = (a.lines + NL - 1) / NL;
  if (blocks == 0) return;
  static const std::string cls = std::string(SIGN < 0 ? "fft_row_fwd_" : "fft_row_inv_") + arith_tag<C>();
  LS_LAUNCH(cls.c_str(), st, k_row_pass<C, L, SIGN, PR><<<(unsigned)blocks, NT, smem, st>>>(a));
}
template <typename C, int L, int SIGN> void launch_row_L(const RowPassArgs& a, cudaStream_t st) {
  const bool half = SIGN < 0 ? a.n_in * 2 == L : a.n_out * 2 == L;
  if (half) {
    launch_row_LP<C, L, SIGN, true>(a, st);
  } else {
    if constexpr (std::is_same<C, double2>::value) launch_row_LP<C, L, SIGN, false>(a, st);
    else LS_FAIL(EINVAL_, "row pass: only the half-length form in this arithmetic");
  }
}

template <typename C, int L, int MODE, bool PR> void launch_col_LP(const ColPassArgs& a, cudaStream_t st) {
  constexpr int NT = ColShape<C, L>::NT, TC = ColShape<C, L>::TC;
  const size_t smem = (size_t)SLay<C, L, TC>::SIZE * sizeof(C);
  static std::atomic<bool> attr{false};  // set once per process; repeats are harmless
  if (!attr.load(std::memory_order_acquire)) {
    LS_CUDA(cudaFuncSetAttribute(k_col_pass<C, L, MODE, PR>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    attr.store(true, std::memory_order_release);
  }
  const long tiles = (a.inner + TC - 1) / TC;
  const long blocks = tiles * a.outer;
  if (blocks == 0) return;
  static const std::string cls =
      std::string(MODE == 0 ? "fft_col_fwd_" : MODE == 1 ? "fft_col_inv_" : "fft_col_sym_") + arith_tag<C>();
  LS_LAUNCH(cls.c_str(), st, k_col_pass<C, L, MODE, PR><<<(unsigned)blocks, NT, smem, st>>>(a));
}
template <typename C, int L, int MODE> void launch_col_L(const ColPassArgs& a, cudaStream_t st) {
  const bool in_half = a.n_in * 2 == L, out_half = a.n_out * 2 == L;
  const bool half = MODE == 0 ? in_half : (MODE == 1 ? out_half : in_half && out_half);
  if (half) {
    launch_col_LP<C, L, MODE, true>(a, st);
  } else {
    if constexpr (std::is_same<C, double2>::value) launch_col_LP<C, L, MODE, false>(a, st);
    else LS_FAIL(EINVAL_, "column pass: only the half-length form in this arithmetic");
  }
}

#define LS_FOR_L(X) X(16) X(32) X(48) X(64) X(96) X(128) X(256) X(512) X(1024) X(2048) X(4096)

// Explicit instantiation (PREFIX empty) or instantiation declaration (PREFIX extern) of the
// five launchers of one arithmetic C and one length LL: the float-float passes spread their
// lengths over several translation units, which compile in parallel.
#define LS_PASS_INST(PREFIX, C, LL)                                                \
  PREFIX template void launch_row_L<C, LL, -1>(const RowPassArgs&, cudaStream_t); \
  PREFIX template void launch_row_L<C, LL, 1>(const RowPassArgs&, cudaStream_t);  \
  PREFIX template void launch_col_L<C, LL, 0>(const ColPassArgs&, cudaStream_t);  \
  PREFIX template void launch_col_L<C, LL, 1>(const ColPassArgs&, cudaStream_t);  \
  PREFIX template void launch_col_L<C, LL, 2>(const ColPassArgs&, cudaStream_t);

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

}  // namespace ls
