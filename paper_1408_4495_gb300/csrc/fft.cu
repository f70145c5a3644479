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
#include "fft_plan.h"
#include "kernels.h"
#include "prof.h"

namespace ls {

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
                     void* scratch1, void* scratch2, cudaStream_t st, const void* phase = nullptr) {
  const int n = p.n, L = 2 * n, d = p.d;
  const long rows = (d == 2) ? (long)n : (long)n * n;  // lines of one grid along the last axis
  C* T1 = reinterpret_cast<C*>(scratch1);
  RowPassArgs r{};
  r.in = u; r.out = T1; r.lines = (long)nrhs * rows; r.n_in = n; r.n_out = L;
  r.in_ls = n; r.out_ls = L; r.pw = w2m; r.pw_lines = rows; r.tw = tw;
  r.plane_dirs = plane_dirs; r.d = d; r.n = n; r.omega = p.omega; r.h = p.h; r.in64 = in64;
  r.pw64 = p.w2m64; r.phase = phase;
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

// phase[(rhs * d + a) * n + k] = exp(i omega h (k + 1) dir_a) as float-float complex (FP64
// sincos, once per right-hand side, axis and index): the plane wave exp(i omega x . dir) at
// x = h (i + 1) is the product of one factor per axis
__global__ void k_phase_table(const double* __restrict__ dirs, int nrhs, int d, int n, double omega, double h,
                              ffc* __restrict__ phase) {
  const long tot = (long)nrhs * d * n;
  for (long t = blockIdx.x * (long)blockDim.x + threadIdx.x; t < tot; t += (long)gridDim.x * blockDim.x) {
    const long ra = t / n;
    const int k = (int)(t - ra * n);
    double sn, cs;
    sincos(omega * h * ((double)(k + 1) * dirs[ra]), &sn, &cs);
    phase[t] = ffc_from(make_double2(cs, sn));
  }
}

void conv_rhs_ff(const ConvPlan& p, int nrhs, const double* plane_dirs, double2* g, void* scratch1, void* scratch2,
                 void* phase, cudaStream_t st) {
  if (!p.twff || !p.symff) LS_FAIL(ESTATE_, "float-float operator tables missing");
  const long tot = (long)nrhs * p.d * p.n;
  LS_LAUNCH("rhs_phase", st,
            k_phase_table<<<(unsigned)std::min<long>((tot + 255) / 256, 1024), 256, 0, st>>>(
                plane_dirs, nrhs, p.d, p.n, p.omega, p.h, reinterpret_cast<ffc*>(phase)));
  conv_run<ffc>(p, nrhs, nullptr, g, plane_dirs, false, nullptr, 0, 1, p.twff, p.symff, p.w2mff, scratch1, scratch2,
                st, phase);
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

void fft_twiddles(int L, std::vector<double2>& tw) {
  tw.assign((size_t)tw_table_size(L), make_double2(0.0, 0.0));
  for (int NS = 1; NS < L; NS *= pass_radix(L, NS)) {
    const int R = pass_radix(L, NS);
    if (NS == 1) continue;  // the first pass has no factors
    double2* t = tw.data() + tw_pass_offset(L, NS);
    for (int k = 0; k < NS; ++k)
      for (int r = 0; r < R; ++r) {
        // w^{r k}, w = exp(-2 pi i / (NS R)); the exponent reduced mod NS R
        const long e = ((long)r * k) % ((long)NS * R);
        const double a = -2.0 * M_PI * (double)e / (double)(NS * R);
        t[(size_t)k * R + r] = make_double2(std::cos(a), std::sin(a));
      }
  }
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
