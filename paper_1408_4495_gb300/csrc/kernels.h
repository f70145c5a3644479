// Internal interfaces between the translation units of libls (not part of the C-ABI).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <vector>

namespace ls {

// ---------------------------------------------------------------- FFT passes (fft.cu)
struct RowPassArgs {
  const void* in;      // lines of complex (path precision), line stride in_ls
  void* out;           // line stride out_ls
  long lines;
  int n_in, n_out;     // entries read (zero padded to L) / entries written
  long in_ls, out_ls;
  const void* pw;      // real weights [(line % pw_lines) * n_in + e], or null
  long pw_lines;
  const void* tw;      // twiddles exp(-2 pi i m / L), m < L
  const double* plane_dirs;  // right-hand-side prologue (FP64 and float-float passes), or null
  const double* pw64;  // omega^2 m in FP64 for that prologue
  const void* phase;   // float-float passes: the prologue's phase factors as float-float
                       // complex [rhs][axis][k] = exp(i omega h (k + 1) dir_axis), or null
  int d, n;
  double omega, h;
  const void* addv;    // epilogue: out += addv[line * add_ls + e], or null
  long add_ls;
  const void* subv;    // epilogue: out = subv - (...), or null (float-float passes only)
  int in64, out64;     // float-float passes: in / out, addv, subv are FP64 complex
};

struct ColPassArgs {
  const void* in;
  void* out;
  long outer, inner;   // lines = outer * inner, inner index contiguous in memory
  long in_os, in_es, out_os, out_es;
  int n_in, n_out;
  const void* sym;     // symbol quadrant (n+1)^d for the symbol pass
  int n, d;
  const void* tw;
};

struct ConvPlan {
  int d, n;
  double omega, h;
  const float2* tw32;
  const double2* tw64;
  const float2* sym32;
  const double2* sym64;
  const float* w2m32;   // omega^2 m, n^d
  const double* w2m64;
  const void* twff;     // float-float copies (two floats per real) of tw64, sym64, w2m64
  const void* symff;
  const void* w2mff;
};

template <typename C> void row_pass(int L, int sign, const RowPassArgs& a, cudaStream_t st);
template <typename C> void col_pass(int L, int mode, const ColPassArgs& a, cudaStream_t st);
template <typename C>
void conv_apply(const ConvPlan& p, int nrhs, const C* u, C* y, const double* plane_dirs, bool add_u,
                void* scratch1, void* scratch2, cudaStream_t st);
// y = (I + K omega^2 m) u in float-float arithmetic with FP64 input and output; with
// sub != null, y = sub - (I + K omega^2 m) u (the residual)
void conv_apply_ff(const ConvPlan& p, int nrhs, const double2* u, double2* y, const double2* sub, void* scratch1,
                   void* scratch2, cudaStream_t st);
// g = K(-omega^2 m u_inc) for plane waves (the right-hand side), float-float passes, FP64 g
// phase: scratch of nrhs * d * n float-float complex entries (4 floats each)
void conv_rhs_ff(const ConvPlan& p, int nrhs, const double* plane_dirs, double2* g, void* scratch1, void* scratch2,
                 void* phase, cudaStream_t st);
// C -= A B on the complex FP32 fronts of a level on the tensor cores (tc_gemm.cu): A, B, C
// are the blocks [r0,r1)x[k0,k1), [k0,k1)x[c0,c1), [r0,r1)x[c0,c1) of each column-major
// front (ld = fmax, fstride elements apart); *err = 2 if a bounded wait expired
void tc_cgemm(float2* F, long fstride, int fmax, int nf, int r0, int r1, int c0, int c1, int k0, int k1, int* err,
              cudaStream_t st);
// C[z] = A[z] B[z] on every front z of a level, A = rows [r0, r1) x columns [k0, k1) of the
// front, B and C dense per front outside it (tc_gemm.cu); launches counted under cls
// (k range split nsplit ways, ksz columns each, partial products split_stride apart)
void tc_sweep_gemm(const float2* F, long fstride, int fmax, int nf, int r0, int r1, int k0, int k1, const float2* B,
                   long bstride, int ldb, float2* C, long cstride, int ldc, int ncols, int nsplit, int ksz,
                   long split_stride, int* err, cudaStream_t st, const char* cls);
// tensor-core products on (LS_TC=0 in the environment turns them off, for comparisons)
bool tc_enabled();
// float-float copy of count FP64 reals (dst: 2 * count floats)
void to_ff(const double* src, void* dst, long count, cudaStream_t st);
size_t conv_scratch1_elems(int d, int n, int nrhs);
// the FP32 passes' per-pass twiddle table for lines of length L (layout in fft_plan.h),
// computed in FP64
void fft_twiddles(int L, std::vector<double2>& tw);
size_t conv_scratch2_elems(int d, int n, int nrhs);
void build_kernel_table(int d, int n, double omega, double h, double2* ktq, cudaStream_t st);
// Sec. 5: g_r = q_r K delta_{p_r} / h^d for nrhs point sources (pts: nrhs x d grid indices;
// q: nrhs complex strengths or null for 1), from the quadrant table ktq.
// far-field pattern u_inf(theta_k; r) of the scattered fields us (nrhs x N) of the plane waves
// dirs (nrhs x d) in the directions obs (nobs x d); out: nrhs x nobs
void far_field(int d, int n, int nrhs, int nobs, const double2* us, const double* dirs, const double* obs,
               const double* w, double omega, double h, double2* out, cudaStream_t st);
void point_source(int d, int n, int nrhs, const int* pts, const double2* q, const double2* ktq, double h, double2* g,
                  cudaStream_t st);
void build_symbol(const ConvPlan& p, const double2* ktq, double2* sym64, float2* sym32, double2* work,
                  cudaStream_t st);

// ---------------------------------------------------------------- stencils (setup.cpp)
// alpha for all 3^d classes (3^d x 3^d, zero outside mu) and C for the interior class,
// computed on the host in FP64 from the (n+1)^d quadrant of k_t.
void compute_stencils(int d, int n, int b, const std::vector<double2>& ktq, std::vector<double2>& alpha,
                      std::vector<double2>& cint);

// ---------------------------------------------------------------- stencil apply (stencil.cu)
// r[i * rs_i + rhs * rs_r] = sum_t alpha_cls(i)(t) v[rhs * N + i + t]; v in the input
// precision Cin, r in Cout.
template <typename Cin, typename Cout>
void stencil_apply(int d, int n, int nrhs, const Cin* v, Cout* r, long rs_i, long rs_r, const void* alpha,
                   cudaStream_t st);
// the same with a stencil per point: alpha_pt is N x 3^d in Cout (general domains, Sec. 4.1)
template <typename Cin, typename Cout>
void stencil_apply_pt(int d, int n, int nrhs, const Cin* v, Cout* r, long rs_i, long rs_r, const void* alpha_pt,
                      cudaStream_t st);
// r2 = [A;B] v - M z (FP32), the residual of a preconditioner application (class stencils)
void pre_resid(int d, int n, int nrhs, const float2* v, const float2* z, float2* r2, const float2* alpha32,
               const double2* cint64, const float* w2m32, cudaStream_t st);
// 2D, FP32: [A;B] v (z == nullptr) or [A;B] v - M z written straight into the solve's item
// layout T[group][N][rc] (right-hand sides past nrhs zero; rc = nd_item_width(nrhs))
void stencil_items_2d(int n, int nrhs, int rc, const float2* v, const float2* z, float2* T, const float2* alpha32,
                      const double2* cint64, const float* w2m32, cudaStream_t st);

// ---------------------------------------------------------------- nested dissection (nd.cu)
struct NdPlan;  // opaque: host symbolic + device index arrays
NdPlan* nd_build(int d, int n, cudaStream_t st);
void nd_free(NdPlan* p);
struct NdInfo {
  int levels, fronts, max_front;
  int64_t factor_entries;
  double factor_flops, solve_bytes;
  // entries (not bytes) touched by one forward / backward sweep: factor blocks, and
  // vector entries per right-hand side
  double fwd_factor_entries, fwd_vec_entries, bwd_factor_entries, bwd_vec_entries;
};
NdInfo nd_info(const NdPlan* p);
// factors: assembles M into the fronts and factors them, in C (float2 or double2);
// alpha, cint: FP64 stencil tables, w2m: FP64 omega^2 m.  nd_factor = nd_prepare (device
// allocations, returns true if it allocated) + nd_factor_launch (stream-ordered launches
// only, capturable in a CUDA graph) + nd_factor_check (reads the singular-pivot flag).
template <typename C>
void nd_factor(NdPlan* p, const void* alpha_T, const void* cint_T, const void* w2m_T, cudaStream_t st);
template <typename C> bool nd_prepare(NdPlan* p, cudaStream_t st);
template <typename C>
// top_levels (may be null): recorded on st where the levels with at most 32 fronts begin;
// alpha_pt (FP64, N x 3^d) and inter_pt (N bytes), when not null, give every point its own
// stencil and interior flag (general domains, Sec. 4) in place of the class tables
void nd_factor_launch(NdPlan* p, const void* alpha_T, const void* cint_T, const void* w2m_T, cudaStream_t st,
                      cudaEvent_t top_levels, const void* alpha_pt = nullptr, const unsigned char* inter_pt = nullptr);
void nd_factor_check(NdPlan* p, cudaStream_t st);
// FP32 Schur-complement products on the tensor cores (3xTF32, the default) or on the CUDA cores
void nd_set_tensor_cores(NdPlan* p, bool on);
// Launch-shape choices of the factorization and of the solve sweeps.  The defaults were
// chosen by measurement on 2D n = 256; ls_autotune times the alternatives per grid and
// precision and keeps the fastest.
struct NdTune {
  double two_level_min = 8.0e6;  // trailing-matrix entries of a level from which the blocked
                                 // LU updates in two levels (outer blocks of 4 panels)
  int tc_min_rows = 64;          // FP32 Schur products with at least this many rows (and 16
                                 // inner columns) run on the tensor cores
  int sweep_ctas = 2;            // CTAs per SM that the split of a sweep level's columns aims at
  int gj_max_own = 16;           // fronts with at most this many own rows: Gauss-Jordan in one CTA
  int tcs_min_rows = -1;         // FP32 forward-sweep levels whose products have at least this
                                 // many rows (and 16 inner columns) run on the tensor cores;
                                 // -1: automatic (nd_tcs_min_rows)
  int tcs_bwd_min_rows = -1;     // the same for the backward sweep
  int small_max_k = -1;          // FP32 sweep levels with at most 64 product rows and this many
                                 // columns (up to 256) run one CTA per front (0: none; -1:
                                 // automatic, nd_small_max_k)
};
// The automatic values, per solve (ng groups of 16 right-hand sides): tensor-core solve levels
// from 64 rows in 3D or with at least two groups, none for one group in 2D (their 16-column
// products lose to the CUDA-core sweep there); one-CTA-per-front levels up to 256 columns with
// at least two groups, up to 64 with one.
int nd_tcs_min_rows(int d, int ng, int tune_value);
int nd_small_max_k(int ng, int tune_value);
constexpr int SWEEP_CTAS_MAX = 4;  // the solve's partial-sum buffers are sized for this target
void nd_set_tune(NdPlan* p, const NdTune& t);
NdTune nd_get_tune(const NdPlan* p);
// x = M^{-1} r (accumulate: x += M^{-1} r) for nrhs vectors; r and x in layout [nrhs][N]
// (path precision)
template <typename C> void nd_solve(NdPlan* p, int nrhs, const C* r, C* x, cudaStream_t st, bool accumulate = false);
// The solve's item buffer T[group][N][RC] (grid points in grid order, RC right-hand sides
// per group) for up to nd_items_max() right-hand sides: a producer that writes it directly
// then runs nd_solve_items instead of nd_solve (x = M^{-1} r, or x += M^{-1} r).
void* nd_items(NdPlan* p);
int nd_item_width(int nrhs);
int nd_items_max();
template <typename C> void nd_solve_items(NdPlan* p, int nrhs, C* x, cudaStream_t st, bool accumulate);
size_t nd_device_bytes(const NdPlan* p, int elem_bytes);
// bytes of the factored fronts (the factorization's whole state), and their copy to / from a
// host array of that size (synchronous on st)
size_t nd_factor_bytes(const NdPlan* p);
size_t nd_factor_elems(const NdPlan* p);  // front entries, whether or not the storage exists yet
void nd_copy_factors(NdPlan* p, void* host, bool to_host, cudaStream_t st);

}  // namespace ls
