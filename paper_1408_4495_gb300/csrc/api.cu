// C-ABI of libls (include/ls.h) and the GMRES driver of Sec. 3.3.
//
// ls_solve runs right-preconditioned GMRES(restart) on (I + K omega^2 m) u = g for all
// right-hand sides at once: each launch processes the whole batch, each right-hand side
// keeps its own Krylov space, Hessenberg matrix and stopping point.  Under LS_PREC_MIXED an
// iteration applies the FP32 stencil + ND solve (preconditioner) and the FP32 FFT operator,
// and orthogonalises in FP64 (flexible GMRES: the preconditioned vectors Z are kept, in
// FP32); every cycle ends with the FP64 residual g - A u (FP64 FFT apply), which decides
// convergence and restarts the next cycle (iterative refinement).  Under LS_PREC_FP64 the
// same loop runs with FP64 everywhere.
#include <cuda_runtime.h>
#include <type_traits>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <complex>
#include <cstdlib>
#include <cstring>
#include <map>
#include <mutex>
#include <new>
#include <string>
#include <tuple>
#include <vector>

#include "alloc.h"
#include "common.cuh"
#include "kernels.h"
#include "ffloat.cuh"
#include "krylov.h"
#include "ls.h"
#include "prof.h"
#include "trace.h"

using ls::Error;
using ls::ffc;
using cd = std::complex<double>;

struct DevBuf {
  void* p = nullptr;
  size_t bytes = 0;
};

// A captured launch sequence: replayed while the buffers it was captured on are unchanged
// (generation counter of the context), re-captured otherwise.
struct GraphEntry {
  cudaGraphExec_t exec = nullptr;
  std::map<std::string, long> tally;  // kernel launches per class in one replay
  uint64_t gen = 0;
  bool seen = false;
};

struct ls_ctx {
  ls_grid g{};
  int d = 0, n = 0, L = 0, b = 2, restart = 50, max_iter = 500;
  long N = 0;
  double omega = 0, h = 0;
  bool laplace = false;  // Sec. 5 kernel 1/(4 pi r), potential V in place of omega^2 m
  ls_prec prec = LS_PREC_MIXED;
  cudaStream_t st = nullptr;
  bool own_stream = false;
  int device = 0;  // the device current at setup: every device array of the context lives there
  std::string err;
  double* w2m64 = nullptr;
  float* w2m32 = nullptr;
  float2* tw32 = nullptr;
  double2* tw64 = nullptr;
  double2* ktq = nullptr;
  float2* sym32 = nullptr;
  double2* sym64 = nullptr;
  float2* ffbuf = nullptr;  // float-float twiddles, symbol and omega^2 m
  double2* alpha64 = nullptr;
  float2* alpha32 = nullptr;
  double2* cint64 = nullptr;
  std::vector<double2> alpha_h, cint_h;
  // general domain (Sec. 4), set by ls_general_setup: a stencil per point (N x 3^d) and the
  // interior flag per point, replacing the class tables in the assembly and the stencil apply
  bool general = false;
  double2* apt64 = nullptr;
  float2* apt32 = nullptr;
  unsigned char* inter_pt = nullptr;
  ls::NdPlan* nd = nullptr;
  bool factored = false;
  bool factor_pending = false;  // enqueued, its error flag not read yet
  cudaStream_t st2 = nullptr;   // side stream: right-hand sides that overlap the factorization
  cudaEvent_t ev_factor = nullptr;  // recorded on st where the factorization's top levels begin
  std::map<std::string, DevBuf> bufs;
  std::vector<double2*> V;
  std::vector<void*> Z;
  int Z_elem = 0;
  long basis_cap = 0;  // elements per basis vector allocated
  double2** dV = nullptr;
  void** dZ = nullptr;
  ls::ConvPlan plan{};
  uint64_t gen = 1;  // bumped whenever a device buffer is (re)allocated
  uint64_t medium_hash = 0;  // FNV-1a of the FP64 potential, the identity of exported factors
  bool use_graphs = true;
  // one step of iterative refinement inside each FP32 preconditioner application of the
  // GMRES iterations: -1 = not yet known for this factorization (measured in its first
  // iteration), 0 = off, 1 = on
  int pre_refine = -1;
  int pre_refine_mode = -1;  // ls_set_precond_refine: -1 automatic, 0 off, 1 on
  double pre_err = -1.0;     // |[A;B] v - M z| / |[A;B] v| of the first application after a factorization (-1: none)
  std::map<std::string, GraphEntry> graphs;
};

namespace {

std::mutex g_mu;
std::string g_setup_err;

struct StencilKey {
  int d, n, b;
  double omega;
  int k0_rule;  // C = alpha K(mu, mu) holds k_0
  bool operator<(const StencilKey& o) const {
    return std::tie(d, n, b, omega, k0_rule) < std::tie(o.d, o.n, o.b, o.omega, o.k0_rule);
  }
};
std::map<StencilKey, std::pair<std::vector<double2>, std::vector<double2>>> g_stencil_cache;

bool is_device_ptr(const void* p) {
  cudaPointerAttributes a;
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

template <typename T> T* dalloc(size_t count) {
  return (T*)ls::dev_alloc(std::max<size_t>(1, count) * sizeof(T));
}

template <typename T> T* buf(ls_ctx* c, const std::string& name, size_t count) {
  DevBuf& b = c->bufs[name];
  const size_t need = std::max<size_t>(1, count) * sizeof(T);
  if (b.bytes < need) {
    if (b.p) {
      LS_CUDA(cudaStreamSynchronize(c->st));
      ls::dev_free(b.p);
    }
    b.p = nullptr;
    b.bytes = 0;
    b.p = dalloc<unsigned char>(need);
    b.bytes = need;
    ++c->gen;
  }
  return (T*)b.p;
}

// Runs `body` (stream-ordered work on c->st only, no allocation and no synchronisation)
// through a cached CUDA graph: eager the first time a key is met with the current
// buffers, captured the second time, replayed afterwards.  Bypassed while launches are
// being timed individually.
template <typename F> void run_graph(ls_ctx* c, const std::string& key, F&& body) {
  if (!c->use_graphs || ls::prof_timing_active()) {
    body();
    return;
  }
  GraphEntry& e = c->graphs[key];
  if (e.exec && e.gen == c->gen) {
    LS_CUDA(cudaGraphLaunch(e.exec, c->st));
    ls::prof_count_replay(e.tally);
    return;
  }
  if (e.exec) {
    cudaGraphExecDestroy(e.exec);
    e.exec = nullptr;
  }
  if (!e.seen || e.gen != c->gen) {
    e.seen = true;
    e.gen = c->gen;
    body();
    return;
  }
  e.tally.clear();
  cudaGraph_t g = nullptr;
  LS_CUDA(cudaStreamBeginCapture(c->st, cudaStreamCaptureModeThreadLocal));
  ls::prof_capture_begin(&e.tally);
  try {
    body();
  } catch (...) {
    ls::prof_capture_end();
    cudaStreamEndCapture(c->st, &g);
    if (g) cudaGraphDestroy(g);
    cudaGetLastError();
    throw;
  }
  ls::prof_capture_end();
  LS_CUDA(cudaStreamEndCapture(c->st, &g));
  const cudaError_t ie = cudaGraphInstantiate(&e.exec, g, 0);
  cudaGraphDestroy(g);
  if (ie != cudaSuccess) {
    e.exec = nullptr;
    LS_CUDA(ie);
  }
  LS_CUDA(cudaGraphLaunch(e.exec, c->st));
  ls::prof_count_replay(e.tally);
}

// copy count complex doubles (or doubles) between a caller array and a device buffer
void copy_in(ls_ctx* c, void* dst, const void* src, size_t bytes, cudaStream_t st = nullptr) {
  LS_CUDA(cudaMemcpyAsync(dst, src, bytes, is_device_ptr(src) ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice,
                          st ? st : c->st));
}
void copy_out(ls_ctx* c, void* dst, const void* src, size_t bytes, cudaStream_t st = nullptr) {
  LS_CUDA(cudaMemcpyAsync(dst, src, bytes, is_device_ptr(dst) ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost,
                          st ? st : c->st));
}

// waits for an enqueued factorization and reads its error flag (throws on failure)
void factor_wait(ls_ctx* c) {
  if (!c->factor_pending) return;
  c->factor_pending = false;
  try {
    ls::nd_factor_check(c->nd, c->st);
  } catch (...) {
    c->factored = false;
    throw;
  }
}

void ensure_basis(ls_ctx* c, int nvec, int nrhs, int z_elem) {
  const long need = (long)nrhs * c->N;
  if (need > c->basis_cap || z_elem != c->Z_elem) {
    LS_CUDA(cudaStreamSynchronize(c->st));
    for (auto p : c->V) ls::dev_free(p);
    for (auto p : c->Z) ls::dev_free(p);
    c->V.clear();
    c->Z.clear();
    c->basis_cap = need;
    c->Z_elem = z_elem;
  }
  bool grew = false;
  while ((int)c->V.size() < nvec) {
    c->V.push_back(dalloc<double2>(c->basis_cap));
    grew = true;
  }
  while ((int)c->Z.size() < nvec) {
    c->Z.push_back(dalloc<unsigned char>((size_t)c->basis_cap * z_elem));
    grew = true;
  }
  if (grew || !c->dV) {
    ++c->gen;
    LS_CUDA(cudaStreamSynchronize(c->st));
    if (c->dV) ls::dev_free(c->dV);
    if (c->dZ) ls::dev_free(c->dZ);
    c->dV = dalloc<double2*>(c->V.size());
    c->dZ = dalloc<void*>(c->Z.size());
    LS_CUDA(cudaMemcpy(c->dV, c->V.data(), c->V.size() * sizeof(double2*), cudaMemcpyHostToDevice));
    LS_CUDA(cudaMemcpy(c->dZ, c->Z.data(), c->Z.size() * sizeof(void*), cudaMemcpyHostToDevice));
  }
}

template <typename C> void op_apply(ls_ctx* c, int nrhs, const C* u, C* y) {
  const size_t s1 = ls::conv_scratch1_elems(c->d, c->n, nrhs), s2 = ls::conv_scratch2_elems(c->d, c->n, nrhs);
  void* t1 = buf<C>(c, sizeof(C) == 8 ? "conv1_32" : "conv1_64", s1);
  void* t2 = s2 ? buf<C>(c, sizeof(C) == 8 ? "conv2_32" : "conv2_64", s2) : nullptr;
  ls::conv_apply<C>(c->plan, nrhs, u, y, nullptr, true, t1, t2, c->st);
}

// y = (I + K omega^2 m) u, or y = sub - (I + K omega^2 m) u, in float-float arithmetic
// (16-byte intermediates: the FP64 scratch buffers)
void op_apply_ff(ls_ctx* c, int nrhs, const double2* u, double2* y, const double2* sub) {
  const size_t s1 = ls::conv_scratch1_elems(c->d, c->n, nrhs), s2 = ls::conv_scratch2_elems(c->d, c->n, nrhs);
  void* t1 = buf<double2>(c, "conv1_64", s1);
  void* t2 = s2 ? buf<double2>(c, "conv2_64", s2) : nullptr;
  ls::conv_apply_ff(c->plan, nrhs, u, y, sub, t1, t2, c->st);
}

// z = M^{-1} [A;B] v for FP64 input v; z in the factor precision C
// z = M^{-1} [A;B] v for v in FP64 or FP32 pairs; z in the factor precision C
template <typename C, typename Cv = double2> void precond_apply(ls_ctx* c, int nrhs, const Cv* v, C* z) {
  if constexpr (sizeof(C) == 8 && std::is_same<Cv, float2>::value) {
    if (c->d == 2 && !c->general && c->pre_refine >= 0 && nrhs <= ls::nd_items_max()) {
      // 2D FP32 after the estimate: the stencil sums go straight into the solve's items
      const int rc = ls::nd_item_width(nrhs);
      float2* T = static_cast<float2*>(ls::nd_items(c->nd));
      ls::stencil_items_2d(c->n, nrhs, rc, v, nullptr, T, c->alpha32, nullptr, nullptr, c->st);
      ls::nd_solve_items<C>(c->nd, nrhs, z, c->st, false);
      if (c->pre_refine == 1) {
        // z += M^{-1} ([A;B] v - M z)
        ls::stencil_items_2d(c->n, nrhs, rc, v, z, T, c->alpha32, c->cint64, c->w2m32, c->st);
        ls::nd_solve_items<C>(c->nd, nrhs, z, c->st, true);
      }
      return;
    }
  }
  C* r = buf<C>(c, sizeof(C) == 8 ? "pre_r32" : "pre_r64", (size_t)nrhs * c->N);
  if (c->general) {
    const void* apt = sizeof(C) == 8 ? (const void*)c->apt32 : (const void*)c->apt64;
    ls::stencil_apply_pt<Cv, C>(c->d, c->n, nrhs, v, r, 1, c->N, apt, c->st);
  } else {
    const void* alpha = sizeof(C) == 8 ? (const void*)c->alpha32 : (const void*)c->alpha64;
    ls::stencil_apply<Cv, C>(c->d, c->n, nrhs, v, r, 1, c->N, alpha, c->st);
  }
  ls::nd_solve<C>(c->nd, nrhs, r, z, c->st);
  if constexpr (sizeof(C) == 8 && std::is_same<Cv, float2>::value) {
    if (c->pre_refine == 1 && !c->general) {
      // one step of iterative refinement of z = M^{-1} [A;B] v with the FP32 factors:
      // z += M^{-1} ([A;B] v - M z), the correction added by the solve's last launch
      C* r2 = buf<C>(c, "pre_r2", (size_t)nrhs * c->N);
      ls::pre_resid(c->d, c->n, nrhs, v, z, r2, c->alpha32, c->cint64, c->w2m32, c->st);
      ls::nd_solve<C>(c->nd, nrhs, r2, z, c->st, true);
    }
  }
}

// |[A;B] v - M z|^2 and |[A;B] v|^2 of the first right-hand side of the last preconditioner
// application (FP32 path), into out[0].x and out[1].x
void precond_error(ls_ctx* c, const float2* v, const float2* z, double2* partial, double2* out) {
  const float2* sv = buf<float2>(c, "pre_r32", (size_t)c->N);  // [A;B] v of that application
  float2* r2 = buf<float2>(c, "pre_est", (size_t)c->N);
  ls::pre_resid(c->d, c->n, 1, v, z, r2, c->alpha32, c->cint64, c->w2m32, c->st);
  ls::norms2<float2>(r2, c->N, 1, partial, out, 1, c->st);
  ls::norms2<float2>(sv, c->N, 1, partial, out + 1, 1, c->st);
}

ls_status fail(ls_ctx* c, const Error& e) {
  if (c) c->err = e.msg;
  return (ls_status)e.code;
}

void check_ctx(ls_ctx* c) {
  if (!c) throw Error{ls::ESTATE_, "NULL context"};
}

// ---------------------------------------------------------------------------------------
// GMRES cycles (Sec. 3.3), batched over right-hand sides
// ---------------------------------------------------------------------------------------
// FP32 preconditioner residual |[A;B] v - M z| / |[A;B] v| above which every application is
// refined once.  GMRES contracts the residual by about max(rho, e) per iteration (rho: the
// rate of the exact preconditioner, e this residual), so e = 0.1 costs about twice the
// iterations of e < 0.01, while a refined application (e^2) costs one more forward and
// backward sweep (about a quarter of an iteration on the 2D workloads).  Measured on GB300:
// 2D n = 1024, omega = 2 pi 128: 0.13 (6 iterations, 3-4 refined; FP64: 3); 2D n = 256 and
// 3D n = 64 Helmholtz: 1e-5 (no refinement).
constexpr double PRE_REFINE_ABOVE = 0.02;

template <typename CZ>
void solve_impl(ls_ctx* c, int nrhs, const double2* g, double tol, double2* u, ls_info* info) {
  const long N = c->N, tot = N * nrhs;
  const int R = c->restart;
  const bool mixed = sizeof(CZ) == 8;
  ensure_basis(c, 2, nrhs, sizeof(CZ));
  double2* w = buf<double2>(c, "w64", tot);
  double2* r = buf<double2>(c, "r64", tot);
  double2* Au = mixed ? nullptr : buf<double2>(c, "Au64", tot);
  CZ* wz = mixed ? buf<CZ>(c, "w32", tot) : nullptr;
  const int nblk = ls::dots_blocks(N);
  double2* partial = buf<double2>(c, "partial", (size_t)nrhs * (R + 2) * nblk);
  double2* hd = buf<double2>(c, "hcol", (size_t)nrhs * (R + 2) * 2);
  double* sd = buf<double>(c, "scale", nrhs);
  ffc* hff = mixed ? buf<ffc>(c, "h_ff", (size_t)nrhs * (R + 2) * 2) : nullptr;
  double2* yd = buf<double2>(c, "ycoef", (size_t)nrhs * R);
  double2* est = mixed ? buf<double2>(c, "pre_err", 2) : nullptr;

  LS_CUDA(cudaMemsetAsync(u, 0, tot * sizeof(double2), c->st));
  std::vector<double2> hh((size_t)nrhs * (R + 2) * 2);
  ls::norms2<double2>(g, N, nrhs, partial, hd, 1, c->st);
  LS_CUDA(cudaMemcpyAsync(hh.data(), hd, nrhs * sizeof(double2), cudaMemcpyDeviceToHost, c->st));
  LS_CUDA(cudaStreamSynchronize(c->st));
  std::vector<double> gn(nrhs), rn(nrhs);
  for (int j = 0; j < nrhs; ++j) gn[j] = rn[j] = std::sqrt(hh[j].x);
  std::vector<int> iters(nrhs, 0), cycles(nrhs, 0);
  std::vector<char> conv(nrhs, 0);
  for (int j = 0; j < nrhs; ++j) conv[j] = rn[j] <= tol * gn[j];
  // the first cycle's residual is g itself (u = 0): it is read in place, r holds the later ones
  const double2* r0 = g;

  std::vector<cd> H((size_t)nrhs * (R + 1) * R), sn((size_t)nrhs * R), s((size_t)nrhs * (R + 1));
  std::vector<double> cs((size_t)nrhs * R), sc(nrhs);
  std::vector<int> kdone(nrhs);
  std::vector<char> act(nrhs);
  std::vector<double2> Y((size_t)nrhs * R);
  const double inner = mixed ? 0.5 : 1.0;
  // subsets of right-hand sides that are still iterating
  std::vector<int> live_ix(nrhs);
  int* dlive = buf<int>(c, "live_idx", nrhs);
  double2* vlive = buf<double2>(c, "live_v", tot);
  CZ* zlive = buf<CZ>(c, "live_z", tot);
  void* wlive = buf<double2>(c, "live_w", tot);

  while (true) {
    ls::Range cycle_range("gmres_cycle");
    bool any = false;
    for (int j = 0; j < nrhs; ++j) {
      act[j] = !conv[j] && iters[j] < c->max_iter;
      any |= act[j];
    }
    if (!any) break;
    // V_0 = r / |r|
    for (int j = 0; j < nrhs; ++j) {
      sc[j] = act[j] && rn[j] > 0 ? 1.0 / rn[j] : 0.0;
      kdone[j] = 0;
      s[(size_t)j * (R + 1)] = act[j] ? rn[j] : 0.0;
    }
    LS_CUDA(cudaMemcpyAsync(sd, sc.data(), nrhs * sizeof(double), cudaMemcpyHostToDevice, c->st));
    if (mixed) ls::scale_f<double2>(r0, (float2*)c->V[0], sd, N, nrhs, c->st);
    else ls::scale(r0, c->V[0], sd, N, nrhs, c->st);
    int k = 0;
    for (; k < R; ++k) {
      bool live = false;
      for (int j = 0; j < nrhs; ++j) live |= act[j] && kdone[j] == 0;
      if (!live) break;
      ensure_basis(c, k + 2, nrhs, sizeof(CZ));
      CZ* zk = (CZ*)c->Z[k];
      // right-hand sides still iterating; the others carry zero vectors (their scale was 0)
      int nlive = 0;
      for (int j = 0; j < nrhs; ++j)
        if (act[j] && kdone[j] == 0) live_ix[nlive++] = j;
      const bool compact = nlive < nrhs;
      if (compact) LS_CUDA(cudaMemcpyAsync(dlive, live_ix.data(), nlive * sizeof(int), cudaMemcpyHostToDevice, c->st));
      // z_k = P v_k (stencil + nested-dissection solve), w = A z_k (FFT operator), on the
      // live right-hand sides only
      // the FP32 path measures its preconditioner's residual in the first iteration after a
      // factorization and refines every later application when it is large (FGMRES allows
      // the preconditioner to change from one iteration to the next)
      const bool estimate = mixed && c->pre_refine < 0 && !c->general;
      run_graph(c, "iter:" + std::to_string(k) + ":" + std::to_string(nrhs) + ":" + std::to_string(nlive) +
                       (mixed ? ":m" : ":d") + (estimate ? ":e" : (c->pre_refine == 1 ? ":r" : "")),
                [&] {
                  if (!compact) {
                    if (mixed) precond_apply<CZ, float2>(c, nrhs, (const float2*)c->V[k], zk);
                    else precond_apply<CZ>(c, nrhs, c->V[k], zk);
                    if constexpr (sizeof(CZ) == 8)
                      if (estimate) precond_error(c, (const float2*)c->V[k], zk, partial, est);
                    if (mixed) op_apply<CZ>(c, nrhs, zk, wz);
                    else op_apply<double2>(c, nrhs, (const double2*)zk, w);
                    return;
                  }
                  if (mixed) {
                    ls::rhs_gather<float2>((const float2*)c->V[k], (float2*)vlive, dlive, nlive, N, c->st);
                    precond_apply<CZ, float2>(c, nlive, (const float2*)vlive, zlive);
                    if constexpr (sizeof(CZ) == 8)
                      if (estimate) precond_error(c, (const float2*)vlive, zlive, partial, est);
                  } else {
                    ls::rhs_gather<double2>(c->V[k], vlive, dlive, nlive, N, c->st);
                    precond_apply<CZ>(c, nlive, vlive, zlive);
                  }
                  LS_CUDA(cudaMemsetAsync(zk, 0, tot * sizeof(CZ), c->st));
                  ls::rhs_scatter<CZ>(zlive, zk, dlive, nlive, N, c->st);
                  if (mixed) {
                    op_apply<CZ>(c, nlive, zlive, (CZ*)wlive);
                    LS_CUDA(cudaMemsetAsync(wz, 0, tot * sizeof(CZ), c->st));
                    ls::rhs_scatter<CZ>((const CZ*)wlive, wz, dlive, nlive, N, c->st);
                  } else {
                    op_apply<double2>(c, nlive, (const double2*)zlive, (double2*)wlive);
                    LS_CUDA(cudaMemsetAsync(w, 0, tot * sizeof(double2), c->st));
                    ls::rhs_scatter<double2>((const double2*)wlive, w, dlive, nlive, N, c->st);
                  }
                });
      const double2* const* dV = c->dV;
      // CGS2 against V[0..k]
      double2* hd2 = hd + (size_t)nrhs * (R + 2);
      if (mixed) {
        // the basis and w stored as FP32 complex, every product and sum in float-float on
        // the FP32 pipes; the second projection also gives |w|^2
        const float2* const* dVf = reinterpret_cast<const float2* const*>(dV);
        float2* wf = reinterpret_cast<float2*>(w);
        ffc* hff2 = hff + (size_t)nrhs * (R + 2);
        ls::dots_f(dVf, k + 1, (const float2*)wz, N, nrhs, partial, hd, hff, R + 2, c->st);
        ls::sub_proj_f(dVf, k + 1, (const float2*)wz, wf, hff, R + 2, N, nrhs, partial, nullptr, 0, c->st);
        ls::dots_f(dVf, k + 1, wf, N, nrhs, partial, hd2, hff2, R + 2, c->st);
        ls::sub_proj_f(dVf, k + 1, wf, wf, hff2, R + 2, N, nrhs, partial, hd2 + (k + 1), R + 2, c->st);
      } else {
        ls::dots<double2>(dV, k + 1, w, N, nrhs, partial, hd, R + 2, false, c->st);
        ls::sub_proj<double2>(dV, k + 1, w, w, hd, R + 2, N, nrhs, c->st);
        ls::dots<double2>(dV, k + 1, w, N, nrhs, partial, hd2, R + 2, false, c->st);
        ls::sub_proj<double2>(dV, k + 1, w, w, hd2, R + 2, N, nrhs, c->st);
        ls::norms2<double2>(w, N, nrhs, partial, hd2 + (k + 1), R + 2, c->st);
      }
      LS_CUDA(cudaMemcpyAsync(hh.data(), hd, hh.size() * sizeof(double2), cudaMemcpyDeviceToHost, c->st));
      double2 est_h[2] = {};
      if (estimate) LS_CUDA(cudaMemcpyAsync(est_h, est, sizeof est_h, cudaMemcpyDeviceToHost, c->st));
      LS_CUDA(cudaStreamSynchronize(c->st));
      if (estimate) {
        c->pre_err = est_h[1].x > 0 ? std::sqrt(est_h[0].x / est_h[1].x) : 0.0;
        c->pre_refine = c->pre_err > PRE_REFINE_ABOVE ? 1 : 0;
      }
      for (int j = 0; j < nrhs; ++j) {
        sc[j] = 0.0;
        if (!act[j] || kdone[j]) continue;
        cd* Hj = &H[(size_t)j * (R + 1) * R];
        cd* col = Hj + (size_t)k * (R + 1);
        const double2* h1 = &hh[(size_t)j * (R + 2)];
        const double2* h2 = &hh[(size_t)(nrhs + j) * (R + 2)];
        for (int i = 0; i <= k; ++i) col[i] = cd(h1[i].x + h2[i].x, h1[i].y + h2[i].y);
        const double beta = std::sqrt(std::max(0.0, h2[k + 1].x));
        col[k + 1] = beta;
        double* csj = &cs[(size_t)j * R];
        cd* snj = &sn[(size_t)j * R];
        cd* sj = &s[(size_t)j * (R + 1)];
        for (int i = 0; i < k; ++i) {
          const cd a = col[i], bb = col[i + 1];
          col[i] = csj[i] * a + snj[i] * bb;
          col[i + 1] = -std::conj(snj[i]) * a + csj[i] * bb;
        }
        const cd a = col[k], bb = col[k + 1];
        const double rr = std::hypot(std::abs(a), std::abs(bb));
        if (std::abs(a) == 0.0) { csj[k] = 0.0; snj[k] = 1.0; }
        else { csj[k] = std::abs(a) / rr; snj[k] = (a / std::abs(a)) * std::conj(bb) / rr; }
        col[k] = csj[k] * a + snj[k] * bb;
        col[k + 1] = 0.0;
        sj[k + 1] = -std::conj(snj[k]) * sj[k];
        sj[k] = csj[k] * sj[k];
        iters[j] += 1;
        const double res = std::abs(sj[k + 1]);
        if (res <= inner * tol * gn[j] || beta == 0.0 || iters[j] >= c->max_iter) kdone[j] = k + 1;
        else sc[j] = 1.0 / beta;
      }
      LS_CUDA(cudaMemcpyAsync(sd, sc.data(), nrhs * sizeof(double), cudaMemcpyHostToDevice, c->st));
      if (mixed) ls::scale_f<float2>((const float2*)w, (float2*)c->V[k + 1], sd, N, nrhs, c->st);
      else ls::scale(w, c->V[k + 1], sd, N, nrhs, c->st);
    }
    // least squares: H(0:k, 0:k) y = s(0:k), per right-hand side
    int kmax = 0;
    std::fill(Y.begin(), Y.end(), make_double2(0, 0));
    for (int j = 0; j < nrhs; ++j) {
      if (!act[j]) continue;
      const int kj = kdone[j] ? kdone[j] : k;
      kmax = std::max(kmax, kj);
      const cd* Hj = &H[(size_t)j * (R + 1) * R];
      std::vector<cd> y(kj);
      for (int i = kj - 1; i >= 0; --i) {
        cd acc = s[(size_t)j * (R + 1) + i];
        for (int l = i + 1; l < kj; ++l) acc -= Hj[(size_t)l * (R + 1) + i] * y[l];
        y[i] = acc / Hj[(size_t)i * (R + 1) + i];
      }
      for (int i = 0; i < kj; ++i) Y[(size_t)j * R + i] = make_double2(y[i].real(), y[i].imag());
      cycles[j] += 1;
    }
    if (kmax > 0) {
      LS_CUDA(cudaMemcpyAsync(yd, Y.data(), Y.size() * sizeof(double2), cudaMemcpyHostToDevice, c->st));
      if (mixed) ls::update_u_f((const float2* const*)c->dZ, kmax, yd, R, u, N, nrhs, c->st);
      else ls::update_u<CZ>((const CZ* const*)c->dZ, kmax, yd, R, u, N, nrhs, c->st);
    }
    // residual r = g - A u in FP64 storage; the operator in float-float arithmetic on the
    // mixed path (GB300's FP64 rate is a small fraction of its FP32 rate), FP64 otherwise
    ls::Range resid_range("true_residual");
    run_graph(c, "resid:" + std::to_string(nrhs), [&] {
      if (mixed) {
        op_apply_ff(c, nrhs, u, r, g);
      } else {
        op_apply<double2>(c, nrhs, u, Au);
        ls::residual(g, Au, r, tot, c->st);
      }
      ls::norms2<double2>(r, N, nrhs, partial, hd, 1, c->st);
    });
    LS_CUDA(cudaMemcpyAsync(hh.data(), hd, nrhs * sizeof(double2), cudaMemcpyDeviceToHost, c->st));
    LS_CUDA(cudaStreamSynchronize(c->st));
    for (int j = 0; j < nrhs; ++j) {
      rn[j] = std::sqrt(hh[j].x);
      conv[j] = rn[j] <= tol * gn[j];
    }
    r0 = r;
  }
  bool all = true;
  for (int j = 0; j < nrhs; ++j) {
    if (info) {
      info[j].iters = iters[j];
      info[j].refinements = std::max(0, cycles[j] - 1);
      info[j].rel_resid = gn[j] > 0 ? rn[j] / gn[j] : 0.0;
      info[j].converged = conv[j] ? 1 : 0;
    }
    all &= conv[j] != 0;
  }
  if (!all) throw Error{ls::ENOCONV_, "GMRES did not reach the tolerance for every right-hand side"};
}

bool pow2(int x) { return x > 0 && (x & (x - 1)) == 0; }

}  // namespace

// =======================================================================================
// C-ABI
// =======================================================================================
// FNV-1a (64 bit) of a byte array
static uint64_t fnv1a(const void* data, size_t bytes) {
  const unsigned char* q = static_cast<const unsigned char*>(data);
  uint64_t h = 1469598103934665603ull;
  for (size_t i = 0; i < bytes; ++i) {
    h ^= q[i];
    h *= 1099511628211ull;
  }
  return h;
}

// Medium of a context (Sec. 2.1): the host copy of m (host or device pointer) is checked --
// finite, 1 - m > 0 (Helmholtz), zero within b + 1 layers of the boundary -- and turned into
// the potential omega^2 m (V itself for a Laplace context) in FP64 and FP32.
static void medium_weights(const ls_ctx* c, const double* m, std::vector<double>& w64, std::vector<float>& w32) {
  const long N = c->N;
  const int n = c->n;
  std::vector<double> mh(N);
  if (is_device_ptr(m)) LS_CUDA(cudaMemcpy(mh.data(), m, N * sizeof(double), cudaMemcpyDeviceToHost));
  else std::memcpy(mh.data(), m, N * sizeof(double));
  const int wl = c->b + 1;
  for (long i = 0; i < N; ++i) {
    if (!std::isfinite(mh[i])) throw Error{ls::EINVAL_, "the medium must be finite"};
    if (!c->laplace && !(1.0 - mh[i] > 0)) throw Error{ls::EINVAL_, "m must satisfy 1 - m > 0"};
    long q = i;
    bool edge = false;
    for (int a = 0; a < c->d; ++a) {
      const long ia = q % n;
      q /= n;
      if (ia < wl || ia >= n - wl) edge = true;
    }
    if (edge && mh[i] != 0.0) throw Error{ls::EBUFFER_, "the medium must vanish within b+1 layers of the boundary"};
  }
  w64.resize(N);
  w32.resize(N);
  const double w2 = c->laplace ? 1.0 : c->omega * c->omega;
  for (long i = 0; i < N; ++i) {
    w64[i] = c->laplace ? mh[i] : w2 * mh[i];
    w32[i] = (float)w64[i];
  }
}

extern "C" {

// ---------------------------------------------------------------------------------------
// Autotuner: the launch-shape choices of the factorization and of the solve sweeps (ls::NdTune)
// per (d, n, precision, kernel), timed on a context and kept process-wide; with LS_TUNE_FILE
// set, the table is read from that file at the first setup and rewritten after each tuning.
// ---------------------------------------------------------------------------------------
struct TuneKey {
  int d, n, prec, laplace;
  bool operator<(const TuneKey& o) const {
    return std::tie(d, n, prec, laplace) < std::tie(o.d, o.n, o.prec, o.laplace);
  }
};
static std::mutex g_tune_mu;
static std::map<TuneKey, ls::NdTune> g_tune;
static bool g_tune_loaded = false;

static TuneKey tune_key(const ls_ctx* c) { return TuneKey{c->d, c->n, (int)c->prec, c->laplace ? 1 : 0}; }

// one line per entry, the format tune_save writes
static void tune_load_locked() {
  if (g_tune_loaded) return;
  g_tune_loaded = true;
  const char* path = std::getenv("LS_TUNE_FILE");
  if (!path || !*path) return;
  FILE* f = std::fopen(path, "r");
  if (!f) return;
  char line[512];
  while (std::fgets(line, sizeof line, f)) {
    TuneKey k{};
    ls::NdTune t;
    if (std::sscanf(line,
                    "{\"d\": %d, \"n\": %d, \"prec\": %d, \"laplace\": %d, \"two_level_min\": %lf, "
                    "\"tc_min_rows\": %d, \"sweep_ctas\": %d, \"gj_max_own\": %d, \"tcs_min_rows\": %d, "
                    "\"tcs_bwd_min_rows\": %d, \"small_max_k\": %d}",
                    &k.d, &k.n, &k.prec, &k.laplace, &t.two_level_min, &t.tc_min_rows, &t.sweep_ctas,
                    &t.gj_max_own, &t.tcs_min_rows, &t.tcs_bwd_min_rows, &t.small_max_k) == 11)
      g_tune[k] = t;
  }
  std::fclose(f);
}

static void tune_save_locked() {
  const char* path = std::getenv("LS_TUNE_FILE");
  if (!path || !*path) return;
  const std::string tmp = std::string(path) + ".tmp";
  FILE* f = std::fopen(tmp.c_str(), "w");
  if (!f) return;
  for (const auto& kv : g_tune)
    std::fprintf(f,
                 "{\"d\": %d, \"n\": %d, \"prec\": %d, \"laplace\": %d, \"two_level_min\": %.17g, "
                 "\"tc_min_rows\": %d, \"sweep_ctas\": %d, \"gj_max_own\": %d, \"tcs_min_rows\": %d, "
                 "\"tcs_bwd_min_rows\": %d, \"small_max_k\": %d}\n",
                 kv.first.d, kv.first.n, kv.first.prec, kv.first.laplace, kv.second.two_level_min,
                 kv.second.tc_min_rows, kv.second.sweep_ctas, kv.second.gj_max_own, kv.second.tcs_min_rows,
                 kv.second.tcs_bwd_min_rows, kv.second.small_max_k);
  std::fclose(f);
  std::rename(tmp.c_str(), path);
}

static bool tune_lookup(const TuneKey& k, ls::NdTune* t) {
  std::lock_guard<std::mutex> lk(g_tune_mu);
  tune_load_locked();
  auto it = g_tune.find(k);
  if (it == g_tune.end()) return false;
  *t = it->second;
  return true;
}

static std::string tune_json(const ls::NdTune& t) {
  char b[256];
  std::snprintf(b, sizeof b,
                "{\"two_level_min\": %.6g, \"tc_min_rows\": %d, \"sweep_ctas\": %d, \"gj_max_own\": %d, "
                "\"tcs_min_rows\": %d, \"tcs_bwd_min_rows\": %d, \"small_max_k\": %d}",
                t.two_level_min, t.tc_min_rows, t.sweep_ctas, t.gj_max_own, t.tcs_min_rows, t.tcs_bwd_min_rows,
                t.small_max_k);
  return b;
}

static void write_report(const std::string& r, char* out, int capacity) {
  if (!out || capacity <= 0) return;
  const size_t n = std::min(r.size(), (size_t)capacity - 1);
  std::memcpy(out, r.data(), n);
  out[n] = '\0';
}

// Shared by ls_setup (Helmholtz kernel, medium m, potential omega^2 m) and ls_setup_laplace
// (Sec. 5: Laplace kernel, potential V given directly; omega = 0 selects the kernel).
static ls_status setup_common(const ls_grid* g, double omega, const double* m, bool laplace, void* stream,
                              ls_ctx** out) {
  if (out) *out = nullptr;
  ls_ctx* c = nullptr;
  ls::Range range(laplace ? "ls_setup_laplace" : "ls_setup");
  try {
    if (!g || !m || !out) throw Error{ls::EINVAL_, "NULL argument"};
    if (g->dim != 2 && g->dim != 3) throw Error{ls::EINVAL_, "dim must be 2 or 3"};
    if (laplace && g->dim != 3) throw Error{ls::EINVAL_, "the Laplace variant is three-dimensional (Sec. 5)"};
    const int n = g->n;
    if (!pow2(2 * n) && 2 * n != 48 && 2 * n != 96)
      throw Error{ls::EINVAL_, "2n must be a power of two, 48 or 96 (the FFT lengths of the passes)"};
    if (g->dim == 2 && (n < 16 || n > 2048)) throw Error{ls::EINVAL_, "2D needs 16 <= n <= 2048"};
    if (g->dim == 3 && (n < 8 || n > 128)) throw Error{ls::EINVAL_, "3D needs 8 <= n <= 128"};
    if (!laplace && (!(omega > 0) || !std::isfinite(omega))) throw Error{ls::EINVAL_, "omega must be positive"};
    const int b = g->buffer_b > 0 ? g->buffer_b : 2;
    if (n <= 2 * (b + 1)) throw Error{ls::EINVAL_, "n too small for the buffer layers"};
    if (g->prec != LS_PREC_FP64 && g->prec != LS_PREC_MIXED) throw Error{ls::EINVAL_, "unknown precision"};
    if (g->k0_rule != LS_K0_BALL && g->k0_rule != LS_K0_CORRECTED) throw Error{ls::EINVAL_, "unknown k0_rule"};
    if (g->front_fmt == LS_FRONT_TF32 || g->front_fmt == LS_FRONT_BF16)
      throw Error{ls::EINVAL_, "TF32 and BF16 fronts are not built (LS_FRONT_3XTF32 or LS_FRONT_FP32)"};
    if (g->front_fmt != LS_FRONT_3XTF32 && g->front_fmt != LS_FRONT_FP32) throw Error{ls::EINVAL_, "unknown front_fmt"};
    c = new ls_ctx;
    c->g = *g;
    c->d = g->dim;
    c->n = n;
    c->L = 2 * n;
    c->b = b;
    c->restart = g->restart > 0 ? g->restart : 50;
    c->max_iter = g->max_iter > 0 ? g->max_iter : 500;
    c->prec = g->prec;
    c->N = c->d == 2 ? (long)n * n : (long)n * n * n;
    c->laplace = laplace;
    c->omega = laplace ? 0.0 : omega;
    c->h = 1.0 / (n + 1);
    LS_CUDA(cudaGetDevice(&c->device));
    // LS_GRAPHS=0 runs every launch eagerly (for debugging and per-launch timing)
    if (const char* e = std::getenv("LS_GRAPHS")) c->use_graphs = std::strcmp(e, "0") != 0;
    if (stream) c->st = (cudaStream_t)stream;
    else {
      LS_CUDA(cudaStreamCreateWithFlags(&c->st, cudaStreamNonBlocking));
      c->own_stream = true;
    }
    LS_CUDA(cudaStreamCreateWithFlags(&c->st2, cudaStreamNonBlocking));
    LS_CUDA(cudaEventCreateWithFlags(&c->ev_factor, cudaEventDisableTiming));
    std::vector<double> w64;
    std::vector<float> w32;
    medium_weights(c, m, w64, w32);
    c->medium_hash = fnv1a(w64.data(), w64.size() * sizeof(double));
    c->w2m64 = dalloc<double>(c->N);
    c->w2m32 = dalloc<float>(c->N);
    LS_CUDA(cudaMemcpyAsync(c->w2m64, w64.data(), c->N * sizeof(double), cudaMemcpyHostToDevice, c->st));
    LS_CUDA(cudaMemcpyAsync(c->w2m32, w32.data(), c->N * sizeof(float), cudaMemcpyHostToDevice, c->st));
    // twiddles: exp(-2 pi i m / L) for the FP64 and float-float passes, the per-pass table of
    // the FP32 passes (fft_plan.h)
    const int L = c->L;
    std::vector<double2> t64(L), tp;
    for (int q = 0; q < L; ++q) {
      const double a = -2.0 * M_PI * (double)q / (double)L;
      t64[q] = make_double2(std::cos(a), std::sin(a));
    }
    ls::fft_twiddles(L, tp);
    std::vector<float2> t32(tp.size());
    for (size_t q = 0; q < tp.size(); ++q) t32[q] = make_float2((float)tp[q].x, (float)tp[q].y);
    c->tw64 = dalloc<double2>(L);
    c->tw32 = dalloc<float2>(t32.size());
    LS_CUDA(cudaMemcpyAsync(c->tw64, t64.data(), L * sizeof(double2), cudaMemcpyHostToDevice, c->st));
    LS_CUDA(cudaMemcpyAsync(c->tw32, t32.data(), t32.size() * sizeof(float2), cudaMemcpyHostToDevice, c->st));
    // Nystrom table quadrant and symbol (Sec. 2.1)
    const long n1 = n + 1;
    const long nq = c->d == 2 ? n1 * n1 : n1 * n1 * n1;
    c->ktq = dalloc<double2>(nq);
    c->sym64 = dalloc<double2>(nq);
    c->sym32 = dalloc<float2>(nq);
    ls::build_kernel_table(c->d, n, c->omega, c->h, c->ktq, c->st);
    // the higher-order weight of the singular point replaces k_0 = ktq[0] (Sec. 2.1); the
    // stream is synchronised below, before k0w goes out of scope
    double k0w[2] = {0.0, 0.0};
    if (g->k0_rule == LS_K0_CORRECTED) {
      if (ls_k0_weight(c->d, c->omega, c->h, LS_K0_CORRECTED, k0w) != LS_OK)
        throw Error{ls::EINVAL_, "k_0 weight undefined for these arguments"};
      LS_CUDA(cudaMemcpyAsync(c->ktq, k0w, sizeof(double2), cudaMemcpyHostToDevice, c->st));
    }
    c->plan.d = c->d;
    c->plan.n = n;
    c->plan.omega = c->omega;
    c->plan.h = c->h;
    c->plan.tw32 = c->tw32;
    c->plan.tw64 = c->tw64;
    c->plan.w2m32 = c->w2m32;
    c->plan.w2m64 = c->w2m64;
    {
      const long Ld = c->d == 2 ? (long)L * L : (long)L * L * L;
      double2* work = dalloc<double2>(Ld);
      try {
        ls::build_symbol(c->plan, c->ktq, c->sym64, c->sym32, work, c->st);
        LS_CUDA(cudaStreamSynchronize(c->st));
      } catch (...) {
        ls::dev_free(work);
        throw;
      }
      ls::dev_free(work);
    }
    c->plan.sym32 = c->sym32;
    c->plan.sym64 = c->sym64;
    {
      const size_t ntwf = 2 * (size_t)L, nsy = 2 * (size_t)nq;  // FP64 components: one float pair each
      c->ffbuf = dalloc<float2>(ntwf + nsy + (size_t)c->N);
      ls::to_ff(reinterpret_cast<const double*>(c->tw64), c->ffbuf, (long)ntwf, c->st);
      ls::to_ff(reinterpret_cast<const double*>(c->sym64), c->ffbuf + ntwf, (long)nsy, c->st);
      ls::to_ff(c->w2m64, c->ffbuf + ntwf + nsy, c->N, c->st);
      c->plan.twff = c->ffbuf;
      c->plan.symff = c->ffbuf + ntwf;
      c->plan.w2mff = c->ffbuf + ntwf + nsy;
    }
    // stencils (Sec. 3.1), cached per (d, n, b, omega); omega = 0 is the Laplace kernel
    {
      StencilKey key{c->d, n, b, c->omega, g->k0_rule};
      bool hit = false;
      {
        std::lock_guard<std::mutex> lk(g_mu);
        auto it = g_stencil_cache.find(key);
        if (it != g_stencil_cache.end()) {
          c->alpha_h = it->second.first;
          c->cint_h = it->second.second;
          hit = true;
        }
      }
      if (!hit) {
        std::vector<double2> kh(nq);
        LS_CUDA(cudaMemcpy(kh.data(), c->ktq, nq * sizeof(double2), cudaMemcpyDeviceToHost));
        ls::compute_stencils(c->d, n, b, kh, c->alpha_h, c->cint_h);
        std::lock_guard<std::mutex> lk(g_mu);
        g_stencil_cache[key] = {c->alpha_h, c->cint_h};
      }
    }
    const size_t na = c->alpha_h.size();
    std::vector<float2> a32(na);
    for (size_t i = 0; i < na; ++i) a32[i] = make_float2((float)c->alpha_h[i].x, (float)c->alpha_h[i].y);
    c->alpha64 = dalloc<double2>(na);
    c->alpha32 = dalloc<float2>(na);
    c->cint64 = dalloc<double2>(c->cint_h.size());
    LS_CUDA(cudaMemcpyAsync(c->alpha64, c->alpha_h.data(), na * sizeof(double2), cudaMemcpyHostToDevice, c->st));
    LS_CUDA(cudaMemcpyAsync(c->alpha32, a32.data(), na * sizeof(float2), cudaMemcpyHostToDevice, c->st));
    LS_CUDA(cudaMemcpyAsync(c->cint64, c->cint_h.data(), c->cint_h.size() * sizeof(double2), cudaMemcpyHostToDevice, c->st));
    // nested-dissection structure (Sec. 3.2)
    c->nd = ls::nd_build(c->d, n, c->st);
    {
      ls::NdTune t;
      if (tune_lookup(tune_key(c), &t)) ls::nd_set_tune(c->nd, t);
    }
    ls::nd_set_tensor_cores(c->nd, g->front_fmt == LS_FRONT_3XTF32);
    LS_CUDA(cudaStreamSynchronize(c->st));
    *out = c;
    return LS_OK;
  } catch (const Error& e) {
    std::lock_guard<std::mutex> lk(g_mu);
    g_setup_err = e.msg;
    if (c) ls_free(c);
    return (ls_status)e.code;
  } catch (const std::bad_alloc&) {
    std::lock_guard<std::mutex> lk(g_mu);
    g_setup_err = "host allocation failed";
    if (c) ls_free(c);
    return LS_ENOMEM;
  }
}

ls_status ls_setup(const ls_grid* g, double omega, const double* m, void* stream, ls_ctx** out) {
  return setup_common(g, omega, m, false, stream, out);
}

ls_status ls_setup_laplace(const ls_grid* g, const double* V, void* stream, ls_ctx** out) {
  return setup_common(g, 0.0, V, true, stream, out);
}

ls_status ls_factor(ls_ctx* c) {
  ls::Range range("ls_factor");
  try {
    check_ctx(c);
    c->factored = false;
    const bool mixed = c->prec == LS_PREC_MIXED;
    if (mixed ? ls::nd_prepare<float2>(c->nd, c->st) : ls::nd_prepare<double2>(c->nd, c->st)) ++c->gen;
    const void* apt = c->general ? (const void*)c->apt64 : nullptr;
    const unsigned char* inter = c->general ? c->inter_pt : nullptr;
    run_graph(c, "factor", [&] {
      if (mixed) ls::nd_factor_launch<float2>(c->nd, c->alpha64, c->cint64, c->w2m64, c->st, c->ev_factor, apt, inter);
      else ls::nd_factor_launch<double2>(c->nd, c->alpha64, c->cint64, c->w2m64, c->st, c->ev_factor, apt, inter);
    });
    c->factored = true;
    c->factor_pending = true;
    c->pre_refine = c->pre_refine_mode;
    c->pre_err = -1.0;
    return LS_OK;
  } catch (const Error& e) {
    return fail(c, e);
  } catch (const std::bad_alloc&) {
    return fail(c, Error{ls::ENOMEM_, "host allocation failed"});
  }
}

ls_status ls_rhs_plane_wave(ls_ctx* c, int nrhs, const double* dirs, double* g_out) {
  ls::Range range("ls_rhs_plane_wave");
  try {
    check_ctx(c);
    if (c->laplace) throw Error{ls::ESTATE_, "plane waves need the Helmholtz kernel (omega > 0)"};
    if (nrhs < 1 || !dirs || !g_out) throw Error{ls::EINVAL_, "bad arguments"};
    const size_t tot = (size_t)nrhs * c->N;
    double* dd = buf<double>(c, "dirs", (size_t)nrhs * c->d);
    double2* gd = buf<double2>(c, "rhs_out", tot);
    const size_t s1 = ls::conv_scratch1_elems(c->d, c->n, nrhs), s2 = ls::conv_scratch2_elems(c->d, c->n, nrhs);
    void* t1 = buf<double2>(c, "conv1_64", s1);
    void* t2 = s2 ? buf<double2>(c, "conv2_64", s2) : nullptr;
    // With a factorization in flight, run on the side stream from the point where its top
    // levels begin (they occupy few SMs; every earlier use of these buffers is before that
    // point in stream order), so that the two overlap; it uses none of the factorization's
    // data.
    cudaStream_t st = c->st;
    if (c->factor_pending) {
      st = c->st2;
      LS_CUDA(cudaStreamWaitEvent(st, c->ev_factor, 0));
    }
    copy_in(c, dd, dirs, (size_t)nrhs * c->d * sizeof(double), st);
    // float-float passes on the mixed path, FP64 on the plain path
    if (c->prec == LS_PREC_MIXED)
      ls::conv_rhs_ff(c->plan, nrhs, dd, gd, t1, t2, buf<ffc>(c, "rhs_phase", (size_t)nrhs * c->d * c->n), st);
    else ls::conv_apply<double2>(c->plan, nrhs, (const double2*)nullptr, gd, dd, false, t1, t2, st);
    copy_out(c, g_out, gd, tot * sizeof(double2), st);
    LS_CUDA(cudaStreamSynchronize(st));
    return LS_OK;
  } catch (const Error& e) {
    return fail(c, e);
  }
}

ls_status ls_rhs_point_source(ls_ctx* c, int nrhs, const int* points, const double* strengths, double* g_out) {
  try {
    check_ctx(c);
    if (nrhs < 1 || !points || !g_out) throw Error{ls::EINVAL_, "bad arguments"};
    const size_t np = (size_t)nrhs * c->d;
    std::vector<int> ph(np);
    if (is_device_ptr(points)) LS_CUDA(cudaMemcpy(ph.data(), points, np * sizeof(int), cudaMemcpyDeviceToHost));
    else std::memcpy(ph.data(), points, np * sizeof(int));
    for (size_t i = 0; i < np; ++i)
      if (ph[i] < 0 || ph[i] >= c->n) throw Error{ls::EINVAL_, "source point outside the grid"};
    const size_t tot = (size_t)nrhs * c->N;
    int* pd = buf<int>(c, "src_points", np);
    double2* qd = strengths ? buf<double2>(c, "src_strengths", nrhs) : nullptr;
    double2* gd = buf<double2>(c, "rhs_out", tot);
    // with a factorization in flight, on the side stream (it reads only the kernel table)
    cudaStream_t st = c->st;
    if (c->factor_pending) {
      st = c->st2;
      LS_CUDA(cudaStreamWaitEvent(st, c->ev_factor, 0));
    }
    LS_CUDA(cudaMemcpyAsync(pd, ph.data(), np * sizeof(int), cudaMemcpyHostToDevice, st));
    if (qd) copy_in(c, qd, strengths, (size_t)nrhs * sizeof(double2), st);
    ls::point_source(c->d, c->n, nrhs, pd, qd, c->ktq, c->h, gd, st);
    copy_out(c, g_out, gd, tot * sizeof(double2), st);
    LS_CUDA(cudaStreamSynchronize(st));
    return LS_OK;
  } catch (const Error& e) {
    return fail(c, e);
  }
}

ls_status ls_far_field(ls_ctx* c, int nrhs, const double* dirs, const double* us, int nobs, const double* obs,
                       double* out) {
  try {
    check_ctx(c);
    if (c->laplace) throw Error{ls::ESTATE_, "the far-field pattern needs the Helmholtz kernel (omega > 0)"};
    if (nrhs < 1 || nobs < 1 || !dirs || !us || !obs || !out) throw Error{ls::EINVAL_, "bad arguments"};
    const size_t tot = (size_t)nrhs * c->N;
    double* dd = buf<double>(c, "ff_dirs", (size_t)nrhs * c->d);
    double* od = buf<double>(c, "ff_obs", (size_t)nobs * c->d);
    double2* ud = buf<double2>(c, "ff_u", tot);
    double2* fd = buf<double2>(c, "ff_out", (size_t)nrhs * nobs);
    copy_in(c, dd, dirs, (size_t)nrhs * c->d * sizeof(double));
    copy_in(c, od, obs, (size_t)nobs * c->d * sizeof(double));
    copy_in(c, ud, us, tot * sizeof(double2));
    ls::far_field(c->d, c->n, nrhs, nobs, ud, dd, od, c->w2m64, c->omega, c->h, fd, c->st);
    copy_out(c, out, fd, (size_t)nrhs * nobs * sizeof(double2));
    LS_CUDA(cudaStreamSynchronize(c->st));
    return LS_OK;
  } catch (const Error& e) {
    return fail(c, e);
  }
}

ls_status ls_solve(ls_ctx* c, int nrhs, const double* rhs, double tol, double* u_out, ls_info* info) {
  ls::Range range("ls_solve");
  try {
    check_ctx(c);
    if (!c->factored) throw Error{ls::ESTATE_, "ls_solve before ls_factor"};
    factor_wait(c);
    if (nrhs < 1 || !rhs || !u_out || !(tol > 0)) throw Error{ls::EINVAL_, "bad arguments"};
    const size_t tot = (size_t)nrhs * c->N;
    double2* g = buf<double2>(c, "solve_g", tot);
    double2* u = buf<double2>(c, "solve_u", tot);
    copy_in(c, g, rhs, tot * sizeof(double2));
    ls_status st = LS_OK;
    try {
      if (c->prec == LS_PREC_MIXED) solve_impl<float2>(c, nrhs, g, tol, u, info);
      else solve_impl<double2>(c, nrhs, g, tol, u, info);
    } catch (const Error& e) {
      if (e.code != ls::ENOCONV_) throw;
      c->err = e.msg;
      st = LS_ENOCONV;
    }
    copy_out(c, u_out, u, tot * sizeof(double2));
    LS_CUDA(cudaStreamSynchronize(c->st));
    return st;
  } catch (const Error& e) {
    return fail(c, e);
  } catch (const std::bad_alloc&) {
    return fail(c, Error{ls::ENOMEM_, "host allocation failed"});
  }
}

const char* ls_last_error(const ls_ctx* c) {
  if (!c) return g_setup_err.c_str();
  return c->err.c_str();
}

void ls_free(ls_ctx* c) {
  if (!c) return;
  if (c->st) cudaStreamSynchronize(c->st);
  if (c->st2) cudaStreamSynchronize(c->st2);
  for (void* p : {(void*)c->w2m64, (void*)c->w2m32, (void*)c->tw32, (void*)c->tw64, (void*)c->ktq, (void*)c->sym32,
                  (void*)c->sym64, (void*)c->ffbuf, (void*)c->alpha64, (void*)c->alpha32, (void*)c->cint64, (void*)c->dV, (void*)c->dZ,
                  (void*)c->apt64, (void*)c->apt32, (void*)c->inter_pt})
    if (p) ls::dev_free(p);
  for (auto p : c->V) ls::dev_free(p);
  for (auto p : c->Z) ls::dev_free(p);
  for (auto& kv : c->bufs)
    if (kv.second.p) ls::dev_free(kv.second.p);
  for (auto& kv : c->graphs)
    if (kv.second.exec) cudaGraphExecDestroy(kv.second.exec);
  if (c->nd) ls::nd_free(c->nd);
  if (c->own_stream && c->st) cudaStreamDestroy(c->st);
  if (c->st2) cudaStreamDestroy(c->st2);
  if (c->ev_factor) cudaEventDestroy(c->ev_factor);
  cudaGetLastError();
  delete c;
}

ls_status ls_kernel_table(ls_ctx* c, double* out) {
  try {
    check_ctx(c);
    if (!out) throw Error{ls::EINVAL_, "NULL out"};
    const long n1 = c->n + 1;
    const long nq = c->d == 2 ? n1 * n1 : n1 * n1 * n1;
    copy_out(c, out, c->ktq, nq * sizeof(double2));
    LS_CUDA(cudaStreamSynchronize(c->st));
    return LS_OK;
  } catch (const Error& e) {
    return fail(c, e);
  }
}

ls_status ls_stencils(ls_ctx* c, double* alpha_out, double* c_out) {
  try {
    check_ctx(c);
    if (alpha_out) std::memcpy(alpha_out, c->alpha_h.data(), c->alpha_h.size() * sizeof(double2));
    if (c_out) std::memcpy(c_out, c->cint_h.data(), c->cint_h.size() * sizeof(double2));
    return LS_OK;
  } catch (const Error& e) {
    return fail(c, e);
  }
}

ls_status ls_apply(ls_ctx* c, int nrhs, const double* in, double* out, ls_prec prec) {
  try {
    check_ctx(c);
    if (nrhs < 1 || !in || !out) throw Error{ls::EINVAL_, "bad arguments"};
    const size_t tot = (size_t)nrhs * c->N;
    double2* x = buf<double2>(c, "io_in", tot);
    double2* y = buf<double2>(c, "io_out", tot);
    copy_in(c, x, in, tot * sizeof(double2));
    if (prec == LS_PREC_MIXED) {
      float2* x32 = buf<float2>(c, "io_in32", tot);
      float2* y32 = buf<float2>(c, "io_out32", tot);
      ls::cast<double2, float2>(x, x32, tot, c->st);
      op_apply<float2>(c, nrhs, x32, y32);
      ls::cast<float2, double2>(y32, y, tot, c->st);
    } else if (prec == LS_PREC_FF) {
      op_apply_ff(c, nrhs, x, y, nullptr);
    } else if (prec == LS_PREC_FP64) {
      op_apply<double2>(c, nrhs, x, y);
    } else {
      throw Error{ls::EINVAL_, "unknown precision"};
    }
    copy_out(c, out, y, tot * sizeof(double2));
    LS_CUDA(cudaStreamSynchronize(c->st));
    return LS_OK;
  } catch (const Error& e) {
    return fail(c, e);
  }
}

// A new medium on the context's grid, frequency and kernel: the potential tables (FP64,
// FP32, float-float) are rewritten in place, so the stencils, the symbol, the
// nested-dissection structure, the buffers and the captured graphs stay valid; the
// factorization and a general-domain preconditioner (whose stencils depend on the medium)
// are dropped.
ls_status ls_set_medium(ls_ctx* c, const double* m) {
  try {
    check_ctx(c);
    if (!m) throw Error{ls::EINVAL_, "NULL medium"};
    std::vector<double> w64;
    std::vector<float> w32;
    medium_weights(c, m, w64, w32);
    LS_CUDA(cudaStreamSynchronize(c->st));  // nothing in flight reads the old tables
    c->medium_hash = fnv1a(w64.data(), w64.size() * sizeof(double));
    c->factor_pending = false;
    c->factored = false;
    if (c->general) {
      c->general = false;
      ++c->gen;  // captured graphs hold the per-point tables
    }
    LS_CUDA(cudaMemcpyAsync(c->w2m64, w64.data(), c->N * sizeof(double), cudaMemcpyHostToDevice, c->st));
    LS_CUDA(cudaMemcpyAsync(c->w2m32, w32.data(), c->N * sizeof(float), cudaMemcpyHostToDevice, c->st));
    // the float-float copy where the setup placed it (after the twiddles and the symbol)
    ls::to_ff(c->w2m64, const_cast<float2*>(static_cast<const float2*>(c->plan.w2mff)), c->N, c->st);
    LS_CUDA(cudaStreamSynchronize(c->st));
    return LS_OK;
  } catch (const Error& e) {
    return fail(c, e);
  } catch (const std::bad_alloc&) {
    return fail(c, Error{ls::ENOMEM_, "host allocation failed"});
  }
}

// Checkpoint of a factorization (the serving cache spilled to host memory): a header that
// identifies grid, frequency, kernel, formats and medium, then the factored fronts.
struct FactorHeader {
  char magic[8];
  int32_t d, n, b, prec, k0_rule, front_fmt, laplace, reserved;
  double omega;
  uint64_t medium_hash, bytes;
};
static const char FACTOR_MAGIC[8] = {'L', 'S', 'F', 'A', 'C', 'T', '1', '\0'};

static FactorHeader factor_header(const ls_ctx* c) {
  FactorHeader h{};
  std::memcpy(h.magic, FACTOR_MAGIC, sizeof h.magic);
  h.d = c->d;
  h.n = c->n;
  h.b = c->b;
  h.prec = (int32_t)c->prec;
  h.k0_rule = c->g.k0_rule;
  h.front_fmt = c->g.front_fmt;
  h.laplace = c->laplace ? 1 : 0;
  h.omega = c->omega;
  h.medium_hash = c->medium_hash;
  h.bytes = ls::nd_factor_bytes(c->nd);
  return h;
}

ls_status ls_export_factors(ls_ctx* c, void* out, size_t capacity, size_t* size) {
  try {
    check_ctx(c);
    if (!size) throw Error{ls::EINVAL_, "NULL size"};
    if (!c->factored) throw Error{ls::ESTATE_, "no factorization to export"};
    if (c->general) throw Error{ls::ESTATE_, "general-domain factorizations are not exported"};
    factor_wait(c);
    const FactorHeader h = factor_header(c);
    *size = sizeof(FactorHeader) + h.bytes;
    if (!out) return LS_OK;
    if (capacity < *size) throw Error{ls::EINVAL_, "capacity below the exported size"};
    if (is_device_ptr(out)) throw Error{ls::EINVAL_, "out must be a host array"};
    std::memcpy(out, &h, sizeof h);
    ls::nd_copy_factors(c->nd, static_cast<unsigned char*>(out) + sizeof h, true, c->st);
    return LS_OK;
  } catch (const Error& e) {
    return fail(c, e);
  }
}

ls_status ls_import_factors(ls_ctx* c, const void* in, size_t size) {
  try {
    check_ctx(c);
    if (!in || size < sizeof(FactorHeader)) throw Error{ls::EINVAL_, "bad arguments"};
    if (is_device_ptr(in)) throw Error{ls::EINVAL_, "in must be a host array"};
    if (c->general) throw Error{ls::ESTATE_, "general-domain factorizations are not imported"};
    FactorHeader h;
    std::memcpy(&h, in, sizeof h);
    if (std::memcmp(h.magic, FACTOR_MAGIC, sizeof h.magic) != 0)
      throw Error{ls::EINVAL_, "not an exported factorization"};
    const FactorHeader mine = factor_header(c);
    if (h.d != mine.d || h.n != mine.n || h.b != mine.b || h.prec != mine.prec || h.k0_rule != mine.k0_rule ||
        h.front_fmt != mine.front_fmt || h.laplace != mine.laplace || h.omega != mine.omega)
      throw Error{ls::EINVAL_, "factorization of another grid, frequency, kernel or format"};
    if (h.medium_hash != mine.medium_hash) throw Error{ls::EINVAL_, "factorization of another medium"};
    // checked before anything is dropped: a refused import leaves an existing factorization
    const size_t want = ls::nd_factor_elems(c->nd) * (c->prec == LS_PREC_MIXED ? sizeof(float2) : sizeof(double2));
    if (h.bytes != want || size < sizeof h + h.bytes)
      throw Error{ls::EINVAL_, "size of the exported factorization does not match"};
    LS_CUDA(cudaStreamSynchronize(c->st));
    c->factored = false;
    c->factor_pending = false;
    const bool mixed = c->prec == LS_PREC_MIXED;
    if (mixed ? ls::nd_prepare<float2>(c->nd, c->st) : ls::nd_prepare<double2>(c->nd, c->st)) ++c->gen;
    ls::nd_copy_factors(c->nd, const_cast<unsigned char*>(static_cast<const unsigned char*>(in)) + sizeof h, false,
                        c->st);
    c->factored = true;
    c->pre_refine = c->pre_refine_mode;
    c->pre_err = -1.0;
    return LS_OK;
  } catch (const Error& e) {
    return fail(c, e);
  }
}

// Sec. 4: switches the context to the general-domain preconditioner.  Per grid point i:
// off the unknowns the identity row (alpha_i = e_0, so M and [A;B] act as I there and the
// unknowns decouple from the rest); a boundary point of the unknowns its own stencil from
// ls_general_boundary_stencils; an interior point the rectangular interior stencil and C.
ls_status ls_general_setup(ls_ctx* c, const unsigned char* mask, const double* alpha, const int* boundary) {
  try {
    check_ctx(c);
    if (!mask || !alpha || !boundary) throw Error{ls::EINVAL_, "bad arguments"};
    if (is_device_ptr(mask) || is_device_ptr(alpha) || is_device_ptr(boundary))
      throw Error{ls::EINVAL_, "mask, alpha and boundary are host arrays"};
    const long N = c->N;
    const int P3 = c->d == 2 ? 9 : 27, centre = (P3 - 1) / 2;  // offset 0; also the interior class
    if (c->alpha_h.size() != (size_t)P3 * P3) throw Error{ls::ESTATE_, "stencil tables missing"};
    std::vector<double2> a64((size_t)N * P3);
    std::vector<float2> a32((size_t)N * P3);
    std::vector<unsigned char> inter(N, 0);
    if (ls_general_rows(c->d, c->n, mask, alpha, boundary,
                        reinterpret_cast<const double*>(c->alpha_h.data() + (size_t)centre * P3),
                        reinterpret_cast<double*>(a64.data()), inter.data()) != LS_OK)
      throw Error{ls::EINVAL_, "inconsistent general-domain stencils (an interior point with a neighbour off the "
                               "unknowns, or a boundary stencil without its positive centre)"};
    for (size_t e = 0; e < a64.size(); ++e) a32[e] = make_float2((float)a64[e].x, (float)a64[e].y);
    LS_CUDA(cudaStreamSynchronize(c->st));
    if (!c->apt64) {
      c->apt64 = dalloc<double2>((size_t)N * P3);
      c->apt32 = dalloc<float2>((size_t)N * P3);
      c->inter_pt = dalloc<unsigned char>(N);
    }
    LS_CUDA(cudaMemcpy(c->apt64, a64.data(), a64.size() * sizeof(double2), cudaMemcpyHostToDevice));
    LS_CUDA(cudaMemcpy(c->apt32, a32.data(), a32.size() * sizeof(float2), cudaMemcpyHostToDevice));
    LS_CUDA(cudaMemcpy(c->inter_pt, inter.data(), N, cudaMemcpyHostToDevice));
    c->general = true;
    c->factored = false;
    ++c->gen;  // captured graphs hold the class tables
    return LS_OK;
  } catch (const Error& e) {
    return fail(c, e);
  } catch (const std::bad_alloc&) {
    return fail(c, Error{ls::ENOMEM_, "host allocation failed"});
  }
}

// Sec. 4.1: the sketch T = (K omega^2 m) R on the unknowns of a general domain.  The columns
// of R go through the FP64 operator apply in groups of up to 16 (y = x + K omega^2 m x on the
// device), and T = y - x is read off at the unknowns on the host.
ls_status ls_general_sketch(ls_ctx* c, const unsigned char* mask, int r, const double* R, double* T) {
  try {
    check_ctx(c);
    if (r < 1 || !mask || !R || !T) throw Error{ls::EINVAL_, "bad arguments"};
    if (is_device_ptr(mask) || is_device_ptr(R) || is_device_ptr(T))
      throw Error{ls::EINVAL_, "mask, R and T are host arrays"};
    const long N = c->N;
    std::vector<long> idx;
    for (long i = 0; i < N; ++i)
      if (mask[i]) idx.push_back(i);
    const long nu = (long)idx.size();
    if (nu == 0) return LS_OK;
    constexpr int GROUP = 16;
    const int g = std::min(r, GROUP);
    const size_t tot = (size_t)g * N;
    std::vector<double2> x(tot), y(tot);
    double2* xd = buf<double2>(c, "io_in", tot);
    double2* yd = buf<double2>(c, "io_out", tot);
    for (int q0 = 0; q0 < r; q0 += GROUP) {
      const int w = std::min(GROUP, r - q0);
      std::fill(x.begin(), x.end(), make_double2(0.0, 0.0));
      for (long k = 0; k < nu; ++k)
        for (int q = 0; q < w; ++q) {
          const size_t s = 2 * ((size_t)k * r + q0 + q);
          x[(size_t)q * N + idx[k]] = make_double2(R[s], R[s + 1]);
        }
      LS_CUDA(cudaMemcpyAsync(xd, x.data(), (size_t)w * N * sizeof(double2), cudaMemcpyHostToDevice, c->st));
      op_apply<double2>(c, w, xd, yd);
      LS_CUDA(cudaMemcpyAsync(y.data(), yd, (size_t)w * N * sizeof(double2), cudaMemcpyDeviceToHost, c->st));
      LS_CUDA(cudaStreamSynchronize(c->st));
      for (long k = 0; k < nu; ++k)
        for (int q = 0; q < w; ++q) {
          const size_t e = (size_t)q * N + idx[k], t = 2 * ((size_t)k * r + q0 + q);
          T[t] = y[e].x - x[e].x;
          T[t + 1] = y[e].y - x[e].y;
        }
    }
    return LS_OK;
  } catch (const Error& e) {
    return fail(c, e);
  } catch (const std::bad_alloc&) {
    return fail(c, Error{ls::ENOMEM_, "host allocation failed"});
  }
}

ls_status ls_stencil_apply(ls_ctx* c, int nrhs, const double* in, double* out, ls_prec prec) {
  try {
    check_ctx(c);
    if (nrhs < 1 || !in || !out) throw Error{ls::EINVAL_, "bad arguments"};
    const size_t tot = (size_t)nrhs * c->N;
    double2* x = buf<double2>(c, "io_in", tot);
    double2* y = buf<double2>(c, "io_out", tot);
    copy_in(c, x, in, tot * sizeof(double2));
    if (prec == LS_PREC_MIXED) {
      float2* y32 = buf<float2>(c, "io_out32", tot);
      if (c->general) {
        ls::stencil_apply_pt<double2, float2>(c->d, c->n, nrhs, x, y32, 1, c->N, c->apt32, c->st);
      } else if (c->d == 2) {
        // FP32 input, as in the solver (the 2D FP32 stencil kernel)
        float2* x32 = buf<float2>(c, "io_in32", tot);
        ls::cast<double2, float2>(x, x32, tot, c->st);
        ls::stencil_apply<float2, float2>(c->d, c->n, nrhs, x32, y32, 1, c->N, c->alpha32, c->st);
      } else {
        ls::stencil_apply<double2, float2>(c->d, c->n, nrhs, x, y32, 1, c->N, c->alpha32, c->st);
      }
      ls::cast<float2, double2>(y32, y, tot, c->st);
    } else {
      if (c->general) ls::stencil_apply_pt<double2, double2>(c->d, c->n, nrhs, x, y, 1, c->N, c->apt64, c->st);
      else ls::stencil_apply<double2, double2>(c->d, c->n, nrhs, x, y, 1, c->N, c->alpha64, c->st);
    }
    copy_out(c, out, y, tot * sizeof(double2));
    LS_CUDA(cudaStreamSynchronize(c->st));
    return LS_OK;
  } catch (const Error& e) {
    return fail(c, e);
  }
}

ls_status ls_precond(ls_ctx* c, int nrhs, const double* in, double* out) {
  ls::Range range("ls_precond");
  try {
    check_ctx(c);
    if (!c->factored) throw Error{ls::ESTATE_, "ls_precond before ls_factor"};
    factor_wait(c);
    if (nrhs < 1 || !in || !out) throw Error{ls::EINVAL_, "bad arguments"};
    const size_t tot = (size_t)nrhs * c->N;
    double2* x = buf<double2>(c, "io_in", tot);
    double2* y = buf<double2>(c, "io_out", tot);
    copy_in(c, x, in, tot * sizeof(double2));
    if (c->prec == LS_PREC_MIXED) {
      float2* z32 = buf<float2>(c, "io_out32", tot);
      if (c->pre_refine == 1 && !c->general) {
        // the refined application takes FP32 input, as in the solver
        float2* x32 = buf<float2>(c, "io_in32", tot);
        ls::cast<double2, float2>(x, x32, tot, c->st);
        precond_apply<float2, float2>(c, nrhs, x32, z32);
      } else {
        precond_apply<float2>(c, nrhs, x, z32);
      }
      ls::cast<float2, double2>(z32, y, tot, c->st);
    } else {
      precond_apply<double2>(c, nrhs, x, y);
    }
    copy_out(c, out, y, tot * sizeof(double2));
    LS_CUDA(cudaStreamSynchronize(c->st));
    return LS_OK;
  } catch (const Error& e) {
    return fail(c, e);
  }
}

ls_status ls_get_nd_stats(ls_ctx* c, ls_nd_stats* out) {
  try {
    check_ctx(c);
    if (!out) throw Error{ls::EINVAL_, "NULL out"};
    const ls::NdInfo i = ls::nd_info(c->nd);
    const int eb = c->prec == LS_PREC_MIXED ? 8 : 16;
    out->levels = i.levels;
    out->fronts = i.fronts;
    out->max_front = i.max_front;
    out->factor_entries = i.factor_entries;
    out->factor_flops = i.factor_flops;
    out->solve_bytes = i.solve_bytes * eb;
    out->fwd_factor_bytes = i.fwd_factor_entries * eb;
    out->fwd_bytes_per_rhs = i.fwd_vec_entries * eb;
    out->bwd_factor_bytes = i.bwd_factor_entries * eb;
    out->bwd_bytes_per_rhs = i.bwd_vec_entries * eb;
    return LS_OK;
  } catch (const Error& e) {
    return fail(c, e);
  }
}

}  // extern "C"

// Context accessors for ls_apply_noalloc (noalloc.cu).
namespace ls {
const ConvPlan* ctx_plan(const ls_ctx* c) { return &c->plan; }
cudaStream_t ctx_stream(const ls_ctx* c) { return c->st; }
int ctx_device(const ls_ctx* c) { return c->device; }
void ctx_set_error(ls_ctx* c, const char* msg) { c->err = msg; }
}  // namespace ls

extern "C" {

// ls_autotune: see include/ls.h.  Coordinate search: each choice in turn takes the candidate
// that beats the current best by more than 2 %, the factorization choices timed on
// ls_factor's launches (no graph, no overlap), the sweep choice on preconditioner solves of
// nrhs right-hand sides; every timing is the fastest of its repeats (CUDA events).
ls_status ls_autotune(ls_ctx* c, int nrhs, char* report, int capacity) {
  try {
    check_ctx(c);
    if (nrhs < 1) throw Error{ls::EINVAL_, "nrhs must be >= 1"};
    factor_wait(c);
    const bool mixed = c->prec == LS_PREC_MIXED;
    if (mixed ? ls::nd_prepare<float2>(c->nd, c->st) : ls::nd_prepare<double2>(c->nd, c->st)) ++c->gen;
    const void* apt = c->general ? (const void*)c->apt64 : nullptr;
    const unsigned char* inter = c->general ? c->inter_pt : nullptr;
    cudaEvent_t e0, e1;
    LS_CUDA(cudaEventCreate(&e0));
    LS_CUDA(cudaEventCreate(&e1));
    auto timed = [&](auto&& body, int reps) {
      float best = 1e30f;
      for (int r = 0; r < reps; ++r) {
        LS_CUDA(cudaEventRecord(e0, c->st));
        body();
        LS_CUDA(cudaEventRecord(e1, c->st));
        LS_CUDA(cudaEventSynchronize(e1));
        float ms = 0;
        LS_CUDA(cudaEventElapsedTime(&ms, e0, e1));
        best = std::min(best, ms);
      }
      return (double)best;
    };
    auto factor_ms = [&](const ls::NdTune& t) {
      ls::nd_set_tune(c->nd, t);
      const double ms = timed([&] {
        if (mixed) ls::nd_factor_launch<float2>(c->nd, c->alpha64, c->cint64, c->w2m64, c->st, nullptr, apt, inter);
        else ls::nd_factor_launch<double2>(c->nd, c->alpha64, c->cint64, c->w2m64, c->st, nullptr, apt, inter);
      }, 2);
      ls::nd_factor_check(c->nd, c->st);
      return ms;
    };
    const size_t tot = (size_t)nrhs * c->N;
    void* rb = mixed ? (void*)buf<float2>(c, "tune_r", tot) : (void*)buf<double2>(c, "tune_r", tot);
    void* zb = mixed ? (void*)buf<float2>(c, "tune_z", tot) : (void*)buf<double2>(c, "tune_z", tot);
    LS_CUDA(cudaMemsetAsync(rb, 0x3c, tot * (mixed ? sizeof(float2) : sizeof(double2)), c->st));
    auto solve_ms = [&](const ls::NdTune& t) {
      ls::nd_set_tune(c->nd, t);
      return timed([&] {
        if (mixed) ls::nd_solve<float2>(c->nd, nrhs, (const float2*)rb, (float2*)zb, c->st);
        else ls::nd_solve<double2>(c->nd, nrhs, (const double2*)rb, (double2*)zb, c->st);
      }, 3);
    };
    std::string log = "{\"factor_ms\": [";
    ls::NdTune best = ls::nd_get_tune(c->nd);
    double fb = factor_ms(best);
    log += "[" + tune_json(best) + ", " + std::to_string(fb) + "]";
    auto try_factor = [&](ls::NdTune t) {
      const double f = factor_ms(t);
      log += ", [" + tune_json(t) + ", " + std::to_string(f) + "]";
      if (f < 0.98 * fb) {
        best = t;
        fb = f;
      }
    };
    for (double v : {2.0e6, 3.2e7, 1e30}) {
      ls::NdTune t = best;
      t.two_level_min = v;
      try_factor(t);
    }
    if (mixed)
      for (int v : {128, 256}) {
        ls::NdTune t = best;
        t.tc_min_rows = v;
        try_factor(t);
      }
    {
      ls::NdTune t = best;
      t.gj_max_own = best.gj_max_own == 16 ? 32 : 16;
      try_factor(t);
    }
    // the factors the sweeps read: those of the chosen factorization
    factor_ms(best);
    log += "], \"solve_ms\": [";
    double sb = solve_ms(best);
    log += "[" + tune_json(best) + ", " + std::to_string(sb) + "]";
    auto try_solve = [&](ls::NdTune t) {
      const double sm = solve_ms(t);
      log += ", [" + tune_json(t) + ", " + std::to_string(sm) + "]";
      if (sm < 0.98 * sb) {
        best = t;
        sb = sm;
      }
    };
    const int sweep_base = best.sweep_ctas;
    for (int v : {1, 2, 4}) {
      if (v == sweep_base) continue;
      ls::NdTune t = best;
      t.sweep_ctas = v;
      try_solve(t);
    }
    if (mixed) {
      // forward and backward solve levels on the tensor cores: automatic (the default), from
      // 32, 64, 128 or 256 rows, or none
      for (int bwd = 0; bwd < 2; ++bwd) {
        const int base = bwd ? best.tcs_bwd_min_rows : best.tcs_min_rows;
        for (int v : {-1, 32, 64, 128, 256, 1 << 30}) {
          if (v == base) continue;
          ls::NdTune t = best;
          (bwd ? t.tcs_bwd_min_rows : t.tcs_min_rows) = v;
          try_solve(t);
        }
      }
      // the bottom levels one CTA per front: automatic (the default), up to 32, 64, 128 or
      // 256 columns, or none
      const int small_base = best.small_max_k;
      for (int v : {-1, 0, 32, 64, 128, 256}) {
        if (v == small_base) continue;
        ls::NdTune t = best;
        t.small_max_k = v;
        try_solve(t);
      }
    }
    ls::nd_set_tune(c->nd, best);
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    ++c->gen;  // the captured graphs hold the old launch sequences
    c->factored = true;
    c->factor_pending = false;
    c->pre_refine = c->pre_refine_mode;
    c->pre_err = -1.0;
    {
      std::lock_guard<std::mutex> lk(g_tune_mu);
      tune_load_locked();
      g_tune[tune_key(c)] = best;
      tune_save_locked();
    }
    char head[160];
    std::snprintf(head, sizeof head, "{\"d\": %d, \"n\": %d, \"prec\": %d, \"laplace\": %d, \"nrhs\": %d, ", c->d, c->n,
                  (int)c->prec, c->laplace ? 1 : 0, nrhs);
    write_report(std::string(head) + "\"choice\": " + tune_json(best) + ", " + log.substr(1) + "]}", report, capacity);
    return LS_OK;
  } catch (const Error& e) {
    return fail(c, e);
  }
}

ls_status ls_tune_info(const ls_ctx* c, char* report, int capacity) {
  if (!c) return LS_ESTATE;
  write_report(tune_json(ls::nd_get_tune(c->nd)), report, capacity);
  return LS_OK;
}

// the number after "key": in a flat JSON object, if the key is present
static bool json_number(const char* js, const char* key, double* v) {
  const std::string k = std::string("\"") + key + "\"";
  const char* p = std::strstr(js, k.c_str());
  if (!p) return false;
  p = std::strchr(p + k.size(), ':');
  if (!p) return false;
  char* end = nullptr;
  const double x = std::strtod(p + 1, &end);
  if (end == p + 1) return false;
  *v = x;
  return true;
}

ls_status ls_set_precond_refine(ls_ctx* c, int mode, double* err) {
  try {
    check_ctx(c);
    if (mode < -2 || mode > 1) throw Error{ls::EINVAL_, "precond refine mode " + std::to_string(mode) + " outside -2..1"};
    if (mode >= -1) {
      c->pre_refine_mode = mode;
      if (mode >= 0) c->pre_refine = mode;
      else if (c->pre_err < 0) c->pre_refine = -1;  // estimated at the next solve
      else c->pre_refine = c->pre_err > PRE_REFINE_ABOVE ? 1 : 0;
    }
    if (err) *err = c->pre_err;
    return LS_OK;
  } catch (const Error& e) {
    return fail(c, e);
  }
}

ls_status ls_set_tune(ls_ctx* c, const char* json) {
  try {
    check_ctx(c);
    if (!json) throw Error{ls::EINVAL_, "NULL tune object"};
    ls::NdTune t = ls::nd_get_tune(c->nd);
    double v;
    if (json_number(json, "two_level_min", &v)) {
      if (!(v > 0)) throw Error{ls::EINVAL_, "two_level_min must be > 0"};
      t.two_level_min = v;
    }
    auto int_key = [&](const char* key, int lo, int hi, int* dst) {
      if (!json_number(json, key, &v)) return;
      if (!(v >= lo && v <= hi) || v != std::floor(v)) throw Error{ls::EINVAL_, std::string(key) + " out of range"};
      *dst = (int)v;
    };
    int_key("tc_min_rows", 1, 1 << 30, &t.tc_min_rows);
    int_key("sweep_ctas", 1, ls::SWEEP_CTAS_MAX, &t.sweep_ctas);
    int_key("gj_max_own", 1, 32, &t.gj_max_own);
    int_key("tcs_min_rows", -1, 1 << 30, &t.tcs_min_rows);
    int_key("tcs_bwd_min_rows", -1, 1 << 30, &t.tcs_bwd_min_rows);
    int_key("small_max_k", -1, 256, &t.small_max_k);
    if (t.tcs_min_rows == 0 || t.tcs_bwd_min_rows == 0)
      throw Error{ls::EINVAL_, "tcs_min_rows / tcs_bwd_min_rows: -1 (automatic) or >= 1"};
    factor_wait(c);
    ls::nd_set_tune(c->nd, t);
    ++c->gen;  // the captured graphs hold the old launch sequences
    return LS_OK;
  } catch (const Error& e) {
    return fail(c, e);
  }
}

ls_status ls_profile_start(const char* timed_class) {
  ls::prof_start(timed_class);
  return LS_OK;
}

ls_status ls_profile_stop(char* report, int capacity) {
  ls::prof_stop(report, capacity);
  return LS_OK;
}

}  // extern "C"
