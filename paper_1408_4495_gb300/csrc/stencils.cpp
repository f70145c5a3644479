// Sparsifying stencils of Sec. 2.2 / Sec. 3.1 (eqs. Fmin, Emin, Cmin and the 3D sets
// I_n, F_n, E_n, C_n), computed on the host in FP64.
//
// For a class of grid points with translated neighbourhood mu(0) and far set J, alpha is
// the unit vector minimising |alpha K(mu(0), J)|: with K(mu, J) = U S V^*, alpha = U(:,end)^*.
// K(mu, J) has |mu| <= 27 rows and up to (2n-1)^d columns, so it is never formed whole:
//   1. X = K(mu, J)^* (tall, |J| x |mu|) is reduced to its R factor by a tall-skinny QR
//      (Householder QR of row chunks, the R factors merged pairwise), chunks spread over
//      host threads.  K = R^* Q^*, so the left singular vectors of K are the right
//      singular vectors of R.
//   2. R is diagonalised by one-sided (Hestenes) Jacobi rotations, R V = U S; alpha is the
//      conjugate of the column of V with the smallest singular value.
// Forming K K^* instead would square the condition number, and sigma_min / sigma_max is
// small by design.  Only one class per number of faces is solved (interior, face, edge,
// corner); the others are its mirror images and axis permutations, since k_t depends on
// |t| only.  The centre coefficient of alpha is made real and positive.
#include <cuda_runtime.h>

#include <algorithm>
#include <array>
#include <cmath>
#include <complex>
#include <thread>
#include <vector>

#include "common.cuh"
#include "kernels.h"
#include "ls.h"

namespace ls {

using cd = std::complex<double>;

namespace {

// In-place Householder QR of a column-major m x c matrix A (leading dimension m); on exit
// the upper triangle of the top c x c block holds R.
void householder_r(cd* A, int m, int c) {
  for (int k = 0; k < c && k < m; ++k) {
    cd* x = A + (size_t)k * m;
    double nx2 = 0;
    for (int i = k; i < m; ++i) nx2 += std::norm(x[i]);
    const double nx = std::sqrt(nx2);
    if (nx == 0) continue;
    const double ax0 = std::abs(x[k]);
    const cd ph = ax0 > 0 ? x[k] / ax0 : cd(1, 0);
    const cd alpha = -ph * nx;
    // v = x - alpha e_k (stored in x[k:m]), |v|^2 = 2 nx (nx + |x_k|)
    x[k] -= alpha;
    const double vn2 = 2.0 * nx * (nx + ax0);
    for (int j = k + 1; j < c; ++j) {
      cd* y = A + (size_t)j * m;
      cd s = 0;
      for (int i = k; i < m; ++i) s += std::conj(x[i]) * y[i];
      s *= 2.0 / vn2;
      for (int i = k; i < m; ++i) y[i] -= s * x[i];
    }
    x[k] = alpha;
    for (int i = k + 1; i < m; ++i) x[i] = 0;
  }
}

// R of [Ra; Rb] (both c x c upper triangular, row-major c x c)
void merge_r(std::vector<cd>& Ra, const std::vector<cd>& Rb, int c) {
  std::vector<cd> S((size_t)2 * c * c);  // column-major 2c x c
  for (int j = 0; j < c; ++j)
    for (int i = 0; i < c; ++i) {
      S[(size_t)j * 2 * c + i] = Ra[(size_t)i * c + j];
      S[(size_t)j * 2 * c + c + i] = Rb[(size_t)i * c + j];
    }
  householder_r(S.data(), 2 * c, c);
  for (int i = 0; i < c; ++i)
    for (int j = 0; j < c; ++j) Ra[(size_t)i * c + j] = j >= i ? S[(size_t)j * 2 * c + i] : cd(0, 0);
}

// One-sided Jacobi: returns singular values sig[c] and V (row-major c x c, column j is the
// right singular vector of sig[j]) of the square matrix R (row-major).
void jacobi_svd(const std::vector<cd>& R, int c, std::vector<double>& sig, std::vector<cd>& V) {
  std::vector<cd> X(R);  // columns orthogonalised in place
  V.assign((size_t)c * c, cd(0, 0));
  for (int i = 0; i < c; ++i) V[(size_t)i * c + i] = 1;
  for (int sweep = 0; sweep < 100; ++sweep) {
    double off = 0;
    for (int p = 0; p < c - 1; ++p)
      for (int q = p + 1; q < c; ++q) {
        double a = 0, b = 0;
        cd g = 0;
        for (int i = 0; i < c; ++i) {
          a += std::norm(X[(size_t)i * c + p]);
          b += std::norm(X[(size_t)i * c + q]);
          g += std::conj(X[(size_t)i * c + p]) * X[(size_t)i * c + q];
        }
        const double ag = std::abs(g);
        if (ag == 0 || ag <= 1e-17 * std::sqrt(a * b)) continue;
        off = std::max(off, ag / std::sqrt(a * b));
        // rotate column q by the phase of g so that the pair's inner product is real,
        // then apply the real Jacobi rotation that zeroes it
        const cd e = std::conj(g) / ag;
        const double zeta = (b - a) / (2 * ag);
        const double t = (zeta >= 0 ? 1.0 : -1.0) / (std::abs(zeta) + std::sqrt(1 + zeta * zeta));
        const double cs = 1 / std::sqrt(1 + t * t), sn = cs * t;
        for (int i = 0; i < c; ++i) {
          const cd xp = X[(size_t)i * c + p], xq = X[(size_t)i * c + q] * e;
          X[(size_t)i * c + p] = cs * xp - sn * xq;
          X[(size_t)i * c + q] = sn * xp + cs * xq;
          const cd vp = V[(size_t)i * c + p], vq = V[(size_t)i * c + q] * e;
          V[(size_t)i * c + p] = cs * vp - sn * vq;
          V[(size_t)i * c + q] = sn * vp + cs * vq;
        }
      }
    if (off < 1e-15) break;
  }
  sig.assign(c, 0);
  for (int j = 0; j < c; ++j) {
    double s = 0;
    for (int i = 0; i < c; ++i) s += std::norm(X[(size_t)i * c + j]);
    sig[j] = std::sqrt(s);
  }
}

// alpha = U(:, end)^* for K = U S V^* given as c rows of length r (row-major K[i * r + j]),
// r >= c: the tall-skinny route of solve_class on a single chunk.  Returns false when the
// smallest singular value is not simple (alpha undetermined).
bool min_left_singular(const cd* K, int c, int r, std::vector<cd>& alpha) {
  std::vector<cd> A((size_t)r * c);  // column-major r x c: K^*
  for (int col = 0; col < c; ++col)
    for (int row = 0; row < r; ++row) A[(size_t)col * r + row] = std::conj(K[(size_t)col * r + row]);
  householder_r(A.data(), r, c);
  std::vector<cd> R((size_t)c * c);
  for (int i = 0; i < c; ++i)
    for (int j = 0; j < c; ++j) R[(size_t)i * c + j] = j >= i ? A[(size_t)j * r + i] : cd(0, 0);
  std::vector<double> sig;
  std::vector<cd> V;
  jacobi_svd(R, c, sig, V);
  int jmin = 0, j2 = -1;
  for (int j = 1; j < c; ++j)
    if (sig[j] < sig[jmin]) jmin = j;
  for (int j = 0; j < c; ++j)
    if (j != jmin && (j2 < 0 || sig[j] < sig[j2])) j2 = j;
  if (j2 >= 0 && sig[jmin] > 0 && sig[j2] / sig[jmin] < 1.0 + 1e-8) return false;
  alpha.resize(c);
  for (int i = 0; i < c; ++i) alpha[i] = std::conj(V[(size_t)i * c + jmin]);
  return true;
}

struct ClassGeom {
  int d;
  std::vector<std::array<int, 3>> mu;  // offsets
  int lo[3], hi[3];                    // far-set range per axis, inclusive
  bool interior;
};

ClassGeom canonical_class(int d, int n, int b, int q) {
  ClassGeom g;
  g.d = d;
  g.interior = (q == 0);
  int mlo[3], mhi[3];
  for (int a = 0; a < 3; ++a) {
    mlo[a] = mhi[a] = 0;
    g.lo[a] = g.hi[a] = 0;
  }
  for (int a = 0; a < d; ++a) {
    if (a < q) {  // high face of axis a: mu in {-1, 0}, far set -n < j < -b
      mlo[a] = -1; mhi[a] = 0;
      g.lo[a] = -(n - 1); g.hi[a] = -b - 1;
    } else {
      mlo[a] = -1; mhi[a] = 1;
      g.lo[a] = -(n - 1); g.hi[a] = n - 1;
    }
  }
  for (int t0 = mlo[0]; t0 <= mhi[0]; ++t0)
    for (int t1 = mlo[1]; t1 <= mhi[1]; ++t1)
      for (int t2 = mlo[2]; t2 <= mhi[2]; ++t2) g.mu.push_back({t0, t1, t2});
  return g;
}

// alpha for a canonical class (offsets in g.mu order)
std::vector<cd> solve_class(const ClassGeom& g, int n, const std::vector<double2>& ktq) {
  const int d = g.d, c = (int)g.mu.size();
  const long n1 = n + 1;
  long ext[3] = {1, 1, 1};
  for (int a = 0; a < d; ++a) ext[a] = g.hi[a] - g.lo[a] + 1;
  const long M = ext[0] * ext[1] * ext[2];
  auto kval = [&](int t0, int t1, int t2) -> cd {
    long idx = std::abs(t0);
    if (d >= 2) idx = idx * n1 + std::abs(t1);
    if (d >= 3) idx = idx * n1 + std::abs(t2);
    const double2 v = ktq[idx];
    return cd(v.x, v.y);
  };
  const int nthreads = std::max(1u, std::min(64u, std::thread::hardware_concurrency()));
  const long chunk = 4096;
  const long nchunks = (M + chunk - 1) / chunk;
  std::vector<std::vector<cd>> Rt(nthreads, std::vector<cd>((size_t)c * c, cd(0, 0)));
  std::vector<char> have(nthreads, 0);
  auto work = [&](int tid) {
    std::vector<cd> A((size_t)chunk * c);
    std::vector<cd> Rc((size_t)c * c);
    for (long ch = tid; ch < nchunks; ch += nthreads) {
      const long r0 = ch * chunk, r1 = std::min(M, r0 + chunk);
      const int m = (int)(r1 - r0);
      // skip far points that coincide with mu (interior class: J = box minus mu)
      int rows = 0;
      for (long r = r0; r < r1; ++r) {
        long q = r;
        int j[3] = {0, 0, 0};
        for (int a = d - 1; a >= 0; --a) {
          j[a] = (int)(q % ext[a]) + g.lo[a];
          q /= ext[a];
        }
        if (g.interior) {
          int mx = 0;
          for (int a = 0; a < d; ++a) mx = std::max(mx, std::abs(j[a]));
          if (mx <= 1) continue;
        }
        for (int col = 0; col < c; ++col) {
          const auto& t = g.mu[col];
          A[(size_t)col * m + rows] = std::conj(kval(t[0] - j[0], t[1] - j[1], t[2] - j[2]));
        }
        ++rows;
      }
      if (rows == 0) continue;
      // compact columns to leading dimension `rows`
      if (rows < m)
        for (int col = 1; col < c; ++col)
          std::copy(A.begin() + (size_t)col * m, A.begin() + (size_t)col * m + rows, A.begin() + (size_t)col * rows);
      householder_r(A.data(), rows, c);
      for (int i = 0; i < c; ++i)
        for (int jj = 0; jj < c; ++jj)
          Rc[(size_t)i * c + jj] = (jj >= i && i < rows) ? A[(size_t)jj * rows + i] : cd(0, 0);
      if (!have[tid]) {
        Rt[tid] = Rc;
        have[tid] = 1;
      } else {
        merge_r(Rt[tid], Rc, c);
      }
    }
  };
  std::vector<std::thread> th;
  for (int t = 1; t < nthreads; ++t) th.emplace_back(work, t);
  work(0);
  for (auto& t : th) t.join();
  std::vector<cd> R;
  bool first = true;
  for (int t = 0; t < nthreads; ++t) {
    if (!have[t]) continue;
    if (first) { R = Rt[t]; first = false; }
    else merge_r(R, Rt[t], c);
  }
  if (first) LS_FAIL(EINVAL_, "empty far set (n too small for buffer b)");
  std::vector<double> sig;
  std::vector<cd> V;
  jacobi_svd(R, c, sig, V);
  int jmin = 0, j2 = -1;
  for (int j = 1; j < c; ++j)
    if (sig[j] < sig[jmin]) jmin = j;
  for (int j = 0; j < c; ++j)
    if (j != jmin && (j2 < 0 || sig[j] < sig[j2])) j2 = j;
  if (sig[jmin] > 0 && sig[j2] / sig[jmin] < 1.0 + 1e-8)
    LS_FAIL(EINVAL_, "smallest singular value of K(mu, far) is not simple; stencil undetermined");
  std::vector<cd> alpha(c);
  for (int i = 0; i < c; ++i) alpha[i] = std::conj(V[(size_t)i * c + jmin]);
  // centre coefficient real and positive
  int ci = -1;
  for (int i = 0; i < c; ++i)
    if (g.mu[i][0] == 0 && g.mu[i][1] == 0 && g.mu[i][2] == 0) ci = i;
  const cd ph = alpha[ci] / std::abs(alpha[ci]);
  for (auto& a : alpha) a /= ph;
  return alpha;
}

}  // namespace

void compute_stencils(int d, int n, int b, const std::vector<double2>& ktq, std::vector<double2>& alpha,
                      std::vector<double2>& cint) {
  int p3 = 1;
  for (int a = 0; a < d; ++a) p3 *= 3;
  alpha.assign((size_t)p3 * p3, make_double2(0, 0));
  cint.assign(p3, make_double2(0, 0));
  std::vector<std::vector<cd>> can(d + 1);
  std::vector<ClassGeom> geo;
  for (int q = 0; q <= d; ++q) {
    geo.push_back(canonical_class(d, n, b, q));
    can[q] = solve_class(geo[q], n, ktq);
  }
  // map the canonical solutions onto all 3^d classes
  for (int ci = 0; ci < p3; ++ci) {
    int cls[3] = {0, 0, 0};
    int rem = ci;
    for (int a = d - 1; a >= 0; --a) {
      cls[a] = rem % 3 - 1;
      rem /= 3;
    }
    int perm[3], q = 0;  // perm[a] = canonical axis of class axis a
    for (int a = 0; a < d; ++a)
      if (cls[a] != 0) perm[a] = q++;
    int z = q;
    for (int a = 0; a < d; ++a)
      if (cls[a] == 0) perm[a] = z++;
    const ClassGeom& g = geo[q];
    for (size_t k = 0; k < g.mu.size(); ++k) {
      // canonical offset -> class offset: t[a] = f_a * t_can[perm[a]]
      int t[3] = {0, 0, 0};
      for (int a = 0; a < d; ++a) {
        const int f = cls[a] < 0 ? -1 : 1;
        t[a] = f * g.mu[k][perm[a]];
      }
      int ti = 0;
      for (int a = 0; a < d; ++a) ti = ti * 3 + (t[a] + 1);
      alpha[(size_t)ci * p3 + ti] = make_double2(can[q][k].real(), can[q][k].imag());
    }
  }
  // C(0, t') = sum_{t in mu} alpha_t k_{t - t'} for the interior class
  const long n1 = n + 1;
  const int interior = (p3 - 1) / 2;
  for (int tp = 0; tp < p3; ++tp) {
    int tpv[3] = {0, 0, 0};
    int r = tp;
    for (int a = d - 1; a >= 0; --a) { tpv[a] = r % 3 - 1; r /= 3; }
    cd acc = 0;
    for (int t = 0; t < p3; ++t) {
      int tv[3] = {0, 0, 0};
      int rr = t;
      for (int a = d - 1; a >= 0; --a) { tv[a] = rr % 3 - 1; rr /= 3; }
      long idx = 0;
      for (int a = 0; a < d; ++a) idx = idx * n1 + std::abs(tv[a] - tpv[a]);
      const double2 av = alpha[(size_t)interior * p3 + t];
      acc += cd(av.x, av.y) * cd(ktq[idx].x, ktq[idx].y);
    }
    cint[tp] = make_double2(acc.real(), acc.imag());
  }
}

}  // namespace ls

// ---------------------------------------------------------------------------------------
// Sec. 4, general domains (host, FP64).  The unknowns are the grid points within infinity
// distance b + 1 of supp(m): the support with the buffer that the rectangular method keeps
// at the box boundary, so that a boundary point's objective only sees columns where m
// vanishes nearby, as in the far sets of Sec. 3.1.  A point is interior when all 3^d
// neighbours are unknowns; a boundary point i takes the unit alpha minimising
// |alpha T(mu(i), :)| with T = (K omega^2 m) R the sketch of the rows of K omega^2 m by r
// Gaussian columns and mu(i) its neighbours among the unknowns: alpha = U(:, end)^* of
// T(mu(i), :) = U S V^*, the coefficient at offset 0 made real and positive.
// ---------------------------------------------------------------------------------------

extern "C" ls_status ls_general_support(int dim, int n, const double* m, int b, unsigned char* mask) {
  if ((dim != 2 && dim != 3) || n < 1 || b < 0 || !m || !mask) return LS_EINVAL;
  const long N = dim == 2 ? (long)n * n : (long)n * n * n;
  std::vector<unsigned char> cur(N), nxt(N);
  for (long i = 0; i < N; ++i) cur[i] = m[i] != 0.0;
  const long stride[3] = {dim == 2 ? (long)n : (long)n * n, dim == 2 ? 1L : (long)n, 1L};
  const int w = b + 1;
  // infinity-norm dilation = a running maximum along each axis in turn
  for (int a = 0; a < dim; ++a) {
    for (long i = 0; i < N; ++i) {
      const long c = (i / stride[a]) % n;
      unsigned char v = 0;
      for (int t = -w; t <= w && !v; ++t) {
        const long cc = c + t;
        if (cc >= 0 && cc < n) v = cur[i + t * stride[a]];
      }
      nxt[i] = v;
    }
    cur.swap(nxt);
  }
  std::copy(cur.begin(), cur.end(), mask);
  return LS_OK;
}

extern "C" ls_status ls_general_boundary_stencils(int dim, int n, const unsigned char* mask, const double* T, int r,
                                                  double* alpha, int* boundary) {
  using namespace ls;
  if ((dim != 2 && dim != 3) || n < 1 || !mask || !T || !alpha || !boundary || r < 1) return LS_EINVAL;
  const long N = dim == 2 ? (long)n * n : (long)n * n * n;
  const int P3 = dim == 2 ? 9 : 27;
  if (r < P3) return LS_EINVAL;  // the sketch needs at least as many columns as a stencil has points
  std::vector<long> pos(N, -1), pts;
  for (long i = 0; i < N; ++i)
    if (mask[i]) {
      pos[i] = (long)pts.size();
      pts.push_back(i);
    }
  const long NO = (long)pts.size();
  const cd* Tc = reinterpret_cast<const cd*>(T);
  cd* Ac = reinterpret_cast<cd*>(alpha);
  std::fill(Ac, Ac + (size_t)NO * P3, cd(0, 0));
  const int nthreads = std::max(1u, std::min(64u, std::thread::hardware_concurrency()));
  std::vector<int> bad(nthreads, 0);
  auto work = [&](int tid) {
    std::vector<cd> K;
    std::vector<cd> al;
    for (long k = tid; k < NO; k += nthreads) {
      const long i = pts[k];
      int c[3] = {0, 0, 0};
      long q = i;
      for (int a = dim - 1; a >= 0; --a) {
        c[a] = (int)(q % n);
        q /= n;
      }
      std::vector<int> toff;
      std::vector<long> rows;
      for (int t = 0; t < P3; ++t) {
        int tt = t;
        long j = 0;
        bool in = true;
        int y[3] = {0, 0, 0};
        for (int a = dim - 1; a >= 0; --a) {
          y[a] = c[a] + (tt % 3) - 1;
          tt /= 3;
          if (y[a] < 0 || y[a] >= n) in = false;
        }
        if (!in) continue;
        for (int a = 0; a < dim; ++a) j = j * n + y[a];
        if (pos[j] < 0) continue;
        toff.push_back(t);
        rows.push_back(pos[j]);
      }
      const int cnt = (int)toff.size();
      boundary[k] = cnt < P3 ? 1 : 0;
      if (cnt == P3) continue;
      K.resize((size_t)cnt * r);
      for (int u = 0; u < cnt; ++u)
        for (int j = 0; j < r; ++j) K[(size_t)u * r + j] = Tc[(size_t)rows[u] * r + j];
      if (!min_left_singular(K.data(), cnt, r, al)) {
        bad[tid] = 1;
        continue;
      }
      int ci = -1;
      for (int u = 0; u < cnt; ++u)
        if (toff[u] == (P3 - 1) / 2) ci = u;
      const cd ph = std::abs(al[ci]) > 0 ? al[ci] / std::abs(al[ci]) : cd(1, 0);
      for (int u = 0; u < cnt; ++u) Ac[(size_t)k * P3 + toff[u]] = al[u] / ph;
    }
  };
  std::vector<std::thread> th;
  for (int t = 1; t < nthreads; ++t) th.emplace_back(work, t);
  work(0);
  for (auto& t : th) t.join();
  for (int b : bad)
    if (b) return LS_EINVAL;
  return LS_OK;
}

// Sec. 4: the rows of M and [A;B] per grid point for the general-domain solve in the box
// (identity off the unknowns, alpha_i on their boundary, the interior stencil inside), with
// the checks that an interior point has all 3^d neighbours among the unknowns and that a
// boundary stencil has its positive centre.
extern "C" ls_status ls_general_rows(int dim, int n, const unsigned char* mask, const double* alpha,
                                     const int* boundary, const double* alpha_interior, double* rows,
                                     unsigned char* interior) {
  if ((dim != 2 && dim != 3) || n < 1 || !mask || !alpha || !boundary || !alpha_interior || !rows || !interior)
    return LS_EINVAL;
  const long N = dim == 2 ? (long)n * n : (long)n * n * n;
  const int P3 = dim == 2 ? 9 : 27, centre = (P3 - 1) / 2;
  long k = 0;
  for (long i = 0; i < N; ++i) {
    double* row = rows + 2 * (size_t)i * P3;
    std::fill(row, row + 2 * P3, 0.0);
    interior[i] = 0;
    if (!mask[i]) {
      row[2 * centre] = 1.0;
      continue;
    }
    const double* src = boundary[k] ? alpha + 2 * (size_t)k * P3 : alpha_interior;
    std::copy(src, src + 2 * P3, row);
    if (boundary[k]) {
      if (!(row[2 * centre] > 0.0)) return LS_EINVAL;
    } else {
      interior[i] = 1;
      long q = i;
      int c[3] = {0, 0, 0};
      for (int a = dim - 1; a >= 0; --a) {
        c[a] = (int)(q % n);
        q /= n;
      }
      for (int t = 0; t < P3; ++t) {
        int tt = t, tv[3] = {0, 0, 0};
        for (int a = dim - 1; a >= 0; --a) {
          tv[a] = tt % 3 - 1;
          tt /= 3;
        }
        long j = 0;
        for (int a = 0; a < dim; ++a) {
          const int ca = c[a] + tv[a];
          if (ca < 0 || ca >= n) return LS_EINVAL;
          j = j * n + ca;
        }
        if (!mask[j]) return LS_EINVAL;
      }
    }
    ++k;
  }
  return LS_OK;
}
