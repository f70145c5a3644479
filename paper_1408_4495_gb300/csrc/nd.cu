// Nested-dissection multifrontal LU of M = [A + C omega^2 m ; B] and its multi-right-hand-
// side solves (Sec. 2.2 after eq. PC: nested dissection + multifrontal method; Sec. 3.2:
// O(N^{3/2}) / O(N^2) factorization, O(N log N) / O(N^{4/3}) solve).
//
// Symbolic (host, once per (d, n)): the grid box is split recursively along its longest
// side by a one-point-thick separator slab (the 3^d stencil couples only points at
// infinity-distance <= 1, so the slab disconnects the halves).  A tree node owns its
// separator (a leaf owns its whole box); its front is [own variables ; ring], the ring
// being the grid points adjacent to the node's box (all of them belong to ancestors).
// Nodes at equal depth form one level and are factored by one batch of launches; each
// level stores its fronts densely as nf x fmax x fmax (column major), fmax = smax + bmax,
// with smaller fronts padded (identity on padded own positions, zero ring positions).
//
// Numeric (device, per medium), level by level from the leaves:
//   assemble original entries -> extend-add children's Schur complements -> blocked
//   right-looking partial LU of the own columns, pivot rows restricted to the own rows:
//   panel (pivot, swap whole rows, scale, rank-1) / TRSM of the block row / GEMM update of
//   the trailing block (which ends as the Schur complement F22 - L21 U12 for the parent).
// Solve: forward y = L^{-1} P b from the leaves (children's update vectors extend-added
// into the parent's front vector), backward x = U^{-1}(y - U12 x_ring) from the root.
#include <algorithm>
#include <cstring>
#include <vector>

#include "common.cuh"
#include "kernels.h"
#include "prof.h"

namespace ls {

namespace {

struct Node {
  int lo[3], hi[3];
  int depth = 0, parent = -1, nchild = 0, slot = -1, kidx = -1;
  int child[2] = {-1, -1};
  std::vector<int> own, ring;
};

struct LevelDev {
  int nf = 0, smax = 0, bmax = 0, fmax = 0;
  size_t F_off = 0, W_off = 0;
  int *own = nullptr, *ring = nullptr, *child = nullptr, *parent = nullptr, *kidx = nullptr, *ea = nullptr;
  int *piv = nullptr, *perm = nullptr, *iperm = nullptr;
};

template <typename C> struct LevelK {
  C* F;
  C* W;
  int nf, smax, bmax, fmax;
  const int *own, *ring, *child, *parent, *kidx, *ea;
  int *piv, *perm, *iperm;
};

constexpr int NB = 32;          // panel width
constexpr int SOLVE_CHUNK = 64; // right-hand sides per solve launch

}  // namespace

struct NdPlan {
  int d = 0, n = 0;
  long N = 0;
  std::vector<Node> nodes;
  std::vector<std::vector<int>> lev_nodes;
  std::vector<LevelDev> lev;
  long n_asm = 0, n_pad = 0;
  int64_t* d_asm_off = nullptr;
  int* d_asm_row = nullptr;
  unsigned char* d_asm_t = nullptr;
  int64_t* d_pad_off = nullptr;
  size_t F_elems = 0, W_elems = 0;
  void* F = nullptr;
  int F_bytes = 0;
  void* W = nullptr;
  int W_bytes = 0;
  int* d_err = nullptr;
  std::vector<void*> allocs;
  NdInfo info{};
};

namespace {

template <typename T> T* upload(NdPlan* p, const std::vector<T>& v, cudaStream_t st) {
  T* d = nullptr;
  const size_t bytes = std::max<size_t>(1, v.size()) * sizeof(T);
  if (cudaMalloc(&d, bytes) != cudaSuccess) LS_FAIL(ENOMEM_, "cudaMalloc(%zu) failed for the ND plan", bytes);
  p->allocs.push_back(d);
  if (!v.empty()) LS_CUDA(cudaMemcpyAsync(d, v.data(), v.size() * sizeof(T), cudaMemcpyHostToDevice, st));
  return d;
}

void build_tree(NdPlan* p, int leaf_max) {
  const int d = p->d, n = p->n;
  struct Item { int lo[3], hi[3], depth, parent, kidx; };
  std::vector<Item> stack;
  Item root{};
  for (int a = 0; a < 3; ++a) { root.lo[a] = 0; root.hi[a] = a < d ? n : 1; }
  root.depth = 0; root.parent = -1; root.kidx = -1;
  stack.push_back(root);
  auto flat = [&](int i0, int i1, int i2) -> int {
    return d == 2 ? i0 * n + i1 : (i0 * n + i1) * n + i2;
  };
  while (!stack.empty()) {
    Item it = stack.back();
    stack.pop_back();
    const int id = (int)p->nodes.size();
    p->nodes.emplace_back();
    Node& nd = p->nodes.back();
    for (int a = 0; a < 3; ++a) { nd.lo[a] = it.lo[a]; nd.hi[a] = it.hi[a]; }
    nd.depth = it.depth;
    nd.parent = it.parent;
    nd.kidx = it.kidx;
    if (it.parent >= 0) {
      Node& par = p->nodes[it.parent];
      par.child[it.kidx] = id;
      par.nchild = std::max(par.nchild, it.kidx + 1);
    }
    int size[3], vol = 1, ax = 0;
    for (int a = 0; a < 3; ++a) { size[a] = it.hi[a] - it.lo[a]; vol *= size[a]; }
    for (int a = 1; a < d; ++a)
      if (size[a] > size[ax]) ax = a;
    const bool leaf = vol <= leaf_max || size[ax] < 3;
    int mid = -1;
    if (!leaf) mid = it.lo[ax] + size[ax] / 2;
    for (int i0 = it.lo[0]; i0 < it.hi[0]; ++i0)
      for (int i1 = it.lo[1]; i1 < it.hi[1]; ++i1)
        for (int i2 = it.lo[2]; i2 < it.hi[2]; ++i2) {
          const int c[3] = {i0, i1, i2};
          if (leaf || c[ax] == mid) nd.own.push_back(flat(i0, i1, i2));
        }
    // ring: points within infinity-distance 1 of the box, inside the grid, outside the box
    int elo[3], ehi[3];
    for (int a = 0; a < 3; ++a) {
      if (a < d) { elo[a] = std::max(0, it.lo[a] - 1); ehi[a] = std::min(n, it.hi[a] + 1); }
      else { elo[a] = 0; ehi[a] = 1; }
    }
    for (int i0 = elo[0]; i0 < ehi[0]; ++i0)
      for (int i1 = elo[1]; i1 < ehi[1]; ++i1)
        for (int i2 = elo[2]; i2 < ehi[2]; ++i2) {
          const int c[3] = {i0, i1, i2};
          bool inside = true;
          for (int a = 0; a < d; ++a)
            if (c[a] < it.lo[a] || c[a] >= it.hi[a]) inside = false;
          if (!inside) nd.ring.push_back(flat(i0, i1, i2));
        }
    if (!leaf) {
      // push the second child first so that the first child gets the lower node id
      Item c1 = it, c2 = it;
      c1.hi[ax] = mid;
      c2.lo[ax] = mid + 1;
      c1.depth = c2.depth = it.depth + 1;
      c1.parent = c2.parent = id;
      int k = 0;
      const bool has1 = c1.hi[ax] > c1.lo[ax], has2 = c2.hi[ax] > c2.lo[ax];
      if (has1) c1.kidx = k++;
      if (has2) c2.kidx = k++;
      if (has2) stack.push_back(c2);
      if (has1) stack.push_back(c1);
    }
  }
}

}  // namespace

NdPlan* nd_build(int d, int n, cudaStream_t st) {
  NdPlan* p = new NdPlan;
  try {
    p->d = d;
    p->n = n;
    p->N = d == 2 ? (long)n * n : (long)n * n * n;
    build_tree(p, 64);
    int depth = 0;
    for (auto& nd : p->nodes) depth = std::max(depth, nd.depth + 1);
    p->lev_nodes.assign(depth, {});
    p->lev.assign(depth, LevelDev{});
    for (int id = 0; id < (int)p->nodes.size(); ++id) {
      Node& nd = p->nodes[id];
      nd.slot = (int)p->lev_nodes[nd.depth].size();
      p->lev_nodes[nd.depth].push_back(id);
    }
    size_t F_off = 0, W_off = 0;
    double flops = 0, solve_entries = 0;
    int max_front = 0;
    for (int l = 0; l < depth; ++l) {
      LevelDev& L = p->lev[l];
      L.nf = (int)p->lev_nodes[l].size();
      for (int id : p->lev_nodes[l]) {
        L.smax = std::max(L.smax, (int)p->nodes[id].own.size());
        L.bmax = std::max(L.bmax, (int)p->nodes[id].ring.size());
      }
      L.fmax = L.smax + L.bmax;
      L.F_off = F_off;
      L.W_off = W_off;
      F_off += (size_t)L.nf * L.fmax * L.fmax;
      W_off += (size_t)L.nf * SOLVE_CHUNK * L.fmax;
      max_front = std::max(max_front, L.fmax);
      const double f = L.fmax, s = L.smax;
      flops += L.nf * 8.0 * (f * f * f - (f - s) * (f - s) * (f - s)) / 3.0;
      solve_entries += (double)L.nf * (s * s + 2.0 * s * L.bmax);
    }
    p->F_elems = F_off;
    p->W_elems = W_off;
    p->info.levels = depth;
    p->info.fronts = (int)p->nodes.size();
    p->info.max_front = max_front;
    p->info.factor_entries = (int64_t)F_off;
    p->info.factor_flops = flops;
    p->info.solve_bytes = solve_entries;  // scaled by element size by the caller

    // per-level index arrays, assembly list, extend-add maps
    std::vector<int> pos(p->N, -1);
    std::vector<int64_t> asm_off, pad_off;
    std::vector<int> asm_row;
    std::vector<unsigned char> asm_t;
    const int n_ = n;
    auto coords = [&](int g, int* c) {
      if (d == 2) { c[0] = g / n_; c[1] = g % n_; c[2] = 0; }
      else { c[2] = g % n_; c[1] = (g / n_) % n_; c[0] = g / (n_ * n_); }
    };
    auto flat = [&](const int* c) -> int { return d == 2 ? c[0] * n_ + c[1] : (c[0] * n_ + c[1]) * n_ + c[2]; };
    std::vector<std::vector<int>> l_own(depth), l_ring(depth), l_child(depth), l_parent(depth), l_kidx(depth), l_ea(depth);
    for (int l = 0; l < depth; ++l) {
      const LevelDev& L = p->lev[l];
      l_own[l].assign((size_t)L.nf * L.smax, -1);
      l_ring[l].assign((size_t)L.nf * L.bmax, -1);
      l_child[l].assign((size_t)L.nf * 2, -1);
      l_parent[l].assign(L.nf, -1);
      l_kidx[l].assign(L.nf, -1);
      l_ea[l].assign((size_t)L.nf * L.bmax, -1);
    }
    const int t_lo2 = d == 3 ? -1 : 0, t_hi2 = d == 3 ? 1 : 0;
    for (int id = 0; id < (int)p->nodes.size(); ++id) {
      const Node& nd = p->nodes[id];
      const int l = nd.depth;
      const LevelDev& L = p->lev[l];
      const int z = nd.slot;
      const int s = (int)nd.own.size(), b = (int)nd.ring.size();
      for (int q = 0; q < s; ++q) l_own[l][(size_t)z * L.smax + q] = nd.own[q];
      for (int q = 0; q < b; ++q) l_ring[l][(size_t)z * L.bmax + q] = nd.ring[q];
      for (int k = 0; k < 2; ++k)
        if (nd.child[k] >= 0) l_child[l][(size_t)z * 2 + k] = p->nodes[nd.child[k]].slot;
      if (nd.parent >= 0) {
        l_parent[l][z] = p->nodes[nd.parent].slot;
        l_kidx[l][z] = nd.kidx;
      }
      for (int q = 0; q < s; ++q) pos[nd.own[q]] = q;
      for (int q = 0; q < b; ++q) pos[nd.ring[q]] = L.smax + q;
      const size_t base = L.F_off + (size_t)z * L.fmax * L.fmax;
      // rows of own variables: every stencil neighbour present in the front
      for (int q = 0; q < s; ++q) {
        int c[3];
        coords(nd.own[q], c);
        for (int t0 = -1; t0 <= 1; ++t0)
          for (int t1 = -1; t1 <= 1; ++t1)
            for (int t2 = t_lo2; t2 <= t_hi2; ++t2) {
              const int cc[3] = {c[0] + t0, c[1] + t1, c[2] + t2};
              bool in = true;
              for (int a = 0; a < d; ++a)
                if (cc[a] < 0 || cc[a] >= n_) in = false;
              if (!in) continue;
              const int j = flat(cc);
              if (pos[j] < 0) continue;
              asm_off.push_back((int64_t)(base + (size_t)pos[j] * L.fmax + q));
              asm_row.push_back(nd.own[q]);
              asm_t.push_back((unsigned char)(d == 2 ? (t0 + 1) * 3 + (t1 + 1) : ((t0 + 1) * 3 + (t1 + 1)) * 3 + (t2 + 1)));
            }
      }
      // rows of ring variables: columns of own variables only
      for (int q = 0; q < b; ++q) {
        int c[3];
        coords(nd.ring[q], c);
        for (int t0 = -1; t0 <= 1; ++t0)
          for (int t1 = -1; t1 <= 1; ++t1)
            for (int t2 = t_lo2; t2 <= t_hi2; ++t2) {
              const int cc[3] = {c[0] + t0, c[1] + t1, c[2] + t2};
              bool in = true;
              for (int a = 0; a < d; ++a)
                if (cc[a] < 0 || cc[a] >= n_) in = false;
              if (!in) continue;
              const int j = flat(cc);
              if (pos[j] < 0 || pos[j] >= L.smax) continue;
              asm_off.push_back((int64_t)(base + (size_t)pos[j] * L.fmax + L.smax + q));
              asm_row.push_back(nd.ring[q]);
              asm_t.push_back((unsigned char)(d == 2 ? (t0 + 1) * 3 + (t1 + 1) : ((t0 + 1) * 3 + (t1 + 1)) * 3 + (t2 + 1)));
            }
      }
      for (int q = s; q < L.smax; ++q) pad_off.push_back((int64_t)(base + (size_t)q * L.fmax + q));
      // extend-add maps of the children: child ring variable -> position in this front
      for (int k = 0; k < 2; ++k) {
        const int cid = nd.child[k];
        if (cid < 0) continue;
        const Node& ch = p->nodes[cid];
        const LevelDev& Lc = p->lev[l + 1];
        for (int a = 0; a < (int)ch.ring.size(); ++a) {
          const int ps = pos[ch.ring[a]];
          if (ps < 0) LS_FAIL(EINVAL_, "nested dissection: child ring variable missing from parent front");
          l_ea[l + 1][(size_t)ch.slot * Lc.bmax + a] = ps;
        }
      }
      for (int q = 0; q < s; ++q) pos[nd.own[q]] = -1;
      for (int q = 0; q < b; ++q) pos[nd.ring[q]] = -1;
    }
    for (int l = 0; l < depth; ++l) {
      LevelDev& L = p->lev[l];
      L.own = upload(p, l_own[l], st);
      L.ring = upload(p, l_ring[l], st);
      L.child = upload(p, l_child[l], st);
      L.parent = upload(p, l_parent[l], st);
      L.kidx = upload(p, l_kidx[l], st);
      L.ea = upload(p, l_ea[l], st);
      std::vector<int> zeros((size_t)L.nf * L.smax, 0);
      L.piv = upload(p, zeros, st);
      L.perm = upload(p, zeros, st);
      L.iperm = upload(p, zeros, st);
    }
    p->n_asm = (long)asm_off.size();
    p->n_pad = (long)pad_off.size();
    p->d_asm_off = upload(p, asm_off, st);
    p->d_asm_row = upload(p, asm_row, st);
    p->d_asm_t = upload(p, asm_t, st);
    p->d_pad_off = upload(p, pad_off, st);
    std::vector<int> zero1(1, 0);
    p->d_err = upload(p, zero1, st);
    LS_CUDA(cudaStreamSynchronize(st));
  } catch (...) {
    nd_free(p);
    throw;
  }
  return p;
}

void nd_free(NdPlan* p) {
  if (!p) return;
  for (void* a : p->allocs) cudaFree(a);
  if (p->F) cudaFree(p->F);
  if (p->W) cudaFree(p->W);
  delete p;
}

NdInfo nd_info(const NdPlan* p) { return p->info; }

size_t nd_device_bytes(const NdPlan* p, int elem_bytes) {
  return (p->F_elems + p->W_elems) * (size_t)elem_bytes;
}

// ---------------------------------------------------------------------------------------
// numeric factorization kernels
// ---------------------------------------------------------------------------------------

template <typename C>
__global__ void k_assemble(C* F, long n_asm, const int64_t* __restrict__ off, const int* __restrict__ row,
                           const unsigned char* __restrict__ tcode, int d, int n, const double2* __restrict__ alpha,
                           const double2* __restrict__ cint, const double* __restrict__ w2m) {
  const int P3 = d == 2 ? 9 : 27;
  for (long e = blockIdx.x * (long)blockDim.x + threadIdx.x; e < n_asm; e += (long)gridDim.x * blockDim.x) {
    const int i = row[e];
    const int t = tcode[e];
    int c[3] = {0, 0, 0}, tv[3] = {0, 0, 0};
    int q = i, tt = t;
    for (int a = d - 1; a >= 0; --a) {
      c[a] = q % n;
      q /= n;
      tv[a] = tt % 3 - 1;
      tt /= 3;
    }
    int cls = 0;
    bool interior = true;
    for (int a = 0; a < d; ++a) {
      const int ca = c[a] == 0 ? 0 : (c[a] == n - 1 ? 2 : 1);
      if (ca != 1) interior = false;
      cls = cls * 3 + ca;
    }
    double2 v = alpha[cls * P3 + t];
    if (interior) {
      long j = 0;
      for (int a = 0; a < d; ++a) j = j * n + (c[a] + tv[a]);
      const double w = w2m[j];
      v.x += cint[t].x * w;
      v.y += cint[t].y * w;
    }
    F[off[e]] = ccast<C>(v);
  }
}

template <typename C> __global__ void k_set_pad(C* F, long n_pad, const int64_t* __restrict__ off) {
  for (long e = blockIdx.x * (long)blockDim.x + threadIdx.x; e < n_pad; e += (long)gridDim.x * blockDim.x) {
    C one;
    one.x = 1;
    one.y = 0;
    F[off[e]] = one;
  }
}

// Schur complements of the children with child index k into their parents' fronts.
template <typename C> __global__ void k_extend_add(LevelK<C> P, LevelK<C> Ch, int k) {
  const int c = blockIdx.y;
  if (Ch.kidx[c] != k) return;
  const int pz = Ch.parent[c];
  C* Fp = P.F + (size_t)pz * P.fmax * P.fmax;
  const C* Fc = Ch.F + (size_t)c * Ch.fmax * Ch.fmax;
  const int* ea = Ch.ea + (size_t)c * Ch.bmax;
  const long tot = (long)Ch.bmax * Ch.bmax;
  for (long idx = blockIdx.x * (long)blockDim.x + threadIdx.x; idx < tot; idx += (long)gridDim.x * blockDim.x) {
    const int a = (int)(idx % Ch.bmax), b = (int)(idx / Ch.bmax);
    const int pa = ea[a], pb = ea[b];
    if (pa < 0 || pb < 0) continue;
    const C v = Fc[(size_t)(Ch.smax + b) * Ch.fmax + Ch.smax + a];
    C& dst = Fp[(size_t)pb * P.fmax + pa];
    dst = cadd(dst, v);
  }
}

// Panel [k0, k1): pivot search over the own rows, whole-row swaps, scaling, rank-1 updates.
template <typename C> __global__ void __launch_bounds__(256) k_panel(LevelK<C> L, int k0, int k1, int* err) {
  using Rl = typename RealOf<C>::T;
  const int z = blockIdx.x, tid = threadIdx.x, NT = blockDim.x;
  const int fmax = L.fmax, smax = L.smax;
  C* A = L.F + (size_t)z * fmax * fmax;
  __shared__ Rl rv[256];
  __shared__ int ri[256];
  for (int j = k0; j < k1; ++j) {
    Rl best = -1;
    int bi = j;
    for (int r = j + tid; r < smax; r += NT) {
      const Rl v = cabs2(A[(size_t)j * fmax + r]);
      if (v > best) { best = v; bi = r; }
    }
    rv[tid] = best;
    ri[tid] = bi;
    __syncthreads();
    for (int s = NT / 2; s > 0; s >>= 1) {
      if (tid < s) {
        const Rl o = rv[tid + s];
        const int oi = ri[tid + s];
        if (o > rv[tid] || (o == rv[tid] && oi < ri[tid])) { rv[tid] = o; ri[tid] = oi; }
      }
      __syncthreads();
    }
    const int pr = ri[0];
    const Rl pv = rv[0];
    __syncthreads();
    if (tid == 0) {
      L.piv[(size_t)z * smax + j] = pr;
      if (!(pv > 0)) atomicExch(err, 1);
    }
    if (pr != j)
      for (int col = tid; col < fmax; col += NT) {
        C& x = A[(size_t)col * fmax + j];
        C& y = A[(size_t)col * fmax + pr];
        const C t = x;
        x = y;
        y = t;
      }
    __syncthreads();
    const C dg = A[(size_t)j * fmax + j];
    const Rl den = cabs2(dg);
    C inv;
    inv.x = den > 0 ? dg.x / den : (Rl)0;
    inv.y = den > 0 ? -dg.y / den : (Rl)0;
    for (int r = j + 1 + tid; r < fmax; r += NT) {
      C& x = A[(size_t)j * fmax + r];
      x = cmul(x, inv);
    }
    __syncthreads();
    const int ncol = k1 - j - 1, nrow = fmax - j - 1;
    for (int idx = tid; idx < ncol * nrow; idx += NT) {
      const int col = j + 1 + idx / nrow, r = j + 1 + idx % nrow;
      C& x = A[(size_t)col * fmax + r];
      x = cfms(x, A[(size_t)j * fmax + r], A[(size_t)col * fmax + j]);
    }
    __syncthreads();
  }
}

// Block row: F[k0:k1, c] = L_kk^{-1} F[k0:k1, c] for c >= k1 (unit lower L_kk).
template <typename C> __global__ void __launch_bounds__(128) k_trsm_row(LevelK<C> L, int k0, int k1) {
  const int z = blockIdx.y;
  const int fmax = L.fmax, w = k1 - k0;
  C* A = L.F + (size_t)z * fmax * fmax;
  __shared__ C Ld[NB][NB + 1];
  for (int idx = threadIdx.x; idx < w * w; idx += blockDim.x) {
    const int i = idx % w, l = idx / w;
    Ld[i][l] = A[(size_t)(k0 + l) * fmax + k0 + i];
  }
  __syncthreads();
  const int c = k1 + blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= fmax) return;
  C x[NB];
  C* col = A + (size_t)c * fmax + k0;
#pragma unroll
  for (int i = 0; i < NB; ++i)
    if (i < w) x[i] = col[i];
#pragma unroll
  for (int i = 1; i < NB; ++i) {
    if (i < w) {
      C acc = x[i];
#pragma unroll
      for (int l = 0; l < NB; ++l)
        if (l < i) acc = cfms(acc, Ld[i][l], x[l]);
      x[i] = acc;
    }
  }
#pragma unroll
  for (int i = 0; i < NB; ++i)
    if (i < w) col[i] = x[i];
}

// Trailing update F[k1:, k1:] -= F[k1:, k0:k1] F[k0:k1, k1:], 64 x 64 tiles, K chunks of 16.
template <typename C> __global__ void __launch_bounds__(256) k_gemm_update(LevelK<C> L, int k0, int k1) {
  constexpr int TM = 64, TK = 16;
  const int z = blockIdx.y;
  const int fmax = L.fmax, w = k1 - k0;
  const int m = fmax - k1;
  const int nt = (m + TM - 1) / TM;
  const int tr = blockIdx.x % nt, tcb = blockIdx.x / nt;
  const int r0 = k1 + tr * TM, c0 = k1 + tcb * TM;
  C* A = L.F + (size_t)z * fmax * fmax;
  __shared__ C As[TK][TM + 1];
  __shared__ C Bs[TK][TM + 1];
  const int tx = threadIdx.x % 16, ty = threadIdx.x / 16;
  C acc[4][4];
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) acc[i][j] = czero<C>();
  for (int kk = 0; kk < w; kk += TK) {
    const int kw = min(TK, w - kk);
    for (int idx = threadIdx.x; idx < TK * TM; idx += blockDim.x) {
      const int l = idx / TM, rr = idx % TM;
      C va = czero<C>(), vb = czero<C>();
      if (l < kw) {
        if (r0 + rr < fmax) va = A[(size_t)(k0 + kk + l) * fmax + r0 + rr];
      }
      As[l][rr] = va;
      const int l2 = idx % TK, cc = idx / TK;
      if (l2 < kw && c0 + cc < fmax) vb = A[(size_t)(c0 + cc) * fmax + k0 + kk + l2];
      Bs[l2][cc] = vb;
    }
    __syncthreads();
    for (int l = 0; l < kw; ++l) {
      C a[4], b[4];
#pragma unroll
      for (int i = 0; i < 4; ++i) a[i] = As[l][tx + 16 * i];
#pragma unroll
      for (int j = 0; j < 4; ++j) b[j] = Bs[l][ty + 16 * j];
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[i][j] = cfma(acc[i][j], a[i], b[j]);
    }
    __syncthreads();
  }
#pragma unroll
  for (int j = 0; j < 4; ++j) {
    const int c = c0 + ty + 16 * j;
    if (c >= fmax) continue;
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      const int r = r0 + tx + 16 * i;
      if (r >= fmax) continue;
      C& x = A[(size_t)c * fmax + r];
      x = csub(x, acc[i][j]);
    }
  }
}

__global__ void k_perm(const int* piv, int* perm, int* iperm, int nf, int smax) {
  const int z = blockIdx.x * blockDim.x + threadIdx.x;
  if (z >= nf) return;
  int* pm = perm + (size_t)z * smax;
  const int* pv = piv + (size_t)z * smax;
  for (int q = 0; q < smax; ++q) pm[q] = q;
  for (int j = 0; j < smax; ++j) {
    const int q = pv[j];
    const int t = pm[j];
    pm[j] = pm[q];
    pm[q] = t;
  }
  for (int q = 0; q < smax; ++q) iperm[(size_t)z * smax + pm[q]] = q;
}

template <typename C> LevelK<C> level_k(NdPlan* p, int l) {
  const LevelDev& D = p->lev[l];
  LevelK<C> k;
  k.F = reinterpret_cast<C*>(p->F) + D.F_off;
  k.W = reinterpret_cast<C*>(p->W) + D.W_off;
  k.nf = D.nf; k.smax = D.smax; k.bmax = D.bmax; k.fmax = D.fmax;
  k.own = D.own; k.ring = D.ring; k.child = D.child; k.parent = D.parent; k.kidx = D.kidx; k.ea = D.ea;
  k.piv = D.piv; k.perm = D.perm; k.iperm = D.iperm;
  return k;
}

static void ensure_buffers(NdPlan* p, int elem_bytes) {
  if (p->F && p->F_bytes == elem_bytes) return;
  if (p->F) { cudaFree(p->F); p->F = nullptr; }
  if (p->W) { cudaFree(p->W); p->W = nullptr; }
  if (cudaMalloc(&p->F, p->F_elems * elem_bytes) != cudaSuccess)
    LS_FAIL(ENOMEM_, "cudaMalloc of %zu bytes for the fronts failed", p->F_elems * elem_bytes);
  if (cudaMalloc(&p->W, std::max<size_t>(1, p->W_elems) * elem_bytes) != cudaSuccess)
    LS_FAIL(ENOMEM_, "cudaMalloc of %zu bytes for the front vectors failed", p->W_elems * elem_bytes);
  p->F_bytes = p->W_bytes = elem_bytes;
}

template <typename C>
void nd_factor(NdPlan* p, const void* alpha64, const void* cint64, const void* w2m64, cudaStream_t st) {
  ensure_buffers(p, sizeof(C));
  LS_CUDA(cudaMemsetAsync(p->F, 0, p->F_elems * sizeof(C), st));
  LS_CUDA(cudaMemsetAsync(p->d_err, 0, sizeof(int), st));
  const bool f32 = sizeof(C) == 8;
  LS_LAUNCH(f32 ? "nd_assemble_c64" : "nd_assemble_c128", st,
            k_assemble<C><<<1024, 256, 0, st>>>(reinterpret_cast<C*>(p->F), p->n_asm, p->d_asm_off, p->d_asm_row,
                                                p->d_asm_t, p->d, p->n, (const double2*)alpha64,
                                                (const double2*)cint64, (const double*)w2m64));
  if (p->n_pad > 0)
    LS_LAUNCH(f32 ? "nd_pad_c64" : "nd_pad_c128", st,
              k_set_pad<C><<<256, 256, 0, st>>>(reinterpret_cast<C*>(p->F), p->n_pad, p->d_pad_off));
  const int depth = (int)p->lev.size();
  for (int l = depth - 1; l >= 0; --l) {
    LevelK<C> L = level_k<C>(p, l);
    if (l + 1 < depth) {
      LevelK<C> Ch = level_k<C>(p, l + 1);
      const long tot = (long)Ch.bmax * Ch.bmax;
      const unsigned bx = (unsigned)std::min<long>((tot + 255) / 256, 64);
      for (int k = 0; k < 2; ++k) {
        LS_LAUNCH(f32 ? "nd_extend_add_c64" : "nd_extend_add_c128", st,
                  k_extend_add<C><<<dim3(bx, Ch.nf), 256, 0, st>>>(L, Ch, k));
      }
    }
    for (int k0 = 0; k0 < L.smax; k0 += NB) {
      const int k1 = std::min(k0 + NB, L.smax);
      LS_LAUNCH(f32 ? "nd_panel_c64" : "nd_panel_c128", st, k_panel<C><<<L.nf, 256, 0, st>>>(L, k0, k1, p->d_err));
      const int m = L.fmax - k1;
      if (m > 0) {
        LS_LAUNCH(f32 ? "nd_trsm_c64" : "nd_trsm_c128", st,
                  k_trsm_row<C><<<dim3((m + 127) / 128, L.nf), 128, 0, st>>>(L, k0, k1));
        const int nt = (m + 63) / 64;
        LS_LAUNCH(f32 ? "nd_gemm_c64" : "nd_gemm_c128", st,
                  k_gemm_update<C><<<dim3(nt * nt, L.nf), 256, 0, st>>>(L, k0, k1));
      }
    }
    LS_LAUNCH("nd_perm", st, k_perm<<<(L.nf + 127) / 128, 128, 0, st>>>(L.piv, L.perm, L.iperm, L.nf, L.smax));
  }
  int err = 0;
  LS_CUDA(cudaMemcpyAsync(&err, p->d_err, sizeof(int), cudaMemcpyDeviceToHost, st));
  LS_CUDA(cudaStreamSynchronize(st));
  if (err) LS_FAIL(EINVAL_, "nested-dissection factorization met an exactly singular front");
}

// ---------------------------------------------------------------------------------------
// solves
// ---------------------------------------------------------------------------------------

template <typename C>
__global__ void __launch_bounds__(256) k_nd_fwd(LevelK<C> L, LevelK<C> Ch, int has_child, const C* __restrict__ r,
                                                int nrhs, long N) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  C* yb = reinterpret_cast<C*>(smem_raw);  // [nrhs][NB]
  const int z = blockIdx.x, tid = threadIdx.x, NT = blockDim.x;
  const int fmax = L.fmax, smax = L.smax;
  C* W = L.W + (size_t)z * nrhs * fmax;
  const C* A = L.F + (size_t)z * fmax * fmax;
  for (int idx = tid; idx < nrhs * fmax; idx += NT) {
    const int rhs = idx / fmax, q = idx % fmax;
    C v = czero<C>();
    if (q < smax) {
      const int o = L.perm[(size_t)z * smax + q];
      const int g = L.own[(size_t)z * smax + o];
      if (g >= 0) v = r[(size_t)rhs * N + g];
    }
    W[idx] = v;
  }
  __syncthreads();
  if (has_child) {
    for (int k = 0; k < 2; ++k) {
      const int c = L.child[(size_t)z * 2 + k];
      if (c < 0) continue;
      const C* Wc = Ch.W + (size_t)c * nrhs * Ch.fmax;
      const int* ea = Ch.ea + (size_t)c * Ch.bmax;
      for (int idx = tid; idx < nrhs * Ch.bmax; idx += NT) {
        const int rhs = idx / Ch.bmax, a = idx % Ch.bmax;
        const int ps = ea[a];
        if (ps < 0) continue;
        const int dst = ps < smax ? L.iperm[(size_t)z * smax + ps] : ps;
        C& x = W[(size_t)rhs * fmax + dst];
        x = cadd(x, Wc[(size_t)rhs * Ch.fmax + Ch.smax + a]);
      }
      __syncthreads();
    }
  }
  for (int j0 = 0; j0 < smax; j0 += NB) {
    const int w = min(NB, smax - j0);
    for (int rhs = tid; rhs < nrhs; rhs += NT) {
      C* Wr = W + (size_t)rhs * fmax;
      C* y = yb + rhs * NB;
      for (int i = 0; i < w; ++i) {
        C acc = Wr[j0 + i];
        for (int l = 0; l < i; ++l) acc = cfms(acc, A[(size_t)(j0 + l) * fmax + j0 + i], y[l]);
        y[i] = acc;
        Wr[j0 + i] = acc;
      }
    }
    __syncthreads();
    const int cnt = fmax - j0 - w;
    for (int idx = tid; idx < cnt * nrhs; idx += NT) {
      const int rhs = idx / cnt, i = j0 + w + idx % cnt;
      const C* y = yb + rhs * NB;
      C acc = czero<C>();
      for (int l = 0; l < w; ++l) acc = cfma(acc, A[(size_t)(j0 + l) * fmax + i], y[l]);
      C& x = W[(size_t)rhs * fmax + i];
      x = csub(x, acc);
    }
    __syncthreads();
  }
}

template <typename C>
__global__ void __launch_bounds__(256) k_nd_bwd(LevelK<C> L, C* __restrict__ X, int nrhs, long N) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  C* xb = reinterpret_cast<C*>(smem_raw);  // [nrhs][NB]
  const int z = blockIdx.x, tid = threadIdx.x, NT = blockDim.x;
  const int fmax = L.fmax, smax = L.smax, bmax = L.bmax;
  C* W = L.W + (size_t)z * nrhs * fmax;
  const C* A = L.F + (size_t)z * fmax * fmax;
  for (int idx = tid; idx < nrhs * bmax; idx += NT) {
    const int rhs = idx / bmax, q = idx % bmax;
    const int g = L.ring[(size_t)z * bmax + q];
    W[(size_t)rhs * fmax + smax + q] = g >= 0 ? X[(size_t)rhs * N + g] : czero<C>();
  }
  __syncthreads();
  // y_own -= U12 x_ring
  for (int idx = tid; idx < nrhs * smax; idx += NT) {
    const int rhs = idx / smax, q = idx % smax;
    const C* xr = W + (size_t)rhs * fmax + smax;
    C acc = czero<C>();
    for (int b = 0; b < bmax; ++b) acc = cfma(acc, A[(size_t)(smax + b) * fmax + q], xr[b]);
    C& x = W[(size_t)rhs * fmax + q];
    x = csub(x, acc);
  }
  __syncthreads();
  for (int jend = smax; jend > 0; jend -= NB) {
    const int j0 = max(0, jend - NB), w = jend - j0;
    for (int rhs = tid; rhs < nrhs; rhs += NT) {
      C* Wr = W + (size_t)rhs * fmax;
      C* x = xb + rhs * NB;
      for (int i = w - 1; i >= 0; --i) {
        C acc = Wr[j0 + i];
        for (int l = i + 1; l < w; ++l) acc = cfms(acc, A[(size_t)(j0 + l) * fmax + j0 + i], x[l]);
        acc = cdiv(acc, A[(size_t)(j0 + i) * fmax + j0 + i]);
        x[i] = acc;
        Wr[j0 + i] = acc;
      }
    }
    __syncthreads();
    for (int idx = tid; idx < j0 * nrhs; idx += NT) {
      const int rhs = idx / j0, i = idx % j0;
      const C* x = xb + rhs * NB;
      C acc = czero<C>();
      for (int l = 0; l < w; ++l) acc = cfma(acc, A[(size_t)(j0 + l) * fmax + i], x[l]);
      C& y = W[(size_t)rhs * fmax + i];
      y = csub(y, acc);
    }
    __syncthreads();
  }
  for (int idx = tid; idx < nrhs * smax; idx += NT) {
    const int rhs = idx / smax, q = idx % smax;
    const int g = L.own[(size_t)z * smax + q];
    if (g >= 0) X[(size_t)rhs * N + g] = W[(size_t)rhs * fmax + q];
  }
}

template <typename C> void nd_solve(NdPlan* p, int nrhs, const C* r, C* x, cudaStream_t st) {
  if (!p->F || p->F_bytes != (int)sizeof(C)) LS_FAIL(ESTATE_, "preconditioner not factored in this precision");
  const int depth = (int)p->lev.size();
  for (int c0 = 0; c0 < nrhs; c0 += SOLVE_CHUNK) {
    const int nr = std::min(SOLVE_CHUNK, nrhs - c0);
    const C* rr = r + (size_t)c0 * p->N;
    C* xx = x + (size_t)c0 * p->N;
    const size_t smem = (size_t)nr * NB * sizeof(C);
    for (int l = depth - 1; l >= 0; --l) {
      LevelK<C> L = level_k<C>(p, l);
      LevelK<C> Ch = l + 1 < depth ? level_k<C>(p, l + 1) : L;
      LS_LAUNCH(sizeof(C) == 8 ? "nd_fwd_c64" : "nd_fwd_c128", st,
                k_nd_fwd<C><<<L.nf, 256, smem, st>>>(L, Ch, l + 1 < depth ? 1 : 0, rr, nr, p->N));
    }
    for (int l = 0; l < depth; ++l) {
      LevelK<C> L = level_k<C>(p, l);
      LS_LAUNCH(sizeof(C) == 8 ? "nd_bwd_c64" : "nd_bwd_c128", st, k_nd_bwd<C><<<L.nf, 256, smem, st>>>(L, xx, nr, p->N));
    }
  }
}

template void nd_factor<float2>(NdPlan*, const void*, const void*, const void*, cudaStream_t);
template void nd_factor<double2>(NdPlan*, const void*, const void*, const void*, cudaStream_t);
template void nd_solve<float2>(NdPlan*, int, const float2*, float2*, cudaStream_t);
template void nd_solve<double2>(NdPlan*, int, const double2*, double2*, cudaStream_t);

}  // namespace ls
