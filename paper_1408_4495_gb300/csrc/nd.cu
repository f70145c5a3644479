// Nested-dissection multifrontal factorization of M = [A + C omega^2 m ; B] and its
// multi-right-hand-side solves (Sec. 2.2 after eq. PC: nested dissection + multifrontal
// method; Sec. 3.2: O(N^{3/2}) / O(N^2) factorization, O(N log N) / O(N^{4/3}) solve).
//
// Symbolic (host, once per (d, n)): the grid box is split recursively along its longest
// side by a one-point-thick separator slab (the 3^d stencil couples only points at
// infinity-distance <= 1, so the slab disconnects the halves).  A tree node owns its
// separator (a leaf owns its whole box); its front is [own variables ; ring], the ring
// being the grid points adjacent to the node's box (all of them belong to ancestors).
// Nodes at equal depth form one level and are processed by one batch of launches; each
// level stores its fronts densely as nf x fmax x ncols (column major, ld = fmax),
// fmax = smax + bmax, ncols = fmax + smax, smaller fronts padded (identity on padded own
// positions, zero ring positions).
//
// Numeric (device, per medium), level by level from the leaves.  Each front is augmented
// by an identity block on its own rows:
//       [ F11  F12  I ]        own rows (s)
//       [ F21  F22  0 ]        ring rows (b)
// and eliminated in two sweeps:
//   1. blocked right-looking partial LU of the whole front over the own columns (pivot rows
//      restricted to the own rows; panel / row-swap + unit-lower TRSM of the block row / GEMM
//      of the trailing block), the ring rows included: their panel entries become the
//      multipliers L21 = F21 U11^{-1} (forward substitution with each panel's U block) and
//      one GEMM with them leaves the Schur complement S = F22 - L21 U12 in the ring block and
//      Y = -L21 L11^{-1} P = -F21 F11^{-1} in the ring rows of the identity columns -- the
//      backward-stable LU form (forming them as F21 [H | F11^{-1}] from the explicit inverse
//      amplifies rounding by cond(F11), which weakened the FP32 preconditioner on large
//      fronts); the small fronts (up to 16 own rows) eliminate Gauss-Jordan style in shared
//      memory and form [S | Y] from the inverse;
//   2. blocked backward substitution with U11 on the own rows of [F12 I] (Gauss-Jordan),
//      which leaves H = F11^{-1} F12 and F11^{-1} there.
// S is extend-added into the parent.  The solve then needs no triangular recurrences:
//   forward (leaves to root):  update for the parent  u_ring = w_ring + Y w_own
//   backward (root to leaves): x_own = F11^{-1} w_own - H x_ring
// two batched multi-right-hand-side matrix-vector products per level, every factor entry
// read once per sweep.
#include <atomic>
#include <cooperative_groups.h>

#include <algorithm>
#include <cstring>
#include <map>
#include <memory>
#include <mutex>
#include <vector>

#include "alloc.h"
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
  int nf = 0, smax = 0, bmax = 0, fmax = 0, ncols = 0;
  size_t F_off = 0, W_off = 0;
  int *own = nullptr, *ring = nullptr, *child = nullptr, *parent = nullptr, *kidx = nullptr, *ea = nullptr;
  int* piv = nullptr;
  int* fsrc = nullptr;  // per front position: the two children's W items that add into it (-1: none)
};

template <typename C> struct LevelK {
  C* F;
  C* W;
  int nf, smax, bmax, fmax, ncols;
  const int *own, *ring, *child, *parent, *kidx, *ea;
  int* piv;
};

constexpr int NB = 32;           // panel / block width
constexpr int SOLVE_CHUNK = 64;  // right-hand sides per solve launch

}  // namespace

struct NdPlan {
  int d = 0, n = 0;
  long N = 0;
  std::vector<LevelDev> lev;
  long n_asm = 0, n_one = 0;
  int64_t* d_asm_off = nullptr;
  int* d_asm_row = nullptr;
  unsigned char* d_asm_t = nullptr;
  int64_t* d_one_off = nullptr;
  size_t F_elems = 0, W_elems = 0;
  void* F = nullptr;
  int F_bytes = 0;
  void* W = nullptr;
  int W_bytes = 0;
  void* T = nullptr;  // grid-point items of the solve (N x SOLVE_CHUNK)
  int* swp = nullptr;  // per-front row permutation of the current panel (register sweeps)
  void* part = nullptr;  // solve: partial sums of split column ranges
  // solve levels on the tensor cores (FP32): the gathered vector operands and the products,
  // sized for every level with at least TCS_MIN_ROWS rows
  float2* tcs_B = nullptr;
  float2* tcs_C = nullptr;
  size_t tcs_B_elems = 0, tcs_C_elems = 0;
  size_t part_elems = 0;
  unsigned* cnt = nullptr;  // solve: per-item arrival counters
  int* d_err = nullptr;
  bool use_tc = true;  // FP32 Schur products on the tensor cores (3xTF32) where they qualify
  NdTune tune{};       // launch-shape choices (defaults, or the autotuner's)
  void* blob = nullptr;  // every index array of the plan, one device allocation
  NdInfo info{};
};

namespace {

// Host result of the symbolic analysis for one (d, n): level shapes and every index array,
// packed in one blob (16-byte aligned pieces) that each context copies to the device once.
struct NdHost {
  int d = 0, n = 0;
  long N = 0;
  std::vector<LevelDev> lev;  // shapes and offsets; pointers are set per context
  struct Off {
    size_t own, ring, child, parent, kidx, ea, piv, fsrc;
  };
  std::vector<Off> off;
  size_t asm_off_o = 0, asm_row_o = 0, asm_t_o = 0, one_off_o = 0, err_o = 0;
  long n_asm = 0, n_one = 0;
  size_t F_elems = 0, W_elems = 0;
  NdInfo info{};
  std::vector<unsigned char> blob;
};

template <typename T> size_t put(std::vector<unsigned char>& blob, const std::vector<T>& v) {
  const size_t o = (blob.size() + 15) / 16 * 16;
  blob.resize(o + std::max<size_t>(1, v.size()) * sizeof(T), 0);
  if (!v.empty()) std::memcpy(blob.data() + o, v.data(), v.size() * sizeof(T));
  return o;
}

struct TreeBuild {
  int d = 0, n = 0;
  std::vector<Node> nodes;
};

void build_tree(TreeBuild* p, int leaf_max) {
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

std::shared_ptr<NdHost> host_symbolic(int d, int n) {
  auto H = std::make_shared<NdHost>();
  NdHost* p = H.get();
  TreeBuild T;
  {
    p->d = d;
    p->n = n;
    p->N = d == 2 ? (long)n * n : (long)n * n * n;
    T.d = d;
    T.n = n;
    build_tree(&T, d == 2 ? 16 : 27);
    int depth = 0;
    for (auto& nd : T.nodes) depth = std::max(depth, nd.depth + 1);
    std::vector<std::vector<int>> lev_nodes(depth);
    p->lev.assign(depth, LevelDev{});
    for (int id = 0; id < (int)T.nodes.size(); ++id) {
      Node& nd = T.nodes[id];
      nd.slot = (int)lev_nodes[nd.depth].size();
      lev_nodes[nd.depth].push_back(id);
    }
    size_t F_off = 0, W_off = 0;
    double flops = 0, solve_entries = 0;
    int max_front = 0;
    for (int l = 0; l < depth; ++l) {
      LevelDev& L = p->lev[l];
      L.nf = (int)lev_nodes[l].size();
      for (int id : lev_nodes[l]) {
        L.smax = std::max(L.smax, (int)T.nodes[id].own.size());
        L.bmax = std::max(L.bmax, (int)T.nodes[id].ring.size());
      }
      L.fmax = L.smax + L.bmax;
      L.ncols = L.fmax + L.smax;
      L.F_off = F_off;
      L.W_off = W_off;
      F_off += (size_t)L.nf * L.fmax * L.ncols;
      W_off += (size_t)L.nf * SOLVE_CHUNK * L.fmax;
      max_front = std::max(max_front, L.fmax);
      // complex multiply-adds of the two sweeps on the padded shapes, 8 real flops each
      double cm = 0;
      for (int j = 0; j < L.smax; ++j) cm += (double)(L.smax - j - 1) * (L.ncols - j - 1) + (double)j * (L.ncols - L.smax);
      cm += (double)L.bmax * L.smax * (L.ncols - L.smax);
      flops += 8.0 * cm * L.nf;
      solve_entries += (double)L.nf * ((double)L.smax * L.smax + 2.0 * L.smax * L.bmax);
      // forward: Y (bmax x smax) once; per right-hand side: r at the own points, the front
      // vector written (fmax); backward: [H | F11^-1] (smax x (bmax + smax)) once; per
      // right-hand side: x at the ring points, w_own, x written at the own points
      p->info.fwd_factor_entries += (double)L.nf * L.bmax * L.smax;
      p->info.fwd_vec_entries += (double)L.nf * ((double)L.smax + L.fmax);
      p->info.bwd_factor_entries += (double)L.nf * L.smax * ((double)L.bmax + L.smax);
      p->info.bwd_vec_entries += (double)L.nf * ((double)L.bmax + 2.0 * L.smax);
    }
    // the children's update vectors read by the parents' forward step
    for (int l = 1; l < depth; ++l) p->info.fwd_vec_entries += (double)p->lev[l].nf * p->lev[l].bmax;
    p->F_elems = F_off;
    p->W_elems = W_off;
    p->info.levels = depth;
    p->info.fronts = (int)T.nodes.size();
    p->info.max_front = max_front;
    p->info.factor_entries = (int64_t)F_off;
    p->info.factor_flops = flops;
    p->info.solve_bytes = solve_entries;  // entries; scaled by the element size by the caller

    // per-level index arrays, assembly list, extend-add maps
    std::vector<int> pos(p->N, -1);
    std::vector<int64_t> asm_off, one_off;
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
    auto tcode = [&](int t0, int t1, int t2) -> unsigned char {
      return (unsigned char)(d == 2 ? (t0 + 1) * 3 + (t1 + 1) : ((t0 + 1) * 3 + (t1 + 1)) * 3 + (t2 + 1));
    };
    for (int id = 0; id < (int)T.nodes.size(); ++id) {
      const Node& nd = T.nodes[id];
      const int l = nd.depth;
      const LevelDev& L = p->lev[l];
      const int z = nd.slot;
      const int s = (int)nd.own.size(), b = (int)nd.ring.size();
      for (int q = 0; q < s; ++q) l_own[l][(size_t)z * L.smax + q] = nd.own[q];
      for (int q = 0; q < b; ++q) l_ring[l][(size_t)z * L.bmax + q] = nd.ring[q];
      for (int k = 0; k < 2; ++k)
        if (nd.child[k] >= 0) l_child[l][(size_t)z * 2 + k] = T.nodes[nd.child[k]].slot;
      if (nd.parent >= 0) {
        l_parent[l][z] = T.nodes[nd.parent].slot;
        l_kidx[l][z] = nd.kidx;
      }
      for (int q = 0; q < s; ++q) pos[nd.own[q]] = q;
      for (int q = 0; q < b; ++q) pos[nd.ring[q]] = L.smax + q;
      const size_t base = L.F_off + (size_t)z * L.fmax * L.ncols;
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
              if (pos[j] < 0) continue;  // eliminated in a descendant
              asm_off.push_back((int64_t)(base + (size_t)pos[j] * L.fmax + q));
              asm_row.push_back(nd.own[q]);
              asm_t.push_back(tcode(t0, t1, t2));
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
              asm_t.push_back(tcode(t0, t1, t2));
            }
      }
      // ones: identity on padded own positions and in the augmented block
      for (int q = s; q < L.smax; ++q) one_off.push_back((int64_t)(base + (size_t)q * L.fmax + q));
      for (int q = 0; q < L.smax; ++q) one_off.push_back((int64_t)(base + (size_t)(L.fmax + q) * L.fmax + q));
      // extend-add maps of the children: child ring variable -> position in this front
      for (int k = 0; k < 2; ++k) {
        const int cid = nd.child[k];
        if (cid < 0) continue;
        const Node& ch = T.nodes[cid];
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
    p->off.resize(depth);
    for (int l = 0; l < depth; ++l) {
      const LevelDev& L = p->lev[l];
      NdHost::Off& o = p->off[l];
      o.own = put(p->blob, l_own[l]);
      o.ring = put(p->blob, l_ring[l]);
      o.child = put(p->blob, l_child[l]);
      o.parent = put(p->blob, l_parent[l]);
      o.kidx = put(p->blob, l_kidx[l]);
      o.ea = put(p->blob, l_ea[l]);
      o.piv = put(p->blob, std::vector<int>((size_t)L.nf * L.smax, 0));
      // forward-solve sources: child k's ring entry a lands at position ea[a] of the parent
      std::vector<int> fsrc((size_t)L.nf * L.fmax * 2, -1);
      if (l + 1 < depth) {
        const LevelDev& Lc = p->lev[l + 1];
        for (int z = 0; z < L.nf; ++z)
          for (int k = 0; k < 2; ++k) {
            const int c = l_child[l][(size_t)z * 2 + k];
            if (c < 0) continue;
            for (int a = 0; a < Lc.bmax; ++a) {
              const int ps = l_ea[l + 1][(size_t)c * Lc.bmax + a];
              if (ps >= 0) fsrc[((size_t)z * L.fmax + ps) * 2 + k] = c * Lc.fmax + Lc.smax + a;
            }
          }
      }
      o.fsrc = put(p->blob, fsrc);
    }
    p->n_asm = (long)asm_off.size();
    p->n_one = (long)one_off.size();
    p->asm_off_o = put(p->blob, asm_off);
    p->asm_row_o = put(p->blob, asm_row);
    p->asm_t_o = put(p->blob, asm_t);
    p->one_off_o = put(p->blob, one_off);
    p->err_o = put(p->blob, std::vector<int>(1, 0));
  }
  return H;
}

}  // namespace

NdPlan* nd_build(int d, int n, cudaStream_t st) {
  static std::mutex mu;
  static std::map<std::pair<int, int>, std::shared_ptr<NdHost>> cache;
  std::shared_ptr<NdHost> H;
  {
    std::lock_guard<std::mutex> lk(mu);
    auto it = cache.find({d, n});
    if (it != cache.end()) H = it->second;
  }
  if (!H) {
    H = host_symbolic(d, n);
    std::lock_guard<std::mutex> lk(mu);
    cache[{d, n}] = H;
  }
  NdPlan* p = new NdPlan;
  try {
    p->d = d;
    p->n = n;
    p->N = H->N;
    p->lev = H->lev;
    p->n_asm = H->n_asm;
    p->n_one = H->n_one;
    p->F_elems = H->F_elems;
    p->W_elems = H->W_elems;
    p->info = H->info;
    p->blob = dev_alloc(H->blob.size());
    LS_CUDA(cudaMemcpyAsync(p->blob, H->blob.data(), H->blob.size(), cudaMemcpyHostToDevice, st));
    unsigned char* b = static_cast<unsigned char*>(p->blob);
    for (size_t l = 0; l < p->lev.size(); ++l) {
      LevelDev& L = p->lev[l];
      const NdHost::Off& o = H->off[l];
      L.own = reinterpret_cast<int*>(b + o.own);
      L.ring = reinterpret_cast<int*>(b + o.ring);
      L.child = reinterpret_cast<int*>(b + o.child);
      L.parent = reinterpret_cast<int*>(b + o.parent);
      L.kidx = reinterpret_cast<int*>(b + o.kidx);
      L.ea = reinterpret_cast<int*>(b + o.ea);
      L.piv = reinterpret_cast<int*>(b + o.piv);
      L.fsrc = reinterpret_cast<int*>(b + o.fsrc);
    }
    p->d_asm_off = reinterpret_cast<int64_t*>(b + H->asm_off_o);
    p->d_asm_row = reinterpret_cast<int*>(b + H->asm_row_o);
    p->d_asm_t = b + H->asm_t_o;
    p->d_one_off = reinterpret_cast<int64_t*>(b + H->one_off_o);
    p->d_err = reinterpret_cast<int*>(b + H->err_o);
    LS_CUDA(cudaStreamSynchronize(st));
  } catch (...) {
    nd_free(p);
    throw;
  }
  return p;
}

void nd_free(NdPlan* p) {
  if (!p) return;
  if (p->blob) dev_free(p->blob);
  if (p->F) dev_free(p->F);
  if (p->W) dev_free(p->W);
  if (p->T) dev_free(p->T);
  if (p->swp) dev_free(p->swp);
  if (p->part) dev_free(p->part);
  if (p->cnt) dev_free(p->cnt);
  if (p->tcs_B) dev_free(p->tcs_B);
  if (p->tcs_C) dev_free(p->tcs_C);
  delete p;
}

NdInfo nd_info(const NdPlan* p) { return p->info; }

// rows of a sweep level's product from which it may run on the tensor cores, and its
// operand sizes for SOLVE_CHUNK right-hand sides (mode 0 forward, 1 backward)
constexpr int TCS_MIN_ROWS = 32;
static int tcs_rows(const LevelDev& D, int mode) { return mode == 0 ? D.bmax : D.smax; }
static int tcs_k(const LevelDev& D, int mode) { return mode == 0 ? D.smax : D.bmax + D.smax; }
// split of a level's k range over CTAs: enough CTAs for three per SM (the tensor-core GEMM's
// residency) with at least 64 columns (8 chunks) per split
struct TcsSplit {
  int nsplit, ksz;
};
static TcsSplit tcs_split(const LevelDev& D, int mode) {
  const int K = tcs_k(D, mode), rows = tcs_rows(D, mode);
  const long base = (long)D.nf * ((rows + 127) / 128);
  int ns = 1;
  while (base * ns < 3L * 152 && (K + 2 * ns - 1) / (2 * ns) >= 64) ns *= 2;
  const int ksz = ((K + ns - 1) / ns + 7) / 8 * 8;
  return {(K + ksz - 1) / ksz, ksz};
}
static void tcs_sizes(const std::vector<LevelDev>& lev, size_t* b, size_t* c) {
  *b = *c = 0;
  for (const LevelDev& D : lev)
    for (int mode = 0; mode < 2; ++mode)
      if (tcs_rows(D, mode) >= TCS_MIN_ROWS) {
        *b = std::max(*b, (size_t)D.nf * tcs_k(D, mode) * SOLVE_CHUNK);
        *c = std::max(*c, (size_t)D.nf * tcs_rows(D, mode) * SOLVE_CHUNK * tcs_split(D, mode).nsplit);
      }
}

size_t nd_device_bytes(const NdPlan* p, int elem_bytes) {
  size_t b = 0, c = 0;
  if (elem_bytes == 8) tcs_sizes(p->lev, &b, &c);
  return (p->F_elems + p->W_elems + (size_t)p->N * SOLVE_CHUNK + b + c) * (size_t)elem_bytes;
}

// The factorization's whole state is the front storage F: the solve reads the factored
// fronts and the static index arrays only (the panel pivots are consumed inside the
// factorization).  0 when F is not allocated.
size_t nd_factor_bytes(const NdPlan* p) { return p->F ? p->F_elems * (size_t)p->F_bytes : 0; }
size_t nd_factor_elems(const NdPlan* p) { return p->F_elems; }

void nd_copy_factors(NdPlan* p, void* host, bool to_host, cudaStream_t st) {
  const size_t bytes = nd_factor_bytes(p);
  if (!bytes) LS_FAIL(ESTATE_, "front storage not prepared");
  if (to_host) LS_CUDA(cudaMemcpyAsync(host, p->F, bytes, cudaMemcpyDeviceToHost, st));
  else LS_CUDA(cudaMemcpyAsync(p->F, host, bytes, cudaMemcpyHostToDevice, st));
  LS_CUDA(cudaStreamSynchronize(st));
}

// ---------------------------------------------------------------------------------------
// factorization kernels
// ---------------------------------------------------------------------------------------

template <typename C>
__global__ void k_assemble(C* F, long n_asm, const int64_t* __restrict__ off, const int* __restrict__ row,
                           const unsigned char* __restrict__ tcode, int d, int n, const double2* __restrict__ alpha,
                           const double2* __restrict__ cint, const double* __restrict__ w2m,
                           const double2* __restrict__ alpha_pt, const unsigned char* __restrict__ inter_pt) {
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
    // M(i, i+t) = alpha_cls(i)(t) + [i interior] c(t) omega^2 m_{i+t}   (eq. PC); general
    // domains (Sec. 4) give a stencil and an interior flag per point instead of per class
    double2 v;
    if (alpha_pt) {
      v = alpha_pt[(long)i * P3 + t];
      interior = inter_pt[i] != 0;
    } else {
      v = alpha[cls * P3 + t];
    }
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

template <typename C> __global__ void k_set_one(C* F, long n_one, const int64_t* __restrict__ off) {
  for (long e = blockIdx.x * (long)blockDim.x + threadIdx.x; e < n_one; e += (long)gridDim.x * blockDim.x) {
    C one;
    one.x = 1;
    one.y = 0;
    F[off[e]] = one;
  }
}

// Schur complements of the children with child index k into their parents' fronts.
template <typename C> __global__ void __launch_bounds__(256) k_extend_add(LevelK<C> P, LevelK<C> Ch, int k) {
  const int c = blockIdx.x;
  if (Ch.kidx[c] != k) return;
  const int pz = Ch.parent[c];
  C* Fp = P.F + (size_t)pz * P.fmax * P.ncols;
  const C* Fc = Ch.F + (size_t)c * Ch.fmax * Ch.ncols;
  const int* ea = Ch.ea + (size_t)c * Ch.bmax;
  const int cb = Ch.bmax;
  const long tot = (long)cb * cb;
  // four entries per thread: index, child and parent loads in flight before the stores
  constexpr int B = 4;
  const long step = (long)gridDim.y * blockDim.x;
  for (long base = blockIdx.y * (long)blockDim.x + threadIdx.x; base < tot; base += step * B) {
    C v[B], o[B];
    long dst[B];
#pragma unroll
    for (int u = 0; u < B; ++u) {
      const long idx = base + u * step;
      dst[u] = -1;
      if (idx < tot) {
        const int a = (int)(idx % cb), b = (int)(idx / cb);
        const int pa = ea[a], pb = ea[b];
        if (pa >= 0 && pb >= 0) {
          dst[u] = (long)pb * P.fmax + pa;
          v[u] = Fc[(size_t)(Ch.smax + b) * Ch.fmax + Ch.smax + a];
        }
      }
    }
#pragma unroll
    for (int u = 0; u < B; ++u)
      if (dst[u] >= 0) o[u] = Fp[dst[u]];
#pragma unroll
    for (int u = 0; u < B; ++u)
      if (dst[u] >= 0) Fp[dst[u]] = cadd(o[u], v[u]);
  }
}

// (max |.|^2, smallest index) over a CTA; every thread gets the result
template <typename Rl>
__device__ __forceinline__ void argmax_block(Rl& v, int& i, Rl* sv, int* si) {
  for (int o = 16; o > 0; o >>= 1) {
    const Rl ov = __shfl_down_sync(0xffffffffu, v, o);
    const int oi = __shfl_down_sync(0xffffffffu, i, o);
    if (ov > v || (ov == v && oi < i)) { v = ov; i = oi; }
  }
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
  if (lane == 0) { sv[wid] = v; si[wid] = i; }
  __syncthreads();
  if (wid == 0) {
    v = lane < nw ? sv[lane] : (Rl)-1;
    i = lane < nw ? si[lane] : 0x7fffffff;
    for (int o = 16; o > 0; o >>= 1) {
      const Rl ov = __shfl_down_sync(0xffffffffu, v, o);
      const int oi = __shfl_down_sync(0xffffffffu, i, o);
      if (ov > v || (ov == v && oi < i)) { v = ov; i = oi; }
    }
    if (lane == 0) { sv[0] = v; si[0] = i; }
  }
  __syncthreads();
  v = sv[0];
  i = si[0];
  __syncthreads();
}

// Panel [k0, k1) held in shared memory (rows k0..fmax): pivot search over the own rows,
// row swaps within the panel, scaling, rank-1 updates.  Rows above k0 are final U entries.
template <typename C, bool SMEM>
__global__ void __launch_bounds__(512) k_panel(LevelK<C> L, int k0, int k1, int* err) {
  using Rl = typename RealOf<C>::T;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ Rl sv[32];
  __shared__ int si[32];
  const int z = blockIdx.x, tid = threadIdx.x, NT = blockDim.x;
  const int fmax = L.fmax, smax = L.smax;
  const int R = smax - k0, w = k1 - k0, srow = smax - k0;
  C* A = L.F + (size_t)z * fmax * L.ncols;
  C* P;
  int ld;
  if constexpr (SMEM) {
    P = reinterpret_cast<C*>(smem_raw);
    ld = R;
    for (int idx = tid; idx < R * w; idx += NT) {
      const int c = idx / R, r = idx - c * R;
      P[idx] = A[(size_t)(k0 + c) * fmax + k0 + r];
    }
    __syncthreads();
  } else {
    P = A + (size_t)k0 * fmax + k0;
    ld = fmax;
  }
  for (int j = 0; j < w; ++j) {
    Rl best = -1;
    int bi = 0x7fffffff;
    for (int r = j + tid; r < srow; r += NT) {
      const Rl v = cabs2(P[(size_t)j * ld + r]);
      if (v > best) { best = v; bi = r; }
    }
    argmax_block(best, bi, sv, si);
    if (bi == 0x7fffffff) bi = j;
    if (tid == 0) {
      L.piv[(size_t)z * smax + k0 + j] = k0 + bi;
      if (!(best > 0)) atomicCAS(err, 0, 1);
    }
    if (bi != j)
      for (int c = tid; c < w; c += NT) {
        C& x = P[(size_t)c * ld + j];
        C& y = P[(size_t)c * ld + bi];
        const C t = x;
        x = y;
        y = t;
      }
    __syncthreads();
    const C dg = P[(size_t)j * ld + j];
    const Rl den = cabs2(dg);
    C inv;
    inv.x = den > 0 ? dg.x / den : (Rl)0;
    inv.y = den > 0 ? -dg.y / den : (Rl)0;
    for (int r = j + 1 + tid; r < R; r += NT) {
      C& x = P[(size_t)j * ld + r];
      x = cmul(x, inv);
    }
    __syncthreads();
    const int ncol = w - j - 1, nrow = R - j - 1;
    for (int idx = tid; idx < ncol * nrow; idx += NT) {
      const int c = j + 1 + idx / nrow, r = j + 1 + idx % nrow;
      C& x = P[(size_t)c * ld + r];
      x = cfms(x, P[(size_t)j * ld + r], P[(size_t)c * ld + j]);
    }
    __syncthreads();
  }
  if constexpr (SMEM) {
    for (int idx = tid; idx < R * w; idx += NT) {
      const int c = idx / R, r = idx - c * R;
      A[(size_t)(k0 + c) * fmax + k0 + r] = P[idx];
    }
  }
}

// Columns c in [k1, ncols): apply the panel's row swaps, then F[k0:k1, c] = L_kk^{-1} F[k0:k1, c].
template <typename C> __global__ void __launch_bounds__(128) k_trsm_lower(LevelK<C> L, int k0, int k1) {
  const int z = blockIdx.x;
  const int fmax = L.fmax, w = k1 - k0;
  C* A = L.F + (size_t)z * fmax * L.ncols;
  __shared__ C Ld[NB][NB + 1];
  // net effect of the panel's row swaps: position pos[i] receives original row src[i];
  // positions k0..k1-1 first, then the pivot rows below k1 that were swapped up
  __shared__ int pos[2 * NB], src[2 * NB], npos, pv[NB];
  for (int idx = threadIdx.x; idx < w * w; idx += blockDim.x) {
    const int i = idx % w, l = idx / w;
    Ld[i][l] = A[(size_t)(k0 + l) * fmax + k0 + i];
  }
  for (int j = threadIdx.x; j < w; j += blockDim.x) pv[j] = L.piv[(size_t)z * L.smax + k0 + j];
  __syncthreads();
  if (threadIdx.x == 0) {
    int cnt = w;
    for (int i = 0; i < w; ++i) { pos[i] = k0 + i; src[i] = k0 + i; }
    for (int j = 0; j < w; ++j) {
      const int q = pv[j];
      if (q == k0 + j) continue;
      int iq = -1;
      for (int i = 0; i < cnt; ++i)
        if (pos[i] == q) { iq = i; break; }
      if (iq < 0) { iq = cnt++; pos[iq] = q; src[iq] = q; }
      const int t = src[j];
      src[j] = src[iq];
      src[iq] = t;
    }
    npos = cnt;
  }
  __syncthreads();
  const int c = k1 + blockIdx.y * blockDim.x + threadIdx.x;
  if (c >= L.ncols) return;
  C* col = A + (size_t)c * fmax;
  const int np = npos;
  C x[NB];
#pragma unroll
  for (int i = 0; i < NB; ++i)
    if (i < w) x[i] = col[src[i]];
  {
    C extra[NB];
#pragma unroll
    for (int i = 0; i < NB; ++i)
      if (w + i < np) extra[i] = col[src[w + i]];
#pragma unroll
    for (int i = 0; i < NB; ++i)
      if (w + i < np) col[pos[w + i]] = extra[i];
  }
  // column-oriented (right-looking): x_i final, then every x_r below it updated at once
#pragma unroll
  for (int i = 0; i < NB - 1; ++i) {
    if (i < w) {
#pragma unroll
      for (int r = i + 1; r < NB; ++r)
        if (r < w) x[r] = cfms(x[r], Ld[r][i], x[i]);
    }
  }
#pragma unroll
  for (int i = 0; i < NB; ++i)
    if (i < w) col[k0 + i] = x[i];
}

// Columns c in [smax, ncols): F[j0:j1, c] = U_blk^{-1} F[j0:j1, c] (non-unit upper).
// Column-oriented (right-looking) substitution: once x_i is final, every x_l above it takes
// its update at once, so a thread's dependent chain is one product per row (the dot-product
// form chains up to 31 products per row); the reciprocals of the diagonal are formed once
// per CTA.
template <typename C> __global__ void __launch_bounds__(128) k_trsm_upper(LevelK<C> L, int j0, int j1) {
  const int z = blockIdx.x;
  const int fmax = L.fmax, w = j1 - j0;
  C* A = L.F + (size_t)z * fmax * L.ncols;
  __shared__ C Ud[NB][NB + 1];
  __shared__ C rdg[NB];
  for (int idx = threadIdx.x; idx < w * w; idx += blockDim.x) {
    const int i = idx % w, l = idx / w;
    Ud[i][l] = A[(size_t)(j0 + l) * fmax + j0 + i];
  }
  __syncthreads();
  if (threadIdx.x < w) {
    C one;
    one.x = 1;
    one.y = 0;
    rdg[threadIdx.x] = cdiv(one, Ud[threadIdx.x][threadIdx.x]);
  }
  __syncthreads();
  const int c = L.smax + blockIdx.y * blockDim.x + threadIdx.x;
  if (c >= L.ncols) return;
  C* col = A + (size_t)c * fmax;
  C x[NB];
#pragma unroll
  for (int i = 0; i < NB; ++i)
    if (i < w) x[i] = col[j0 + i];
#pragma unroll
  for (int i = NB - 1; i >= 0; --i) {
    if (i < w) {
      x[i] = cmul(x[i], rdg[i]);
#pragma unroll
      for (int l = 0; l < i; ++l) x[l] = cfms(x[l], Ud[l][i], x[i]);
    }
  }
#pragma unroll
  for (int i = 0; i < NB; ++i)
    if (i < w) col[j0 + i] = x[i];
}

// Ring rows r in [smax, fmax) of every front, panel columns [k0, k1): the multipliers
// L21 = F21 U_kk^{-1}, by forward substitution along the panel with its upper triangle U_kk
// (rows k0..k1 of the panel after the panel kernel; the ring rows are never permuted).  With
// the ring rows also in the trailing updates, the forward elimination of the own columns is
// the partial LU of the whole front, so the Schur complement S = F22 - L21 U12 and
// Y = -L21 L11^{-1} P are formed backward stably (the product F21 [H | F11^{-1}] of the
// explicit inverse would amplify rounding by cond(F11)).  One thread per ring row; U_kk and
// its reciprocal pivots in shared memory.
template <typename C> __global__ void __launch_bounds__(256) k_ring_trsm(LevelK<C> L, int k0, int k1) {
  using Rl = typename RealOf<C>::T;
  __shared__ C u[NB][NB + 1];  // u[j][i] = U_kk(i, j)
  __shared__ C invd[NB];
  const int z = blockIdx.x, w = k1 - k0, fmax = L.fmax;
  C* A = L.F + (size_t)z * fmax * L.ncols;
  for (int e = threadIdx.x; e < w * w; e += blockDim.x) {
    const int i = e % w, j = e / w;
    u[j][i] = A[(size_t)(k0 + j) * fmax + k0 + i];
  }
  __syncthreads();
  for (int j = threadIdx.x; j < w; j += blockDim.x) {
    const C dg = u[j][j];
    const Rl den = cabs2(dg);
    C inv;
    inv.x = den > 0 ? dg.x / den : (Rl)0;
    inv.y = den > 0 ? -dg.y / den : (Rl)0;
    invd[j] = inv;
  }
  __syncthreads();
  const int r = L.smax + blockIdx.y * blockDim.x + threadIdx.x;
  if (r >= fmax) return;
  C* row = A + (size_t)k0 * fmax + r;
  C f[NB];
#pragma unroll
  for (int c = 0; c < NB; ++c) f[c] = c < w ? row[(size_t)c * fmax] : czero<C>();
  // column-oriented (right-looking): f_c final, then every f_c2 right of it updated at once
#pragma unroll
  for (int c = 0; c < NB; ++c) {
    if (c < w) {
      f[c] = cmul(f[c], invd[c]);
#pragma unroll
      for (int c2 = c + 1; c2 < NB; ++c2)
        if (c2 < w) f[c2] = cfms(f[c2], f[c], u[c2][c]);
    }
  }
#pragma unroll
  for (int c = 0; c < NB; ++c)
    if (c < w) row[(size_t)c * fmax] = f[c];
}

template <typename C> static void launch_ring_trsm(const LevelK<C>& L, int k0, int k1, cudaStream_t st) {
  if (L.bmax <= 0) return;
  LS_LAUNCH(sizeof(C) == 8 ? "nd_trsm_c64" : "nd_trsm_c128", st,
            k_ring_trsm<C><<<dim3(L.nf, (L.bmax + 255) / 256), 256, 0, st>>>(L, k0, k1));
}

// ---------------------------------------------------------------------------------------
// Register-resident blocked factorization for fronts with at most 32 * RPL own rows.
// Sweep 1 (LU of F11 with partial pivoting over the own rows, [F12 | I] carried along):
// per panel of NB columns one CTA factors the panel with one own row per thread held in
// registers (k_panel_reg), then one warp per trailing column (in registers) applies the
// panel's row permutation, the forward substitution with the unit lower L_kk and the update
// of the rows below.  Sweep 2 (U11 X = B on the own rows of [F12 | I]): one warp per column
// runs the whole backward substitution with its column in registers, the U11 columns staged
// in shared memory 32 at a time.  The blocked path of larger fronts uses the same panels
// (and, from 513 to 4096 rows, their cluster form) with tensor-core trailing GEMMs.
// ---------------------------------------------------------------------------------------
constexpr int SWP_STRIDE = 1 + 4 * NB;  // per front: count, then (position, source) pairs
constexpr int OB_PANELS = 4;            // panels per outer block of the blocked path

// dst[e] = src(e) for e < n over the CTA's threads, B loads in flight per thread before the
// first store (the loads do not wait on the stores of earlier iterations)
template <int B, typename T, typename F> __device__ __forceinline__ void stage_copy(T* dst, int n, F src) {
  for (int base = threadIdx.x; base < n; base += blockDim.x * B) {
    T v[B];
#pragma unroll
    for (int u = 0; u < B; ++u) {
      const int e = base + u * blockDim.x;
      if (e < n) v[u] = src(e);
    }
#pragma unroll
    for (int u = 0; u < B; ++u) {
      const int e = base + u * blockDim.x;
      if (e < n) dst[e] = v[u];
    }
  }
}

// 1 / x, correctly rounded
__device__ __forceinline__ float recip(float x) { return __frcp_rn(x); }
__device__ __forceinline__ double recip(double x) { return 1.0 / x; }

template <typename C> __device__ __forceinline__ C shfl_c(C v, int src) {
  v.x = __shfl_sync(0xffffffffu, v.x, src);
  v.y = __shfl_sync(0xffffffffu, v.y, src);
  return v;
}

// Panel [k0, k1) on at most 512 own rows (256 in FP64), one row per thread held in registers
// (the column loops are unrolled, so every register index is a constant).  Per column one
// barrier: each warp's best live row publishes its key, the reciprocal of its pivot entry
// and the rest of its row to a parity-double-buffered slot before the barrier; after it
// every thread picks the winning warp and updates its own row from the winner's slot with
// broadcast shared-memory reads.  Pivot key: |re| + |im| as an FP32 bit pattern cut to 14
// mantissa bits, packed above (1023 - row) so that one max reduction finds the largest
// entry and, among entries equal to 14 bits, the lowest row (partial pivoting up to a
// relative 2^-14, as stable as an exact search).  The panel rows are then written to their
// logical positions (local to k0): pivot j to position j; the rows at positions < w that
// were not chosen fill, in increasing order, the positions >= w whose rows were chosen.
// Any consistent row order is valid: the same permutation, recorded in swp, is applied to
// the trailing columns and to the identity block.
template <typename C> __host__ __device__ constexpr int panel_reg_rows() { return sizeof(C) == 8 ? 512 : 256; }

template <typename C>
__global__ void __launch_bounds__(panel_reg_rows<C>()) k_panel_reg(LevelK<C> L, int k0, int k1, int* __restrict__ swp,
                                                                  int* err) {
  using Rl = typename RealOf<C>::T;
  constexpr int MW = panel_reg_rows<C>() / 32;
  __shared__ __align__(16) C slot[2][MW][NB];
  __shared__ unsigned skey[2][MW];
  __shared__ int vac[NB];
  __shared__ int wcnt[MW];
  __shared__ int cnt;
  const int z = blockIdx.x, r = threadIdx.x, lane = r & 31, wid = r >> 5, nw = blockDim.x >> 5;
  const int fmax = L.fmax, R = L.smax - k0, w = k1 - k0;
  C* A = L.F + (size_t)z * fmax * L.ncols + (size_t)k0 * fmax + k0;  // local (r, c) at A[c * fmax + r]
  const bool has = r < R;
  C a[NB];
#pragma unroll
  for (int c = 0; c < NB; ++c) a[c] = (has && c < w) ? A[(size_t)c * fmax + r] : czero<C>();
  if (r == 0) cnt = 0;
  if (r < NB) vac[r] = r;
  bool live = has;
  int jp = -1;  // the column at which this row was chosen as pivot
#pragma unroll
  for (int j = 0; j < NB; ++j) {
    if (j < w) {
      const int par = j & 1;
      const unsigned mag = __float_as_uint((float)(fabs(a[j].x) + fabs(a[j].y)));
      const unsigned key = live ? ((mag >> 9) << 10) | (1023u - (unsigned)r) : 0u;
      const unsigned kw = __reduce_max_sync(0xffffffffu, key);
      if (live && key == kw) {
        const Rl den = cabs2(a[j]);
        const Rl rden = den > 0 ? recip(den) : (Rl)0;
        C inv;
        inv.x = a[j].x * rden;
        inv.y = -a[j].y * rden;
        slot[par][wid][j] = inv;
#pragma unroll
        for (int c = j + 1; c < NB; ++c) slot[par][wid][c] = a[c];
      }
      if (lane == 0) skey[par][wid] = kw;
      __syncthreads();
      const unsigned km = __reduce_max_sync(0xffffffffu, lane < nw ? skey[par][lane] : 0u);
      if (km == 0u) {  // no live row left (cannot happen while j < R)
        if (r == 0) atomicCAS(err, 0, 1);
        continue;
      }
      if ((km >> 10) == 0u && r == 0) atomicCAS(err, 0, 1);  // zero pivot
      const int bi = 1023 - (int)(km & 1023u);
      if (r == bi) {
        live = false;
        jp = j;
      }
      if (live) {
        const C* pr = slot[par][bi >> 5];
        const C m = cmul(a[j], pr[j]);
        a[j] = m;
#pragma unroll
        for (int c = j + 1; c < NB; ++c) a[c] = cfms(a[c], m, pr[c]);
      }
    }
  }
  // positions >= w vacated by pivots, in increasing order
  const bool vp = jp >= 0 && r >= w;
  const unsigned bv = __ballot_sync(0xffffffffu, vp);
  if (lane == 0) wcnt[wid] = __popc(bv);
  __syncthreads();
  const unsigned lt = (1u << lane) - 1u;
  if (vp) {
    int before = 0;
    for (int q = 0; q < wid; ++q) before += wcnt[q];
    vac[before + __popc(bv & lt)] = r;
  }
  __syncthreads();
  // rows at positions < w not chosen (all in warp 0) take the vacated positions in order
  const bool dp = has && jp < 0 && r < w;
  const unsigned bd = __ballot_sync(0xffffffffu, dp);
  const int pos = jp >= 0 ? jp : (dp ? min(vac[__popc(bd & lt)], R - 1) : r);
  if (has) {
#pragma unroll
    for (int c = 0; c < NB; ++c)
      if (c < w) A[(size_t)c * fmax + pos] = a[c];
    if (pos != r) {
      const int q = atomicAdd(&cnt, 1);
      if (q < 2 * NB) {
        swp[(size_t)z * SWP_STRIDE + 1 + 2 * q] = pos;
        swp[(size_t)z * SWP_STRIDE + 2 + 2 * q] = r;
      }
    }
  }
  __syncthreads();
  if (r == 0) swp[(size_t)z * SWP_STRIDE] = min(cnt, 2 * NB);
}

// Panel [k0, k1) of a front with up to PC_CTAS * 512 own rows (FP32): the register panel
// spread over a thread-block cluster, one own row per thread, 512 rows per CTA.  Per column:
// each warp's best live row publishes its key, reciprocal pivot and row to its CTA's
// parity-double-buffered slot (as in k_panel_reg), the CTA reduces its warps' keys, one
// cluster barrier makes every CTA's best key and slots visible, and each warp reads the
// CTAs' keys and then the winning row through distributed shared memory.  Keys carry the
// magnitude |re| + |im| cut to 12 mantissa bits above (4095 - row).  At the end CTA 0 gathers the pivot
// sequence from every CTA and places the rows above w that were not chosen; the rows are
// written to their logical positions and swp holds, per front, the pairs (position, source)
// local to k0: pivot j in pair j, the displaced rows in pairs w.. (count = w + displaced).
constexpr int PC_ROWS = 512, PC_CTAS = 8;
template <typename C>
__global__ void __launch_bounds__(PC_ROWS) k_panel_cluster(LevelK<C> L, int k0, int k1, int* __restrict__ swp,
                                                          int* err) {
  namespace cg = cooperative_groups;
  using Rl = typename RealOf<C>::T;
  constexpr int MW = PC_ROWS / 32;
  cg::cluster_group cl = cg::this_cluster();
  __shared__ __align__(16) C slot[2][MW][NB];
  __shared__ unsigned wkey[2][MW];
  __shared__ unsigned ckey[2];
  __shared__ int pivrow[NB];  // the row chosen at each step when it lives in this CTA, else -1
  __shared__ int pseq[NB], vac[NB];
  const int q = (int)cl.block_rank(), ncta = (int)cl.num_blocks();
  const int z = blockIdx.y, t = threadIdx.x, lane = t & 31, wid = t >> 5;
  const int fmax = L.fmax, R = L.smax - k0, w = k1 - k0;
  const int r = q * PC_ROWS + t;  // own row, local to k0
  C* A = L.F + (size_t)z * fmax * L.ncols + (size_t)k0 * fmax + k0;  // local (r, c) at A[c * fmax + r]
  const bool has = r < R;
  C a[NB];
#pragma unroll
  for (int c = 0; c < NB; ++c) a[c] = (has && c < w) ? A[(size_t)c * fmax + r] : czero<C>();
  if (t < NB) pivrow[t] = -1;
  bool live = has;
  int jp = -1;
#pragma unroll
  for (int j = 0; j < NB; ++j) {
    if (j < w) {
      const int par = j & 1;
      const unsigned mag = __float_as_uint((float)(fabs(a[j].x) + fabs(a[j].y)));
      const unsigned key = live ? ((mag >> 11) << 12) | (4095u - (unsigned)r) : 0u;
      const unsigned kw = __reduce_max_sync(0xffffffffu, key);
      if (live && key == kw) {
        const Rl den = cabs2(a[j]);
        const Rl rden = den > 0 ? recip(den) : (Rl)0;
        C inv;
        inv.x = a[j].x * rden;
        inv.y = -a[j].y * rden;
        slot[par][wid][j] = inv;
#pragma unroll
        for (int c = j + 1; c < NB; ++c) slot[par][wid][c] = a[c];
      }
      if (lane == 0) wkey[par][wid] = kw;
      __syncthreads();
      if (wid == 0) {
        const unsigned kc = __reduce_max_sync(0xffffffffu, lane < MW ? wkey[par][lane] : 0u);
        if (lane == 0) ckey[par] = kc;
      }
      cl.sync();
      const unsigned km = __reduce_max_sync(0xffffffffu, lane < ncta ? *cl.map_shared_rank(&ckey[par], lane) : 0u);
      if (km == 0u) {  // no live row left (cannot happen while j < R)
        if (t == 0 && q == 0) atomicCAS(err, 0, 1);
        continue;
      }
      if ((km >> 12) == 0u && t == 0 && q == 0) atomicCAS(err, 0, 1);  // zero pivot
      const int bi = 4095 - (int)(km & 4095u);
      if (r == bi) {
        live = false;
        jp = j;
        pivrow[j] = r;
      }
      if (live) {
        const C* pr = cl.map_shared_rank(&slot[par][(bi % PC_ROWS) >> 5][0], bi / PC_ROWS);
        const C m = cmul(a[j], pr[j]);
        a[j] = m;
#pragma unroll
        for (int c = j + 1; c < NB; ++c) a[c] = cfms(a[c], m, pr[c]);
      }
    }
  }
  cl.sync();  // every CTA's pivrow is final
  if (q == 0 && wid == 0) {
    int pj = -1;
    if (lane < w)
      for (int p = 0; p < ncta; ++p) {
        const int v = *cl.map_shared_rank(&pivrow[lane], p);
        if (v >= 0) pj = v;
      }
    pseq[lane] = pj;
    // positions >= w vacated by pivots, in increasing order (rank among the vacated rows)
    const bool vp = lane < w && pj >= w;
    int rank = 0;
    for (int i = 0; i < 32; ++i) {
      const int o = __shfl_sync(0xffffffffu, pj, i);
      const bool ov = __shfl_sync(0xffffffffu, vp ? 1 : 0, i) != 0;
      if (ov && o < pj) ++rank;
    }
    vac[lane] = lane;  // unused entries stay in range
    __syncwarp();
    if (vp) vac[rank] = pj;
  }
  __syncthreads();
  cl.sync();  // CTA 0 has finished reading the other CTAs' shared memory
  int pos = r;
  if (jp >= 0) pos = jp;
  int* sw = swp + (size_t)z * SWP_STRIDE;
  if (q == 0 && wid == 0) {
    // rows at positions < w that were not chosen (all in warp 0 of CTA 0)
    const bool dp = has && jp < 0 && r < w;
    const unsigned bd = __ballot_sync(0xffffffffu, dp);
    const int k = __popc(bd & ((1u << lane) - 1u));
    if (dp) {
      pos = min(vac[k], R - 1);
      sw[1 + 2 * (w + k)] = pos;
      sw[2 + 2 * (w + k)] = r;
    }
    // a step without a pivot (singular front, flagged in err) keeps its position
    if (lane < w && pseq[lane] < 0) {
      sw[1 + 2 * lane] = lane;
      sw[2 + 2 * lane] = lane;
    }
    if (lane == 0) sw[0] = w + __popc(bd);
  }
  if (jp >= 0) {
    sw[1 + 2 * jp] = jp;
    sw[2 + 2 * jp] = r;
  }
  if (has) {
#pragma unroll
    for (int c = 0; c < NB; ++c)
      if (c < w) A[(size_t)c * fmax + pos] = a[c];
  }
}

// Columns c in [c0, c1): apply the panel's row permutation given as (position, source)
// pairs local to k0 (k_panel_reg / k_panel_cluster; none when swp is null), then
// F[k0:k1, c] = L_kk^{-1} F[k0:k1, c].
template <typename C> __global__ void __launch_bounds__(128) k_trsm_lower_swp(LevelK<C> L, int k0, int k1, int c0,
                                                                              int c1, const int* __restrict__ swp) {
  const int z = blockIdx.x;
  const int fmax = L.fmax, w = k1 - k0, R = L.smax - k0;
  C* A = L.F + (size_t)z * fmax * L.ncols;
  __shared__ C Ld[NB][NB + 1];
  __shared__ int stop[NB], bpos[NB], bsrc[NB], nb;
  for (int idx = threadIdx.x; idx < w * w; idx += blockDim.x) {
    const int i = idx % w, l = idx / w;
    Ld[i][l] = A[(size_t)(k0 + l) * fmax + k0 + i];
  }
  if (threadIdx.x < NB) stop[threadIdx.x] = threadIdx.x;
  __syncthreads();
  if (threadIdx.x == 0) {
    const int* sw = swp ? swp + (size_t)z * SWP_STRIDE : nullptr;
    const int cnt = sw ? min(sw[0], 2 * NB) : 0;
    int m = 0;
    for (int qq = 0; qq < cnt; ++qq) {
      const int ps = sw[1 + 2 * qq], sr = sw[2 + 2 * qq];
      if (ps < 0 || ps >= R || sr < 0 || sr >= R) continue;
      if (ps < w) stop[ps] = sr;
      else if (m < NB) {
        bpos[m] = ps;
        bsrc[m] = sr;
        ++m;
      }
    }
    nb = m;
  }
  __syncthreads();
  const int c = c0 + blockIdx.y * blockDim.x + threadIdx.x;
  if (c >= c1) return;
  C* col = A + (size_t)c * fmax + k0;
  const int np = nb;
  C x[NB];
#pragma unroll
  for (int i = 0; i < NB; ++i)
    if (i < w) x[i] = col[stop[i]];
  {
    C extra[NB];
#pragma unroll
    for (int i = 0; i < NB; ++i)
      if (i < np) extra[i] = col[bsrc[i]];
#pragma unroll
    for (int i = 0; i < NB; ++i)
      if (i < np) col[bpos[i]] = extra[i];
  }
  // column-oriented (right-looking): x_i final, then every x_r below it updated at once
#pragma unroll
  for (int i = 0; i < NB - 1; ++i) {
    if (i < w) {
#pragma unroll
      for (int r = i + 1; r < NB; ++r)
        if (r < w) x[r] = cfms(x[r], Ld[r][i], x[i]);
    }
  }
#pragma unroll
  for (int i = 0; i < NB; ++i)
    if (i < w) col[i] = x[i];
}

// Row permutations of nrec panels applied in order to the columns [c0, c1) (no solve): record
// q holds (position, source) pairs local to k0 + q NB, as written by k_panel_reg /
// k_panel_cluster.  A block takes AP_COLS columns; a thread moves one entry of one column.
constexpr int AP_COLS = 4;
template <typename C>
__global__ void __launch_bounds__(256) k_apply_swp(LevelK<C> L, int k0, int c0, int c1, const int* __restrict__ swp,
                                                   int nrec, long rec_stride) {
  __shared__ C v[AP_COLS][2 * NB];
  __shared__ int sp[2 * NB], ss[2 * NB], cnt;
  const int z = blockIdx.x, R = L.smax - k0;
  C* A = L.F + (size_t)z * L.fmax * L.ncols;
  const int u = threadIdx.x / (2 * NB), e = threadIdx.x % (2 * NB);
  const int c = c0 + blockIdx.y * AP_COLS + u;
  for (int q = 0; q < nrec; ++q) {
    const int kq = k0 + q * NB;
    __syncthreads();
    if (threadIdx.x == 0) cnt = min(swp[q * rec_stride + (size_t)z * SWP_STRIDE], 2 * NB);
    __syncthreads();
    if (threadIdx.x < cnt) {
      const int* sw = swp + q * rec_stride + (size_t)z * SWP_STRIDE;
      const int ps = sw[1 + 2 * threadIdx.x], sr = sw[2 + 2 * threadIdx.x];
      const bool ok = ps >= 0 && sr >= 0 && kq + ps < k0 + R && kq + sr < k0 + R;
      sp[threadIdx.x] = ok ? kq + ps : -1;
      ss[threadIdx.x] = ok ? kq + sr : -1;
    }
    __syncthreads();
    const bool act = u < AP_COLS && c < c1 && e < cnt && sp[e] >= 0;
    if (act) v[u][e] = A[(size_t)c * L.fmax + ss[e]];
    __syncthreads();
    if (act) A[(size_t)c * L.fmax + sp[e]] = v[u][e];
  }
}

// One warp per column c in [k1, ncols): local rows p = 32 q + lane of [k0, smax) in slot q,
// loaded through the panel's permutation; x_p -= L_pi x_i for i < w, p > i (forward
// substitution inside the block, update below it).  The panel L is staged in shared
// memory as lp[i * R32 + p], R32 = R rounded up to 32, rows R..R32 zero, so that only the
// first slot (p < 32) needs the p > i test.
template <typename C, int RPL>
__global__ void __launch_bounds__(256) k_lower_update(LevelK<C> L, int k0, int k1, const int* __restrict__ swp) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int z = blockIdx.x;
  const int fmax = L.fmax, R = L.smax - k0, w = k1 - k0, R32 = (R + 31) & ~31;
  C* lp = reinterpret_cast<C*>(smem_raw);
  int* perm = reinterpret_cast<int*>(lp + (size_t)w * R32);
  const C* P = L.F + (size_t)z * fmax * L.ncols + (size_t)k0 * fmax + k0;
  stage_copy<8>(lp, w * R32, [&](int e) {
    const int i = e / R32, p = e - i * R32;
    return p < R ? P[(size_t)i * fmax + p] : czero<C>();
  });
  for (int p = threadIdx.x; p < R; p += blockDim.x) perm[p] = p;
  __syncthreads();
  const int* sw = swp + (size_t)z * SWP_STRIDE;
  const int cnt = sw[0];
  for (int q = threadIdx.x; q < cnt; q += blockDim.x) perm[sw[1 + 2 * q]] = sw[2 + 2 * q];
  __syncthreads();
  const int lane = threadIdx.x & 31;
  const int c = k1 + blockIdx.y * (blockDim.x >> 5) + (threadIdx.x >> 5);
  if (c >= L.ncols) return;
  C* col = L.F + (size_t)z * fmax * L.ncols + (size_t)c * fmax + k0;
  C x[RPL];
#pragma unroll
  for (int q = 0; q < RPL; ++q) {
    const int p = 32 * q + lane;
    x[q] = p < R ? col[perm[p]] : czero<C>();
  }
  for (int i = 0; i < w; ++i) {
    const C xi = shfl_c(x[0], i);
    const C* li = lp + (size_t)i * R32 + lane;
    if (lane > i) x[0] = cfms(x[0], li[0], xi);
#pragma unroll
    for (int q = 1; q < RPL; ++q)
      if (32 * q < R32) x[q] = cfms(x[q], li[32 * q], xi);
  }
#pragma unroll
  for (int q = 0; q < RPL; ++q) {
    const int p = 32 * q + lane;
    if (p < R) col[p] = x[q];
  }
}

// One warp per column c in [smax, ncols): x = U11^{-1} x over the own rows, the column in
// registers (row 32 q + lane in slot q); U11 columns [i0, i0 + 32) staged per block as
// us[il * rows + p], their reciprocal pivots in invd.
template <typename C, int RPL>
__global__ void __launch_bounds__(256, 1) k_upper_solve(LevelK<C> L) {
  using Rl = typename RealOf<C>::T;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ C invd[32];
  const int z = blockIdx.x, lane = threadIdx.x & 31;
  const int fmax = L.fmax, smax = L.smax;
  C* us = reinterpret_cast<C*>(smem_raw);
  const C* U = L.F + (size_t)z * fmax * L.ncols;
  const int c = smax + blockIdx.y * (blockDim.x >> 5) + (threadIdx.x >> 5);
  const bool active = c < L.ncols;
  C* col = L.F + (size_t)z * fmax * L.ncols + (size_t)(active ? c : smax) * fmax;
  C x[RPL];
#pragma unroll
  for (int q = 0; q < RPL; ++q) {
    const int p = 32 * q + lane;
    x[q] = (active && p < smax) ? col[p] : czero<C>();
  }
#pragma unroll
  for (int qi = RPL - 1; qi >= 0; --qi) {
    const int i0 = 32 * qi;
    if (i0 < smax) {
      const int iw = min(32, smax - i0), rows = i0 + iw;
      __syncthreads();
      stage_copy<8>(us, iw * rows, [&](int e) {
        const int il = e / rows, p = e - il * rows;
        return U[(size_t)(i0 + il) * fmax + p];
      });
      for (int il = threadIdx.x; il < iw; il += blockDim.x) {
        const C dg = U[(size_t)(i0 + il) * fmax + i0 + il];
        const Rl den = cabs2(dg);
        C inv;
        inv.x = den > 0 ? dg.x / den : (Rl)0;
        inv.y = den > 0 ? -dg.y / den : (Rl)0;
        invd[il] = inv;
      }
      __syncthreads();
      if (active)
        for (int li = iw - 1; li >= 0; --li) {
          C xi = cmul(shfl_c(x[qi], li), invd[li]);
          if (lane == li) x[qi] = xi;
          const C* ui = us + (size_t)li * rows + lane;
#pragma unroll
          for (int q = 0; q < qi; ++q) x[q] = cfms(x[q], ui[32 * q], xi);  // rows p < i0 <= i
          if (lane < li) x[qi] = cfms(x[qi], ui[32 * qi], xi);
        }
    }
  }
  if (active)
#pragma unroll
    for (int q = 0; q < RPL; ++q) {
      const int p = 32 * q + lane;
      if (p < smax) col[p] = x[q];
    }
}

// F[r0:r1, c0:c1] -= F[r0:r1, k0:k1] F[k0:k1, c0:c1], 64 x 64 tiles, K chunks of 16.
template <typename C>
__global__ void __launch_bounds__(256) k_gemm(LevelK<C> L, int r0, int r1, int c0, int c1, int k0, int k1) {
  constexpr int TM = 64, TK = 16;
  const int z = blockIdx.x;
  const int fmax = L.fmax, w = k1 - k0;
  const int nt = (r1 - r0 + TM - 1) / TM;
  const int tr = blockIdx.y % nt, tcb = blockIdx.y / nt;
  const int rb = r0 + tr * TM, cb = c0 + tcb * TM;
  C* A = L.F + (size_t)z * fmax * L.ncols;
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
    {
      // all loads of the two tiles in flight before the shared-memory stores
      constexpr int PER = TK * TM / 256;
      C va[PER], vb[PER];
#pragma unroll
      for (int u = 0; u < PER; ++u) {
        const int idx = threadIdx.x + u * 256;
        const int l = idx / TM, rr = idx % TM;
        va[u] = (l < kw && rb + rr < r1) ? A[(size_t)(k0 + kk + l) * fmax + rb + rr] : czero<C>();
        const int l2 = idx % TK, cc = idx / TK;
        vb[u] = (l2 < kw && cb + cc < c1) ? A[(size_t)(cb + cc) * fmax + k0 + kk + l2] : czero<C>();
      }
#pragma unroll
      for (int u = 0; u < PER; ++u) {
        const int idx = threadIdx.x + u * 256;
        As[idx / TM][idx % TM] = va[u];
        Bs[idx % TK][idx / TK] = vb[u];
      }
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
    const int c = cb + ty + 16 * j;
    if (c >= c1) continue;
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      const int r = rb + tx + 16 * i;
      if (r >= r1) continue;
      C& x = A[(size_t)c * fmax + r];
      x = csub(x, acc[i][j]);
    }
  }
}

// One CTA per front (fronts whose own-row block fits in shared memory): extend-add of the
// children's Schur complements, then Gauss-Jordan elimination with partial pivoting over
// the own rows of [F11 | F12 | I] held in shared memory, which leaves [I | H | F11^{-1}]
// with H = F11^{-1} F12; the ring rows are updated by the tiled GEMM afterwards.
// With ring != 0 the CTA also forms the ring rows' [S | Y] = [F22 | 0] - F21 [H | F11^{-1}]
// (what the level's ring GEMM does otherwise): F21 read from global memory, [H | F11^{-1}]
// from the shared-memory block.
template <typename C>
__global__ void __launch_bounds__(256) k_gauss_jordan(LevelK<C> L, LevelK<C> Ch, int has_child, int* err,
                                                     int ring) {
  using Rl = typename RealOf<C>::T;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  C* B = reinterpret_cast<C*>(smem_raw);  // column major, ld = smax
  const int z = blockIdx.x, tid = threadIdx.x, NT = blockDim.x;
  const int s = L.smax, fmax = L.fmax, nc = L.ncols;
  C* A = L.F + (size_t)z * fmax * nc;
  if (has_child) {
    // extend-add: the child's map is staged in shared memory (the front's own-row buffer
    // is not in use yet), then batches of 4 independent loads per thread
    int* eas = reinterpret_cast<int*>(smem_raw);
    for (int k = 0; k < 2; ++k) {
      const int c = L.child[(size_t)z * 2 + k];
      if (c < 0) continue;
      const C* __restrict__ Fc = Ch.F + (size_t)c * Ch.fmax * Ch.ncols + (size_t)Ch.smax * Ch.fmax + Ch.smax;
      const int cb = Ch.bmax;
      for (int a = tid; a < cb; a += NT) eas[a] = Ch.ea[(size_t)c * cb + a];
      __syncthreads();
      const int tot = cb * cb;
      for (int base = tid; base < tot; base += 4 * NT) {
        C v[4];
        int dst[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) {
          const int idx = base + u * NT;
          dst[u] = -1;
          if (idx < tot) {
            const int a = idx % cb, b = idx / cb;
            const int pa = eas[a], pb = eas[b];
            if (pa >= 0 && pb >= 0) {
              dst[u] = pb * fmax + pa;
              v[u] = Fc[(size_t)b * Ch.fmax + a];
            }
          }
        }
        C o[4];
#pragma unroll
        for (int u = 0; u < 4; ++u)
          if (dst[u] >= 0) o[u] = A[dst[u]];
#pragma unroll
        for (int u = 0; u < 4; ++u)
          if (dst[u] >= 0) A[dst[u]] = cadd(o[u], v[u]);
      }
      __syncthreads();
    }
  }
  // Elimination without moving rows: thread (r, g) updates row r on the columns
  // c = g (mod G); a row chosen as pivot is retired from the pivot search but, as Gauss-
  // Jordan requires, still eliminated in later columns.  Pivot = largest |re| + |im| over
  // the live rows (FP32 bit patterns, warp reductions, lowest row on ties).
  __shared__ unsigned skey[2][8], sidx[2][8];
  __shared__ int pseq_s[1024];
  C* prow = B + (size_t)s * nc;  // normalised pivot row, nc entries
  const int G = NT / s, r = tid % s, g = tid / s;
  const bool act = g < G;
  const int lane = tid & 31, wid = tid >> 5, nw = NT >> 5;
  bool live = act && g == 0;  // one thread per row takes part in the pivot search
  // off = (g - j - 1) mod G: this thread's first column after column j
  int off = G > 0 ? ((g - 1) % G + G) % G : 0;
  // own-row block into shared memory: thread (r, g) copies row r on columns g (mod G),
  // four loads in flight before the stores
  if (act)
    for (int c = g; c < nc; c += 4 * G) {
      C v[4];
#pragma unroll
      for (int u = 0; u < 4; ++u)
        if (c + u * G < nc) v[u] = A[(size_t)(c + u * G) * fmax + r];
#pragma unroll
      for (int u = 0; u < 4; ++u)
        if (c + u * G < nc) B[(size_t)(c + u * G) * s + r] = v[u];
    }
  __syncthreads();
  for (int j = 0; j < s; ++j) {
    const int par = j & 1;
    const C bj = B[(size_t)j * s + r];
    const unsigned key = live ? __float_as_uint((float)(fabs(bj.x) + fabs(bj.y))) : 0u;
    const unsigned kw = __reduce_max_sync(0xffffffffu, key);
    const unsigned iw = __reduce_min_sync(0xffffffffu, (live && key == kw) ? (unsigned)r : 0xffffffffu);
    if (lane == 0) { skey[par][wid] = kw; sidx[par][wid] = iw; }
    __syncthreads();
    const unsigned k2 = lane < nw ? skey[par][lane] : 0u;
    const unsigned km = __reduce_max_sync(0xffffffffu, k2);
    const unsigned bu = __reduce_min_sync(0xffffffffu, (lane < nw && k2 == km) ? sidx[par][lane] : 0xffffffffu);
    const int bi = bu == 0xffffffffu ? 0 : (int)bu;
    if (tid == 0) {
      if (km == 0u || bu == 0xffffffffu) atomicCAS(err, 0, 1);
      pseq_s[j] = bi;
    }
    if (live && r == bi) live = false;
    // normalised pivot row (columns j+1..nc-1) by the threads of row bi; column j of the
    // pivot row is left as it is (every thread reads it for the pivot)
    const C dg = B[(size_t)j * s + bi];
    const Rl den = cabs2(dg);
    const Rl rden = den > 0 ? recip(den) : (Rl)0;
    C inv;
    inv.x = dg.x * rden;
    inv.y = -dg.y * rden;
    if (act && r == bi)
      for (int c = j + 1 + off; c < nc; c += G) {
        const C v = cmul(B[(size_t)c * s + bi], inv);
        prow[c] = v;
        B[(size_t)c * s + bi] = v;
      }
    __syncthreads();
    if (act && r != bi) {
      const C mr = bj;  // B[j][r], read before any update of this step
      int c = j + 1 + off;
      for (; c + 3 * G < nc; c += 4 * G) {
        C pv[4], rv[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) { pv[u] = prow[c + u * G]; rv[u] = B[(size_t)(c + u * G) * s + r]; }
#pragma unroll
        for (int u = 0; u < 4; ++u) B[(size_t)(c + u * G) * s + r] = cfms(rv[u], mr, pv[u]);
      }
      for (; c < nc; c += G) B[(size_t)c * s + r] = cfms(B[(size_t)c * s + r], mr, prow[c]);
    }
    off = off == 0 ? G - 1 : off - 1;
    __syncthreads();
  }
  // row ph[i] holds the result for own row i
  int* ph = reinterpret_cast<int*>(prow + nc);
  int* iph = ph + s;
  for (int i = tid; i < s; i += NT) { ph[i] = i; iph[i] = i; }
  __syncthreads();
  if (tid == 0)
    for (int j = 0; j < s; ++j) {
      const int bi = pseq_s[j], pj = ph[j], lb = iph[bi];
      ph[j] = bi;
      iph[bi] = j;
      ph[lb] = pj;
      iph[pj] = lb;
    }
  __syncthreads();
  if (act) {
    const int src = ph[r];
    for (int c = s + g; c < nc; c += G) A[(size_t)c * fmax + r] = B[(size_t)c * s + src];
  }
  if (ring) {
    // ring row i, column c: consecutive threads take consecutive ring rows (coalesced F21
    // and F22 accesses); own row k of [H | F11^{-1}] is row ph[k] of the block
    const int b = fmax - s, nco = nc - s;
    for (int t = tid; t < b * nco; t += NT) {
      const int i = s + t % b, c = s + t / b;
      C acc = A[(size_t)c * fmax + i];
      for (int k = 0; k < s; ++k) acc = cfms(acc, A[(size_t)k * fmax + i], B[(size_t)c * s + ph[k]]);
      A[(size_t)c * fmax + i] = acc;
    }
  }
}

template <typename C> LevelK<C> level_k(NdPlan* p, int l) {
  const LevelDev& D = p->lev[l];
  LevelK<C> k;
  k.F = reinterpret_cast<C*>(p->F) + D.F_off;
  k.W = reinterpret_cast<C*>(p->W) + D.W_off;
  k.nf = D.nf; k.smax = D.smax; k.bmax = D.bmax; k.fmax = D.fmax; k.ncols = D.ncols;
  k.own = D.own; k.ring = D.ring; k.child = D.child; k.parent = D.parent; k.kidx = D.kidx; k.ea = D.ea;
  k.piv = D.piv;
  return k;
}

// Launch shape of one level of a solve sweep: rows per tile, tiles, and how many column
// ranges each tile is split into so that about two CTAs per SM have work (ranges of at
// least 64 columns: below that the extra partial-sum pass costs more than it saves).
struct SweepPlan {
  int K, tr, ntile, nsplit, ksz;
};
static SweepPlan sweep_plan(const LevelDev& D, int mode, int ng, int ctas_per_sm) {
  SweepPlan q;
  q.K = mode == 0 ? D.smax : D.bmax + D.smax;
  const int nrows = mode == 0 ? D.bmax : D.smax;
  q.tr = nrows <= 16 ? 16 : 32;
  q.ntile = std::max(1, (nrows + q.tr - 1) / q.tr);
  const long base = (long)D.nf * q.ntile * ng;
  q.nsplit = 1;
  if (nrows > 0)
    while (base * q.nsplit < (long)ctas_per_sm * 152 && q.K / (q.nsplit * 2) >= 64) q.nsplit *= 2;
  q.ksz = q.K > 0 ? (q.K + q.nsplit - 1) / q.nsplit : 0;
  return q;
}

static bool ensure_buffers(NdPlan* p, int elem_bytes, cudaStream_t st) {
  if (p->F && p->F_bytes == elem_bytes) return false;
  if (p->F) { dev_free(p->F); p->F = nullptr; }
  if (p->W) { dev_free(p->W); p->W = nullptr; }
  if (p->T) { dev_free(p->T); p->T = nullptr; }
  p->F = dev_alloc(p->F_elems * elem_bytes);
  p->W = dev_alloc(std::max<size_t>(1, p->W_elems) * elem_bytes);
  p->T = dev_alloc((size_t)p->N * SOLVE_CHUNK * elem_bytes);
  int nf_max = 1;
  for (const LevelDev& D : p->lev) nf_max = std::max(nf_max, D.nf);
  // solve partial sums: the largest split level, for any number of right-hand-side groups
  size_t part = 1, items = 1;
  for (const LevelDev& D : p->lev)
    for (int mode = 0; mode < 2; ++mode)
      for (int ng = 1; ng <= SOLVE_CHUNK / 16; ++ng) {
        const SweepPlan q = sweep_plan(D, mode, ng, SWEEP_CTAS_MAX);
        items = std::max(items, (size_t)D.nf * q.ntile * ng);
        if (q.nsplit > 1) part = std::max(part, (size_t)D.nf * q.ntile * q.nsplit * q.tr * 16 * ng);
      }
  if (p->part) { dev_free(p->part); p->part = nullptr; }
  if (p->cnt) { dev_free(p->cnt); p->cnt = nullptr; }
  p->part = dev_alloc(part * elem_bytes);
  p->cnt = static_cast<unsigned*>(dev_alloc(items * sizeof(unsigned)));
  if (p->tcs_B) { dev_free(p->tcs_B); p->tcs_B = nullptr; }
  if (p->tcs_C) { dev_free(p->tcs_C); p->tcs_C = nullptr; }
  p->tcs_B_elems = p->tcs_C_elems = 0;
  if (elem_bytes == 8) {
    tcs_sizes(p->lev, &p->tcs_B_elems, &p->tcs_C_elems);
    if (p->tcs_B_elems) p->tcs_B = static_cast<float2*>(dev_alloc(p->tcs_B_elems * sizeof(float2)));
    if (p->tcs_C_elems) p->tcs_C = static_cast<float2*>(dev_alloc(p->tcs_C_elems * sizeof(float2)));
  }
  LS_CUDA(cudaMemsetAsync(p->cnt, 0, items * sizeof(unsigned), st));
  p->part_elems = part;
  if (p->swp) { dev_free(p->swp); p->swp = nullptr; }
  p->swp = static_cast<int*>(dev_alloc((size_t)OB_PANELS * nf_max * SWP_STRIDE * sizeof(int)));
  p->F_bytes = p->W_bytes = elem_bytes;
  return true;
}

// threads for the Gauss-Jordan CTA: about 16 entries of the own-row block per thread
static int gj_threads(int s, int nc) {
  const int t = ((s * nc / 16 + 31) / 32) * 32;
  return std::max((s + 31) / 32 * 32, std::min(256, std::max(32, t)));
}

// shared memory of the Gauss-Jordan CTA: own-row block, normalised pivot row, row order
template <typename C> static size_t gj_smem(int s, int nc) {
  return ((size_t)s * nc + nc) * sizeof(C) + 2 * (size_t)s * sizeof(int);
}

// FP32 products with at least this many rows and k go to the tensor cores (3xTF32)
constexpr int TC_MIN_ROWS = 64, TC_MIN_K = 16;

// tc: the launch-shape choices when the tensor cores may take the product, else null
// whether a Schur product of this many rows and inner columns runs on the tensor cores
template <typename C> static bool gemm_on_tc(int rows, int k, const NdTune* tc) {
  return sizeof(C) == 8 && tc && rows >= std::max(tc->tc_min_rows, TC_MIN_ROWS) && k >= TC_MIN_K && tc_enabled();
}

template <typename C> static void launch_gemm(const LevelK<C>& L, int r0, int r1, int c0, int c1, int k0, int k1,
                                              cudaStream_t st, int* err, const NdTune* tc) {
  if (r1 <= r0 || c1 <= c0 || k1 <= k0) return;
  if constexpr (sizeof(C) == 8) {
    if (gemm_on_tc<C>(r1 - r0, k1 - k0, tc)) {
      tc_cgemm(reinterpret_cast<float2*>(L.F), (long)L.fmax * L.ncols, L.fmax, L.nf, r0, r1, c0, c1, k0, k1, err, st);
      return;
    }
  }
  const int nr = (r1 - r0 + 63) / 64, nc = (c1 - c0 + 63) / 64;
  LS_LAUNCH(sizeof(C) == 8 ? "nd_gemm_c64" : "nd_gemm_c128", st,
            k_gemm<C><<<dim3(L.nf, nr * nc), 256, 0, st>>>(L, r0, r1, c0, c1, k0, k1));
}

template <typename C> bool nd_prepare(NdPlan* p, cudaStream_t st) { return ensure_buffers(p, sizeof(C), st); }

void nd_set_tensor_cores(NdPlan* p, bool on) { p->use_tc = on; }
void nd_set_tune(NdPlan* p, const NdTune& t) { p->tune = t; }
NdTune nd_get_tune(const NdPlan* p) { return p->tune; }

// own rows per lane of the register sweeps (32 * this many own rows at most)
template <typename C> constexpr int reg_rpl_max() { return sizeof(C) == 8 ? 16 : 8; }

template <typename C, int RPL>
static void reg_sweeps(const LevelK<C>& L, int* swp, int* err, const NdTune* tc, cudaStream_t st) {
  const bool f32 = sizeof(C) == 8;
  const size_t smem_max = (size_t)32 * 32 * RPL * sizeof(C) + (size_t)32 * RPL * sizeof(int);
  static std::atomic<bool> attr{false};  // set once per process; repeats are harmless
  if (!attr.load(std::memory_order_acquire)) {
    LS_CUDA(cudaFuncSetAttribute(k_lower_update<C, RPL>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_max));
    LS_CUDA(cudaFuncSetAttribute(k_upper_solve<C, RPL>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_max));
    attr.store(true, std::memory_order_release);
  }
  static_assert(32 * RPL <= panel_reg_rows<C>(), "the register panel holds every own row");
  for (int k0 = 0; k0 < L.smax; k0 += NB) {
    const int k1 = std::min(k0 + NB, L.smax), R = L.smax - k0;
    const int r32 = (R + 31) / 32 * 32;
    LS_LAUNCH(f32 ? "nd_panel_c64" : "nd_panel_c128", st, k_panel_reg<C><<<L.nf, r32, 0, st>>>(L, k0, k1, swp, err));
    launch_ring_trsm<C>(L, k0, k1, st);
    const int m = L.ncols - k1;
    const size_t smem = (size_t)(k1 - k0) * r32 * sizeof(C) + (size_t)R * sizeof(int);
    LS_LAUNCH(f32 ? "nd_trsm_c64" : "nd_trsm_c128", st,
              k_lower_update<C, RPL><<<dim3(L.nf, (m + 7) / 8), 256, smem, st>>>(L, k0, k1, swp));
    // the ring rows' own-column entries right of the panel (the later panels' multipliers)
    launch_gemm<C>(L, L.smax, L.fmax, k1, L.smax, k0, k1, st, err, tc);
  }
  // ring rows: [S | Y] = [F22 | 0] - L21 [U12 | L11^{-1} P], before sweep 2 overwrites the own
  // rows of [F12 | I]
  launch_gemm<C>(L, L.smax, L.fmax, L.smax, L.ncols, 0, L.smax, st, err, tc);
  const int m = L.ncols - L.smax;
  const size_t smem = (size_t)32 * L.smax * sizeof(C);
  LS_LAUNCH(f32 ? "nd_trsm_c64" : "nd_trsm_c128", st, k_upper_solve<C, RPL><<<dim3(L.nf, (m + 7) / 8), 256, smem, st>>>(L));
}

template <typename C>
void nd_factor(NdPlan* p, const void* alpha64, const void* cint64, const void* w2m64, cudaStream_t st) {
  nd_prepare<C>(p, st);
  nd_factor_launch<C>(p, alpha64, cint64, w2m64, st, nullptr, nullptr, nullptr);
  nd_factor_check(p, st);
}

void nd_factor_check(NdPlan* p, cudaStream_t st) {
  int err = 0;
  LS_CUDA(cudaMemcpyAsync(&err, p->d_err, sizeof(int), cudaMemcpyDeviceToHost, st));
  LS_CUDA(cudaStreamSynchronize(st));
  // a singular pivot only claims the flag while it is clear (atomicCAS), an expired wait
  // always takes it (atomicExch): a timeout is reported even when the fronts it left
  // unupdated later give a zero pivot
  if (err == 2) LS_FAIL(ETIMEOUT_, "a bounded wait of the tensor-core front update expired");
  if (err) LS_FAIL(EINVAL_, "nested-dissection factorization met an exactly singular front");
}

// an event other streams can wait on, also from inside a stream capture (as an event node)
static void record_marker(cudaEvent_t ev, cudaStream_t st) {
  cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
  LS_CUDA(cudaStreamIsCapturing(st, &cs));
  if (cs == cudaStreamCaptureStatusActive) LS_CUDA(cudaEventRecordWithFlags(ev, st, cudaEventRecordExternal));
  else LS_CUDA(cudaEventRecord(ev, st));
}

template <typename C>
void nd_factor_launch(NdPlan* p, const void* alpha64, const void* cint64, const void* w2m64, cudaStream_t st,
                      cudaEvent_t top_levels, const void* alpha_pt64, const unsigned char* inter_pt) {
  if (!p->F || p->F_bytes != (int)sizeof(C)) LS_FAIL(ESTATE_, "front storage not prepared for this precision");
  const bool f32 = sizeof(C) == 8;
  LS_CUDA(cudaMemsetAsync(p->F, 0, p->F_elems * sizeof(C), st));
  LS_CUDA(cudaMemsetAsync(p->d_err, 0, sizeof(int), st));
  LS_LAUNCH(f32 ? "nd_assemble_c64" : "nd_assemble_c128", st,
            k_assemble<C><<<1024, 256, 0, st>>>(reinterpret_cast<C*>(p->F), p->n_asm, p->d_asm_off, p->d_asm_row,
                                                p->d_asm_t, p->d, p->n, (const double2*)alpha64,
                                                (const double2*)cint64, (const double*)w2m64,
                                                (const double2*)alpha_pt64, inter_pt));
  LS_LAUNCH(f32 ? "nd_ones_c64" : "nd_ones_c128", st,
            k_set_one<C><<<256, 256, 0, st>>>(reinterpret_cast<C*>(p->F), p->n_one, p->d_one_off));
  const int depth = (int)p->lev.size();
  constexpr size_t PANEL_SMEM_MAX = 200 * 1024;
  constexpr int REG_MAX_COLS = 1024;
  constexpr size_t GJ_SMEM_MAX = 160 * 1024;
  static std::atomic<bool> attr{false};  // set once per process; repeats are harmless
  if (!attr.load(std::memory_order_acquire)) {
    LS_CUDA(cudaFuncSetAttribute(k_panel<C, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)PANEL_SMEM_MAX));
    LS_CUDA(cudaFuncSetAttribute(k_gauss_jordan<C>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)GJ_SMEM_MAX));
    attr.store(true, std::memory_order_release);
  }
  bool marked = top_levels == nullptr;
  const NdTune* tcp = p->use_tc ? &p->tune : nullptr;
  for (int l = depth - 1; l >= 0; --l) {
    prof_tag(l);
    LevelK<C> L = level_k<C>(p, l);
    const bool has_child = l + 1 < depth;
    LevelK<C> Ch = has_child ? level_k<C>(p, l + 1) : L;
    if (!marked && L.nf <= 32) {
      // the levels from here to the root run on few SMs: work on other streams may start
      record_marker(top_levels, st);
      marked = true;
    }
    // own rows: [F11 | F12 | I] -> [* | H | F11^{-1}]
    const size_t gjm = gj_smem<C>(L.smax, L.ncols);
    // the children's Schur complements: by a GPU-wide kernel, or inside the Gauss-Jordan
    // CTA when they are small (one CTA per front would serialise large ones)
    // Gauss-Jordan in one CTA for the small fronts (up to 16 own rows); the register sweeps,
    // whose trailing updates spread over many CTAs, for the larger ones (measured on 2D
    // n = 256: 1 % faster with the 32-row levels on the register path, 6 % slower with
    // the 8- and 16-row levels there too)
    const bool gj = gjm <= GJ_SMEM_MAX && (L.smax <= p->tune.gj_max_own || L.smax > 32 * reg_rpl_max<C>());
    const bool fused_ea = gj && has_child && Ch.bmax < 48;
    if (has_child && !fused_ea) {
      const long tot = (long)Ch.bmax * Ch.bmax;
      const unsigned bx = (unsigned)std::max<long>(1, std::min<long>((tot + 1023) / 1024, 64));
      for (int k = 0; k < 2; ++k)
        LS_LAUNCH(f32 ? "nd_extend_add_c64" : "nd_extend_add_c128", st,
                  k_extend_add<C><<<dim3(Ch.nf, bx), 256, 0, st>>>(L, Ch, k));
    }
    if (gj) {
      // one CTA per front: Gauss-Jordan in shared memory (with the extend-add if fused), and
      // the ring rows' product in the same CTA unless it goes to the tensor cores
      const bool ring_tc = gemm_on_tc<C>(L.bmax, L.smax, tcp);
      LS_LAUNCH(f32 ? "nd_gauss_jordan_c64" : "nd_gauss_jordan_c128", st,
                k_gauss_jordan<C><<<L.nf, gj_threads(L.smax, L.ncols), gjm, st>>>(L, Ch, fused_ea ? 1 : 0,
                                                                                   p->d_err, ring_tc ? 0 : 1));
      if (ring_tc) launch_gemm<C>(L, L.smax, L.fmax, L.smax, L.ncols, 0, L.smax, st, p->d_err, tcp);
      continue;
    }
    // The register sweeps update every trailing column on CUDA cores from a panel staged per
    // block; fronts with many columns (3D levels with thousands of ring rows) take the
    // blocked path, whose trailing updates are tensor-core GEMMs.
    if (L.smax <= 32 * reg_rpl_max<C>() && L.ncols <= REG_MAX_COLS) {
      // both sweeps with the fronts' own rows in registers
      const int rpl = (L.smax + 31) / 32;
      if (rpl <= 4) reg_sweeps<C, 4>(L, p->swp, p->d_err, tcp, st);
      else if (rpl <= 8) reg_sweeps<C, 8>(L, p->swp, p->d_err, tcp, st);
      else reg_sweeps<C, reg_rpl_max<C>()>(L, p->swp, p->d_err, tcp, st);
    } else {
      // sweep 1: blocked LU of the own columns on the own rows (pivot rows restricted to
      // them), the block rows of [F12 | I] carried along.  Outer blocks of OB_PANELS panels:
      // when the block's panels record their permutations as pairs (register panel up to
      // panel_reg_rows rows, cluster panel up to PC_CTAS * PC_ROWS rows in FP32), the columns
      // right of the block receive all the block's permutations, then the triangular solve
      // with the block's unit lower L11 panel by panel, then one trailing GEMM with
      // K = OB_PANELS * NB (a quarter of the passes over the trailing matrix); otherwise
      // (the shared- or global-memory panel with LAPACK-style swaps) every panel updates
      // all trailing columns.
      const long rs = (long)L.nf * SWP_STRIDE;  // one swp record per panel of an outer block
      for (int K0 = 0; K0 < L.smax; K0 += OB_PANELS * NB) {
        const int K1 = std::min(K0 + OB_PANELS * NB, L.smax), R0 = L.smax - K0;
        const bool pairs = R0 <= panel_reg_rows<C>() || (f32 && (R0 + PC_ROWS - 1) / PC_ROWS <= PC_CTAS);
        if (!pairs) {
          for (int k0 = K0; k0 < K1; k0 += NB) {
            const int k1 = std::min(k0 + NB, L.smax), R = L.smax - k0, m = L.ncols - k1;
            const size_t psm = (size_t)R * (k1 - k0) * sizeof(C);
            if (psm <= PANEL_SMEM_MAX)
              LS_LAUNCH(f32 ? "nd_panel_c64" : "nd_panel_c128", st,
                        k_panel<C, true><<<L.nf, 512, psm, st>>>(L, k0, k1, p->d_err));
            else
              LS_LAUNCH(f32 ? "nd_panel_c64" : "nd_panel_c128", st,
                        k_panel<C, false><<<L.nf, 512, 0, st>>>(L, k0, k1, p->d_err));
            launch_ring_trsm<C>(L, k0, k1, st);
            LS_LAUNCH(f32 ? "nd_trsm_c64" : "nd_trsm_c128", st,
                      k_trsm_lower<C><<<dim3(L.nf, (m + 127) / 128), 128, 0, st>>>(L, k0, k1));
            launch_gemm<C>(L, k1, L.smax, k1, L.ncols, k0, k1, st, p->d_err, tcp);
            launch_gemm<C>(L, L.smax, L.fmax, k1, L.smax, k0, k1, st, p->d_err, tcp);
          }
          continue;
        }
        // two levels only where the trailing matrix is large: below about 8 M entries per
        // level the extra launches cost more than the passes they save (2D n = 1024)
        const bool two = (double)L.nf * R0 * (L.ncols - K0) >= p->tune.two_level_min;
        int np = 0;
        for (int k0 = K0; k0 < K1; k0 += NB, ++np) {
          const int k1 = std::min(k0 + NB, K1), R = L.smax - k0;
          int* rec = p->swp + (two ? np : 0) * rs;
          if (R <= panel_reg_rows<C>()) {
            LS_LAUNCH(f32 ? "nd_panel_c64" : "nd_panel_c128", st,
                      k_panel_reg<C><<<L.nf, (R + 31) / 32 * 32, 0, st>>>(L, k0, k1, rec, p->d_err));
          } else if constexpr (sizeof(C) == 8) {
            const int ncta = (R + PC_ROWS - 1) / PC_ROWS;
            cudaLaunchConfig_t cfg = {};
            cfg.gridDim = dim3(ncta, L.nf);
            cfg.blockDim = dim3(PC_ROWS);
            cfg.stream = st;
            cudaLaunchAttribute at[1];
            at[0].id = cudaLaunchAttributeClusterDimension;
            at[0].val.clusterDim.x = ncta;
            at[0].val.clusterDim.y = 1;
            at[0].val.clusterDim.z = 1;
            cfg.attrs = at;
            cfg.numAttrs = 1;
            LS_LAUNCH("nd_panel_c64", st, LS_CUDA(cudaLaunchKernelEx(&cfg, k_panel_cluster<C>, L, k0, k1, rec, p->d_err)));
          }
          launch_ring_trsm<C>(L, k0, k1, st);
          if (!two) {
            // one level: permutation and forward substitution of every trailing column, then
            // the trailing GEMM with K = NB
            LS_LAUNCH(f32 ? "nd_trsm_c64" : "nd_trsm_c128", st,
                      k_trsm_lower_swp<C><<<dim3(L.nf, (L.ncols - k1 + 127) / 128), 128, 0, st>>>(L, k0, k1, k1,
                                                                                                 L.ncols, rec));
            launch_gemm<C>(L, k1, L.smax, k1, L.ncols, k0, k1, st, p->d_err, tcp);
            launch_gemm<C>(L, L.smax, L.fmax, k1, L.smax, k0, k1, st, p->d_err, tcp);
            continue;
          }
          // the block's earlier L columns follow this panel's permutation
          if (k0 > K0)
            LS_LAUNCH(f32 ? "nd_trsm_c64" : "nd_trsm_c128", st,
                      k_apply_swp<C><<<dim3(L.nf, (k0 - K0 + AP_COLS - 1) / AP_COLS), 256, 0, st>>>(L, k0, K0, k0, rec,
                                                                                                    1, rs));
          // the rest of the block: permutation, forward substitution, update below
          if (k1 < K1) {
            LS_LAUNCH(f32 ? "nd_trsm_c64" : "nd_trsm_c128", st,
                      k_trsm_lower_swp<C><<<dim3(L.nf, (K1 - k1 + 127) / 128), 128, 0, st>>>(L, k0, k1, k1, K1, rec));
            launch_gemm<C>(L, k1, L.fmax, k1, K1, k0, k1, st, p->d_err, tcp);
          }
        }
        if (two && K1 < L.ncols) {
          const int m = L.ncols - K1;
          LS_LAUNCH(f32 ? "nd_trsm_c64" : "nd_trsm_c128", st,
                    k_apply_swp<C><<<dim3(L.nf, (m + AP_COLS - 1) / AP_COLS), 256, 0, st>>>(L, K0, K1, L.ncols, p->swp,
                                                                                             np, rs));
          for (int q = 0; q < np; ++q) {
            const int k0 = K0 + q * NB, k1 = std::min(k0 + NB, K1);
            LS_LAUNCH(f32 ? "nd_trsm_c64" : "nd_trsm_c128", st,
                      k_trsm_lower_swp<C><<<dim3(L.nf, (m + 127) / 128), 128, 0, st>>>(L, k0, k1, K1, L.ncols,
                                                                                       (const int*)nullptr));
            launch_gemm<C>(L, k1, K1, K1, L.ncols, k0, k1, st, p->d_err, tcp);
          }
          launch_gemm<C>(L, K1, L.smax, K1, L.ncols, K0, K1, st, p->d_err, tcp);
          launch_gemm<C>(L, L.smax, L.fmax, K1, L.smax, K0, K1, st, p->d_err, tcp);
        }
      }
      // ring rows: [S | Y] = [F22 | 0] - L21 [U12 | L11^{-1} P], before sweep 2 overwrites the
      // own rows of [F12 | I]
      launch_gemm<C>(L, L.smax, L.fmax, L.smax, L.ncols, 0, L.smax, st, p->d_err, tcp);
      // sweep 2: backward substitution with U11 on the own rows of [F12 | I], in outer
      // blocks of OB_PANELS row blocks: inside a block each 32-row solve updates the block's
      // rows above it, then one GEMM with K = OB_PANELS * NB updates the rows above the block
      const int nblk = (L.smax + NB - 1) / NB;
      const int m2 = L.ncols - L.smax;
      for (int ob = (nblk - 1) / OB_PANELS; ob >= 0; --ob) {
        const int J0 = ob * OB_PANELS * NB, J1 = std::min(J0 + OB_PANELS * NB, L.smax);
        for (int jb = (J1 - 1) / NB; jb >= J0 / NB; --jb) {
          const int j0 = jb * NB, j1 = std::min(j0 + NB, L.smax);
          LS_LAUNCH(f32 ? "nd_trsm_c64" : "nd_trsm_c128", st,
                    k_trsm_upper<C><<<dim3(L.nf, (m2 + 127) / 128), 128, 0, st>>>(L, j0, j1));
          launch_gemm<C>(L, J0, j0, L.smax, L.ncols, j0, j1, st, p->d_err, tcp);
        }
        launch_gemm<C>(L, 0, J0, L.smax, L.ncols, J0, J1, st, p->d_err, tcp);
      }
    }
  }
  if (!marked) record_marker(top_levels, st);
  prof_tag(-1);
}

// ---------------------------------------------------------------------------------------
// solves
// ---------------------------------------------------------------------------------------
// The two sweeps of the multifrontal solve with the factored fronts, one launch per level:
//   forward (leaves to root):  w_own  = r_own + the children's updates at the own positions,
//                              u_ring = the children's updates at the ring positions + Y w_own;
//   backward (root to leaves): x_own  = F11^{-1} w_own - H x_ring.
// Vectors move as items: the RC right-hand sides of one grid point or one front position
// are contiguous (RC * sizeof(C) bytes, copied as 16-byte pieces).  T holds r at the grid
// points on the way down and x on the way up: every grid point is own in exactly one front
// and the backward sweep reads only ring points, which ancestors own and have written.
// W holds, per level, group of RC right-hand sides and front, [w_own | u_ring].
// Every launch of a solve is a programmatic dependent of the one before: its prologue
// (index loads and the first chunk of the factor tile, all written by the factorization,
// which completed before the solve's first kernel started) overlaps the previous level's
// tail, and griddepcontrol.wait orders every read of T and W after the previous level.
// Reads of T and W bypass L1 (ld.global.cg).

template <typename C> struct Piece;
template <> struct Piece<float2> { using T = float4; };
template <> struct Piece<double2> { using T = double2; };

__device__ __forceinline__ float4 padd(float4 a, float4 b) {
  return make_float4(a.x + b.x, a.y + b.y, a.z + b.z, a.w + b.w);
}
__device__ __forceinline__ double2 padd(double2 a, double2 b) { return make_double2(a.x + b.x, a.y + b.y); }
template <typename P> __device__ __forceinline__ P pzero() {
  P p;
  memset(&p, 0, sizeof(P));
  return p;
}

__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;\n" ::: "memory"); }
__device__ __forceinline__ void pdl_trigger() { asm volatile("griddepcontrol.launch_dependents;\n" ::: "memory"); }

// asynchronous global -> shared copy of one element; a row outside the tile is zero-filled
template <int B> __device__ __forceinline__ void cp_async_elem(void* dst, const void* src, bool valid) {
  const unsigned s = (unsigned)__cvta_generic_to_shared(dst);
  const int nb = valid ? B : 0;
  if constexpr (B == 16)
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;\n" ::"r"(s), "l"(src), "r"(nb) : "memory");
  else
    asm volatile("cp.async.ca.shared.global [%0], [%1], %2, %3;\n" ::"r"(s), "l"(src), "n"(B), "r"(nb) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
template <int N> __device__ __forceinline__ void cp_async_wait() { asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory"); }

template <typename C> struct SweepK {
  const C* F;       // factored fronts of this level
  C* W;             // front vectors of this level
  const C* Wc;      // front vectors of the child level (forward)
  C* T;             // grid-point items
  const int *own, *ring, *fsrc;
  int nf, smax, bmax, fmax, ncols;
  int nf_c, fmax_c;  // child level: fronts and front size (group stride of Wc)
  int ntile;         // row tiles per front
  int nsplit;        // column ranges per row tile; their partial sums are added in range
                     // order by the CTA that finishes last
  int ksz;           // columns per range
  int kv;            // items of the vector operand held in shared memory at once
  int ng;            // groups of RC right-hand sides: the CTAs of one front's groups are
                     // adjacent in the grid (x = front * ng + group), so that its factor tile
                     // is read from DRAM once and from L2 by the other groups
  C* part;           // nsplit > 1: partial sums [item][nsplit][tile rows x RC]
  unsigned* cnt;     // nsplit > 1: CTAs finished per item (the last one resets it)
  long N;
};

// columns of the factor tile per chunk, and the largest vector operand staged whole
template <typename C> __host__ __device__ constexpr int sweep_ka() { return sizeof(C) == 8 ? 128 : 64; }
constexpr size_t SWEEP_VS_MAX = 64 * 1024;
constexpr size_t SWEEP_SMEM_MAX = 200 * 1024;

struct SweepShape {
  int kv, kg, nbuf, kc0;
  size_t region0, smem;  // region0 in elements
};

// shared-memory layout of one CTA working on a column range of ksz columns; TR rows per
// tile (32: one row per lane, all RC right-hand sides per thread; 16: lanes 0-15 and 16-31
// take the two halves of the right-hand sides)
template <typename C, int RC, int TR, int MODE> __host__ __device__ SweepShape sweep_shape(int ksz, int kg_in) {
  SweepShape s;
  constexpr int KA = sweep_ka<C>();
  constexpr int RCT = RC * TR / 32;
  s.kc0 = ksz < KA ? ksz : KA;
  s.nbuf = ksz > KA ? 2 : 1;
  s.kv = (size_t)ksz * RC * sizeof(C) <= SWEEP_VS_MAX ? ksz : KA;
  if (kg_in > 0) s.kg = kg_in;
  // one warp up to 32 columns (its sums are final, no cross-warp reduction), else about
  // 16 columns per warp up to 8 warps
  else s.kg = ksz > KA ? 8 : (ksz <= 32 ? 1 : (ksz / 16 > 8 ? 8 : ksz / 16));
  const size_t a = (size_t)s.nbuf * s.kc0 * TR + (size_t)s.kv * RC;
  const size_t red = (size_t)s.kg * 32 * (RCT + 1);
  s.region0 = a > red ? a : red;
  const size_t wt = MODE == 0 ? (size_t)TR * RC : 0;
  const size_t idx = MODE == 0 ? 3 * (size_t)s.kv + 2 * TR : (size_t)s.kv + TR;
  s.smem = (s.region0 + wt) * sizeof(C) + idx * sizeof(int);
  return s;
}

// vector operand items [c0, c0 + kc) of one front into dst (item-major, RC per item);
// forward: w_own (also stored to W by the first row tile); backward: [x_ring | w_own].
// ixs: the staged indices of these items, or null (read from the index arrays)
template <typename C, int RC, int MODE>
__device__ __forceinline__ void sweep_gather(const SweepK<C>& S, int z, int g, int c0, int kc, const int* ixs,
                                             C* dst, bool write_own) {
  using P = typename Piece<C>::T;
  constexpr int NV = RC * (int)sizeof(C) / 16;
  constexpr int B = 4;  // pieces per thread with their loads in flight together
  const size_t wrow = (size_t)g * S.nf * S.fmax + (size_t)z * S.fmax;
  const size_t cg = (size_t)g * S.nf_c * S.fmax_c;
  const int tot = kc * NV;
  for (int base = threadIdx.x; base < tot; base += blockDim.x * B) {
    P s[B];
#pragma unroll
    for (int q = 0; q < B; ++q) {
      const int u = base + q * blockDim.x;
      s[q] = pzero<P>();
      if (u >= tot) continue;
      const int ci = u / NV, v = u % NV, c = c0 + ci;
      if (MODE == 0) {
        int pt, s0, s1;
        if (ixs) {
          pt = ixs[3 * ci];
          s0 = ixs[3 * ci + 1];
          s1 = ixs[3 * ci + 2];
        } else {
          pt = __ldg(S.own + (size_t)z * S.smax + c);
          s0 = __ldg(S.fsrc + ((size_t)z * S.fmax + c) * 2);
          s1 = __ldg(S.fsrc + ((size_t)z * S.fmax + c) * 2 + 1);
        }
        P a = pzero<P>(), b = pzero<P>(), r = pzero<P>();
        if (pt >= 0) r = __ldcg(reinterpret_cast<const P*>(S.T + ((size_t)g * S.N + pt) * RC) + v);
        if (s0 >= 0) a = __ldcg(reinterpret_cast<const P*>(S.Wc + (cg + s0) * RC) + v);
        if (s1 >= 0) b = __ldcg(reinterpret_cast<const P*>(S.Wc + (cg + s1) * RC) + v);
        s[q] = padd(padd(r, a), b);
      } else if (c < S.bmax) {
        const int pt = ixs ? ixs[ci] : __ldg(S.ring + (size_t)z * S.bmax + c);
        if (pt >= 0) s[q] = __ldcg(reinterpret_cast<const P*>(S.T + ((size_t)g * S.N + pt) * RC) + v);
      } else {
        s[q] = __ldcg(reinterpret_cast<const P*>(S.W + (wrow + c - S.bmax) * RC) + v);
      }
    }
#pragma unroll
    for (int q = 0; q < B; ++q) {
      const int u = base + q * blockDim.x;
      if (u >= tot) continue;
      reinterpret_cast<P*>(dst)[u] = s[q];
      if (MODE == 0 && write_own) reinterpret_cast<P*>(S.W + (wrow + c0 + u / NV) * RC)[u % NV] = s[q];
    }
  }
}

// One level of either sweep.  grid (fronts x groups of RC right-hand sides, row tiles x
// column ranges); the kg warps split the columns of each chunk and add their partial
// sums in a fixed order.  Forward rows are the ring rows of Y (the identity columns of the
// augmented front); backward rows are the own rows of [H | F11^{-1}].
template <typename C, int RC, int TR, int MODE> __global__ void __launch_bounds__(256) k_sweep(SweepK<C> S) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ int last_s;
  constexpr int KA = sweep_ka<C>();
  constexpr int RCT = RC * TR / 32;
  const int z = blockIdx.x / S.ng, g = blockIdx.x - (blockIdx.x / S.ng) * S.ng;
  const int tile = blockIdx.y / S.nsplit, sp = blockIdx.y - tile * S.nsplit;
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, kg = blockDim.x >> 5, NT = blockDim.x;
  const int row = TR == 32 ? lane : (lane & 15);
  const int j0 = TR == 32 ? 0 : (lane >> 4) * RCT;
  const int smax = S.smax, bmax = S.bmax, fmax = S.fmax;
  const int K = MODE == 0 ? smax : bmax + smax;
  const int kb = sp * S.ksz, ke = min(K, kb + S.ksz), Kr = ke - kb;
  const SweepShape sh = sweep_shape<C, RC, TR, MODE>(S.ksz, kg);
  const int kv = S.kv, t0 = tile * TR;
  const int nrows = MODE == 0 ? bmax : smax;
  const int rvalid = min(TR, nrows - t0);
  const int kvr = min(kv, Kr);  // items gathered up front
  C* as = reinterpret_cast<C*>(smem_raw);             // [nbuf][kc0][TR] factor tile chunks
  C* vs = as + (size_t)sh.nbuf * sh.kc0 * TR;         // [kv][RC] vector operand
  C* wt = reinterpret_cast<C*>(smem_raw) + sh.region0;  // forward: [TR][RC] ring-tile updates
  int* ixs = reinterpret_cast<int*>(wt + (MODE == 0 ? TR * RC : 0));
  const C* A = S.F + (size_t)z * fmax * S.ncols + (size_t)(MODE == 0 ? fmax : smax) * fmax +
               (MODE == 0 ? smax : 0) + t0;
  auto load_chunk = [&](int ch) {
    const int cb = kb + ch * KA, kc = min(KA, ke - cb);
    C* dst = as + (size_t)(ch % sh.nbuf) * sh.kc0 * TR;
    if (rvalid > 0)
      for (int e = threadIdx.x; e < kc * TR; e += NT) {
        const int c = e / TR, i = e - c * TR;
        cp_async_elem<sizeof(C)>(dst + e, i < rvalid ? A + (size_t)(cb + c) * fmax + i : A, i < rvalid);
      }
    cp_async_commit();
  };

  // ---- prologue: static data only
  if (MODE == 0) {
    for (int c = threadIdx.x; c < kvr; c += NT) {
      const int col = kb + c;
      ixs[3 * c] = __ldg(S.own + (size_t)z * smax + col);
      ixs[3 * c + 1] = __ldg(S.fsrc + ((size_t)z * fmax + col) * 2);
      ixs[3 * c + 2] = __ldg(S.fsrc + ((size_t)z * fmax + col) * 2 + 1);
    }
    for (int i = threadIdx.x; i < TR; i += NT) {
      const int p = smax + t0 + i;
      const bool on = sp == 0 && i < rvalid;
      ixs[3 * kv + 2 * i] = on ? __ldg(S.fsrc + ((size_t)z * fmax + p) * 2) : -1;
      ixs[3 * kv + 2 * i + 1] = on ? __ldg(S.fsrc + ((size_t)z * fmax + p) * 2 + 1) : -1;
    }
  } else {
    for (int c = threadIdx.x; c < kvr; c += NT) {
      const int col = kb + c;
      ixs[c] = col < bmax ? __ldg(S.ring + (size_t)z * bmax + col) : -1;
    }
    for (int i = threadIdx.x; i < TR; i += NT) ixs[kv + i] = i < rvalid ? __ldg(S.own + (size_t)z * smax + t0 + i) : -1;
  }
  const int nch = (Kr + KA - 1) / KA;
  if (Kr > 0) load_chunk(0);

  // ---- after the previous level
  pdl_wait();
  pdl_trigger();
  __syncthreads();
  const bool write_own = MODE == 0 && tile == 0;
  if (Kr > 0) sweep_gather<C, RC, MODE>(S, z, g, kb, kvr, ixs, vs, write_own);
  if (MODE == 0 && sp == 0) {
    using P = typename Piece<C>::T;
    constexpr int NV = RC * (int)sizeof(C) / 16;
    const size_t cg = (size_t)g * S.nf_c * S.fmax_c;
    constexpr int B = 4;
    for (int base = threadIdx.x; base < TR * NV; base += NT * B) {
      P sv[B];
#pragma unroll
      for (int q = 0; q < B; ++q) {
        const int u = base + q * NT;
        sv[q] = pzero<P>();
        if (u >= TR * NV) continue;
        const int i = u / NV, v = u % NV;
        const int s0 = ixs[3 * kv + 2 * i], s1 = ixs[3 * kv + 2 * i + 1];
        P a = pzero<P>(), b = pzero<P>();
        if (s0 >= 0) a = __ldcg(reinterpret_cast<const P*>(S.Wc + (cg + s0) * RC) + v);
        if (s1 >= 0) b = __ldcg(reinterpret_cast<const P*>(S.Wc + (cg + s1) * RC) + v);
        sv[q] = padd(a, b);
      }
#pragma unroll
      for (int q = 0; q < B; ++q) {
        const int u = base + q * NT;
        if (u < TR * NV) reinterpret_cast<P*>(wt)[u] = sv[q];
      }
    }
  }

  C acc[RCT];
#pragma unroll
  for (int j = 0; j < RCT; ++j) acc[j] = czero<C>();
  for (int ch = 0; ch < nch; ++ch) {
    const int cb = kb + ch * KA, kc = min(KA, ke - cb);
    if (ch + 1 < nch) {
      load_chunk(ch + 1);
      cp_async_wait<1>();
    } else {
      cp_async_wait<0>();
    }
    // the staged vector operand covers [vb, vb + kv); when it is smaller than the range it
    // is refilled chunk by chunk (kv == KA then)
    const int vb = kv >= Kr ? kb : cb;
    if (kv < Kr && ch > 0) {
      __syncthreads();
      sweep_gather<C, RC, MODE>(S, z, g, cb, kc, nullptr, vs, write_own);
    }
    __syncthreads();
    if (rvalid > 0) {
      const C* ab = as + (size_t)(ch % sh.nbuf) * sh.kc0 * TR;
      const int per = (kc + kg - 1) / kg;
      const int k0 = w * per, k1 = min(kc, k0 + per);
      for (int k = k0; k < k1; ++k) {
        C a = ab[k * TR + row];
        if (MODE == 1 && cb + k < bmax) {
          a.x = -a.x;
          a.y = -a.y;
        }
        const C* vv = vs + (size_t)(cb + k - vb) * RC + j0;
#pragma unroll
        for (int j = 0; j < RCT; ++j) acc[j] = cfma(acc[j], a, vv[j]);
      }
    }
    __syncthreads();
  }
  if (rvalid <= 0) return;
  if (kg == 1 && S.nsplit == 1) {
    // one warp over all columns: every thread holds the finished sums of its row and
    // right-hand sides and stores them directly (RCT consecutive entries of one item)
    __syncthreads();  // wt complete when no column chunk ran
    if (row >= rvalid) return;
    C* dst;
    if (MODE == 0) {
      dst = S.W + ((size_t)g * S.nf * fmax + (size_t)z * fmax + smax + t0 + row) * RC + j0;
      if (sp == 0) {
#pragma unroll
        for (int j = 0; j < RCT; ++j) acc[j] = cadd(acc[j], wt[row * RC + j0 + j]);
      }
    } else {
      const int pt = ixs[kv + row];
      if (pt < 0) return;
      dst = S.T + ((size_t)g * S.N + pt) * RC + j0;
    }
    if constexpr (sizeof(C) == 8 && RCT % 2 == 0) {
#pragma unroll
      for (int j = 0; j < RCT; j += 2)
        reinterpret_cast<float4*>(dst)[j / 2] = make_float4(acc[j].x, acc[j].y, acc[j + 1].x, acc[j + 1].y);
    } else {
#pragma unroll
      for (int j = 0; j < RCT; ++j) dst[j] = acc[j];
    }
    return;
  }
  C* red = reinterpret_cast<C*>(smem_raw);
#pragma unroll
  for (int j = 0; j < RCT; ++j) red[((size_t)w * 32 + lane) * (RCT + 1) + j] = acc[j];
  __syncthreads();
  const size_t item = ((size_t)g * S.nf + z) * S.ntile + tile;
  auto store = [&](int i, int j, C s) {
    if (MODE == 0) {
      S.W[((size_t)g * S.nf * fmax + (size_t)z * fmax + smax + t0 + i) * RC + j] = s;
    } else {
      const int pt = ixs[kv + i];
      if (pt >= 0) S.T[((size_t)g * S.N + pt) * RC + j] = s;
    }
  };
  for (int o = threadIdx.x; o < TR * RC; o += NT) {
    const int i = o / RC, j = o % RC;
    if (i >= rvalid) continue;
    const int ln = TR == 32 ? i : i + 16 * (j / RCT), sl = TR == 32 ? j : j % RCT;
    C s = MODE == 0 && sp == 0 ? wt[i * RC + j] : czero<C>();
    for (int q = 0; q < kg; ++q) s = cadd(s, red[((size_t)q * 32 + ln) * (RCT + 1) + sl]);
    if (S.nsplit == 1) store(i, j, s);
    else S.part[(item * S.nsplit + sp) * TR * RC + o] = s;
  }
  if (S.nsplit == 1) return;
  // the CTA that completes the item last adds the ranges' partial sums in range order
  __threadfence();
  __syncthreads();
  if (threadIdx.x == 0) last_s = atomicAdd(S.cnt + item, 1u) == (unsigned)(S.nsplit - 1);
  __syncthreads();
  if (!last_s) return;
  __threadfence();
  for (int o = threadIdx.x; o < TR * RC; o += NT) {
    const int i = o / RC, j = o % RC;
    if (i >= rvalid) continue;
    C s = czero<C>();
    for (int q = 0; q < S.nsplit; ++q) s = cadd(s, __ldcg(S.part + (item * S.nsplit + q) * TR * RC + o));
    store(i, j, s);
  }
  if (threadIdx.x == 0) S.cnt[item] = 0u;
}

// r[rhs][N] -> T[group][N][RC] (right-hand sides past nr are zero)
template <typename C, int RC> __global__ void __launch_bounds__(256) k_items_in(const C* __restrict__ r, C* T, int nr, long N) {
  constexpr int TP = 512 / RC;
  __shared__ C s[RC][TP + 1];
  pdl_wait();
  pdl_trigger();
  const long i0 = (long)blockIdx.x * TP;
  const int g = blockIdx.y;
  for (int e = threadIdx.x; e < TP * RC; e += blockDim.x) {
    const int j = e / TP, ii = e % TP;
    const long i = i0 + ii;
    const int rhs = g * RC + j;
    s[j][ii] = (i < N && rhs < nr) ? __ldcg(r + (size_t)rhs * N + i) : czero<C>();
  }
  __syncthreads();
  for (int e = threadIdx.x; e < TP * RC; e += blockDim.x) {
    const int ii = e / RC, j = e % RC;
    const long i = i0 + ii;
    if (i < N) T[((size_t)g * N + i) * RC + j] = s[j][ii];
  }
}

// T[group][N][RC] -> x[rhs][N] for the nr right-hand sides (ACC: x += T)
template <typename C, int RC, bool ACC>
__global__ void __launch_bounds__(256) k_items_out(const C* T, C* __restrict__ x, int nr, long N) {
  constexpr int TP = 512 / RC;
  __shared__ C s[RC][TP + 1];
  pdl_wait();
  pdl_trigger();
  const long i0 = (long)blockIdx.x * TP;
  const int g = blockIdx.y;
  for (int e = threadIdx.x; e < TP * RC; e += blockDim.x) {
    const int ii = e / RC, j = e % RC;
    const long i = i0 + ii;
    s[j][ii] = i < N ? __ldcg(T + ((size_t)g * N + i) * RC + j) : czero<C>();
  }
  __syncthreads();
  for (int e = threadIdx.x; e < TP * RC; e += blockDim.x) {
    const int j = e / TP, ii = e % TP;
    const long i = i0 + ii;
    const int rhs = g * RC + j;
    if (i < N && rhs < nr) {
      if constexpr (ACC) x[(size_t)rhs * N + i] = cadd(x[(size_t)rhs * N + i], s[j][ii]);
      else x[(size_t)rhs * N + i] = s[j][ii];
    }
  }
}

// launch as a programmatic dependent of the previous kernel in the stream
template <typename... KArgs, typename... Args>
static void launch_pdl(void (*kern)(KArgs...), dim3 grid, dim3 block, size_t smem, cudaStream_t st, Args... args) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = grid;
  cfg.blockDim = block;
  cfg.dynamicSmemBytes = smem;
  cfg.stream = st;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  at[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = at;
  cfg.numAttrs = 1;
  LS_CUDA(cudaLaunchKernelEx(&cfg, kern, args...));
}

template <typename C, int RC, int TR, int MODE>
static void launch_sweep_tr(NdPlan* p, int l, C* T, int ng, const SweepPlan& q, cudaStream_t st) {
  const LevelDev& D = p->lev[l];
  const int depth = (int)p->lev.size();
  const SweepShape sh = sweep_shape<C, RC, TR, MODE>(q.ksz, 0);
  if (sh.smem > SWEEP_SMEM_MAX) LS_FAIL(EINVAL_, "front too large for the solve kernels (%zu bytes of shared memory)", sh.smem);
  static std::atomic<bool> attr{false};  // set once per process; repeats are harmless
  if (!attr.load(std::memory_order_acquire)) {
    LS_CUDA(cudaFuncSetAttribute(k_sweep<C, RC, TR, MODE>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)SWEEP_SMEM_MAX));
    attr.store(true, std::memory_order_release);
  }
  SweepK<C> S;
  S.F = reinterpret_cast<const C*>(p->F) + D.F_off;
  S.W = reinterpret_cast<C*>(p->W) + D.W_off;
  const bool has_child = l + 1 < depth;
  S.Wc = has_child ? reinterpret_cast<const C*>(p->W) + p->lev[l + 1].W_off : S.W;
  S.T = T;
  S.own = D.own;
  S.ring = D.ring;
  S.fsrc = D.fsrc;
  S.nf = D.nf;
  S.smax = D.smax;
  S.bmax = D.bmax;
  S.fmax = D.fmax;
  S.ncols = D.ncols;
  S.nf_c = has_child ? p->lev[l + 1].nf : 0;
  S.fmax_c = has_child ? p->lev[l + 1].fmax : 0;
  S.ntile = q.ntile;
  S.nsplit = q.nsplit;
  S.ksz = q.ksz;
  S.kv = sh.kv;
  S.ng = ng;
  S.part = reinterpret_cast<C*>(p->part);
  S.cnt = p->cnt;
  S.N = p->N;
  const dim3 grid((unsigned)((long)D.nf * ng), q.ntile * q.nsplit, 1);
  const bool f32 = sizeof(C) == 8;
  LS_LAUNCH(MODE == 0 ? (f32 ? "nd_fwd_c64" : "nd_fwd_c128") : (f32 ? "nd_bwd_c64" : "nd_bwd_c128"), st,
            launch_pdl(k_sweep<C, RC, TR, MODE>, grid, dim3(32 * sh.kg), sh.smem, st, S));
}

// ---- sweep levels on the tensor cores (FP32, 16 right-hand sides per group): the level's
// product of k_sweep as one batched GEMM (tc_sweep_gemm, 3xTF32) between a gather of the
// vector operand into B[z][k][n] and a scatter of C[z][row][n], n = group * 16 + j < ncols
//   forward:  B = w_own (r at the own points + the children's updates, also stored to W),
//             C = Y w_own, stored to the ring part of W with the children's ring updates added;
//   backward: B = [-x_ring; w_own], C = [H | F11^-1] B = x_own, stored to T at the own points.
// One thread moves two right-hand sides (16 bytes) of one k or row.
template <int MODE>
__global__ void __launch_bounds__(256) k_tcs_gather(SweepK<float2> S, float2* __restrict__ B, int K, int ncols) {
  const int z = blockIdx.x, pairs = ncols / 2;
  float2* Bz = B + (size_t)z * K * ncols;
  for (int t = blockIdx.y * blockDim.x + threadIdx.x; t < K * pairs; t += gridDim.y * blockDim.x) {
    const int k = t / pairs, n = 2 * (t - k * pairs), g = n >> 4, j = n & 15;
    const size_t wrow = (size_t)g * S.nf * S.fmax + (size_t)z * S.fmax;
    float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
    if (MODE == 0) {
      const int pt = __ldg(S.own + (size_t)z * S.smax + k);
      const int s0 = __ldg(S.fsrc + ((size_t)z * S.fmax + k) * 2), s1 = __ldg(S.fsrc + ((size_t)z * S.fmax + k) * 2 + 1);
      const size_t cg = (size_t)g * S.nf_c * S.fmax_c;
      if (pt >= 0) v = padd(v, __ldcg(reinterpret_cast<const float4*>(S.T + ((size_t)g * S.N + pt) * 16 + j)));
      if (s0 >= 0) v = padd(v, __ldcg(reinterpret_cast<const float4*>(S.Wc + (cg + s0) * 16 + j)));
      if (s1 >= 0) v = padd(v, __ldcg(reinterpret_cast<const float4*>(S.Wc + (cg + s1) * 16 + j)));
      *reinterpret_cast<float4*>(S.W + (wrow + k) * 16 + j) = v;
    } else if (k < S.bmax) {
      const int pt = __ldg(S.ring + (size_t)z * S.bmax + k);
      if (pt >= 0) {
        v = __ldcg(reinterpret_cast<const float4*>(S.T + ((size_t)g * S.N + pt) * 16 + j));
        v = make_float4(-v.x, -v.y, -v.z, -v.w);
      }
    } else {
      v = __ldcg(reinterpret_cast<const float4*>(S.W + (wrow + k - S.bmax) * 16 + j));
    }
    *reinterpret_cast<float4*>(Bz + (size_t)k * ncols + n) = v;
  }
}

// the k-range splits' partial products are added in split order (nsplit arrays split_stride
// apart)
template <int MODE>
__global__ void __launch_bounds__(256) k_tcs_scatter(SweepK<float2> S, const float2* __restrict__ Cm, int rows,
                                                     int ncols, int nsplit, long split_stride) {
  const int z = blockIdx.x, pairs = ncols / 2;
  const float2* Cz = Cm + (size_t)z * rows * ncols;
  for (int t = blockIdx.y * blockDim.x + threadIdx.x; t < rows * pairs; t += gridDim.y * blockDim.x) {
    const int i = t / pairs, n = 2 * (t - i * pairs), g = n >> 4, j = n & 15;
    float4 v = __ldcg(reinterpret_cast<const float4*>(Cz + (size_t)i * ncols + n));
    for (int sp = 1; sp < nsplit; ++sp)
      v = padd(v, __ldcg(reinterpret_cast<const float4*>(Cz + sp * split_stride + (size_t)i * ncols + n)));
    if (MODE == 0) {
      const int p0 = S.smax + i;
      const int s0 = __ldg(S.fsrc + ((size_t)z * S.fmax + p0) * 2), s1 = __ldg(S.fsrc + ((size_t)z * S.fmax + p0) * 2 + 1);
      const size_t cg = (size_t)g * S.nf_c * S.fmax_c;
      if (s0 >= 0) v = padd(v, __ldcg(reinterpret_cast<const float4*>(S.Wc + (cg + s0) * 16 + j)));
      if (s1 >= 0) v = padd(v, __ldcg(reinterpret_cast<const float4*>(S.Wc + (cg + s1) * 16 + j)));
      *reinterpret_cast<float4*>(S.W + ((size_t)g * S.nf * S.fmax + (size_t)z * S.fmax + p0) * 16 + j) = v;
    } else {
      const int pt = __ldg(S.own + (size_t)z * S.smax + i);
      if (pt >= 0) *reinterpret_cast<float4*>(S.T + ((size_t)g * S.N + pt) * 16 + j) = v;
    }
  }
}

// ---- small sweep levels (the bottom of the tree: at most 64 product rows and SMALL_MAX_K
// columns, FP32, 16 right-hand sides per item): one CTA per front, one warp per group of 16
// right-hand sides (ng warps).  Before the programmatic-dependent wait the CTA stages the
// front's indices and copies the first SMALL_KCH columns of its factor tile (shared by the
// groups) into shared memory with cp.async, overlapping the previous level's tail; after it,
// column chunk by chunk, every warp gathers its group's vector operand (16 right-hand sides
// per column; index and data loads of four pieces in flight) and accumulates.  Lane l holds
// row l (and l + 32 when RP = 64) for all 16 right-hand sides, or, when RP = 16, row l & 15
// for 8 of them (lanes 16-31 the second half).  Forward: rows are the ring rows of Y, the
// children's ring updates added at the store.
constexpr int SMALL_FPC = 4;   // warps per CTA at most (groups of 16 of SOLVE_CHUNK)
constexpr int SMALL_KCH = 64;  // columns of the factor tile and operand staged at once
// bytes of the CTA's shared memory: factor chunk (RP x KC complex, RP = 16, 32 or 64 rows,
// KC = min(K, SMALL_KCH) columns), indices (3 K + 2 RP ints, padded to 16 bytes), then ng
// operand chunks (KC x 16 complex)
__host__ __device__ constexpr int small_kc(int K) { return K < SMALL_KCH ? K : SMALL_KCH; }
__host__ __device__ constexpr size_t small_head_bytes(int K, int rp) {
  return ((size_t)rp * small_kc(K) * sizeof(float2) + ((size_t)3 * K + 2 * rp) * sizeof(int) + 15) / 16 * 16;
}
__host__ __device__ constexpr size_t small_smem_bytes(int K, int rp, int ng) {
  return small_head_bytes(K, rp) + (size_t)ng * small_kc(K) * 16 * sizeof(float2);
}
template <int MODE, int RP, bool MULTI>
__global__ void __launch_bounds__(32 * SMALL_FPC) k_sweep_small(SweepK<float2> S) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  constexpr int NJ = RP == 16 ? 8 : 16, NRB = RP == 64 ? 2 : 1;
  const int lane = threadIdx.x & 31, g = threadIdx.x >> 5, NT = blockDim.x;
  const int z = blockIdx.x;
  const int smax = S.smax, bmax = S.bmax, fmax = S.fmax;
  const int K = MODE == 0 ? smax : bmax + smax;
  const int rows = MODE == 0 ? bmax : smax;
  const int kcap = small_kc(K);
  float2* As = reinterpret_cast<float2*>(smem_raw);  // [kcap][RP]
  int* ix = reinterpret_cast<int*>(As + (size_t)RP * kcap);  // [3 K] item sources, [2 RP] rows
  float2* vs = reinterpret_cast<float2*>(smem_raw + small_head_bytes(K, RP)) + (size_t)g * kcap * 16;
  const float2* A = S.F + (size_t)z * fmax * S.ncols + (size_t)(MODE == 0 ? fmax : smax) * fmax +
                    (MODE == 0 ? smax : 0);
  auto load_chunk = [&](int kc) {
    const int kw = min(SMALL_KCH, K - kc);
    for (int e = threadIdx.x; e < kw * RP; e += NT) {
      const int k = e / RP, r = e - k * RP;
      cp_async_elem<8>(As + e, r < rows ? A + (size_t)(kc + k) * fmax + r : A, r < rows);
    }
    cp_async_commit();
  };
  // ---- prologue: static data only
  load_chunk(0);
  for (int c = threadIdx.x; c < K; c += NT) {
    if (MODE == 0) {
      ix[3 * c] = __ldg(S.own + (size_t)z * smax + c);
      ix[3 * c + 1] = __ldg(S.fsrc + ((size_t)z * fmax + c) * 2);
      ix[3 * c + 2] = __ldg(S.fsrc + ((size_t)z * fmax + c) * 2 + 1);
    } else {
      ix[3 * c] = c < bmax ? __ldg(S.ring + (size_t)z * bmax + c) : -1;
    }
  }
  for (int r = threadIdx.x; r < RP; r += NT) {
    if (MODE == 0) {
      const bool rv = r < rows;
      ix[3 * K + 2 * r] = rv ? __ldg(S.fsrc + ((size_t)z * fmax + smax + r) * 2) : -1;
      ix[3 * K + 2 * r + 1] = rv ? __ldg(S.fsrc + ((size_t)z * fmax + smax + r) * 2 + 1) : -1;
    } else {
      ix[3 * K + 2 * r] = r < rows ? __ldg(S.own + (size_t)z * smax + r) : -1;
    }
  }
  pdl_wait();
  pdl_trigger();
  __syncthreads();  // indices
  const size_t wrow = (size_t)g * S.nf * fmax + (size_t)z * fmax;
  const size_t cg = (size_t)g * S.nf_c * S.fmax_c;
  const int row0 = RP == 16 ? (lane & 15) : lane, j0 = RP == 16 ? (lane >> 4) * 8 : 0;
  float2 acc[NRB][NJ];
#pragma unroll
  for (int b = 0; b < NRB; ++b)
#pragma unroll
    for (int j = 0; j < NJ; ++j) acc[b][j] = make_float2(0.f, 0.f);
  constexpr int GB = 4;
  // MULTI: more than one column chunk (K > SMALL_KCH); else the loop runs once
  for (int kc = 0; kc < (MULTI ? K : 1); kc += SMALL_KCH) {
    const int kw = MULTI ? min(SMALL_KCH, K - kc) : K;
    if (MULTI && kc > 0) {
      __syncthreads();  // every warp is done with the previous chunk
      load_chunk(kc);
    }
    for (int p0 = lane; p0 < kw * 8; p0 += 32 * GB) {
      float4 x[GB];
#pragma unroll
      for (int u = 0; u < GB; ++u) {
        const int p = p0 + 32 * u, c = kc + (p >> 3), v = p & 7;
        x[u] = make_float4(0.f, 0.f, 0.f, 0.f);
        if (p >= kw * 8) continue;
        if (MODE == 0) {
          const int pt = ix[3 * c], s0 = ix[3 * c + 1], s1 = ix[3 * c + 2];
          if (pt >= 0) x[u] = padd(x[u], __ldcg(reinterpret_cast<const float4*>(S.T + ((size_t)g * S.N + pt) * 16) + v));
          if (s0 >= 0) x[u] = padd(x[u], __ldcg(reinterpret_cast<const float4*>(S.Wc + (cg + s0) * 16) + v));
          if (s1 >= 0) x[u] = padd(x[u], __ldcg(reinterpret_cast<const float4*>(S.Wc + (cg + s1) * 16) + v));
        } else if (c < bmax) {
          const int pt = ix[3 * c];
          if (pt >= 0) {
            const float4 t = __ldcg(reinterpret_cast<const float4*>(S.T + ((size_t)g * S.N + pt) * 16) + v);
            x[u] = make_float4(-t.x, -t.y, -t.z, -t.w);  // the H columns enter with a minus sign
          }
        } else {
          x[u] = __ldcg(reinterpret_cast<const float4*>(S.W + (wrow + c - bmax) * 16) + v);
        }
      }
#pragma unroll
      for (int u = 0; u < GB; ++u) {
        const int p = p0 + 32 * u, c = kc + (p >> 3), v = p & 7;
        if (p >= kw * 8) continue;
        if (MODE == 0) reinterpret_cast<float4*>(S.W + (wrow + c) * 16)[v] = x[u];
        reinterpret_cast<float4*>(vs)[p] = x[u];
      }
    }
    cp_async_wait<0>();
    __syncthreads();  // the factor chunk (every thread's copies) and this warp's operand
#pragma unroll 4
    for (int k = 0; k < kw; ++k) {
      const float4* vv = reinterpret_cast<const float4*>(vs + (size_t)k * 16 + j0);
#pragma unroll
      for (int b = 0; b < NRB; ++b) {
        const float2 a = As[k * RP + row0 + 32 * b];
#pragma unroll
        for (int j = 0; j < NJ / 2; ++j) {
          const float4 v4 = vv[j];
          acc[b][2 * j] = cfma(acc[b][2 * j], a, make_float2(v4.x, v4.y));
          acc[b][2 * j + 1] = cfma(acc[b][2 * j + 1], a, make_float2(v4.z, v4.w));
        }
      }
    }
  }
#pragma unroll
  for (int b = 0; b < NRB; ++b) {
    const int row = row0 + 32 * b;
    if (row >= rows) continue;
    float2* dst;
    if (MODE == 0) {
      const int s0 = ix[3 * K + 2 * row], s1 = ix[3 * K + 2 * row + 1];
#pragma unroll
      for (int j = 0; j < NJ; j += 2) {
        float4 x = make_float4(acc[b][j].x, acc[b][j].y, acc[b][j + 1].x, acc[b][j + 1].y);
        if (s0 >= 0) x = padd(x, __ldcg(reinterpret_cast<const float4*>(S.Wc + (cg + s0) * 16 + j0 + j)));
        if (s1 >= 0) x = padd(x, __ldcg(reinterpret_cast<const float4*>(S.Wc + (cg + s1) * 16 + j0 + j)));
        acc[b][j] = make_float2(x.x, x.y);
        acc[b][j + 1] = make_float2(x.z, x.w);
      }
      dst = S.W + (wrow + smax + row) * 16 + j0;
    } else {
      const int pt = ix[3 * K + 2 * row];
      if (pt < 0) continue;
      dst = S.T + ((size_t)g * S.N + pt) * 16 + j0;
    }
#pragma unroll
    for (int j = 0; j < NJ; j += 2)
      reinterpret_cast<float4*>(dst)[j / 2] =
          make_float4(acc[b][j].x, acc[b][j].y, acc[b][j + 1].x, acc[b][j + 1].y);
  }
}

constexpr int SMALL_MAX_K = 256;
// the automatic values of the solve-level choices (measured: 2D n = 256 with 16 right-hand
// sides solves 1.9x faster with neither tensor-core levels nor one-CTA-per-front levels past
// 64 columns than with the 64-right-hand-side choices; 3D n = 64 with 8 keeps its
// tensor-core levels)
int nd_tcs_min_rows(int d, int ng, int v) { return v >= 0 ? v : ((d == 3 || ng >= 2) ? 64 : (1 << 30)); }
int nd_small_max_k(int ng, int v) { return v >= 0 ? v : (ng >= 2 ? SMALL_MAX_K : 64); }

static bool small_level(const NdPlan* p, int l, int mode, int ng) {
  const LevelDev& D = p->lev[l];
  const int rows = mode == 0 ? D.bmax : D.smax, K = mode == 0 ? D.smax : D.bmax + D.smax;
  return rows > 0 && rows <= 64 && K > 0 && K <= std::min(SMALL_MAX_K, nd_small_max_k(ng, p->tune.small_max_k));
}

template <int MODE> static void launch_sweep_small(NdPlan* p, int l, float2* T, int ng, cudaStream_t st) {
  const LevelDev& D = p->lev[l];
  const int depth = (int)p->lev.size();
  SweepK<float2> S{};
  S.F = reinterpret_cast<const float2*>(p->F) + D.F_off;
  S.W = reinterpret_cast<float2*>(p->W) + D.W_off;
  const bool has_child = l + 1 < depth;
  S.Wc = has_child ? reinterpret_cast<const float2*>(p->W) + p->lev[l + 1].W_off : S.W;
  S.T = T;
  S.own = D.own;
  S.ring = D.ring;
  S.fsrc = D.fsrc;
  S.nf = D.nf;
  S.smax = D.smax;
  S.bmax = D.bmax;
  S.fmax = D.fmax;
  S.ncols = D.ncols;
  S.nf_c = has_child ? p->lev[l + 1].nf : 0;
  S.fmax_c = has_child ? p->lev[l + 1].fmax : 0;
  S.ng = ng;
  S.N = p->N;
  const int K = MODE == 0 ? D.smax : D.bmax + D.smax;
  const int rows = MODE == 0 ? D.bmax : D.smax;
  const int rp = rows > 32 ? 64 : (rows > 16 ? 32 : 16);
  const size_t smem = small_smem_bytes(K, rp, ng);
  const size_t smem_max = small_smem_bytes(SMALL_MAX_K, 64, SMALL_FPC);
  static std::atomic<bool> attr{false};  // set once per process; repeats are harmless
  if (!attr.load(std::memory_order_acquire)) {
    LS_CUDA(cudaFuncSetAttribute(k_sweep_small<MODE, 16, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_max));
    LS_CUDA(cudaFuncSetAttribute(k_sweep_small<MODE, 32, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_max));
    LS_CUDA(cudaFuncSetAttribute(k_sweep_small<MODE, 64, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_max));
    LS_CUDA(cudaFuncSetAttribute(k_sweep_small<MODE, 16, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_max));
    LS_CUDA(cudaFuncSetAttribute(k_sweep_small<MODE, 32, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_max));
    LS_CUDA(cudaFuncSetAttribute(k_sweep_small<MODE, 64, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_max));
    attr.store(true, std::memory_order_release);
  }
  // one CTA per front, one warp per group
  const dim3 grid((unsigned)D.nf), block(32 * ng);
  const char* cls = MODE == 0 ? "nd_fwd_c64" : "nd_bwd_c64";
  const bool multi = K > SMALL_KCH;
#define LS_SMALL(RP_, M_) LS_LAUNCH(cls, st, launch_pdl(k_sweep_small<MODE, RP_, M_>, grid, block, smem, st, S))
  if (rp == 64) { if (multi) LS_SMALL(64, true); else LS_SMALL(64, false); }
  else if (rp == 32) { if (multi) LS_SMALL(32, true); else LS_SMALL(32, false); }
  else { if (multi) LS_SMALL(16, true); else LS_SMALL(16, false); }
#undef LS_SMALL
}

// whether level l's sweep product of this mode runs on the tensor cores
static bool tcs_level(const NdPlan* p, int l, int mode, int ng) {
  const LevelDev& D = p->lev[l];
  const int rows = tcs_rows(D, mode);
  const int min_rows = nd_tcs_min_rows(p->d, ng, mode == 0 ? p->tune.tcs_min_rows : p->tune.tcs_bwd_min_rows);
  return p->use_tc && tc_enabled() && p->tcs_B && p->tcs_C && rows >= std::max(TCS_MIN_ROWS, min_rows) &&
         tcs_k(D, mode) >= TC_MIN_K && (size_t)D.nf * tcs_k(D, mode) * ng * 16 <= p->tcs_B_elems &&
         (size_t)D.nf * rows * ng * 16 * tcs_split(D, mode).nsplit <= p->tcs_C_elems;
}

template <int MODE> static void launch_sweep_tc(NdPlan* p, int l, float2* T, int ng, cudaStream_t st) {
  const LevelDev& D = p->lev[l];
  const int depth = (int)p->lev.size();
  SweepK<float2> S{};
  S.F = reinterpret_cast<const float2*>(p->F) + D.F_off;
  S.W = reinterpret_cast<float2*>(p->W) + D.W_off;
  const bool has_child = l + 1 < depth;
  S.Wc = has_child ? reinterpret_cast<const float2*>(p->W) + p->lev[l + 1].W_off : S.W;
  S.T = T;
  S.own = D.own;
  S.ring = D.ring;
  S.fsrc = D.fsrc;
  S.nf = D.nf;
  S.smax = D.smax;
  S.bmax = D.bmax;
  S.fmax = D.fmax;
  S.ncols = D.ncols;
  S.nf_c = has_child ? p->lev[l + 1].nf : 0;
  S.fmax_c = has_child ? p->lev[l + 1].fmax : 0;
  S.N = p->N;
  const int K = tcs_k(D, MODE), rows = tcs_rows(D, MODE), ncols = ng * 16;
  const char* cls = MODE == 0 ? "nd_fwd_c64" : "nd_bwd_c64";
  const int gy_b = std::min(64, (K * ncols / 2 + 255) / 256), gy_c = std::min(64, (rows * ncols / 2 + 255) / 256);
  LS_LAUNCH(cls, st, k_tcs_gather<MODE><<<dim3(D.nf, gy_b), 256, 0, st>>>(S, p->tcs_B, K, ncols));
  // forward: A = Y (ring rows smax.., identity columns fmax..); backward: A = [H | F11^-1]
  // (own rows, columns smax..ncols)
  const int r0 = MODE == 0 ? D.smax : 0, k0 = MODE == 0 ? D.fmax : D.smax;
  const TcsSplit sp = tcs_split(D, MODE);
  const long split_stride = (long)D.nf * rows * ncols;
  tc_sweep_gemm(reinterpret_cast<const float2*>(p->F) + D.F_off, (long)D.fmax * D.ncols, D.fmax, D.nf, r0, r0 + rows,
                k0, k0 + K, p->tcs_B, (long)K * ncols, ncols, p->tcs_C, (long)rows * ncols, ncols, ncols, sp.nsplit,
                sp.ksz, split_stride, p->d_err, st, cls);
  LS_LAUNCH(cls, st,
            k_tcs_scatter<MODE><<<dim3(D.nf, gy_c), 256, 0, st>>>(S, p->tcs_C, rows, ncols, sp.nsplit, split_stride));
}

template <typename C, int RC, int MODE> static void launch_sweep(NdPlan* p, int l, C* T, int ng, cudaStream_t st) {
  if constexpr (sizeof(C) == 8 && RC == 16) {
    if (tcs_level(p, l, MODE, ng)) {
      launch_sweep_tc<MODE>(p, l, reinterpret_cast<float2*>(T), ng, st);
      return;
    }
    if (small_level(p, l, MODE, ng)) {
      launch_sweep_small<MODE>(p, l, reinterpret_cast<float2*>(T), ng, st);
      return;
    }
  }
  const SweepPlan q = sweep_plan(p->lev[l], MODE, ng, std::min(std::max(p->tune.sweep_ctas, 1), SWEEP_CTAS_MAX));
  if (q.K <= 0) return;
  if (q.nsplit > 1 && (size_t)p->lev[l].nf * q.ntile * q.nsplit * q.tr * RC * ng > p->part_elems)
    LS_FAIL(EINVAL_, "solve partial-sum buffer too small");
  if (q.tr == 16) launch_sweep_tr<C, RC, 16, MODE>(p, l, T, ng, q, st);
  else launch_sweep_tr<C, RC, 32, MODE>(p, l, T, ng, q, st);
}

template <typename C, int RC>
static void solve_chunk(NdPlan* p, int nr, const C* r, C* x, cudaStream_t st, bool acc) {
  const int depth = (int)p->lev.size();
  const int ng = (nr + RC - 1) / RC;
  const bool f32 = sizeof(C) == 8;
  C* T = reinterpret_cast<C*>(p->T);
  constexpr int TP = 512 / RC;
  const dim3 tgrid((unsigned)((p->N + TP - 1) / TP), ng);
  if (r != nullptr)  // (else the items are in T already)
    LS_LAUNCH(f32 ? "nd_items_c64" : "nd_items_c128", st,
              launch_pdl(k_items_in<C, RC>, tgrid, dim3(256), 0, st, r, T, nr, p->N));
  for (int l = depth - 1; l >= 0; --l) {
    prof_tag(l);
    launch_sweep<C, RC, 0>(p, l, T, ng, st);
  }
  for (int l = 0; l < depth; ++l) {
    prof_tag(l);
    launch_sweep<C, RC, 1>(p, l, T, ng, st);
  }
  prof_tag(-1);
  // (its own class: one launch per application, whether or not the items came from k_items_in)
  if (acc)
    LS_LAUNCH(f32 ? "nd_items_out_c64" : "nd_items_out_c128", st,
              launch_pdl(k_items_out<C, RC, true>, tgrid, dim3(256), 0, st, (const C*)T, x, nr, p->N));
  else
    LS_LAUNCH(f32 ? "nd_items_out_c64" : "nd_items_out_c128", st,
              launch_pdl(k_items_out<C, RC, false>, tgrid, dim3(256), 0, st, (const C*)T, x, nr, p->N));
}

// x = M^{-1} r, or x += M^{-1} r (accumulate: the refinement step's correction)
template <typename C> void nd_solve(NdPlan* p, int nrhs, const C* r, C* x, cudaStream_t st, bool accumulate) {
  if (!p->F || p->F_bytes != (int)sizeof(C)) LS_FAIL(ESTATE_, "preconditioner not factored in this precision");
  for (int c0 = 0; c0 < nrhs; c0 += SOLVE_CHUNK) {
    const int nr = std::min(SOLVE_CHUNK, nrhs - c0);
    const C* rr = r + (size_t)c0 * p->N;
    C* xx = x + (size_t)c0 * p->N;
    if (nd_item_width(nr) == 4) solve_chunk<C, 4>(p, nr, rr, xx, st, accumulate);
    else solve_chunk<C, 16>(p, nr, rr, xx, st, accumulate);
  }
}

template void nd_factor<float2>(NdPlan*, const void*, const void*, const void*, cudaStream_t);
template void nd_factor<double2>(NdPlan*, const void*, const void*, const void*, cudaStream_t);
template bool nd_prepare<float2>(NdPlan*, cudaStream_t);
template bool nd_prepare<double2>(NdPlan*, cudaStream_t);
template void nd_factor_launch<float2>(NdPlan*, const void*, const void*, const void*, cudaStream_t, cudaEvent_t,
                                       const void*, const unsigned char*);
template void nd_factor_launch<double2>(NdPlan*, const void*, const void*, const void*, cudaStream_t, cudaEvent_t,
                                        const void*, const unsigned char*);
void* nd_items(NdPlan* p) { return p->T; }
int nd_item_width(int nrhs) { return nrhs <= 4 ? 4 : 16; }
int nd_items_max() { return SOLVE_CHUNK; }

template <typename C> void nd_solve_items(NdPlan* p, int nrhs, C* x, cudaStream_t st, bool accumulate) {
  if (!p->F || p->F_bytes != (int)sizeof(C)) LS_FAIL(ESTATE_, "preconditioner not factored in this precision");
  if (nrhs < 1 || nrhs > SOLVE_CHUNK) LS_FAIL(EINVAL_, "nd_solve_items: %d right-hand sides (1..%d)", nrhs, SOLVE_CHUNK);
  if (nd_item_width(nrhs) == 4) solve_chunk<C, 4>(p, nrhs, nullptr, x, st, accumulate);
  else solve_chunk<C, 16>(p, nrhs, nullptr, x, st, accumulate);
}

template void nd_solve_items<float2>(NdPlan*, int, float2*, cudaStream_t, bool);
template void nd_solve_items<double2>(NdPlan*, int, double2*, cudaStream_t, bool);
template void nd_solve<float2>(NdPlan*, int, const float2*, float2*, cudaStream_t, bool);
template void nd_solve<double2>(NdPlan*, int, const double2*, double2*, cudaStream_t, bool);

}  // namespace ls
