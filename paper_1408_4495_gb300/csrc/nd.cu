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
//   1. blocked right-looking LU of the own columns (pivot rows restricted to the own rows;
//      panel / row-swap + unit-lower TRSM of the block row / GEMM of the trailing block),
//      which leaves the Schur complement S = F22 - F21 F11^{-1} F12 in the ring block and
//      Y = -F21 F11^{-1} in the ring rows of the identity columns;
//   2. blocked backward substitution with U11 on the own rows of [F12 I] (Gauss-Jordan),
//      which leaves H = F11^{-1} F12 and F11^{-1} there.
// S is extend-added into the parent.  The solve then needs no triangular recurrences:
//   forward (leaves to root):  update for the parent  u_ring = w_ring + Y w_own
//   backward (root to leaves): x_own = F11^{-1} w_own - H x_ring
// two batched multi-right-hand-side matrix-vector products per level, every factor entry
// read once per sweep.
#include <algorithm>
#include <cstring>
#include <map>
#include <memory>
#include <mutex>
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
  int nf = 0, smax = 0, bmax = 0, fmax = 0, ncols = 0;
  size_t F_off = 0, W_off = 0;
  int *own = nullptr, *ring = nullptr, *child = nullptr, *parent = nullptr, *kidx = nullptr, *ea = nullptr;
  int* piv = nullptr;
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
  int* d_err = nullptr;
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
    size_t own, ring, child, parent, kidx, ea, piv;
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
    if (cudaMalloc(&p->blob, H->blob.size()) != cudaSuccess) {
      cudaGetLastError();
      LS_FAIL(ENOMEM_, "cudaMalloc(%zu) failed for the ND plan", H->blob.size());
    }
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
  if (p->blob) cudaFree(p->blob);
  if (p->F) cudaFree(p->F);
  if (p->W) cudaFree(p->W);
  delete p;
}

NdInfo nd_info(const NdPlan* p) { return p->info; }

size_t nd_device_bytes(const NdPlan* p, int elem_bytes) { return (p->F_elems + p->W_elems) * (size_t)elem_bytes; }

// ---------------------------------------------------------------------------------------
// factorization kernels
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
    // M(i, i+t) = alpha_cls(i)(t) + [i interior] c(t) omega^2 m_{i+t}   (eq. PC)
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

template <typename C> __global__ void k_set_one(C* F, long n_one, const int64_t* __restrict__ off) {
  for (long e = blockIdx.x * (long)blockDim.x + threadIdx.x; e < n_one; e += (long)gridDim.x * blockDim.x) {
    C one;
    one.x = 1;
    one.y = 0;
    F[off[e]] = one;
  }
}

// Schur complements of the children with child index k into their parents' fronts.
template <typename C> __global__ void k_extend_add(LevelK<C> P, LevelK<C> Ch, int k) {
  const int c = blockIdx.x;
  if (Ch.kidx[c] != k) return;
  const int pz = Ch.parent[c];
  C* Fp = P.F + (size_t)pz * P.fmax * P.ncols;
  const C* Fc = Ch.F + (size_t)c * Ch.fmax * Ch.ncols;
  const int* ea = Ch.ea + (size_t)c * Ch.bmax;
  const long tot = (long)Ch.bmax * Ch.bmax;
  for (long idx = blockIdx.y * (long)blockDim.x + threadIdx.x; idx < tot; idx += (long)gridDim.y * blockDim.x) {
    const int a = (int)(idx % Ch.bmax), b = (int)(idx / Ch.bmax);
    const int pa = ea[a], pb = ea[b];
    if (pa < 0 || pb < 0) continue;
    const C v = Fc[(size_t)(Ch.smax + b) * Ch.fmax + Ch.smax + a];
    C& dst = Fp[(size_t)pb * P.fmax + pa];
    dst = cadd(dst, v);
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
      if (!(best > 0)) atomicExch(err, 1);
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
    if (i < w) col[k0 + i] = x[i];
}

// Columns c in [smax, ncols): F[j0:j1, c] = U_blk^{-1} F[j0:j1, c] (non-unit upper).
template <typename C> __global__ void __launch_bounds__(128) k_trsm_upper(LevelK<C> L, int j0, int j1) {
  const int z = blockIdx.x;
  const int fmax = L.fmax, w = j1 - j0;
  C* A = L.F + (size_t)z * fmax * L.ncols;
  __shared__ C Ud[NB][NB + 1];
  for (int idx = threadIdx.x; idx < w * w; idx += blockDim.x) {
    const int i = idx % w, l = idx / w;
    Ud[i][l] = A[(size_t)(j0 + l) * fmax + j0 + i];
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
      C acc = x[i];
#pragma unroll
      for (int l = 0; l < NB; ++l)
        if (l > i && l < w) acc = cfms(acc, Ud[i][l], x[l]);
      x[i] = cdiv(acc, Ud[i][i]);
    }
  }
#pragma unroll
  for (int i = 0; i < NB; ++i)
    if (i < w) col[j0 + i] = x[i];
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
    for (int idx = threadIdx.x; idx < TK * TM; idx += blockDim.x) {
      const int l = idx / TM, rr = idx % TM;
      C va = czero<C>(), vb = czero<C>();
      if (l < kw && rb + rr < r1) va = A[(size_t)(k0 + kk + l) * fmax + rb + rr];
      As[l][rr] = va;
      const int l2 = idx % TK, cc = idx / TK;
      if (l2 < kw && cb + cc < c1) vb = A[(size_t)(cb + cc) * fmax + k0 + kk + l2];
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
template <typename C>
__global__ void __launch_bounds__(256) k_gauss_jordan(LevelK<C> L, LevelK<C> Ch, int has_child, int* err) {
  using Rl = typename RealOf<C>::T;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  C* B = reinterpret_cast<C*>(smem_raw);  // column major, ld = smax
  __shared__ Rl sv[32];
  __shared__ int si[32];
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
  for (int idx = tid; idx < s * nc; idx += NT) {
    const int c = idx / s, r = idx - c * s;
    B[idx] = A[(size_t)c * fmax + r];
  }
  __syncthreads();
  for (int j = 0; j < s; ++j) {
    Rl best = -1;
    int bi = 0x7fffffff;
    for (int r = j + tid; r < s; r += NT) {
      const Rl v = cabs2(B[(size_t)j * s + r]);
      if (v > best) { best = v; bi = r; }
    }
    argmax_block(best, bi, sv, si);
    if (bi == 0x7fffffff) bi = j;
    if (tid == 0 && !(best > 0)) atomicExch(err, 1);
    if (bi != j)
      for (int c = j + tid; c < nc; c += NT) {
        C& x = B[(size_t)c * s + j];
        C& y = B[(size_t)c * s + bi];
        const C t = x;
        x = y;
        y = t;
      }
    __syncthreads();
    const C dg = B[(size_t)j * s + j];
    const Rl den = cabs2(dg);
    C inv;
    inv.x = den > 0 ? dg.x / den : (Rl)0;
    inv.y = den > 0 ? -dg.y / den : (Rl)0;
    for (int c = j + 1 + tid; c < nc; c += NT) {
      C& x = B[(size_t)c * s + j];
      x = cmul(x, inv);
    }
    __syncthreads();
    const int ncol = nc - j - 1;
    for (int idx = tid; idx < ncol * s; idx += NT) {
      const int cq = idx / s, r = idx - cq * s;
      if (r == j) continue;
      const int c = j + 1 + cq;
      C& x = B[(size_t)c * s + r];
      x = cfms(x, B[(size_t)j * s + r], B[(size_t)c * s + j]);
    }
    __syncthreads();
  }
  for (int idx = tid; idx < s * (nc - s); idx += NT) {
    const int cq = idx / s, r = idx - cq * s;
    A[(size_t)(s + cq) * fmax + r] = B[(size_t)(s + cq) * s + r];
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

static bool ensure_buffers(NdPlan* p, int elem_bytes) {
  if (p->F && p->F_bytes == elem_bytes) return false;
  if (p->F) { cudaFree(p->F); p->F = nullptr; }
  if (p->W) { cudaFree(p->W); p->W = nullptr; }
  if (cudaMalloc(&p->F, p->F_elems * elem_bytes) != cudaSuccess) {
    cudaGetLastError();
    LS_FAIL(ENOMEM_, "cudaMalloc of %zu bytes for the fronts failed", p->F_elems * elem_bytes);
  }
  if (cudaMalloc(&p->W, std::max<size_t>(1, p->W_elems) * elem_bytes) != cudaSuccess) {
    cudaGetLastError();
    LS_FAIL(ENOMEM_, "cudaMalloc of %zu bytes for the front vectors failed", p->W_elems * elem_bytes);
  }
  p->F_bytes = p->W_bytes = elem_bytes;
  return true;
}

// threads for the Gauss-Jordan CTA: about 16 entries of the own-row block per thread
static int gj_threads(int s, int nc) {
  const int t = ((s * nc / 16 + 31) / 32) * 32;
  return std::max(32, std::min(256, t));
}

template <typename C> static void launch_gemm(const LevelK<C>& L, int r0, int r1, int c0, int c1, int k0, int k1,
                                              cudaStream_t st) {
  if (r1 <= r0 || c1 <= c0 || k1 <= k0) return;
  const int nr = (r1 - r0 + 63) / 64, nc = (c1 - c0 + 63) / 64;
  LS_LAUNCH(sizeof(C) == 8 ? "nd_gemm_c64" : "nd_gemm_c128", st,
            k_gemm<C><<<dim3(L.nf, nr * nc), 256, 0, st>>>(L, r0, r1, c0, c1, k0, k1));
}

template <typename C> bool nd_prepare(NdPlan* p) { return ensure_buffers(p, sizeof(C)); }

template <typename C>
void nd_factor(NdPlan* p, const void* alpha64, const void* cint64, const void* w2m64, cudaStream_t st) {
  nd_prepare<C>(p);
  nd_factor_launch<C>(p, alpha64, cint64, w2m64, st);
  nd_factor_check(p, st);
}

void nd_factor_check(NdPlan* p, cudaStream_t st) {
  int err = 0;
  LS_CUDA(cudaMemcpyAsync(&err, p->d_err, sizeof(int), cudaMemcpyDeviceToHost, st));
  LS_CUDA(cudaStreamSynchronize(st));
  if (err) LS_FAIL(EINVAL_, "nested-dissection factorization met an exactly singular front");
}

template <typename C>
void nd_factor_launch(NdPlan* p, const void* alpha64, const void* cint64, const void* w2m64, cudaStream_t st) {
  if (!p->F || p->F_bytes != (int)sizeof(C)) LS_FAIL(ESTATE_, "front storage not prepared for this precision");
  const bool f32 = sizeof(C) == 8;
  LS_CUDA(cudaMemsetAsync(p->F, 0, p->F_elems * sizeof(C), st));
  LS_CUDA(cudaMemsetAsync(p->d_err, 0, sizeof(int), st));
  LS_LAUNCH(f32 ? "nd_assemble_c64" : "nd_assemble_c128", st,
            k_assemble<C><<<1024, 256, 0, st>>>(reinterpret_cast<C*>(p->F), p->n_asm, p->d_asm_off, p->d_asm_row,
                                                p->d_asm_t, p->d, p->n, (const double2*)alpha64,
                                                (const double2*)cint64, (const double*)w2m64));
  LS_LAUNCH(f32 ? "nd_ones_c64" : "nd_ones_c128", st,
            k_set_one<C><<<256, 256, 0, st>>>(reinterpret_cast<C*>(p->F), p->n_one, p->d_one_off));
  const int depth = (int)p->lev.size();
  constexpr size_t PANEL_SMEM_MAX = 200 * 1024;
  constexpr size_t GJ_SMEM_MAX = 160 * 1024;
  static bool attr = false;
  if (!attr) {
    LS_CUDA(cudaFuncSetAttribute(k_panel<C, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)PANEL_SMEM_MAX));
    LS_CUDA(cudaFuncSetAttribute(k_gauss_jordan<C>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)GJ_SMEM_MAX));
    attr = true;
  }
  for (int l = depth - 1; l >= 0; --l) {
    prof_tag(l);
    LevelK<C> L = level_k<C>(p, l);
    const bool has_child = l + 1 < depth;
    LevelK<C> Ch = has_child ? level_k<C>(p, l + 1) : L;
    // own rows: [F11 | F12 | I] -> [* | H | F11^{-1}]
    const size_t gjm = (size_t)L.smax * L.ncols * sizeof(C);
    if (gjm <= GJ_SMEM_MAX) {
      // one CTA per front: extend-add, Gauss-Jordan in shared memory, ring rows
      LS_LAUNCH(f32 ? "nd_gauss_jordan_c64" : "nd_gauss_jordan_c128", st,
                k_gauss_jordan<C><<<L.nf, gj_threads(L.smax, L.ncols), gjm, st>>>(L, Ch, has_child ? 1 : 0,
                                                                                   p->d_err));
      launch_gemm<C>(L, L.smax, L.fmax, L.smax, L.ncols, 0, L.smax, st);
      continue;
    }
    if (has_child) {
      const long tot = (long)Ch.bmax * Ch.bmax;
      const unsigned bx = (unsigned)std::max<long>(1, std::min<long>((tot + 255) / 256, 64));
      for (int k = 0; k < 2; ++k)
        LS_LAUNCH(f32 ? "nd_extend_add_c64" : "nd_extend_add_c128", st,
                  k_extend_add<C><<<dim3(Ch.nf, bx), 256, 0, st>>>(L, Ch, k));
    }
    {
      // sweep 1: blocked LU of the own columns on the own rows (pivot rows restricted to
      // them), the block rows of [F12 | I] carried along
      for (int k0 = 0; k0 < L.smax; k0 += NB) {
        const int k1 = std::min(k0 + NB, L.smax);
        const size_t psm = (size_t)(L.smax - k0) * (k1 - k0) * sizeof(C);
        if (psm <= PANEL_SMEM_MAX)
          LS_LAUNCH(f32 ? "nd_panel_c64" : "nd_panel_c128", st,
                    k_panel<C, true><<<L.nf, 512, psm, st>>>(L, k0, k1, p->d_err));
        else
          LS_LAUNCH(f32 ? "nd_panel_c64" : "nd_panel_c128", st,
                    k_panel<C, false><<<L.nf, 512, 0, st>>>(L, k0, k1, p->d_err));
        const int m = L.ncols - k1;
        LS_LAUNCH(f32 ? "nd_trsm_c64" : "nd_trsm_c128", st,
                  k_trsm_lower<C><<<dim3(L.nf, (m + 127) / 128), 128, 0, st>>>(L, k0, k1));
        launch_gemm<C>(L, k1, L.smax, k1, L.ncols, k0, k1, st);
      }
      // sweep 2: backward substitution with U11 on the own rows of [F12 | I]
      const int nblk = (L.smax + NB - 1) / NB;
      for (int jb = nblk - 1; jb >= 0; --jb) {
        const int j0 = jb * NB, j1 = std::min(j0 + NB, L.smax);
        const int m = L.ncols - L.smax;
        LS_LAUNCH(f32 ? "nd_trsm_c64" : "nd_trsm_c128", st,
                  k_trsm_upper<C><<<dim3(L.nf, (m + 127) / 128), 128, 0, st>>>(L, j0, j1));
        launch_gemm<C>(L, 0, j0, L.smax, L.ncols, j0, j1, st);
      }
    }
    // ring rows: [S | Y] = [F22 | 0] - F21 [H | F11^{-1}]
    launch_gemm<C>(L, L.smax, L.fmax, L.smax, L.ncols, 0, L.smax, st);
  }
  prof_tag(-1);
}

// ---------------------------------------------------------------------------------------
// solves
// ---------------------------------------------------------------------------------------

// W[z] = [w_own ; w_ring]: own entries from r plus the children's updates, ring entries
// from the children's updates.
template <typename C>
__global__ void __launch_bounds__(256) k_fwd_gather(LevelK<C> L, LevelK<C> Ch, int has_child, const C* __restrict__ r,
                                                    int nrhs, long N) {
  const int z = blockIdx.x, tid = threadIdx.x, NT = blockDim.x;
  const int fmax = L.fmax, smax = L.smax;
  C* W = L.W + (size_t)z * nrhs * fmax;
  for (int idx = tid; idx < nrhs * fmax; idx += NT) {
    const int rhs = idx / fmax, q = idx % fmax;
    C v = czero<C>();
    if (q < smax) {
      const int g = L.own[(size_t)z * smax + q];
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
        C& x = W[(size_t)rhs * fmax + ps];
        x = cadd(x, Wc[(size_t)rhs * Ch.fmax + Ch.smax + a]);
      }
      __syncthreads();
    }
  }
}

// Forward sweep of one level, gather and product fused (fronts with smax <= FUSED_SMAX):
// a CTA builds w_own (own entries of r plus the children's updates) and the children's
// contributions to its 32 ring rows in shared memory, keeps w_own in W for the backward
// sweep, and writes u_ring = w_ring + Y w_own for its rows.  Columns are split among the
// kg warps and the partial sums added in a fixed order.
constexpr int FUSED_SMAX = 1024;

template <typename C, int RC>
__global__ void __launch_bounds__(sizeof(C) == 8 ? 512 : 256)
    k_fwd(LevelK<C> L, LevelK<C> Ch, int has_child, const C* __restrict__ r, int nrhs, long N) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int z = blockIdx.x, rc0 = blockIdx.z * RC, nr = min(RC, nrhs - rc0);
  const int lane = threadIdx.x & 31, g = threadIdx.x >> 5, kg = blockDim.x >> 5, NT = blockDim.x;
  const int fmax = L.fmax, smax = L.smax;
  const int t0 = smax + blockIdx.y * 32;
  // right-hand-side vectors of one item are RCP = RC + 1 entries apart (odd stride: the
  // per-thread stores of different items fall in different banks)
  constexpr int RCP = RC + 1;
  C* wt = reinterpret_cast<C*>(smem_raw);  // [32][RCP] ring rows of this tile
  C* wo = wt + 32 * RCP;                   // [smax][RCP], later [kg][32][RCP]
  C* W = L.W + (size_t)z * nrhs * fmax;
  const int* own = L.own + (size_t)z * smax;
  // own entries of r: one own variable per thread, its RC right-hand sides loaded together
  for (int q = threadIdx.x; q < smax; q += NT) {
    const int gi = own[q];
    C v[RC];
#pragma unroll
    for (int j = 0; j < RC; ++j) v[j] = (j < nr && gi >= 0) ? r[(size_t)(rc0 + j) * N + gi] : czero<C>();
#pragma unroll
    for (int j = 0; j < RC; ++j) wo[q * RCP + j] = v[j];
  }
  for (int idx = threadIdx.x; idx < 32 * RCP; idx += NT) wt[idx] = czero<C>();
  __syncthreads();
  if (has_child) {
    for (int k = 0; k < 2; ++k) {
      const int c = L.child[(size_t)z * 2 + k];
      if (c < 0) continue;
      const C* Wc = Ch.W + (size_t)c * nrhs * Ch.fmax + Ch.smax;
      const int* ea = Ch.ea + (size_t)c * Ch.bmax;
      for (int a = threadIdx.x; a < Ch.bmax; a += NT) {
        const int ps = ea[a];
        C* dst = ps < 0 ? nullptr : (ps < smax ? &wo[ps * RCP] : ((ps >= t0 && ps < t0 + 32) ? &wt[(ps - t0) * RCP] : nullptr));
        if (!dst) continue;
        C v[RC];
#pragma unroll
        for (int j = 0; j < RC; ++j) v[j] = j < nr ? Wc[(size_t)(rc0 + j) * Ch.fmax + a] : czero<C>();
#pragma unroll
        for (int j = 0; j < RC; ++j) dst[j] = cadd(dst[j], v[j]);
      }
      __syncthreads();
    }
  }
  if (blockIdx.y == 0)
    for (int idx = threadIdx.x; idx < smax * RC; idx += NT) {
      const int q = idx / RC, j = idx % RC;
      if (j < nr) W[(size_t)(rc0 + j) * fmax + q] = wo[q * RCP + j];
    }
  const int row = t0 + lane;
  C acc[RC];
#pragma unroll
  for (int j = 0; j < RC; ++j) acc[j] = czero<C>();
  if (row < fmax) {
    const C* a = L.F + (size_t)z * fmax * L.ncols + (size_t)fmax * fmax + row;  // Y, identity columns
    const int per = (smax + kg - 1) / kg;
    const int k0 = g * per, k1 = min(smax, k0 + per);
    int k = k0;
    for (; k + 4 <= k1; k += 4) {
      const C a0 = a[(size_t)k * fmax], a1 = a[(size_t)(k + 1) * fmax];
      const C a2 = a[(size_t)(k + 2) * fmax], a3 = a[(size_t)(k + 3) * fmax];
      const C* z0 = wo + (size_t)k * RCP;
#pragma unroll
      for (int j = 0; j < RC; ++j) {
        acc[j] = cfma(acc[j], a0, z0[j]);
        acc[j] = cfma(acc[j], a1, z0[RCP + j]);
        acc[j] = cfma(acc[j], a2, z0[2 * RCP + j]);
        acc[j] = cfma(acc[j], a3, z0[3 * RCP + j]);
      }
    }
    for (; k < k1; ++k) {
      const C a0 = a[(size_t)k * fmax];
      const C* z0 = wo + (size_t)k * RCP;
#pragma unroll
      for (int j = 0; j < RC; ++j) acc[j] = cfma(acc[j], a0, z0[j]);
    }
  }
  __syncthreads();
  C* red = wo;
#pragma unroll
  for (int j = 0; j < RC; ++j) red[((size_t)g * 32 + lane) * RCP + j] = acc[j];
  __syncthreads();
  for (int o = threadIdx.x; o < 32 * RC; o += NT) {
    const int ln = o / RC, j = o % RC;
    const int rr = t0 + ln;
    if (rr >= fmax || j >= nr) continue;
    C s = wt[ln * RCP + j];
    for (int q = 0; q < kg; ++q) s = cadd(s, red[((size_t)q * 32 + ln) * RCP + j]);
    W[(size_t)(rc0 + j) * fmax + rr] = s;
  }
}

// Batched multi-right-hand-side products of the solve, one launch per level:
//   MODE 0 (forward):  u_ring = w_ring + Y w_own, Y = -F21 F11^{-1} (ring rows of the
//                      identity columns), written back into the ring part of W;
//   MODE 1 (backward): x_own = F11^{-1} w_own - H x_ring (own rows of [H | F11^{-1}]),
//                      scattered to the solution at the own grid points.
// A CTA takes 32 rows (one warp-wide coalesced segment per column) and splits the columns
// among its kg warps; the kg partial sums are added in a fixed order in shared memory.
// The vector operand (RC right-hand sides) is staged in shared memory, KCH columns at a time.
constexpr int KCH = 256;

template <typename C, int RC, int MODE>
__global__ void __launch_bounds__(sizeof(C) == 8 ? 512 : 256) k_gemv(LevelK<C> L, C* __restrict__ X, int nrhs, long N) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  constexpr int RCP = RC + 1;  // odd item stride, see k_fwd
  C* zs = reinterpret_cast<C*>(smem_raw);  // [KCH][RCP], later [kg][32][RCP]
  const int z = blockIdx.x, rc0 = blockIdx.z * RC, nr = min(RC, nrhs - rc0);
  const int lane = threadIdx.x & 31, g = threadIdx.x >> 5, kg = blockDim.x >> 5;
  const int fmax = L.fmax, smax = L.smax, bmax = L.bmax;
  const int row = (MODE == 0 ? smax : 0) + blockIdx.y * 32 + lane;
  const int rend = MODE == 0 ? fmax : smax;
  const int K = MODE == 0 ? smax : bmax + smax;
  const C* A = L.F + (size_t)z * fmax * L.ncols + (size_t)(MODE == 0 ? fmax : smax) * fmax;
  C* W = L.W + (size_t)z * nrhs * fmax;
  const int* ring = L.ring + (size_t)z * bmax;
  C acc[RC];
#pragma unroll
  for (int j = 0; j < RC; ++j) acc[j] = czero<C>();
  for (int cb = 0; cb < K; cb += KCH) {
    const int kc = min(KCH, K - cb);
    // one column per thread, its RC right-hand sides loaded together
    for (int k = threadIdx.x; k < kc; k += blockDim.x) {
      const int c = cb + k;
      C v[RC];
      if (MODE == 0) {
#pragma unroll
        for (int j = 0; j < RC; ++j) v[j] = j < nr ? W[(size_t)(rc0 + j) * fmax + c] : czero<C>();
      } else if (c < bmax) {
        const int gi = ring[c];
#pragma unroll
        for (int j = 0; j < RC; ++j) {
          C x = czero<C>();
          if (j < nr && gi >= 0) x = X[(size_t)(rc0 + j) * N + gi];
          x.x = -x.x;
          x.y = -x.y;
          v[j] = x;
        }
      } else {
#pragma unroll
        for (int j = 0; j < RC; ++j) v[j] = j < nr ? W[(size_t)(rc0 + j) * fmax + (c - bmax)] : czero<C>();
      }
#pragma unroll
      for (int j = 0; j < RC; ++j) zs[k * RCP + j] = v[j];
    }
    __syncthreads();
    if (row < rend) {
      const int per = (kc + kg - 1) / kg;
      const int k0 = g * per, k1 = min(kc, k0 + per);
      const C* a = A + (size_t)cb * fmax + row;
      int k = k0;
      for (; k + 4 <= k1; k += 4) {
        const C a0 = a[(size_t)k * fmax], a1 = a[(size_t)(k + 1) * fmax];
        const C a2 = a[(size_t)(k + 2) * fmax], a3 = a[(size_t)(k + 3) * fmax];
        const C* z0 = zs + (size_t)k * RCP;
#pragma unroll
        for (int j = 0; j < RC; ++j) {
          acc[j] = cfma(acc[j], a0, z0[j]);
          acc[j] = cfma(acc[j], a1, z0[RCP + j]);
          acc[j] = cfma(acc[j], a2, z0[2 * RCP + j]);
          acc[j] = cfma(acc[j], a3, z0[3 * RCP + j]);
        }
      }
      for (; k < k1; ++k) {
        const C a0 = a[(size_t)k * fmax];
        const C* z0 = zs + (size_t)k * RCP;
#pragma unroll
        for (int j = 0; j < RC; ++j) acc[j] = cfma(acc[j], a0, z0[j]);
      }
    }
    __syncthreads();
  }
#pragma unroll
  for (int j = 0; j < RC; ++j) zs[((size_t)g * 32 + lane) * RCP + j] = acc[j];
  __syncthreads();
  for (int o = threadIdx.x; o < 32 * RC; o += blockDim.x) {
    const int ln = o / RC, j = o % RC;
    const int r = (MODE == 0 ? smax : 0) + blockIdx.y * 32 + ln;
    if (r >= rend || j >= nr) continue;
    C s = czero<C>();
    for (int q = 0; q < kg; ++q) s = cadd(s, zs[((size_t)q * 32 + ln) * RCP + j]);
    if (MODE == 0) {
      C& x = W[(size_t)(rc0 + j) * fmax + r];
      x = cadd(x, s);
    } else {
      const int gi = L.own[(size_t)z * smax + r];
      if (gi >= 0) X[(size_t)(rc0 + j) * N + gi] = s;
    }
  }
}

template <typename C, int RC, int MODE>
static void launch_gemv(const LevelK<C>& L, C* X, int nr, long N, cudaStream_t st) {
  const int rows = MODE == 0 ? L.bmax : L.smax;
  const int K = MODE == 0 ? L.smax : L.bmax + L.smax;
  if (rows <= 0 || K <= 0) return;
  const int kg = std::max(1, std::min(sizeof(C) == 8 ? 16 : 8, K / 16));
  const size_t smem = (size_t)std::max(std::min(KCH, K), kg * 32) * (RC + 1) * sizeof(C);
  static bool attr = false;
  if (!attr) {
    LS_CUDA(cudaFuncSetAttribute(k_gemv<C, RC, MODE>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)((size_t)KCH * 2 * (RC + 1) * sizeof(C))));
    attr = true;
  }
  const dim3 grid(L.nf, (rows + 31) / 32, (nr + RC - 1) / RC);
  const bool f32 = sizeof(C) == 8;
  LS_LAUNCH(MODE == 0 ? (f32 ? "nd_fwd_c64" : "nd_fwd_c128") : (f32 ? "nd_bwd_c64" : "nd_bwd_c128"), st,
            k_gemv<C, RC, MODE><<<grid, 32 * kg, smem, st>>>(L, X, nr, N));
}

constexpr size_t FUSED_SMEM_MAX = 200 * 1024;

template <typename C, int RC> static size_t fwd_fused_smem(int smax) {
  const int kg = std::max(1, std::min(sizeof(C) == 8 ? 16 : 8, smax / 16));
  return (size_t)(32 + std::max(smax, kg * 32)) * (RC + 1) * sizeof(C);
}

template <typename C, int RC>
static void launch_fwd_fused(const LevelK<C>& L, const LevelK<C>& Ch, int has_child, const C* r, int nr, long N,
                             cudaStream_t st) {
  const int kg = std::max(1, std::min(sizeof(C) == 8 ? 16 : 8, L.smax / 16));
  const size_t smem = fwd_fused_smem<C, RC>(L.smax);
  static bool attr = false;
  if (!attr) {
    LS_CUDA(cudaFuncSetAttribute(k_fwd<C, RC>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)FUSED_SMEM_MAX));
    attr = true;
  }
  const dim3 grid(L.nf, std::max(1, (L.bmax + 31) / 32), (nr + RC - 1) / RC);
  LS_LAUNCH(sizeof(C) == 8 ? "nd_fwd_c64" : "nd_fwd_c128", st,
            k_fwd<C, RC><<<grid, 32 * kg, smem, st>>>(L, Ch, has_child, r, nr, N));
}

template <typename C, int RC>
static void solve_chunk(NdPlan* p, int nr, const C* rr, C* xx, cudaStream_t st) {
  const int depth = (int)p->lev.size();
  const bool f32 = sizeof(C) == 8;
  for (int l = depth - 1; l >= 0; --l) {
    prof_tag(l);
    LevelK<C> L = level_k<C>(p, l);
    LevelK<C> Ch = l + 1 < depth ? level_k<C>(p, l + 1) : L;
    if (L.smax <= FUSED_SMAX && fwd_fused_smem<C, RC>(L.smax) <= FUSED_SMEM_MAX) {
      launch_fwd_fused<C, RC>(L, Ch, l + 1 < depth ? 1 : 0, rr, nr, p->N, st);
    } else {
      LS_LAUNCH(f32 ? "nd_fwd_gather_c64" : "nd_fwd_gather_c128", st,
                k_fwd_gather<C><<<L.nf, 256, 0, st>>>(L, Ch, l + 1 < depth ? 1 : 0, rr, nr, p->N));
      launch_gemv<C, RC, 0>(L, xx, nr, p->N, st);
    }
  }
  for (int l = 0; l < depth; ++l) {
    prof_tag(l);
    launch_gemv<C, RC, 1>(level_k<C>(p, l), xx, nr, p->N, st);
  }
  prof_tag(-1);
}

template <typename C> void nd_solve(NdPlan* p, int nrhs, const C* r, C* x, cudaStream_t st) {
  if (!p->F || p->F_bytes != (int)sizeof(C)) LS_FAIL(ESTATE_, "preconditioner not factored in this precision");
  for (int c0 = 0; c0 < nrhs; c0 += SOLVE_CHUNK) {
    const int nr = std::min(SOLVE_CHUNK, nrhs - c0);
    const C* rr = r + (size_t)c0 * p->N;
    C* xx = x + (size_t)c0 * p->N;
    if (nr <= 4) solve_chunk<C, 4>(p, nr, rr, xx, st);
    else solve_chunk<C, 16>(p, nr, rr, xx, st);
  }
}

template void nd_factor<float2>(NdPlan*, const void*, const void*, const void*, cudaStream_t);
template void nd_factor<double2>(NdPlan*, const void*, const void*, const void*, cudaStream_t);
template bool nd_prepare<float2>(NdPlan*);
template bool nd_prepare<double2>(NdPlan*);
template void nd_factor_launch<float2>(NdPlan*, const void*, const void*, const void*, cudaStream_t);
template void nd_factor_launch<double2>(NdPlan*, const void*, const void*, const void*, cudaStream_t);
template void nd_solve<float2>(NdPlan*, int, const float2*, float2*, cudaStream_t);
template void nd_solve<double2>(NdPlan*, int, const double2*, double2*, cudaStream_t);

}  // namespace ls
