// Schur-complement updates of the fronts on the 5th-generation tensor cores (tcgen05):
//
//   C[r0:r1, c0:c1] -= A[r0:r1, k0:k1] B[k0:k1, c0:c1]   (complex FP32, one front per CTA
//                                                         column of the grid)
//
// with A, B, C blocks of the same column-major front (ld = fmax).  The complex product is
// one real product of twice the size,
//   [Re C | Im C] = A' B',  A'[m][2k + {0,1}] = (Re, Im) A[m][k],
//   B' = [[Re B, Im B]; [-Im B, Re B]] (rows 2k, 2k+1),
// and each FP32 operand is split into two TF32 numbers, x = hi + lo, so that
// A'B' ~ A'hi B'hi + A'hi B'lo + A'lo B'hi ("3xTF32": error about 2^-22 relative, the
// accuracy of the FP32 fronts).  A CTA owns a 128-row tile of C and NT = 64 complex columns:
// D = 128 x 128 FP32 accumulators in tensor memory, filled by tcgen05.mma kind::tf32
// (M = 128, N = 128, K = 8 per instruction) from K-major operands in shared memory
// (no-swizzle canonical layout: 8-row x 16-byte core matrices).  The K loop is a two-stage
// pipeline over chunks of KC complex k: while the tensor core runs the MMAs of one chunk, the
// threads convert the next chunk (held in registers) into the other operand stage (3xTF32
// split, canonical layout, conflict-free stores) and load the chunk after it from global
// memory.  One thread issues the MMAs and
// commits each chunk to its stage's mbarrier; 65 KB of shared memory, three CTAs per SM.  All
// waits are bounded and set *err on expiry, and the tensor memory is freed only after the
// last commit has been awaited.
//
// The same kernel, instantiated with EXT, runs the multi-right-hand-side products of the
// solve sweeps on the large fronts: C[z] = A[z] B[z] with A a block of front z (Y on its ring
// rows for the forward sweep, [H | F11^-1] on its own rows for the backward one), B[z] the
// gathered vector operand (k x right-hand side, right-hand sides contiguous) and C[z] a
// dense result (row x right-hand side), both outside the fronts.
#include <atomic>
#include <cuda_runtime.h>

#include <cstdint>
#include <cstdlib>
#include <cstring>

#include "common.cuh"
#include "kernels.h"
#include "prof.h"

namespace ls {

namespace tc {

constexpr int TM = 128;        // rows of C per CTA
constexpr int NT = 64;         // complex columns of C per CTA
constexpr int NP = 2 * NT;     // real columns (Re | Im)
constexpr int KC = 8;          // complex k per chunk
constexpr int KP = 2 * KC;     // real k per chunk
constexpr int KSTEP = 8;       // tf32 k per instruction
constexpr int NSTEP = KP / KSTEP;
constexpr int THREADS = 256;
// one operand slice of KSTEP real k: rows x 32 bytes
constexpr int A_SLICE = TM * KSTEP * 4;   // 4 KB
constexpr int B_SLICE = NP * KSTEP * 4;   // 4 KB
constexpr int A_BYTES = NSTEP * A_SLICE;  // 8 KB (hi or lo)
constexpr int B_BYTES = NSTEP * B_SLICE;  // 8 KB
constexpr int STAGE = 2 * A_BYTES + 2 * B_BYTES;  // hi and lo of A' and B': 32 KB
constexpr int SMEM = 2 * STAGE + 1024;            // two stages + barriers and TMEM address: three CTAs per SM
constexpr long WAIT_LIMIT = 1L << 26;
constexpr long TEST_WAIT_LIMIT = 1L << 10;

__device__ __forceinline__ uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ uint32_t to_tf32(float x) {
  uint32_t r;
  asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
  return r;
}

// byte offset of element (row, k) of a K-major no-swizzle operand slice: core matrices of
// 8 rows x 16 bytes (4 tf32), the two K halves of a row group 128 bytes apart (LBO), row
// groups 256 bytes apart (SBO)
__device__ __forceinline__ int core_off(int row, int k) {
  return ((row >> 3) * 2 + (k >> 2)) * 128 + (row & 7) * 16 + (k & 3) * 4;
}

// shared-memory matrix descriptor: start >> 4 (bits 0-13), LBO >> 4 (16-29), SBO >> 4 (32-45),
// fixed 0b001 (46-48), no swizzle (61-63 = 0)
__device__ __forceinline__ uint64_t sdesc(uint32_t addr) {
  const uint64_t lbo = 128 >> 4, sbo = 256 >> 4;
  return (uint64_t)((addr >> 4) & 0x3FFF) | (lbo << 16) | (sbo << 32) | (1ull << 46);
}

// instruction descriptor, kind::tf32: D F32 (bits 4-5 = 1), A and B TF32 (7-9, 10-12 = 2),
// both K-major, N >> 3 at bits 17-22, M >> 4 at bits 24-28
constexpr uint32_t IDESC = (1u << 4) | (2u << 7) | (2u << 10) | ((uint32_t)(NP >> 3) << 17) | ((uint32_t)(TM >> 4) << 24);

__device__ __forceinline__ void mma_tf32(uint32_t dtmem, uint64_t ad, uint64_t bd, int accumulate) {
  asm volatile(
      "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
      " tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n}\n" ::"r"(dtmem),
      "l"(ad), "l"(bd), "r"(IDESC), "r"(accumulate));
}

__device__ __forceinline__ void mma_commit(uint32_t mbar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];\n" ::"r"(mbar) : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint32_t mbar, uint32_t phase) {
  uint32_t ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(ok)
      : "r"(mbar), "r"(phase)
      : "memory");
  return ok != 0;
}

// waits for the given phase of the barrier; false if the bound expired
__device__ __forceinline__ bool mbar_wait(uint32_t mbar, uint32_t phase, long limit) {
  for (long it = 0; it < limit; ++it)
    if (mbar_try_wait(mbar, phase)) return true;
  return false;
}

}  // namespace tc

struct TcArgs {
  float2* F;         // fronts of the level
  long fstride;      // elements per front (fmax * ncols)
  int fmax;          // leading dimension
  int r0, r1, c0, c1, k0, k1;
  int ntr;           // row tiles (grid.y = ntr * column tiles)
  int* err;
  int test_no_mma;   // test hook: issue no MMA and no commit, so that the bounded waits expire
  long wait_limit;   // iterations of a bounded mbarrier wait
  // EXT: B[z][k][n] = Bx[z * bstride + (k - k0) * ldb + n], C[z][r][n] = Cx[z * cstride +
  // (r - r0) * ldc + n] (written, not accumulated); columns n in [c0, c1).  The k range may be
  // split over grid.z: split s takes k in [k0 + s ksz, k0 + (s + 1) ksz) and writes its
  // partial product to Cx + s * split_stride
  const float2* Bx;
  long bstride;
  int ldb;
  float2* Cx;
  long cstride;
  int ldc;
  int ksz;
  long split_stride;
};

template <bool EXT>
__global__ void __launch_bounds__(tc::THREADS) k_tc_cgemm(TcArgs a) {
  using namespace tc;
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  uint64_t* mbar = reinterpret_cast<uint64_t*>(smem_raw + 2 * STAGE);  // one per stage
  uint32_t* tslot = reinterpret_cast<uint32_t*>(mbar + 2);
  __shared__ int failed;

  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int z = blockIdx.x;
  const int tr = blockIdx.y % a.ntr, tcn = blockIdx.y / a.ntr;
  const int rb = a.r0 + tr * TM, cb = a.c0 + tcn * NT;
  float2* F = a.F + (size_t)z * a.fstride;
  const int fmax = a.fmax;

  if (tid == 0) {
    failed = 0;
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;\n" ::"r"(smem_u32(mbar)) : "memory");
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;\n" ::"r"(smem_u32(mbar + 1)) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;\n" ::"r"(smem_u32(tslot)),
                 "r"(NP)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;\n" ::: "memory");
  }
  asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
  const uint32_t tmem = *tslot;

  const int kbeg = EXT ? (int)blockIdx.z * a.ksz : 0;
  const int K = EXT ? min(a.k1 - a.k0 - kbeg, a.ksz) : a.k1 - a.k0;
  const int nchunk = (K + KC - 1) / KC;
  // global loads of one chunk into registers.  Element u of a thread: idx = u * THREADS + tid,
  // group idx / 32 of 32 entries = 8 consecutive rows (or B columns) x 4 consecutive k, lane
  // bits 0-2 the row, bits 3-4 the k.  Its 32 shared-memory stores (8 bytes each) then fill
  // 8 rows x 16 bytes of two neighbouring core matrices, 256 distinct bytes: no bank
  // conflict; the global loads are 8-row (64-byte) runs of a column of A and 4-entry
  // (32-byte) runs of a column of B
  constexpr int PA = TM * KC / THREADS, PB = NT * KC / THREADS;
  float2 va[PA], vb[PB];
  auto a_of = [&](int u, int& m, int& k) {
    const int idx = u * THREADS + tid, grp = idx >> 5, ln = idx & 31;
    m = (grp >> 1) * 8 + (ln & 7);
    k = (grp & 1) * 4 + (ln >> 3);
  };
  auto b_of = [&](int u, int& n, int& k) {
    const int idx = u * THREADS + tid, grp = idx >> 5, ln = idx & 31;
    n = (grp >> 1) * 8 + (ln & 7);
    k = (grp & 1) * 4 + (ln >> 3);
  };
  auto load = [&](int kc) {
    const int kw = min(KC, K - kc);
#pragma unroll
    for (int u = 0; u < PA; ++u) {
      int m, k;
      a_of(u, m, k);
      va[u] = (k < kw && rb + m < a.r1) ? F[(size_t)(a.k0 + kbeg + kc + k) * fmax + rb + m] : make_float2(0.f, 0.f);
    }
#pragma unroll
    for (int u = 0; u < PB; ++u) {
      int n, k;
      b_of(u, n, k);
      if constexpr (EXT)
        vb[u] = (k < kw && cb + n < a.c1) ? a.Bx[(size_t)z * a.bstride + (size_t)(kbeg + kc + k) * a.ldb + cb + n]
                                          : make_float2(0.f, 0.f);
      else
        vb[u] = (k < kw && cb + n < a.c1) ? F[(size_t)(cb + n) * fmax + a.k0 + kc + k] : make_float2(0.f, 0.f);
    }
  };
  // the registers of one chunk -> stage st: A' (TM x KP): element (m, 2k + p); B' (NP x KP,
  // K-major): column n < NT holds (Re B, -Im B), column NT + n holds (Im B, Re B); each as
  // the TF32 pair hi, lo = x - hi
  auto convert = [&](int st) {
    unsigned char* Ahi = smem_raw + st * STAGE;
    unsigned char* Alo = Ahi + A_BYTES;
    unsigned char* Bhi = Alo + A_BYTES;
    unsigned char* Blo = Bhi + B_BYTES;
#pragma unroll
    for (int u = 0; u < PA; ++u) {
      int m, k;
      a_of(u, m, k);
      const float2 v = va[u];
      const int kr = 2 * k;  // real k within the chunk
      const int s = kr / KSTEP, kk = kr % KSTEP;
      const uint32_t hx = to_tf32(v.x), hy = to_tf32(v.y);
      const uint32_t lx = to_tf32(v.x - __uint_as_float(hx)), ly = to_tf32(v.y - __uint_as_float(hy));
      const int o = s * A_SLICE + core_off(m, kk);
      *reinterpret_cast<uint2*>(Ahi + o) = make_uint2(hx, hy);  // kk even: (2k, 2k+1) adjacent
      *reinterpret_cast<uint2*>(Alo + o) = make_uint2(lx, ly);
    }
#pragma unroll
    for (int u = 0; u < PB; ++u) {
      int n, k;
      b_of(u, n, k);
      const float re = vb[u].x, im = vb[u].y;
      const int kr = 2 * k, s = kr / KSTEP, kk = kr % KSTEP;
      const uint32_t hre = to_tf32(re), him = to_tf32(im), hnim = to_tf32(-im);
      const uint32_t lre = to_tf32(re - __uint_as_float(hre)), lim = to_tf32(im - __uint_as_float(him));
      const uint32_t lnim = to_tf32(-im - __uint_as_float(hnim));
      const int o1 = s * B_SLICE + core_off(n, kk), o2 = s * B_SLICE + core_off(NT + n, kk);
      *reinterpret_cast<uint2*>(Bhi + o1) = make_uint2(hre, hnim);
      *reinterpret_cast<uint2*>(Blo + o1) = make_uint2(lre, lnim);
      *reinterpret_cast<uint2*>(Bhi + o2) = make_uint2(him, hre);
      *reinterpret_cast<uint2*>(Blo + o2) = make_uint2(lim, lre);
    }
  };
  // one thread: the chunk's MMAs on stage st (3 per K step: hi hi, hi lo, lo hi), committed
  // to the stage's barrier
  auto issue = [&](int st, bool first) {
    const unsigned char* Ahi = smem_raw + st * STAGE;
    const unsigned char* Alo = Ahi + A_BYTES;
    const unsigned char* Bhi = Alo + A_BYTES;
    const unsigned char* Blo = Bhi + B_BYTES;
    asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
    if (a.test_no_mma) return;
    for (int s = 0; s < NSTEP; ++s) {
      const uint64_t ah = sdesc(smem_u32(Ahi + s * A_SLICE)), al = sdesc(smem_u32(Alo + s * A_SLICE));
      const uint64_t bh = sdesc(smem_u32(Bhi + s * B_SLICE)), bl = sdesc(smem_u32(Blo + s * B_SLICE));
      mma_tf32(tmem, ah, bh, (!first || s > 0) ? 1 : 0);
      mma_tf32(tmem, ah, bl, 1);
      mma_tf32(tmem, al, bh, 1);
    }
    mma_commit(smem_u32(mbar + st));
  };

  // two-stage pipeline: the registers of chunk ch + 1 load while the MMAs of chunk ch - 1 run
  // and chunk ch is converted into the stage the MMAs of chunk ch - 2 have released
  uint32_t phase[2] = {0u, 0u};
  int last = -1;  // last chunk whose MMAs were issued
  if (nchunk > 0) load(0);
  for (int ch = 0; ch < nchunk; ++ch) {
    const int st = ch & 1;
    if (ch >= 2) {
      if (!tc::mbar_wait(smem_u32(mbar + st), phase[st], a.wait_limit)) {
        if (tid == 0) atomicExch(a.err, 2);
        failed = 1;
      }
      phase[st] ^= 1u;
      __syncthreads();
      if (failed) break;
    }
    convert(st);
    if (ch + 1 < nchunk) load((ch + 1) * KC);
    // generic-proxy writes -> visible to the tensor core's async proxy
    asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
    __syncthreads();
    if (tid == 0) issue(st, ch == 0);
    last = ch;
  }
  // the last commit covers every MMA issued before it.  If it does not arrive within the
  // bound, the error is set and it is awaited once more (bounded) before the tensor memory
  // is freed, so that no MMA issued here can still be writing it
  if (last >= 0) {
    const int st = last & 1;
    if (!tc::mbar_wait(smem_u32(mbar + st), phase[st], a.wait_limit)) {
      if (tid == 0) atomicExch(a.err, 2);
      failed = 1;
      tc::mbar_wait(smem_u32(mbar + st), phase[st], a.wait_limit);
    }
  }
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");

  if (!failed && last >= 0) {
    // ---- epilogue: warp w reads TMEM lanes 32 (w % 4) .., columns of half w / 4 of the Re
    // and the Im blocks, and subtracts from C
    const int q = warp & 3, half = warp >> 2;
    const int m = q * 32 + lane;
    const uint32_t lane_base = (uint32_t)(q * 32) << 16;
    for (int cc = 0; cc < NT / 2; cc += 16) {
      const int col = half * (NT / 2) + cc;
      uint32_t re[16], im[16];
      asm volatile(
          "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];\n"
          : "=r"(re[0]), "=r"(re[1]), "=r"(re[2]), "=r"(re[3]), "=r"(re[4]), "=r"(re[5]), "=r"(re[6]), "=r"(re[7]),
            "=r"(re[8]), "=r"(re[9]), "=r"(re[10]), "=r"(re[11]), "=r"(re[12]), "=r"(re[13]), "=r"(re[14]),
            "=r"(re[15])
          : "r"(tmem + lane_base + (uint32_t)col));
      asm volatile(
          "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];\n"
          : "=r"(im[0]), "=r"(im[1]), "=r"(im[2]), "=r"(im[3]), "=r"(im[4]), "=r"(im[5]), "=r"(im[6]), "=r"(im[7]),
            "=r"(im[8]), "=r"(im[9]), "=r"(im[10]), "=r"(im[11]), "=r"(im[12]), "=r"(im[13]), "=r"(im[14]),
            "=r"(im[15])
          : "r"(tmem + lane_base + (uint32_t)(NT + col)));
      asm volatile("tcgen05.wait::ld.sync.aligned;\n" ::: "memory");
      if constexpr (EXT) {
        // 16 consecutive right-hand sides of one row: 8 16-byte stores
        if (rb + m < a.r1) {
          float2* cr = a.Cx + (size_t)blockIdx.z * a.split_stride + (size_t)z * a.cstride +
                       (size_t)(rb + m - a.r0) * a.ldc + cb + col;
          if (cb + col + 16 <= a.c1) {
#pragma unroll
            for (int j = 0; j < 16; j += 2)
              reinterpret_cast<float4*>(cr)[j / 2] = make_float4(__uint_as_float(re[j]), __uint_as_float(im[j]),
                                                                 __uint_as_float(re[j + 1]), __uint_as_float(im[j + 1]));
          } else {
#pragma unroll
            for (int j = 0; j < 16; ++j)
              if (cb + col + j < a.c1) cr[j] = make_float2(__uint_as_float(re[j]), __uint_as_float(im[j]));
          }
        }
      } else if (rb + m < a.r1) {
#pragma unroll
        for (int j = 0; j < 16; ++j) {
          const int c = cb + col + j;
          if (c < a.c1) {
            float2& x = F[(size_t)c * fmax + rb + m];
            x.x -= __uint_as_float(re[j]);
            x.y -= __uint_as_float(im[j]);
          }
        }
      }
    }
  }
  asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
  __syncthreads();
  if (warp == 0)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;\n" ::"r"(tmem), "r"(NP) : "memory");
}

bool tc_enabled() {
  static const bool on = [] {
    const char* e = std::getenv("LS_TC");
    return !(e && std::strcmp(e, "0") == 0);
  }();
  return on;
}

template <bool EXT> static void tc_smem_attr() {
  static std::atomic<bool> attr{false};  // set once per process; repeats are harmless
  if (!attr.load(std::memory_order_acquire)) {
    LS_CUDA(cudaFuncSetAttribute(k_tc_cgemm<EXT>, cudaFuncAttributeMaxDynamicSharedMemorySize, tc::SMEM));
    attr.store(true, std::memory_order_release);
  }
}

// C -= A B on every front of a level (see the file comment); a no-op for empty ranges
void tc_cgemm(float2* F, long fstride, int fmax, int nf, int r0, int r1, int c0, int c1, int k0, int k1, int* err,
              cudaStream_t st) {
  if (r1 <= r0 || c1 <= c0 || k1 <= k0 || nf <= 0) return;
  tc_smem_attr<false>();
  TcArgs a{};
  // test hook (off unless LS_TEST_TC_TIMEOUT=1): no MMA is issued and the waits are short,
  // so that the bounded waits expire with nothing in flight and ls_factor reports LS_ETIMEOUT
  const char* hook = std::getenv("LS_TEST_TC_TIMEOUT");
  a.test_no_mma = (hook && hook[0] == '1') ? 1 : 0;
  a.wait_limit = a.test_no_mma ? tc::TEST_WAIT_LIMIT : tc::WAIT_LIMIT;
  a.F = F;
  a.fstride = fstride;
  a.fmax = fmax;
  a.r0 = r0; a.r1 = r1; a.c0 = c0; a.c1 = c1; a.k0 = k0; a.k1 = k1;
  a.ntr = (r1 - r0 + tc::TM - 1) / tc::TM;
  a.err = err;
  const int ntc = (c1 - c0 + tc::NT - 1) / tc::NT;
  LS_LAUNCH("nd_gemm_tc_c64", st, k_tc_cgemm<false><<<dim3(nf, a.ntr * ntc), tc::THREADS, tc::SMEM, st>>>(a));
}

// C[z] = A[z] B[z] for the sweeps (see the file comment): A = rows [r0, r1) x columns
// [k0, k1) of front z, B[z] (k1 - k0) x ncols at B + z * bstride (ld ldb), C[z]
// (r1 - r0) x ncols at C + z * cstride (ld ldc); with nsplit > 1 split s of the k range
// (ksz columns each, a multiple of the chunk) writes its partial product at
// C + s * split_stride (the caller adds them)
void tc_sweep_gemm(const float2* F, long fstride, int fmax, int nf, int r0, int r1, int k0, int k1, const float2* B,
                   long bstride, int ldb, float2* C, long cstride, int ldc, int ncols, int nsplit, int ksz,
                   long split_stride, int* err, cudaStream_t st, const char* cls) {
  if (r1 <= r0 || ncols <= 0 || k1 <= k0 || nf <= 0) return;
  if (nsplit < 1 || ksz % tc::KC != 0 || (long)(nsplit - 1) * ksz >= k1 - k0 || (long)nsplit * ksz < k1 - k0)
    LS_FAIL(EINVAL_, "tensor-core sweep: bad split of the k range");
  tc_smem_attr<true>();
  TcArgs a{};
  a.test_no_mma = 0;
  a.wait_limit = tc::WAIT_LIMIT;
  a.F = const_cast<float2*>(F);
  a.fstride = fstride;
  a.fmax = fmax;
  a.r0 = r0; a.r1 = r1; a.c0 = 0; a.c1 = ncols; a.k0 = k0; a.k1 = k1;
  a.ntr = (r1 - r0 + tc::TM - 1) / tc::TM;
  a.err = err;
  a.Bx = B; a.bstride = bstride; a.ldb = ldb;
  a.Cx = C; a.cstride = cstride; a.ldc = ldc;
  a.ksz = ksz; a.split_stride = split_stride;
  const int ntc = (ncols + tc::NT - 1) / tc::NT;
  LS_LAUNCH(cls, st, k_tc_cgemm<true><<<dim3(nf, a.ntr * ntc, nsplit), tc::THREADS, tc::SMEM, st>>>(a));
}

}  // namespace ls
