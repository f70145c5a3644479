// Caching allocator: contexts created and freed in a loop (one medium after another)
// would otherwise pay cudaMalloc / cudaFree of the fronts, the Krylov basis and the FFT
// scratch on every context; freed blocks are kept per (device, size class) and handed to
// the next request of that class.  Size classes: powers of two up to 1 MiB, multiples of
// 2 MiB above.  At most CACHE_MAX bytes stay cached; beyond that blocks go back to the
// driver.
#include "alloc.h"

#include <cuda_runtime.h>

#include <atomic>
#include <map>
#include <mutex>
#include <unordered_map>

#include "common.cuh"
#include "ls.h"

namespace ls {

namespace {

constexpr size_t CACHE_MAX = size_t(16) << 30;

struct Pool {
  std::mutex mu;
  std::unordered_map<void*, std::pair<int, size_t>> live;  // block -> (device, class size)
  std::multimap<std::pair<int, size_t>, void*> idle;
  size_t cached = 0;
};

Pool& pool() {
  static Pool* p = new Pool;  // never destroyed: blocks may be freed during process exit
  return *p;
}

size_t size_class(size_t bytes) {
  if (bytes <= (size_t(1) << 20)) {
    size_t s = 512;
    while (s < bytes) s <<= 1;
    return s;
  }
  const size_t g = size_t(2) << 20;
  return (bytes + g - 1) / g * g;
}

// Host-side fault injection (ls_fault_alloc): the number of device allocations still to
// pass before one is refused; 0 = disarmed.
std::atomic<long> fault_countdown{0};

}  // namespace

void* dev_alloc(size_t bytes) {
  for (long k = fault_countdown.load(); k > 0;) {
    if (fault_countdown.compare_exchange_weak(k, k - 1)) {
      if (k == 1) LS_FAIL(ENOMEM_, "device allocation of %zu bytes refused (injected by ls_fault_alloc)", bytes);
      break;
    }
  }
  int dev = 0;
  LS_CUDA(cudaGetDevice(&dev));
  const size_t cls = size_class(bytes == 0 ? 1 : bytes);
  Pool& P = pool();
  {
    std::lock_guard<std::mutex> lk(P.mu);
    auto it = P.idle.find({dev, cls});
    if (it != P.idle.end()) {
      void* p = it->second;
      P.idle.erase(it);
      P.cached -= cls;
      P.live[p] = {dev, cls};
      return p;
    }
  }
  void* p = nullptr;
  if (cudaMalloc(&p, cls) != cudaSuccess) {
    cudaGetLastError();
    // free the cached blocks of this device (cudaFree) and retry once
    std::multimap<std::pair<int, size_t>, void*> drop;
    {
      std::lock_guard<std::mutex> lk(P.mu);
      for (auto it = P.idle.begin(); it != P.idle.end();) {
        if (it->first.first == dev) {
          P.cached -= it->first.second;
          drop.insert(*it);
          it = P.idle.erase(it);
        } else {
          ++it;
        }
      }
    }
    for (auto& kv : drop) cudaFree(kv.second);
    if (cudaMalloc(&p, cls) != cudaSuccess) {
      cudaGetLastError();
      LS_FAIL(ENOMEM_, "cudaMalloc of %zu bytes failed", cls);
    }
  }
  std::lock_guard<std::mutex> lk(P.mu);
  P.live[p] = {dev, cls};
  return p;
}

void dev_free(void* p) {
  if (!p) return;
  Pool& P = pool();
  std::pair<int, size_t> key;
  {
    std::lock_guard<std::mutex> lk(P.mu);
    auto it = P.live.find(p);
    if (it == P.live.end()) return;
    key = it->second;
    P.live.erase(it);
    if (P.cached + key.second <= CACHE_MAX) {
      P.idle.insert({key, p});
      P.cached += key.second;
      return;
    }
  }
  cudaFree(p);
}

}  // namespace ls

extern "C" ls_status ls_fault_alloc(long k) {
  if (k < 0) return LS_EINVAL;
  ls::fault_countdown.store(k);
  return LS_OK;
}
