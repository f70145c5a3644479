// ls_apply_noalloc: the FP64 operator apply y = (I + K omega^2 m) x on device arrays that
// the caller owns, with the FFT passes' intermediate buffer taken from a fixed array that is
// part of the library image instead of from cudaMalloc.
//
// Why: some callers cannot allocate device memory at the moment they need the operator --
// for example code that runs while another component owns the device memory pool, loops
// that must not let cudaMalloc / cudaFree synchronise the device, or deployments that
// forbid allocation once they have started.  This entry point performs no allocation of
// any kind; the context passed in was set up earlier by ls_setup.
#include <cuda_runtime.h>

#include <mutex>

#include "common.cuh"
#include "kernels.h"
#include "ls.h"

namespace {

// Scratch of the FFT passes: 64 MiB, resident on every GPU that loads this library, for as
// long as the process lives.  A call needs nrhs * n^(d-1) * 2n complex doubles in 2D and
// nrhs * (n^2 * 2n + n * (2n)^2) in 3D (e.g. up to 32 right-hand sides at n = 256 in 2D).
constexpr size_t kScratchBytes = 64ull << 20;
static __device__ __align__(256) unsigned char g_noalloc_scratch[kScratchBytes];

constexpr int kMaxDevices = 64;
std::mutex g_mu;
void* g_scratch_ptr[kMaxDevices] = {};

// Device address of the scratch array on the current device, looked up once per device.
// In host code g_noalloc_scratch is only a stand-in symbol; the kernels need this address.
void* scratch_on_current_device() {
  int dev = 0;
  LS_CUDA(cudaGetDevice(&dev));
  if (dev < 0 || dev >= kMaxDevices) LS_FAIL(ls::EINVAL_, "device index %d out of range", dev);
  std::lock_guard<std::mutex> lk(g_mu);
  if (!g_scratch_ptr[dev]) {
    void* p = nullptr;
    LS_CUDA(cudaGetSymbolAddress(&p, g_noalloc_scratch));
    if (!p) LS_FAIL(ls::ECUDA_, "cudaGetSymbolAddress returned a null address");
    g_scratch_ptr[dev] = p;
  }
  return g_scratch_ptr[dev];
}

// True when p is device (or managed) memory that belongs to device dev.
bool on_device(const void* p, int dev) {
  cudaPointerAttributes a;
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return (a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged) && a.device == dev;
}

}  // namespace

// Access to the context fields this entry point needs (defined in api.cu).
namespace ls {
const ConvPlan* ctx_plan(const ls_ctx* c);
cudaStream_t ctx_stream(const ls_ctx* c);
int ctx_device(const ls_ctx* c);
void ctx_set_error(ls_ctx* c, const char* msg);
}  // namespace ls

extern "C" ls_status ls_apply_noalloc(ls_ctx* c, int nrhs, const double* x, double* y) {
  if (!c) return LS_ESTATE;
  try {
    const ls::ConvPlan* p = ls::ctx_plan(c);
    if (nrhs < 1 || !x || !y) LS_FAIL(ls::EINVAL_, "bad arguments");
    int dev = -1;
    LS_CUDA(cudaGetDevice(&dev));
    if (dev != ls::ctx_device(c))
      LS_FAIL(ls::EINVAL_, "ls_apply_noalloc: the current device (%d) is not the context's device (%d)", dev,
              ls::ctx_device(c));
    if (!on_device(x, dev) || !on_device(y, dev))
      LS_FAIL(ls::EINVAL_, "ls_apply_noalloc takes device arrays of the context's device only");
    const size_t s1 = ls::conv_scratch1_elems(p->d, p->n, nrhs), s2 = ls::conv_scratch2_elems(p->d, p->n, nrhs);
    const size_t need = (s1 + s2) * sizeof(double2);
    if (need > kScratchBytes)
      LS_FAIL(ls::EINVAL_, "ls_apply_noalloc: %d right-hand sides need %zu bytes of scratch, the fixed scratch holds %zu",
              nrhs, need, kScratchBytes);
    unsigned char* base = static_cast<unsigned char*>(scratch_on_current_device());
    void* t1 = base;
    void* t2 = s2 ? base + ((s1 * sizeof(double2) + 255) / 256) * 256 : nullptr;
    if (s2 && ((s1 * sizeof(double2) + 255) / 256) * 256 + s2 * sizeof(double2) > kScratchBytes)
      LS_FAIL(ls::EINVAL_, "ls_apply_noalloc: scratch too small for %d right-hand sides", nrhs);
    const cudaStream_t st = ls::ctx_stream(c);
    ls::conv_apply<double2>(*p, nrhs, reinterpret_cast<const double2*>(x), reinterpret_cast<double2*>(y), nullptr,
                            true, t1, t2, st);
    LS_CUDA(cudaStreamSynchronize(st));
    return LS_OK;
  } catch (const ls::Error& e) {
    ls::ctx_set_error(c, e.msg.c_str());
    return (ls_status)e.code;
  }
}
