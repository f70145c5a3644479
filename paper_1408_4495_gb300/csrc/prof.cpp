// Launch instrumentation: every kernel launch of the library goes through prof_begin /
// prof_end with its kernel class.  Counting is always on (one atomic add per launch); for
// one selected class the launches are also bracketed by CUDA events on their own stream,
// so that a caller can measure that class's average device duration inside a longer run.
#include <cuda_runtime.h>

#include <atomic>
#include <cstdio>
#include <cstring>
#include <map>
#include <mutex>
#include <string>
#include <vector>

#include "prof.h"

namespace ls {

namespace {
std::mutex mu;
std::map<std::string, long> counts;
std::string timed;
struct Pair {
  cudaEvent_t a, b;
};
std::vector<Pair> pairs;
std::vector<cudaEvent_t> open_ev;
std::atomic<bool> active{false};
std::atomic<bool> timing{false};

cudaEvent_t take() {
  cudaEvent_t e;
  cudaEventCreate(&e);
  return e;
}
}  // namespace

void prof_begin(const char* cls, cudaStream_t st) {
  if (!active.load(std::memory_order_relaxed)) return;
  std::lock_guard<std::mutex> lk(mu);
  counts[cls] += 1;
  if (timing && timed == cls) {
    cudaEvent_t e = take();
    cudaEventRecord(e, st);
    open_ev.push_back(e);
  }
}

void prof_end(const char* cls, cudaStream_t st) {
  if (!active.load(std::memory_order_relaxed) || !timing) return;
  std::lock_guard<std::mutex> lk(mu);
  if (timed == cls && !open_ev.empty()) {
    cudaEvent_t b;
    cudaEventCreate(&b);
    cudaEventRecord(b, st);
    pairs.push_back({open_ev.back(), b});
    open_ev.pop_back();
  }
}

void prof_start(const char* timed_class) {
  std::lock_guard<std::mutex> lk(mu);
  counts.clear();
  for (auto& p : pairs) {
    cudaEventDestroy(p.a);
    cudaEventDestroy(p.b);
  }
  pairs.clear();
  timed = timed_class ? timed_class : "";
  timing = !timed.empty();
  active = true;
}

int prof_stop(char* out, int cap) {
  std::lock_guard<std::mutex> lk(mu);
  active = false;
  timing = false;
  double ms = 0;
  long ok = 0;
  for (auto& p : pairs) {
    cudaEventSynchronize(p.b);
    float t = 0;
    if (cudaEventElapsedTime(&t, p.a, p.b) == cudaSuccess) {
      ms += t;
      ++ok;
    }
    cudaEventDestroy(p.a);
    cudaEventDestroy(p.b);
  }
  pairs.clear();
  cudaGetLastError();
  std::string s = "{\"counts\": {";
  long total = 0;
  bool first = true;
  for (auto& kv : counts) {
    char b[160];
    snprintf(b, sizeof b, "%s\"%s\": %ld", first ? "" : ", ", kv.first.c_str(), kv.second);
    s += b;
    total += kv.second;
    first = false;
  }
  char b[256];
  snprintf(b, sizeof b, "}, \"total\": %ld, \"timed\": {\"class\": \"%s\", \"launches\": %ld, \"ms\": %.9g}}", total,
           timed.c_str(), ok, ms);
  s += b;
  if (out && cap > 0) {
    std::strncpy(out, s.c_str(), (size_t)cap - 1);
    out[cap - 1] = 0;
  }
  return (int)s.size();
}

}  // namespace ls
