// Launch instrumentation: every kernel launch of the library goes through prof_begin /
// prof_end with its kernel class.  While a measurement is active the launches are counted
// per class; for one selected class (or all, "*" / "**") the launches are also bracketed by
// CUDA events on their own stream, so that a caller can measure device durations inside a
// longer run.  Launches recorded into a CUDA graph are counted into the graph's own tally
// (prof_capture_begin / prof_capture_end), which is added to the counters at every replay.
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
  std::string cls;
};
std::vector<Pair> pairs;
std::vector<cudaEvent_t> open_ev;
std::atomic<bool> active{false};
std::atomic<bool> timing{false};
thread_local int tag = -1;
thread_local std::map<std::string, long>* capture_sink = nullptr;

bool timed_match(const char* cls) { return timed == cls || timed == "*" || timed == "**"; }
}  // namespace

void prof_tag(int t) { tag = t; }

bool prof_timing_active() { return timing.load(std::memory_order_relaxed); }

void prof_capture_begin(std::map<std::string, long>* sink) { capture_sink = sink; }
void prof_capture_end() { capture_sink = nullptr; }

void prof_count_replay(const std::map<std::string, long>& tally) {
  if (!active.load(std::memory_order_relaxed)) return;
  std::lock_guard<std::mutex> lk(mu);
  for (auto& kv : tally) counts[kv.first] += kv.second;
}

void prof_begin(const char* cls, cudaStream_t st) {
  if (capture_sink) {
    (*capture_sink)[cls] += 1;
    return;
  }
  if (!active.load(std::memory_order_relaxed)) return;
  std::lock_guard<std::mutex> lk(mu);
  counts[cls] += 1;
  if (timing && timed_match(cls)) {
    cudaEvent_t e;
    cudaEventCreate(&e);
    cudaEventRecord(e, st);
    open_ev.push_back(e);
  }
}

void prof_end(const char* cls, cudaStream_t st) {
  if (capture_sink || !active.load(std::memory_order_relaxed) || !timing) return;
  std::lock_guard<std::mutex> lk(mu);
  if (timed_match(cls) && !open_ev.empty()) {
    cudaEvent_t b;
    cudaEventCreate(&b);
    cudaEventRecord(b, st);
    std::string key = cls;
    if (timed == "**" && tag >= 0) key += "@L" + std::to_string(tag);
    pairs.push_back({open_ev.back(), b, key});
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
  std::map<std::string, double> per;
  for (auto& p : pairs) {
    cudaEventSynchronize(p.b);
    float t = 0;
    if (cudaEventElapsedTime(&t, p.a, p.b) == cudaSuccess) {
      ms += t;
      ++ok;
      per[p.cls] += t;
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
  snprintf(b, sizeof b, "}, \"total\": %ld, \"timed\": {\"class\": \"%s\", \"launches\": %ld, \"ms\": %.9g}", total,
           timed.c_str(), ok, ms);
  s += b;
  s += ", \"ms_by_class\": {";
  first = true;
  for (auto& kv : per) {
    char c[160];
    snprintf(c, sizeof c, "%s\"%s\": %.6g", first ? "" : ", ", kv.first.c_str(), kv.second);
    s += c;
    first = false;
  }
  s += "}}";
  if (out && cap > 0) {
    std::strncpy(out, s.c_str(), (size_t)cap - 1);
    out[cap - 1] = 0;
  }
  return (int)s.size();
}

}  // namespace ls
