// Launch instrumentation (prof.cpp).
#pragma once

#include <cuda_runtime.h>

#include <map>
#include <string>

namespace ls {

void prof_tag(int level);  // level tag for "**" timing (-1: none)
void prof_begin(const char* cls, cudaStream_t st);
void prof_end(const char* cls, cudaStream_t st);
void prof_start(const char* timed_class);
int prof_stop(char* out, int cap);
// true while launches are being timed with events (CUDA graphs are then bypassed)
bool prof_timing_active();
// launches issued between these calls (on this thread) are tallied into *sink, not counted
void prof_capture_begin(std::map<std::string, long>* sink);
void prof_capture_end();
// adds a captured graph's tally to the counters (one replay)
void prof_count_replay(const std::map<std::string, long>& tally);

}  // namespace ls

// Launches a kernel of class `cls` on stream `st` and checks the launch.
#define LS_LAUNCH(cls, st, ...)          \
  do {                                   \
    ls::prof_begin(cls, st);             \
    __VA_ARGS__;                         \
    ls::prof_end(cls, st);               \
    LS_CHECK_LAUNCH();                   \
  } while (0)
