// Launch instrumentation (prof.cpp).
#pragma once

#include <cuda_runtime.h>

namespace ls {

void prof_begin(const char* cls, cudaStream_t st);
void prof_end(const char* cls, cudaStream_t st);
void prof_start(const char* timed_class);
int prof_stop(char* out, int cap);

}  // namespace ls

// Launches a kernel of class `cls` on stream `st` and checks the launch.
#define LS_LAUNCH(cls, st, ...)          \
  do {                                   \
    ls::prof_begin(cls, st);             \
    __VA_ARGS__;                         \
    ls::prof_end(cls, st);               \
    LS_CHECK_LAUNCH();                   \
  } while (0)
