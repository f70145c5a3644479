// Process-wide caching allocator for the library's device buffers (alloc.cpp).
#pragma once

#include <cstddef>

namespace ls {

// Device memory of at least `bytes` bytes on the current device: a cached block of the
// same size class when one is free, else cudaMalloc (throws Error{ENOMEM_} on failure).
void* dev_alloc(size_t bytes);
// Returns a block from dev_alloc to the cache (NULL-safe).  The caller guarantees that no
// work still in flight uses it.
void dev_free(void* p);

}  // namespace ls
