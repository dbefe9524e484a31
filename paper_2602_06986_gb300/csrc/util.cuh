// util.cuh -- host-side error state and small device utilities (order-preserving
// compaction, reason counting) shared by the library's translation units.
#pragma once

#include <cuda_runtime.h>
#include <stdarg.h>
#include <stdint.h>

#include "dse.h"

namespace dse {

void set_error(const char *fmt, ...);
void clear_error();

// Returns DSE_ECUDA and records the message if `e` is an error.
dse_status cuda_status(cudaError_t e, const char *what);

#define DSE_CUDA(call)                                        \
  do {                                                        \
    cudaError_t e_ = (call);                                  \
    if (e_ != cudaSuccess) return ::dse::cuda_status(e_, #call); \
  } while (0)

#define DSE_TRY(call)                  \
  do {                                 \
    dse_status s_ = (call);            \
    if (s_ != DSE_OK) return s_;       \
  } while (0)

// Device allocation that records DSE_ENOMEM.  Allocations are stream-ordered
// on the stream installed by the innermost AllocStream guard (each entry point
// installs its descriptor's stream), from the device's cached memory pool.
struct AllocStream {
  explicit AllocStream(cudaStream_t s);
  ~AllocStream();
  cudaStream_t prev;
};
dse_status dmalloc(void **p, size_t bytes, const char *what);
template <typename T>
dse_status dalloc(T **p, size_t count, const char *what) {
  return dmalloc(reinterpret_cast<void **>(p), count * sizeof(T), what);
}
void dfree(void *p);
// Stream-ordered, pool-cached allocation (cudaMallocAsync / cudaFreeAsync).
dse_status dmalloc_async(void **p, size_t bytes, cudaStream_t s, const char *what);
void dfree_async(void *p, cudaStream_t s);

// Order-preserving selection: out[j] = the j-th index p < n with flags[p] == want.
// Writes the count to *count_host (synchronises the stream).
dse_status compact_bytes(const uint8_t *flags, uint64_t n, uint8_t want, uint64_t *out,
                         uint64_t *count_host, cudaStream_t s);

// Same with the count left on the device (*count_dev); no synchronisation.
dse_status compact_bytes_dev(const uint8_t *flags, uint64_t n, uint8_t want, uint64_t *out,
                             unsigned long long *count_dev, cudaStream_t s);

// The calling thread's pinned host staging area of at least `bytes` bytes
// (nullptr and an error message if it cannot be allocated).  Small results
// are copied there asynchronously so that one stream synchronisation covers
// several copies; its contents are valid until the thread's next call.
void *pinned_staging(size_t bytes);

// counts[c] += number of p < n with flags[p] == c, for c < 6 (device counters).
void launch_count_reasons(const uint8_t *flags, uint64_t n, unsigned long long *counts, cudaStream_t s);

// NVTX range around a public call (a no-op unless a profiler is attached),
// so that timelines show the library's phases.
struct NvtxRange {
  explicit NvtxRange(const char *name);
  ~NvtxRange();
};

// Test hook of dse_debug_fail_alloc.
void debug_fail_alloc(int64_t after);

// Process-wide count of kernels the library has launched.
int64_t launches_so_far();

// Check whether a pointer is device memory.
bool is_device_pointer(const void *p);

}  // namespace dse
