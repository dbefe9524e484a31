// util.cu -- error state, allocation wrappers and order-preserving compaction.
#include <atomic>
#include <stdio.h>
#include <string.h>

#include "util.cuh"

#include <nvtx3/nvToolsExt.h>

namespace dse {

static thread_local char g_err[1024] = "";
static unsigned long long g_launches = 0;

void note_launches(int64_t n) { __atomic_fetch_add(&g_launches, (unsigned long long)n, __ATOMIC_RELAXED); }
int64_t launches_so_far() { return (int64_t)__atomic_load_n(&g_launches, __ATOMIC_RELAXED); }

void set_error(const char *fmt, ...) {
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(g_err, sizeof(g_err), fmt, ap);
  va_end(ap);
}
void clear_error() { g_err[0] = 0; }
const char *last_error() { return g_err; }

dse_status cuda_status(cudaError_t e, const char *what) {
  set_error("%s: %s", what, cudaGetErrorString(e));
  return e == cudaErrorMemoryAllocation ? DSE_ENOMEM : DSE_ECUDA;
}

// The stream that dmalloc / dfree order their pool operations on (set by each
// entry point for the duration of the call).
static thread_local cudaStream_t g_alloc_stream = nullptr;

AllocStream::AllocStream(cudaStream_t s) : prev(g_alloc_stream) { g_alloc_stream = s; }
AllocStream::~AllocStream() { g_alloc_stream = prev; }

dse_status dmalloc(void **p, size_t bytes, const char *what) {
  return dmalloc_async(p, bytes, g_alloc_stream, what);
}

void dfree(void *p) { dfree_async(p, g_alloc_stream); }

// Stream-ordered allocation from the device's default memory pool.  The
// pool's release threshold is raised once per device for this process, so
// freed blocks stay cached and a later allocation of a similar size costs no
// driver round trip and no device-wide synchronisation.
static bool g_pool_ready[64] = {false};

// Simulated allocation failure (dse_debug_fail_alloc): the allocation after
// g_fail_after more successful ones fails; negative: off.
static std::atomic<int64_t> g_fail_after{-1};

void debug_fail_alloc(int64_t after) { g_fail_after.store(after); }

NvtxRange::NvtxRange(const char *name) { nvtxRangePushA(name); }
NvtxRange::~NvtxRange() { nvtxRangePop(); }

static bool simulated_failure() {
  int64_t v = g_fail_after.load();
  while (v >= 0) {
    if (g_fail_after.compare_exchange_weak(v, v - 1)) return v == 0;
  }
  return false;
}

dse_status dmalloc_async(void **p, size_t bytes, cudaStream_t s, const char *what) {
  *p = nullptr;
  if (simulated_failure()) {
    set_error("simulated allocation failure for %s (dse_debug_fail_alloc)", what);
    return DSE_ENOMEM;
  }
  if (bytes == 0) bytes = 16;
  int dev = 0;
  cudaGetDevice(&dev);
  if (dev >= 0 && dev < 64 && !g_pool_ready[dev]) {
    cudaMemPool_t pool;
    if (cudaDeviceGetDefaultMemPool(&pool, dev) == cudaSuccess) {
      uint64_t thr = ~0ull;
      cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &thr);
    }
    cudaGetLastError();
    g_pool_ready[dev] = true;
  }
  cudaError_t e = cudaMallocAsync(p, bytes, s);
  if (e != cudaSuccess) {
    cudaGetLastError();
    set_error("cudaMallocAsync(%zu) for %s: %s", bytes, what, cudaGetErrorString(e));
    return e == cudaErrorMemoryAllocation ? DSE_ENOMEM : DSE_ECUDA;
  }
  return DSE_OK;
}

void dfree_async(void *p, cudaStream_t s) {
  if (p) cudaFreeAsync(p, s);
}

// The calling thread's pinned staging area (grown on demand, never shrunk,
// held until the thread exits).
namespace {
struct Pinned {
  void *p = nullptr;
  size_t bytes = 0;
  ~Pinned() {
    if (p) cudaFreeHost(p);
  }
};
thread_local Pinned g_pinned;
}  // namespace

void *pinned_staging(size_t bytes) {
  if (bytes > g_pinned.bytes) {
    size_t want = 4096;
    while (want < bytes) want <<= 1;
    // an asynchronous upload from the old area may still be in flight
    if (g_pinned.p) {
      cudaDeviceSynchronize();
      cudaFreeHost(g_pinned.p);
    }
    g_pinned.p = nullptr;
    g_pinned.bytes = 0;
    if (cudaMallocHost(&g_pinned.p, want) != cudaSuccess) {
      cudaGetLastError();
      g_pinned.p = nullptr;
      set_error("cudaMallocHost(%zu) for staging failed", want);
      return nullptr;
    }
    g_pinned.bytes = want;
  }
  return g_pinned.p;
}

bool is_device_pointer(const void *p) {
  if (!p) return false;
  cudaPointerAttributes a;
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

// ------------------------------------------------------------- compaction

constexpr int kCompactThreads = 256;
constexpr int kCompactPer = 16;  // elements per thread
constexpr int kCompactTile = kCompactThreads * kCompactPer;

__global__ void k_compact_count(const uint8_t *flags, uint64_t n, uint8_t want, unsigned int *block_counts) {
  __shared__ unsigned int red[kCompactThreads / 32];
  uint64_t base = (uint64_t)blockIdx.x * kCompactTile + (uint64_t)threadIdx.x * kCompactPer;
  unsigned int c = 0;
  for (int e = 0; e < kCompactPer; ++e) {
    uint64_t p = base + e;
    if (p < n && flags[p] == want) ++c;
  }
  for (int o = 16; o > 0; o >>= 1) c += __shfl_xor_sync(0xffffffffu, c, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = c;
  __syncthreads();
  if (threadIdx.x == 0) {
    unsigned int t = 0;
    for (int w = 0; w < kCompactThreads / 32; ++w) t += red[w];
    block_counts[blockIdx.x] = t;
  }
}

// Exclusive scan of block counts by one block (loops over chunks).
__global__ void k_compact_scan(const unsigned int *block_counts, uint64_t nb, unsigned long long *offsets,
                               unsigned long long *total) {
  __shared__ unsigned long long part[1024];
  __shared__ unsigned long long carry;
  if (threadIdx.x == 0) carry = 0;
  __syncthreads();
  for (uint64_t c0 = 0; c0 < nb; c0 += 1024) {
    uint64_t i = c0 + threadIdx.x;
    unsigned long long v = i < nb ? block_counts[i] : 0ull;
    part[threadIdx.x] = v;
    __syncthreads();
    for (int o = 1; o < 1024; o <<= 1) {
      unsigned long long t = threadIdx.x >= (unsigned)o ? part[threadIdx.x - o] : 0ull;
      __syncthreads();
      part[threadIdx.x] += t;
      __syncthreads();
    }
    if (i < nb) offsets[i] = carry + part[threadIdx.x] - v;
    __syncthreads();
    if (threadIdx.x == 1023) carry += part[1023];
    __syncthreads();
  }
  if (threadIdx.x == 0) *total = carry;
}

__global__ void k_compact_write(const uint8_t *flags, uint64_t n, uint8_t want,
                                const unsigned long long *offsets, uint64_t *out) {
  __shared__ unsigned int sc[kCompactThreads];
  uint64_t base = (uint64_t)blockIdx.x * kCompactTile + (uint64_t)threadIdx.x * kCompactPer;
  unsigned int c = 0;
  for (int e = 0; e < kCompactPer; ++e) {
    uint64_t p = base + e;
    if (p < n && flags[p] == want) ++c;
  }
  sc[threadIdx.x] = c;
  __syncthreads();
  for (int o = 1; o < kCompactThreads; o <<= 1) {
    unsigned int t = threadIdx.x >= (unsigned)o ? sc[threadIdx.x - o] : 0u;
    __syncthreads();
    sc[threadIdx.x] += t;
    __syncthreads();
  }
  unsigned long long w = offsets[blockIdx.x] + sc[threadIdx.x] - c;
  for (int e = 0; e < kCompactPer; ++e) {
    uint64_t p = base + e;
    if (p < n && flags[p] == want) out[w++] = p;
  }
}

dse_status compact_bytes_dev(const uint8_t *flags, uint64_t n, uint8_t want, uint64_t *out,
                             unsigned long long *count_dev, cudaStream_t s) {
  if (n == 0) {
    DSE_CUDA(cudaMemsetAsync(count_dev, 0, sizeof(unsigned long long), s));
    return DSE_OK;
  }
  uint64_t nb = (n + kCompactTile - 1) / kCompactTile;
  unsigned int *bc = nullptr;
  unsigned long long *off = nullptr;
  DSE_TRY(dalloc(&bc, nb, "compaction counts"));
  dse_status st = dalloc(&off, nb, "compaction offsets");
  if (st != DSE_OK) {
    dfree(bc);
    return st;
  }
  note_launches(3);
  k_compact_count<<<(unsigned)nb, kCompactThreads, 0, s>>>(flags, n, want, bc);
  k_compact_scan<<<1, 1024, 0, s>>>(bc, nb, off, count_dev);
  k_compact_write<<<(unsigned)nb, kCompactThreads, 0, s>>>(flags, n, want, off, out);
  dfree(bc);
  dfree(off);
  DSE_CUDA(cudaGetLastError());
  return DSE_OK;
}

dse_status compact_bytes(const uint8_t *flags, uint64_t n, uint8_t want, uint64_t *out, uint64_t *count_host,
                         cudaStream_t s) {
  *count_host = 0;
  if (n == 0) return DSE_OK;
  uint64_t nb = (n + kCompactTile - 1) / kCompactTile;
  unsigned int *bc = nullptr;
  unsigned long long *off = nullptr;
  DSE_TRY(dalloc(&bc, nb, "compaction counts"));
  dse_status st = dalloc(&off, nb + 1, "compaction offsets");
  if (st != DSE_OK) {
    dfree(bc);
    return st;
  }
  note_launches(3);
  k_compact_count<<<(unsigned)nb, kCompactThreads, 0, s>>>(flags, n, want, bc);
  k_compact_scan<<<1, 1024, 0, s>>>(bc, nb, off, off + nb);
  k_compact_write<<<(unsigned)nb, kCompactThreads, 0, s>>>(flags, n, want, off, out);
  unsigned long long tot = 0;
  cudaError_t e = cudaMemcpyAsync(&tot, off + nb, sizeof(tot), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  dfree(bc);
  dfree(off);
  if (e != cudaSuccess) return cuda_status(e, "compaction");
  *count_host = tot;
  return DSE_OK;
}

__global__ void k_count_reasons(const uint8_t *flags, uint64_t n, unsigned long long *counts) {
  __shared__ unsigned int c[6];
  if (threadIdx.x < 6) c[threadIdx.x] = 0;
  __syncthreads();
  for (uint64_t p = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; p < n; p += (uint64_t)gridDim.x * blockDim.x) {
    uint8_t f = flags[p];
    if (f < 6) atomicAdd(&c[f], 1u);
  }
  __syncthreads();
  if (threadIdx.x < 6 && c[threadIdx.x]) atomicAdd(&counts[threadIdx.x], (unsigned long long)c[threadIdx.x]);
}

void launch_count_reasons(const uint8_t *flags, uint64_t n, unsigned long long *counts, cudaStream_t s) {
  if (n == 0) return;
  uint64_t blocks = (n + 255) / 256;
  if (blocks > 4096) blocks = 4096;
  note_launches(1);
  k_count_reasons<<<(unsigned)blocks, 256, 0, s>>>(flags, n, counts);
}

}  // namespace dse
