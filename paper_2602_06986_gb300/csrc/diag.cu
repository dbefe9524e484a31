// diag.cu -- failure-detection checks that need no fault: the bounded
// device wait that every pipelined kernel uses, run on a barrier that may
// never complete, and the simulated allocation failure hook.
#include "dse_internal.cuh"
#include "util.cuh"

namespace dse {

dse_status check_device();

// One thread initialises an mbarrier expecting one arrival; with `arrive`
// it arrives, otherwise nothing ever does.  It then waits for the phase
// with the same bounded poll loop as the kernels (mbar_wait_bounded) and
// records DSE_ETIMEOUT when the limit runs out.
__global__ void k_wait_probe(uint32_t polls, int arrive, int *status) {
  __shared__ uint64_t bar;
  if (threadIdx.x != 0) return;
  mbar_init(&bar, 1);
  mbar_fence_init();
  if (arrive) asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(&bar)) : "memory");
  *status = mbar_wait_bounded(&bar, 0, polls) ? DSE_OK : DSE_ETIMEOUT;
}

// One bounds check of the checked build on the device: status gets
// DSE_EBOUNDS when index is outside [0, limit), DSE_OK otherwise.
__global__ void k_bounds_probe(int64_t index, int64_t limit, int *status) {
  if (threadIdx.x != 0) return;
  *status = DSE_OK;
  if (DSE_IN_BOUNDS(index, limit, status)) {
  }
}

}  // namespace dse

extern "C" dse_status dse_bounds_probe(int64_t index, int64_t limit, void *stream) {
  using namespace dse;
  clear_error();
#ifndef DSE_CHECK_BOUNDS
  (void)index;
  (void)limit;
  (void)stream;
  set_error("not a bounds-checked build (compile with DSE_CHECK_BOUNDS)");
  return DSE_EINVAL;
#else
  DSE_TRY(check_device());
  cudaStream_t st = (cudaStream_t)stream;
  AllocStream as(st);
  int *d = nullptr;
  DSE_TRY(dmalloc(reinterpret_cast<void **>(&d), sizeof(int), "bounds probe status"));
  int h = DSE_ECUDA;
  note_launches(1);
  k_bounds_probe<<<1, 32, 0, st>>>(index, limit, d);
  cudaError_t e = cudaGetLastError();
  if (!e) e = cudaMemcpyAsync(&h, d, sizeof(int), cudaMemcpyDeviceToHost, st);
  if (!e) e = cudaStreamSynchronize(st);
  dfree(d);
  if (e) return cuda_status(e, "bounds probe");
  if (h == DSE_EBOUNDS) set_error("index %lld outside [0, %lld)", (long long)index, (long long)limit);
  return h;
#endif
}

extern "C" dse_status dse_check_wait(uint32_t polls, int32_t arrive, void *stream) {
  using namespace dse;
  clear_error();
  if (polls == 0) {
    set_error("polls must be positive");
    return DSE_EINVAL;
  }
  DSE_TRY(check_device());
  cudaStream_t st = (cudaStream_t)stream;
  AllocStream as(st);
  int *d = nullptr;
  DSE_TRY(dmalloc(reinterpret_cast<void **>(&d), sizeof(int), "wait probe status"));
  int h = DSE_ECUDA;
  note_launches(1);
  k_wait_probe<<<1, 32, 0, st>>>(polls, arrive ? 1 : 0, d);
  cudaError_t e = cudaGetLastError();
  if (!e) e = cudaMemcpyAsync(&h, d, sizeof(int), cudaMemcpyDeviceToHost, st);
  if (!e) e = cudaStreamSynchronize(st);
  dfree(d);
  if (e) return cuda_status(e, "wait probe");
  if (h == DSE_ETIMEOUT) set_error("a bounded device wait timed out (wait probe, %u polls)", polls);
  return h;
}

extern "C" void dse_debug_fail_alloc(int64_t after) { dse::debug_fail_alloc(after); }
