// peaks.cu -- issue-rate probe of the pipes the CUDA-core kernels are bound
// by: FP32 fused multiply-adds, special-function (MUFU) operations and FP64
// fused multiply-adds, each as independent register-resident chains in
// every lane of enough warps to fill every SM, timed with CUDA events.  The
// rates are the denominators of the ALU rooflines (lane operations per
// second), measured on the part they are reported for.
#include <algorithm>

#include "dse_internal.cuh"
#include "util.cuh"

namespace dse {

dse_status check_device();

namespace {

constexpr int kChains = 8;      // independent dependency chains per thread
constexpr int kPeakIters = 4096;

// FP32: kChains chains of kPeakIters FMAs per thread.
__global__ void __launch_bounds__(256) k_peak_fp32(float seed, float *sink) {
  float a[kChains];
#pragma unroll
  for (int c = 0; c < kChains; ++c) a[c] = seed + (float)(threadIdx.x + c);
  const float m = 0.9999999f, k = 1e-7f;
#pragma unroll 16
  for (int i = 0; i < kPeakIters; ++i)
#pragma unroll
    for (int c = 0; c < kChains; ++c) a[c] = fmaf(a[c], m, k);
  float s = 0.f;
#pragma unroll
  for (int c = 0; c < kChains; ++c) s += a[c];
  if (s == 1234.5f) sink[threadIdx.x] = s;  // (never true: keeps the chains)
}

// MUFU: kChains chains of kPeakIters base-2 exponentials (ex2.approx) per
// thread, each fed back through a multiply that keeps the values bounded.
__global__ void __launch_bounds__(256) k_peak_sfu(float seed, float *sink) {
  float a[kChains];
#pragma unroll
  for (int c = 0; c < kChains; ++c) a[c] = seed * (float)(c + 1) * 1e-3f;
#pragma unroll 16
  for (int i = 0; i < kPeakIters; ++i)
#pragma unroll
    for (int c = 0; c < kChains; ++c) {
      float r;
      asm volatile("ex2.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(a[c]));
      a[c] = r * -0.5f;
    }
  float s = 0.f;
#pragma unroll
  for (int c = 0; c < kChains; ++c) s += a[c];
  if (s == 1234.5f) sink[threadIdx.x] = s;
}

// FP64: kChains chains of kPeakIters / 16 FMAs per thread (the pipe is slow).
__global__ void __launch_bounds__(256) k_peak_fp64(double seed, double *sink) {
  double a[kChains];
#pragma unroll
  for (int c = 0; c < kChains; ++c) a[c] = seed + (double)(threadIdx.x + c);
  const double m = 0.99999999999, k = 1e-13;
#pragma unroll 4
  for (int i = 0; i < kPeakIters / 16; ++i)
#pragma unroll
    for (int c = 0; c < kChains; ++c) a[c] = fma(a[c], m, k);
  double s = 0.0;
#pragma unroll
  for (int c = 0; c < kChains; ++c) s += a[c];
  if (s == 1234.5) sink[threadIdx.x] = s;
}

}  // namespace
}  // namespace dse

extern "C" dse_status dse_measure_peaks(double *fp32_fma_per_s, double *sfu_per_s, double *fp64_fma_per_s,
                                        void *stream) {
  using namespace dse;
  clear_error();
  if (!fp32_fma_per_s || !sfu_per_s || !fp64_fma_per_s) {
    set_error("null argument");
    return DSE_EINVAL;
  }
  DSE_TRY(check_device());
  cudaStream_t st = (cudaStream_t)stream;
  AllocStream as(st);
  int dev = 0, sms = 0;
  DSE_CUDA(cudaGetDevice(&dev));
  DSE_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  void *sink = nullptr;
  DSE_TRY(dmalloc(&sink, 256 * sizeof(double), "peak probe sink"));
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  cudaError_t e = cudaEventCreate(&e0);
  if (!e) e = cudaEventCreate(&e1);
  // 8 blocks of 256 threads per SM: 64 warps, enough to hide each pipe's
  // latency with 8 independent chains per thread
  const unsigned blocks = (unsigned)sms * 8;
  const double threads = (double)blocks * 256.0;
  double best[3] = {0.0, 0.0, 0.0};
  for (int rep = 0; rep < 4 && !e; ++rep) {
    for (int which = 0; which < 3 && !e; ++which) {
      e = cudaEventRecord(e0, st);
      note_launches(1);
      if (which == 0) k_peak_fp32<<<blocks, 256, 0, st>>>(0.5f, static_cast<float *>(sink));
      if (which == 1) k_peak_sfu<<<blocks, 256, 0, st>>>(0.5f, static_cast<float *>(sink));
      if (which == 2) k_peak_fp64<<<blocks, 256, 0, st>>>(0.5, static_cast<double *>(sink));
      if (!e) e = cudaGetLastError();
      if (!e) e = cudaEventRecord(e1, st);
      if (!e) e = cudaEventSynchronize(e1);
      float ms = 0.f;
      if (!e) e = cudaEventElapsedTime(&ms, e0, e1);
      const double ops = threads * kChains * (which == 2 ? kPeakIters / 16 : kPeakIters);
      // the first round warms the clocks and the instruction cache
      if (!e && rep > 0 && ms > 0.f) best[which] = std::max(best[which], ops / (ms * 1e-3));
    }
  }
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  dfree(sink);
  if (e) return cuda_status(e, "peak probe");
  *fp32_fma_per_s = best[0];
  *sfu_per_s = best[1];
  *fp64_fma_per_s = best[2];
  return DSE_OK;
}
