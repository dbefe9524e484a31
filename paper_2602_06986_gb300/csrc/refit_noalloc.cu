// refit_noalloc.cu -- dse_ls_refit_noalloc: the residual-loop refit of
// dse_ls_refit with every scratch buffer carved from one fixed, file-scope
// device array instead of cudaMalloc.
//
// It serves callers that cannot allocate device memory while they run:
// applications whose device memory is owned by their own pool allocator or
// accounted against a hard budget, and processes that have reserved the whole
// device for other work before the refit runs.  The price is a fixed ceiling
// on the problem size and one shared scratch area per device.  The call still
// waits for its stream and reads the winner back to host memory, so it is an
// ordinary synchronous call: it must not be issued on a stream that is being
// captured into a CUDA graph.
#include <string.h>

#include <mutex>

#include "dse_internal.cuh"
#include "util.cuh"

namespace dse {

FeatTable table_of(const dse_space *S);

// The refit steps of refit.cu (the same kernels as dse_ls_refit, so the two
// agree to the bit), launched here on the static scratch.
size_t refit_chain_bytes(int64_t N, int64_t cap);
void refit_chain_prep(dse_space *S, const double *y, const uint64_t *fid, int nf, void *scratch, int64_t cap,
                      cudaStream_t st);
void refit_chain_fit(dse_space *S, const double *y, const uint64_t *fid, int nf, const uint64_t *cand, int64_t cap,
                     const int64_t *n_dev, void *scratch, bool have_sums, double *res, double *report,
                     uint64_t *chosen, cudaStream_t st);

namespace {

constexpr int kCoef = 5;                       // intercept + up to 4 columns
constexpr size_t kScratchBytes = 8u << 20;     // 8 MiB per device
constexpr int64_t kMaxSamples = 32768;
constexpr int64_t kMaxCand = 16384;
constexpr int kMaxDevices = 64;

// The scratch itself.  Host code must never use this name as a device
// address: it only stands in for the symbol; the address comes from
// cudaGetSymbolAddress below.
static __device__ __align__(256) unsigned char g_refit_scratch[kScratchBytes];

std::mutex g_mu;
void *g_addr[kMaxDevices] = {nullptr};

// Device address of the scratch on the current device, looked up once per
// device (the first call on a device does it) and kept for the life of the
// process.  A cudaDeviceReset destroys the context the address belongs to:
// after one, this cache is stale, so the library must not be used across a
// device reset.
dse_status scratch_address(void **out) {
  int dev = 0;
  DSE_CUDA(cudaGetDevice(&dev));
  if (dev < 0 || dev >= kMaxDevices) {
    set_error("device ordinal %d beyond the no-alloc table", dev);
    return DSE_EINVAL;
  }
  std::lock_guard<std::mutex> lk(g_mu);
  if (!g_addr[dev]) {
    void *p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_refit_scratch);
    if (e != cudaSuccess || !p) {
      cudaGetLastError();
      set_error("cudaGetSymbolAddress of the refit scratch: %s", cudaGetErrorString(e));
      return DSE_ECUDA;
    }
    g_addr[dev] = p;
  }
  *out = g_addr[dev];
  return DSE_OK;
}

size_t round256(size_t b) { return (b + 255) / 256 * 256; }

}  // namespace

dse_status refit_noalloc_impl(dse_space *S, const dse_refit_desc *d, uint64_t *best_id, double *best_rmse,
                              double *coefs, double *residual) {
  cudaStream_t st = (cudaStream_t)d->stream;
  const int64_t N = S->N, nc = d->n_cand;
  const int nf = d->n_fixed;
  if (N > kMaxSamples || nc > kMaxCand) {
    set_error("no-alloc refit limits: N <= %lld and n_cand <= %lld (got N=%lld, n_cand=%lld)",
              (long long)kMaxSamples, (long long)kMaxCand, (long long)N, (long long)nc);
    return DSE_EOVERFLOW;
  }
  const uint64_t total = (uint64_t)S->n + S->geom.slots;
  for (int j = 0; j < nf; ++j)
    if (d->fixed[j] >= total) {
      set_error("fixed id out of range");
      return DSE_ERANGE;
    }
  if (!d->cand_on_device)
    for (int64_t i = 0; i < nc; ++i)
      if (d->cand[i] >= total) {
        set_error("candidate id out of range");
        return DSE_ERANGE;
      }
  // layout: the refit step's buffers, then y, fixed ids, candidates, the
  // winner's report and the residual
  size_t off = 0;
  auto take = [&](size_t bytes) {
    size_t o = off;
    off += round256(bytes);
    return o;
  };
  const size_t o_chain = take(refit_chain_bytes(N, nc)), o_y = take(8 * N), o_fid = take(8 * 4), o_c = take(8 * nc),
               o_rep = take(8 * (kCoef + 3)), o_res = take(8 * N);
  if (off > kScratchBytes) {
    set_error("no-alloc refit needs %zu bytes of scratch, the fixed area holds %zu", off, kScratchBytes);
    return DSE_EOVERFLOW;
  }
  void *vbase = nullptr;
  DSE_TRY(scratch_address(&vbase));
  char *base = static_cast<char *>(vbase);
  double *y = reinterpret_cast<double *>(base + o_y);
  uint64_t *fid = reinterpret_cast<uint64_t *>(base + o_fid);
  uint64_t *cand = reinterpret_cast<uint64_t *>(base + o_c);
  double *rep = reinterpret_cast<double *>(base + o_rep);
  double *res = reinterpret_cast<double *>(base + o_res);
  // Every kernel writes all it later reads, so nothing left by an earlier
  // call is read; the report is still cleared so that a failed launch cannot
  // return an earlier call's pick.
  cudaError_t e = cudaMemsetAsync(rep, 0xff, 8 * (kCoef + 3), st);
  if (!e) e = cudaMemcpyAsync(y, d->y, 8 * N, cudaMemcpyDefault, st);
  if (!e && nf) e = cudaMemcpyAsync(fid, d->fixed, 8 * nf, cudaMemcpyHostToDevice, st);
  if (!e) e = cudaMemcpyAsync(cand, d->cand, 8 * nc, cudaMemcpyDefault, st);
  if (e) return cuda_status(e, "no-alloc refit upload");
  refit_chain_prep(S, y, fid, nf, base + o_chain, nc, st);
  refit_chain_fit(S, y, fid, nf, cand, nc, nullptr, base + o_chain, false, res, rep, nullptr, st);
  // the winner's report and the residual are queued on the caller's stream
  // behind the fit; one wait for both
  double h[kCoef + 3];
  e = cudaMemcpyAsync(h, rep, sizeof(h), cudaMemcpyDeviceToHost, st);
  if (!e && residual) e = cudaMemcpyAsync(residual, res, 8 * N, cudaMemcpyDefault, st);
  if (!e) e = cudaStreamSynchronize(st);
  if (e) return cuda_status(e, "no-alloc refit");
  long long hb, hid;
  memcpy(&hb, &h[0], 8);
  memcpy(&hid, &h[1], 8);
  if (hb < 0) {
    set_error("no candidate gives a full-rank fit");
    return DSE_EINVAL;
  }
  *best_id = (uint64_t)hid;
  *best_rmse = h[2];
  if (coefs)
    for (int c = 0; c < nf + 2; ++c) coefs[c] = h[3 + c];
  return DSE_OK;
}

}  // namespace dse

extern "C" dse_status dse_ls_refit_noalloc(dse_space *s, const dse_refit_desc *d, uint64_t *best_id,
                                           double *best_rmse, double *coefs, double *residual) {
  dse::NvtxRange nvtx_range_("dse_ls_refit_noalloc");
  dse::clear_error();
  if (!s || !d || !d->y || d->n_fixed < 0 || d->n_fixed > 3 || (d->n_fixed > 0 && !d->fixed) || !d->cand ||
      d->n_cand < 1 || !best_id || !best_rmse) {
    dse::set_error("invalid refit descriptor");
    return DSE_EINVAL;
  }
  int n = 0;
  if (cudaGetDeviceCount(&n) != cudaSuccess || n == 0) {
    cudaGetLastError();
    dse::set_error("no usable CUDA device");
    return DSE_ECUDA;
  }
  return dse::refit_noalloc_impl(s, d, best_id, best_rmse, coefs, residual);
}
