// refit_noalloc.cu -- dse_ls_refit_noalloc: the residual-loop refit of
// dse_ls_refit with every scratch buffer carved from one fixed, file-scope
// device array instead of cudaMalloc.
//
// It serves callers that must not allocate device memory while they run:
// code between cudaStreamBeginCapture and EndCapture (an allocation there is
// illegal in the capturing stream), applications whose device memory is
// owned by their own pool or accounted against a hard budget, and paths that
// run after the caller has reserved the whole device.  The price is a fixed
// ceiling on the problem size and one shared scratch area per device.
#include <mutex>

#include "dse_internal.cuh"
#include "util.cuh"

namespace dse {

FeatTable table_of(const dse_space *S);

// The refit kernels of refit.cu (same definitions, launched here on the
// static scratch).
__global__ void k_columns(FeatTable F, RungGeom G, int64_t n_stored, const uint64_t *ids, int n, double *out);
__global__ void k_refit(FeatTable F, RungGeom G, int64_t n_stored, const double *y, const double *fixed_cols, int nf,
                        const uint64_t *fixed_ids, const uint64_t *cand, int64_t n_cand, double *rmse_out,
                        double *beta_out);
__global__ void k_argmin(const double *rmse, const uint64_t *cand, int64_t n, int64_t *best, const double *beta,
                         double *report, const int64_t *n_dev, uint64_t *chosen);
__global__ void k_residual(FeatTable F, RungGeom G, int64_t n_stored, const double *y, const double *fixed_cols,
                           int nf, const uint64_t *cand, const int64_t *best, const double *beta_all, double *res);

namespace {

constexpr int kCoef = 5;                       // intercept + up to 4 columns
constexpr size_t kScratchBytes = 4u << 20;     // 4 MiB per device
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
// device (the first call on a device does it).
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
  // layout: y, fixed ids, fixed columns, candidates, rmse, beta, best, residual
  size_t off = 0;
  auto take = [&](size_t bytes) {
    size_t o = off;
    off += round256(bytes);
    return o;
  };
  const size_t o_y = take(8 * N), o_fid = take(8 * 4), o_fc = take(8 * (size_t)N * 4), o_c = take(8 * nc),
               o_r = take(8 * nc), o_b = take(8 * (size_t)nc * kCoef), o_best = take(8), o_res = take(8 * N);
  if (off > kScratchBytes) {
    set_error("no-alloc refit needs %zu bytes of scratch, the fixed area holds %zu", off, kScratchBytes);
    return DSE_EOVERFLOW;
  }
  void *vbase = nullptr;
  DSE_TRY(scratch_address(&vbase));
  char *base = static_cast<char *>(vbase);
  double *y = reinterpret_cast<double *>(base + o_y);
  uint64_t *fid = reinterpret_cast<uint64_t *>(base + o_fid);
  double *fc = reinterpret_cast<double *>(base + o_fc);
  uint64_t *cand = reinterpret_cast<uint64_t *>(base + o_c);
  double *rm = reinterpret_cast<double *>(base + o_r);
  double *beta = reinterpret_cast<double *>(base + o_b);
  int64_t *best = reinterpret_cast<int64_t *>(base + o_best);
  double *res = reinterpret_cast<double *>(base + o_res);
  // Every kernel below writes all it later reads (columns, one RMSE and one
  // coefficient row per candidate, the argmin slot, the residual), so nothing
  // left by an earlier call is read; the argmin slot is still cleared so that
  // a failed launch cannot report an earlier call's pick.
  cudaError_t e = cudaMemsetAsync(best, 0xff, 8, st);
  if (!e) e = cudaMemcpyAsync(y, d->y, 8 * N, cudaMemcpyDefault, st);
  if (!e && nf) e = cudaMemcpyAsync(fid, d->fixed, 8 * nf, cudaMemcpyHostToDevice, st);
  if (!e) e = cudaMemcpyAsync(cand, d->cand, 8 * nc, cudaMemcpyDefault, st);
  if (e) return cuda_status(e, "no-alloc refit upload");
  const FeatTable F = table_of(S);
  note_launches(3 + (nf ? 1 : 0));
  if (nf) k_columns<<<(unsigned)nf, 256, 0, st>>>(F, S->geom, S->n, fid, nf, fc);
  k_refit<<<(unsigned)((nc * 32 + 255) / 256), 256, 0, st>>>(F, S->geom, S->n, y, fc, nf, fid, cand, nc, rm, beta);
  k_argmin<<<1, 1024, 0, st>>>(rm, cand, nc, best, beta, nullptr, nullptr, nullptr);
  k_residual<<<64, 256, 0, st>>>(F, S->geom, S->n, y, fc, nf, cand, best, beta, res);
  int64_t hb = -1;
  e = cudaMemcpyAsync(&hb, best, 8, cudaMemcpyDeviceToHost, st);
  if (!e) e = cudaStreamSynchronize(st);
  if (e) return cuda_status(e, "no-alloc refit");
  if (hb < 0) {
    set_error("no candidate gives a full-rank fit");
    return DSE_EINVAL;
  }
  double hb_beta[kCoef];
  e = cudaMemcpy(best_rmse, rm + hb, 8, cudaMemcpyDeviceToHost);
  if (!e) e = cudaMemcpy(best_id, cand + hb, 8, cudaMemcpyDeviceToHost);
  if (!e) e = cudaMemcpy(hb_beta, beta + hb * kCoef, sizeof(hb_beta), cudaMemcpyDeviceToHost);
  if (!e && residual) e = cudaMemcpy(residual, res, 8 * N, cudaMemcpyDefault);
  if (e) return cuda_status(e, "no-alloc refit fetch");
  if (coefs)
    for (int c = 0; c < nf + 2; ++c) coefs[c] = hb_beta[c];
  return DSE_OK;
}

}  // namespace dse

extern "C" dse_status dse_ls_refit_noalloc(dse_space *s, const dse_refit_desc *d, uint64_t *best_id,
                                           double *best_rmse, double *coefs, double *residual) {
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
