// dedup.cu -- score-based redundancy removal of the SIS lists
// (DSE_FLAG_DEDUP).
//
// Reading of "Design Philosophy and Constraints" (rules that reduce the
// search space) and of SISSO's habit of keeping one feature of a group of
// interchangeable ones: two valid candidates are equivalent when the FP64
// Pearson correlation of their values has |rho| >= 1 - tau; a candidate is
// redundant when an equivalent candidate with a smaller id exists in the
// screened range; each list keeps the top-k of the non-redundant candidates.
//
// For unit vectors a, b with |a.b| >= 1 - tau, | |a.y| - |b.y| | <= |a -+ b| =
// sqrt(2 (1 - |a.b|)) <= sqrt(2 tau): equivalent candidates have scores
// within sqrt(2 tau) of each other.  So the screen is run for a longer list
// (kk entries, sorted by score), and each entry's partners are sought only
// among the entries whose reported scores lie within
//   W = sqrt(2 tau) + 2 * (largest reported bound of the list) + 1e-13
// of its own.  An entry is decided only if the list is complete down to its
// score minus W (else kk grows and the screen runs again).
//
// Kernels (per list chunk):
//   k_dedup_unit     block per entry: FP64 values, centred, scaled to unit
//                    norm (two passes over the operands' FP64 rows)
//   k_dedup_flags    block per entry: window by binary search on the sorted
//                    scores, warps over the partners with a smaller id,
//                    lanes over samples, |z_i . z_j| >= 1 - tau
//   k_dedup_compact  warp per list: ballot scan of the flags in rank order,
//                    first k non-redundant entries out, decidability check
#include <math.h>

#include <algorithm>
#include <vector>

#include "dse_internal.cuh"
#include "eval64.cuh"
#include "util.cuh"

namespace dse {
FeatTable table_of(const dse_space *S);

namespace {

constexpr int kUnitThreads = 128;
constexpr int kFlagThreads = 256;

__device__ __forceinline__ double block_sum128(double v, double *sm) {
  v = warp_sum64(v);
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  if (lane == 0) sm[w] = v;
  __syncthreads();
  double t = 0.0;
  for (int i = 0; i < kUnitThreads / 32; ++i) t += sm[i];
  __syncthreads();
  return t;
}

// z[(l - l0) * kk + i][0..N) = unit centred FP64 values of entry i of list l.
__global__ void __launch_bounds__(kUnitThreads) k_dedup_unit(FeatTable F, RungGeom G, int64_t n_stored,
                                                             const uint64_t *ids, const int64_t *n_list, int64_t kk,
                                                             int l0, double *z) {
  __shared__ double sm[kUnitThreads / 32];
  const int l = l0 + (int)blockIdx.y;
  const int64_t i = blockIdx.x;
  if (i >= n_list[l]) return;
  const uint64_t gid = ids[(int64_t)l * kk + i];
  const int64_t N = F.N;
  double *zi = z + ((int64_t)blockIdx.y * kk + i) * N;
  double s = 0.0;
  for (int64_t t = threadIdx.x; t < N; t += kUnitThreads) {
    const double v = candidate_value64(F, G, n_stored, gid, t);
    zi[t] = v;
    s += v;
  }
  const double mean = block_sum128(s, sm) / (double)N;
  double q = 0.0;
  for (int64_t t = threadIdx.x; t < N; t += kUnitThreads) {
    const double d = zi[t] - mean;
    zi[t] = d;
    q = fma(d, d, q);
  }
  const double inv = 1.0 / sqrt(block_sum128(q, sm));
  for (int64_t t = threadIdx.x; t < N; t += kUnitThreads) zi[t] *= inv;
}

// red[l * kk + i] = 1 if an entry j of list l within the score window of i
// has a smaller id and |z_i . z_j| >= 1 - tau.
__global__ void __launch_bounds__(kFlagThreads) k_dedup_flags(const uint64_t *ids, const double *score,
                                                              const int64_t *n_list, const double *max_eps,
                                                              int64_t kk, int l0, int64_t N, const double *z,
                                                              double tau, double w_tau, uint8_t *red) {
  __shared__ int found;
  const int l = l0 + (int)blockIdx.y;
  const int64_t i = blockIdx.x, n = n_list[l];
  if (i >= n) return;
  const uint64_t *li = ids + (int64_t)l * kk;
  const double *ls = score + (int64_t)l * kk;
  const double si = ls[i], W = w_tau + 2.0 * max_eps[l];
  // scores are sorted descending: lo = first j with ls[j] <= si + W, hi =
  // last j with ls[j] >= si - W (i itself lies in [lo, hi])
  int64_t a = 0, b = i;
  while (a < b) {
    const int64_t m = (a + b) >> 1;
    if (ls[m] <= si + W) b = m; else a = m + 1;
  }
  const int64_t lo = a;
  a = i;
  b = n - 1;
  while (a < b) {
    const int64_t m = (a + b + 1) >> 1;
    if (ls[m] >= si - W) a = m; else b = m - 1;
  }
  const int64_t hi = a;
  if (threadIdx.x == 0) found = 0;
  __syncthreads();
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const uint64_t idi = li[i];
  const double *zi = z + ((int64_t)blockIdx.y * kk + i) * N;
  for (int64_t j = lo + warp; j <= hi; j += kFlagThreads / 32) {
    if (*(volatile int *)&found) break;
    if (li[j] >= idi) continue;
    const double *zj = z + ((int64_t)blockIdx.y * kk + j) * N;
    double d = 0.0;
    for (int64_t t = lane; t < N; t += 32) d = fma(zi[t], zj[t], d);
    d = warp_sum64(d);
    if (fabs(d) >= 1.0 - tau) {
      if (lane == 0) atomicExch(&found, 1);
      break;
    }
  }
  __syncthreads();
  if (threadIdx.x == 0) red[(int64_t)l * kk + i] = (uint8_t)found;
}

// Warp per list: the first k non-redundant entries in rank order into the
// output lists; undecided[l] = 1 if an entry examined before the k-th kept
// one is kept while its score lies within W of the list's last score and
// the list may be incomplete; n_red[l] = redundant entries examined.
__global__ void k_dedup_compact(const uint64_t *ids, const double *score, const double *eps, const int64_t *n_list,
                                const double *max_eps, int64_t kk, int64_t k, int full, double w_tau,
                                const uint8_t *red, uint64_t *o_id, double *o_score, double *o_eps, int64_t *o_n,
                                double *o_max_eps, int *undecided, int64_t *n_red) {
  const int l = blockIdx.x;
  const int lane = threadIdx.x;
  const int64_t n = n_list[l];
  const int64_t base = (int64_t)l * kk;
  const double W = w_tau + 2.0 * max_eps[l];
  const double s_last = n > 0 ? score[base + n - 1] : 0.0;
  const bool may_miss = full && n == kk;
  int64_t kept = 0, nr = 0;
  int und = 0;
  double me = 0.0;
  for (int64_t c = 0; c < n && kept < k; c += 32) {
    const int64_t i = c + lane;
    const bool in = i < n;
    const bool r = in ? red[base + i] != 0 : true;
    const unsigned km = __ballot_sync(0xffffffffu, in && !r);
    const int before = __popc(km & ((1u << lane) - 1u));
    const bool examined = in && (kept + before < k);
    // a redundant entry is settled by its partner; a kept one needs the
    // whole window in the list
    if (examined && !r && may_miss && !(score[base + i] - W > s_last)) und = 1;
    if (examined && !r) {
      const int64_t pos = kept + before;
      o_id[(int64_t)l * k + pos] = ids[base + i];
      o_score[(int64_t)l * k + pos] = score[base + i];
      o_eps[(int64_t)l * k + pos] = eps[base + i];
      me = fmax(me, eps[base + i]);
    }
    nr += __popc(__ballot_sync(0xffffffffu, examined && r));
    kept += __popc(km);
  }
  und = __any_sync(0xffffffffu, und);
  me = warp_max64(me);
  if (lane == 0) {
    o_n[l] = kept < k ? kept : k;
    o_max_eps[l] = me;
    undecided[l] = und;
    n_red[l] = nr;
  }
}

}  // namespace

// Redundancy removal of a finished result (lists of length kk) into lists of
// length k.  On success R holds the new lists (R->k = k) and *undecided
// tells whether some list needs a longer screen.  Synchronises.
dse_status dedup_result(dse_result *R, int64_t k, double tau, bool full, bool *undecided, int64_t *n_redundant) {
  dse_space *sp = R->space;
  cudaStream_t st = R->stream;
  const int L = R->n_lists;
  const int64_t kk = R->k, N = sp->N;
  const double w_tau = sqrt(2.0 * tau) * (1.0 + 1e-9) + 1e-13;
  const FeatTable F = table_of(sp);
  // unit vectors for as many lists at a time as fit in 1 GiB
  const size_t per_list = (size_t)kk * (size_t)N * sizeof(double);
  const int chunk = (int)std::max<size_t>(1, std::min<size_t>((size_t)L, ((size_t)1 << 30) / std::max<size_t>(per_list, 1)));
  double *z = nullptr;
  uint8_t *red = nullptr;
  DSE_TRY(dalloc(&z, (size_t)chunk * kk * N, "dedup unit vectors"));
  DSE_TRY(dalloc(&red, (size_t)L * kk, "dedup flags"));
  DSE_CUDA(cudaMemsetAsync(red, 0, (size_t)L * kk, st));
  for (int l0 = 0; l0 < L; l0 += chunk) {
    const int nl = std::min(chunk, L - l0);
    const dim3 grid((unsigned)kk, (unsigned)nl);
    note_launches(2);
    k_dedup_unit<<<grid, kUnitThreads, 0, st>>>(F, sp->geom, sp->n, R->out_id, R->out_n, kk, l0, z);
    k_dedup_flags<<<grid, kFlagThreads, 0, st>>>(R->out_id, R->out_score, R->out_n, R->max_eps, kk, l0, N, z, tau,
                                                 w_tau, red);
  }
  // new lists: ids, scores, bounds [L][k], lengths, bounds, flags, counts
  const size_t b_id = 8 * (size_t)L * k, b_sc = b_id, b_ep = b_id;
  const size_t off_sc = b_id, off_ep = off_sc + b_sc, off_n = off_ep + b_ep, off_me = off_n + 8 * (size_t)L,
               off_un = off_me + 8 * (size_t)L, off_nr = off_un + 8 * (size_t)L, bytes = off_nr + 8 * (size_t)L;
  char *buf = nullptr;
  DSE_TRY(dalloc(&buf, bytes, "deduplicated lists"));
  uint64_t *o_id = reinterpret_cast<uint64_t *>(buf);
  double *o_sc = reinterpret_cast<double *>(buf + off_sc);
  double *o_ep = reinterpret_cast<double *>(buf + off_ep);
  int64_t *o_n = reinterpret_cast<int64_t *>(buf + off_n);
  double *o_me = reinterpret_cast<double *>(buf + off_me);
  int *o_un = reinterpret_cast<int *>(buf + off_un);
  int64_t *o_nr = reinterpret_cast<int64_t *>(buf + off_nr);
  note_launches(1);
  k_dedup_compact<<<(unsigned)L, 32, 0, st>>>(R->out_id, R->out_score, R->out_eps, R->out_n, R->max_eps, kk, k,
                                              full ? 1 : 0, w_tau, red, o_id, o_sc, o_ep, o_n, o_me, o_un, o_nr);
  dfree(z);
  dfree(red);
  // lengths, bounds, flags and counts back in one copy
  char *h = static_cast<char *>(pinned_staging(bytes - off_n));
  if (!h) {
    dfree(buf);
    return DSE_ENOMEM;
  }
  DSE_CUDA(cudaMemcpyAsync(h, buf + off_n, bytes - off_n, cudaMemcpyDeviceToHost, st));
  DSE_CUDA(cudaStreamSynchronize(st));
  const int64_t *hn = reinterpret_cast<const int64_t *>(h);
  const double *hme = reinterpret_cast<const double *>(h + (off_me - off_n));
  const int *hun = reinterpret_cast<const int *>(h + (off_un - off_n));
  const int64_t *hnr = reinterpret_cast<const int64_t *>(h + (off_nr - off_n));
  bool und = false;
  int64_t nr = 0;
  double me = 0.0;
  for (int l = 0; l < L; ++l) {
    und |= hun[l] != 0;
    nr += hnr[l];
    if (hn[l] > 0) me = std::max(me, hme[l]);
  }
  *undecided = und;
  *n_redundant = nr;
  if (und) {
    dfree(buf);
    return DSE_OK;
  }
  dfree(R->extra);
  R->extra = buf;
  R->out_id = o_id;
  R->out_score = o_sc;
  R->out_eps = o_ep;
  R->out_n = o_n;
  R->max_eps = o_me;
  R->k = k;
  R->h_out_n.assign(hn, hn + L);
  R->host_stats.max_err_bound = me;
  return DSE_OK;
}

}  // namespace dse
