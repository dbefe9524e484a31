// select.cu -- exact top-k selection from the candidate buffers.
//
// Each buffered entry carries an interval [lo, hi] = [s - eps, s + eps] that
// contains its FP64 score.  With L the k-th largest lo and H the (k+1)-th
// largest hi of a list:
//   lo > H          the entry is certainly in the top k;
//   hi < L          it is certainly out (and so is every unbuffered candidate,
//                   whose hi is below the list's threshold <= L);
//   otherwise       it is undecided and re-scored in FP64.
// The retained set (certain + undecided) is ordered by score (FP64 where
// re-scored), then id, and its first k entries are the result: order by score
// descending, then global id ascending (the SIS top-k, SISSO screening).
#include <math.h>

#include "dse_internal.cuh"
#include "eval64.cuh"
#include "screen_common.cuh"
#include "screen_kernels.cuh"
#include "util.cuh"

namespace dse {

__device__ __forceinline__ uint32_t key_lo(float s, float e) {
  float lo = s - e;
  if (!(lo > 0.f)) lo = 0.f;
  return __float_as_uint(lo);
}
__device__ __forceinline__ uint32_t key_hi(float s, float e) {
  float hi = s + e;
  if (!(hi > 0.f)) hi = 0.f;
  return __float_as_uint(hi);
}

// k-th largest key (1-based) among n entries; block-wide radix select.
template <bool HI>
__device__ uint32_t kth_largest(const float *s, const float *e, int64_t n, int64_t k, unsigned *hist) {
  __shared__ uint32_t sh_prefix, sh_mask;
  __shared__ unsigned long long sh_rem;
  if (threadIdx.x == 0) {
    sh_prefix = 0;
    sh_mask = 0;
    sh_rem = (unsigned long long)k;
  }
  __syncthreads();
  for (int shift = 24; shift >= 0; shift -= 8) {
    for (int b = threadIdx.x; b < 256; b += blockDim.x) hist[b] = 0;
    __syncthreads();
    const uint32_t prefix = sh_prefix, mask = sh_mask;
    for (int64_t i = threadIdx.x; i < n; i += blockDim.x) {
      uint32_t key = HI ? key_hi(s[i], e[i]) : key_lo(s[i], e[i]);
      if ((key & mask) == prefix) atomicAdd(&hist[(key >> shift) & 255u], 1u);
    }
    __syncthreads();
    if (threadIdx.x == 0) {
      unsigned long long cum = 0, rem = sh_rem;
      int d = 255;
      for (; d > 0; --d) {
        if (cum + hist[d] >= rem) break;
        cum += hist[d];
      }
      sh_rem = rem - cum;
      sh_prefix = prefix | ((uint32_t)d << shift);
      sh_mask = mask | (255u << shift);
    }
    __syncthreads();
  }
  return sh_prefix;
}

// One block per list: thresholds, classification, retained set, FP64 jobs.
__global__ void __launch_bounds__(1024) k_classify(const SelectArgs S) {
  __shared__ unsigned hist[256];
  __shared__ unsigned sh_rn;
  const int l = blockIdx.x;
  const unsigned cnt = S.B.count[l];
  const int64_t n = (int64_t)cnt < S.B.cap ? (int64_t)cnt : S.B.cap;
  if (threadIdx.x == 0) {
    S.overflow[l] = (int64_t)cnt > S.B.cap ? 1u : 0u;
    sh_rn = 0;
  }
  const size_t base = (size_t)l * S.B.cap;
  const float *sc = S.B.score + base, *ep = S.B.eps + base;
  float L = -1.f, H = -1.f;
  if (n > S.k) {
    L = __uint_as_float(kth_largest<false>(sc, ep, n, S.k, hist));
    H = __uint_as_float(kth_largest<true>(sc, ep, n, S.k + 1, hist));
  }
  __syncthreads();
  for (int64_t i = threadIdx.x; i < n; i += blockDim.x) {
    const float s = sc[i], e = ep[i];
    const float lo = __uint_as_float(key_lo(s, e)), hi = __uint_as_float(key_hi(s, e));
    const bool in = n <= S.k || lo > H;
    const bool und = !in && hi >= L;
    if (!(in || und)) continue;
    const unsigned pos = atomicAdd(&sh_rn, 1u);
    const size_t r = base + pos;
    S.r_id[r] = S.B.id[base + i];
    S.r_s32[r] = s;
    S.r_e32[r] = e;
    const bool need = S.all64 || und || e > kTol * s;
    S.r_need[r] = need ? 1 : 0;
    if (need) {
      unsigned j = atomicAdd(S.n_jobs, 1u);
      S.job[j] = pos;
      S.job_list[j] = (uint32_t)l;
    }
  }
  __syncthreads();
  if (threadIdx.x == 0) S.r_count[l] = sh_rn;
}

// FP64 re-score: one warp per job.
__global__ void k_rescore(const SelectArgs S, const ScreenArgs A) {
  const int lane = threadIdx.x & 31;
  const unsigned nj = *S.n_jobs;
  const uint64_t warps = (uint64_t)gridDim.x * (blockDim.x >> 5);
  const int64_t N = A.N;
  for (uint64_t w = ((uint64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; w < nj; w += warps) {
    const unsigned pos = S.job[w], l = S.job_list[w];
    const size_t r = (size_t)l * S.B.cap + pos;
    const uint64_t gid = S.r_id[r];
    int op;
    int64_t a, b;
    if (gid < (uint64_t)A.n_stored) {
      op = DSE_OP_PRIMARY;
      a = (int64_t)gid;
      b = -1;
    } else {
      decode_flat(A.G, gid - (uint64_t)A.n_stored, &op, &a, &b);
    }
    const double *xa = A.F.v64 + a * A.F.ld;
    const double *xb = A.F.v64 + (b >= 0 ? b : a) * A.F.ld;
    double sum = 0.0;
    for (int64_t s = lane; s < N; s += 32) sum += eval_op64(op, xa[s], xb[s]);
    sum = warp_sum64(sum);
    const double mean = sum / (double)N;
    double sxx = 0.0;
    for (int64_t s = lane; s < N; s += 32) {
      double d = eval_op64(op, xa[s], xb[s]) - mean;
      sxx = fma(d, d, sxx);
    }
    sxx = warp_sum64(sxx);
    const int t_begin = A.mode == DSE_MODE_AGGREGATED ? 0 : (int)l;
    const int t_end = A.mode == DSE_MODE_AGGREGATED ? A.T : (int)l + 1;
    double agg = 0.0;
    for (int t = t_begin; t < t_end; ++t) {
      const double *y = A.y64 + (int64_t)t * A.ldy;
      double sxy = 0.0;
      for (int64_t s = lane; s < N; s += 32) sxy = fma(eval_op64(op, xa[s], xb[s]) - mean, y[s], sxy);
      sxy = warp_sum64(sxy);
      double sc = fabs(sxy) / sqrt(sxx);
      agg += sc * sc;
    }
    double sc = A.mode == DSE_MODE_AGGREGATED ? sqrt(agg / (double)A.T) : sqrt(agg);
    if (lane == 0) {
      S.r_s64[r] = sc;
      S.r_e64[r] = (double)(N / 32 + 40) * 1.1102230246251565e-16 * 8.0 * (sc + 1e-3);
      atomicAdd(&A.stats[ST_RESCORED], 1ull);
    }
  }
}

__device__ __forceinline__ bool before(double ka, uint64_t ia, double kb, uint64_t ib) {
  return ka > kb || (ka == kb && ia < ib);
}

// Bitonic sort (descending key, ascending id) of M (power of two) entries.
__device__ void bitonic(double *key, uint64_t *id, int64_t M) {
  for (int64_t size = 2; size <= M; size <<= 1) {
    for (int64_t stride = size >> 1; stride > 0; stride >>= 1) {
      for (int64_t i = threadIdx.x; i < M; i += blockDim.x) {
        int64_t j = i ^ stride;
        if (j > i) {
          bool up = (i & size) == 0;
          double ki = key[i], kj = key[j];
          uint64_t ii = id[i], ij = id[j];
          bool sw = up ? before(kj, ij, ki, ii) : before(ki, ii, kj, ij);
          if (sw) {
            key[i] = kj;
            key[j] = ki;
            id[i] = ij;
            id[j] = ii;
          }
        }
      }
      __syncthreads();
    }
  }
}

constexpr int64_t kSmemSort = 4096;

// One block per list: order the retained set and write the first k.
__global__ void __launch_bounds__(1024) k_final(const SelectArgs S) {
  extern __shared__ __align__(16) unsigned char sm[];
  const int l = blockIdx.x;
  const int64_t rn = S.r_count[l];
  const size_t base = (size_t)l * S.B.cap;
  int64_t M = 1;
  while (M < rn) M <<= 1;
  double *key;
  uint64_t *id;
  if (M <= kSmemSort) {
    key = reinterpret_cast<double *>(sm);
    id = reinterpret_cast<uint64_t *>(sm + kSmemSort * sizeof(double));
  } else {
    key = S.sort_key + (size_t)l * S.sort_cap;
    id = S.sort_id + (size_t)l * S.sort_cap;
  }
  // id slot holds the retained position; ties are resolved on the real ids
  // below, so sort on (key, global id) pairs directly.
  for (int64_t i = threadIdx.x; i < M; i += blockDim.x) {
    if (i < rn) {
      const size_t r = base + i;
      key[i] = S.r_need[r] ? S.r_s64[r] : (double)S.r_s32[r];
      id[i] = S.r_id[r];
    } else {
      key[i] = -INFINITY;
      id[i] = ~0ull;
    }
  }
  __syncthreads();
  bitonic(key, id, M);
  // look up each output's bound by searching the retained set (rn small
  // relative to the work above; entries are unique by id)
  const int64_t nout = rn < S.k ? rn : S.k;
  for (int64_t i = threadIdx.x; i < nout; i += blockDim.x) {
    S.out_id[(size_t)l * S.k + i] = id[i];
    S.out_score[(size_t)l * S.k + i] = key[i];
  }
  __syncthreads();
  for (int64_t i = threadIdx.x; i < rn; i += blockDim.x) {
    // position of entry i in the sorted order: binary search on (key, id)
    const size_t r = base + i;
    const double k0 = S.r_need[r] ? S.r_s64[r] : (double)S.r_s32[r];
    const uint64_t i0 = S.r_id[r];
    int64_t lo = 0, hi = M;
    while (lo < hi) {
      int64_t mid = (lo + hi) >> 1;
      if (before(key[mid], id[mid], k0, i0)) lo = mid + 1;
      else hi = mid;
    }
    if (lo < nout) S.out_eps[(size_t)l * S.k + lo] = S.r_need[r] ? S.r_e64[r] : (double)S.r_e32[r];
  }
  if (threadIdx.x == 0) S.out_n[l] = nout;
}

dse_status launch_select(const SelectArgs &S, const ScreenArgs &A, int sms, cudaStream_t st) {
  note_launches(3);
  k_classify<<<S.n_lists, 1024, 0, st>>>(S);
  k_rescore<<<sms * 4, 256, 0, st>>>(S, A);
  static bool attr = false;
  if (!attr) {
    DSE_CUDA(cudaFuncSetAttribute(k_final, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  (int)(kSmemSort * (sizeof(double) + sizeof(uint64_t)))));
    attr = true;
  }
  k_final<<<S.n_lists, 1024, kSmemSort * (sizeof(double) + sizeof(uint64_t)), st>>>(S);
  return DSE_OK;
}

}  // namespace dse
