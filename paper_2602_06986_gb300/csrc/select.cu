// select.cu -- exact top-k selection from the candidate buffers.
//
// Each buffered entry carries an interval [lo, hi] = [s - eps, s + eps] that
// contains its FP64 score.  With L the k-th largest lo and H the (k+1)-th
// largest hi of a list:
//   lo > H          the entry is certainly in the top k;
//   hi < L          it is certainly out (and so is every unbuffered candidate,
//                   whose hi is below the list's threshold <= L);
//   otherwise       it is undecided and re-scored (FP32-pair sums, FP64
//                   where they do not apply).
// The retained set (certain + undecided) is ordered by score (FP64 where
// re-scored), then id, and its first k entries are the result: order by score
// descending, then global id ascending (the SIS top-k of SISSO screening).
//
// L and H come from the bound histograms the screen kept while buffering:
// the bin holding the k-th lower bound (resp. (k+1)-th upper bound) is found
// from the counts, and only the entries of that one bin are ranked exactly.
// Every pass over the buffers is spread over the whole GPU.
#include <math.h>

#include <algorithm>

#include "dse_internal.cuh"
#include "df32.cuh"
#include "eval64.cuh"
#include "screen_common.cuh"
#include "screen_kernels.cuh"
#include "util.cuh"

namespace dse {

__device__ __forceinline__ float lo_of(float s, float e) {
  const float lo = iv_lo(s, e);
  return lo > 0.f ? lo : 0.f;
}
__device__ __forceinline__ float hi_of(float s, float e) {
  const float hi = iv_hi(s, e);
  return hi > 0.f ? hi : 0.f;
}

// Highest bin b of h[0..kNumBins) whose suffix count reaches k; *rank = k minus
// the count above b.  One block of 1024 threads: thread t owns kNumBins/1024
// consecutive bins; the suffix sums over threads come from warp shuffles and
// one pass over the 32 warp totals.
__device__ int suffix_bin(const unsigned *h, unsigned long long k, unsigned long long *rank) {
  constexpr int PER = kNumBins / 1024;
  __syncthreads();  // a previous call's result has been read by every thread
  const int t = threadIdx.x, lane = t & 31, w = t >> 5;
  unsigned long long c[PER], tot = 0;
#pragma unroll
  for (int i = 0; i < PER; ++i) {
    c[i] = h[t * PER + i];
    tot += c[i];
  }
  // suffix within the warp (lanes >= this one)
  unsigned long long x = tot;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const unsigned long long v = __shfl_down_sync(0xffffffffu, x, o);
    if (lane + o < 32) x += v;
  }
  __shared__ unsigned long long wsum[32];
  __shared__ int found;
  if (lane == 0) wsum[w] = x;
  if (t == 0) found = -1;
  __syncthreads();
  unsigned long long above_w = 0;  // all bins of the warps above this one
  for (int q = w + 1; q < 32; ++q) above_w += wsum[q];
  // count above this thread's highest bin, then walk its bins downwards
  unsigned long long cum = above_w + (x - tot);
#pragma unroll
  for (int i = PER - 1; i >= 0; --i) {
    if (cum < k && cum + c[i] >= k) {
      found = t * PER + i;
      *rank = k - cum;
    }
    cum += c[i];
  }
  __syncthreads();
  return found;
}

// 1) per list: entry count, overflow flag, bins and in-bin ranks of L and H.
__global__ void __launch_bounds__(1024) k_sel_bins(const SelectArgs S) {
  __shared__ unsigned long long rankL, rankH;
  const int l = blockIdx.x;
  const unsigned cnt = S.B.count[l];
  const int64_t n = (int64_t)cnt < S.B.cap ? (int64_t)cnt : S.B.cap;
  SelState st{};
  st.n = (unsigned)n;
  if (n <= S.k) {
    st.all_in = 1;
    st.binL = st.binH = -1;
  } else {
    st.binL = suffix_bin(S.B.hist + (size_t)l * kNumBins, (unsigned long long)S.k, &rankL);
    st.binH = suffix_bin(S.B.hist_hi + (size_t)l * kNumBins, (unsigned long long)S.k + 1ull, &rankH);
    st.rankL = (unsigned)rankL;
    st.rankH = (unsigned)rankH;
  }
  if (threadIdx.x == 0) {
    S.overflow[l] = (int64_t)cnt > S.B.cap ? 1u : 0u;
    S.state[l] = st;
    S.r_count[l] = 0;
    S.max_eps[l] = 0.0;
  }
}

// 2) entries of the L bin and of the H bin, per list (all blocks, 2-D grid).
__global__ void k_sel_collect(const SelectArgs S) {
  const int l = blockIdx.y;
  const SelState st = S.state[l];
  if (st.all_in) return;
  const size_t base = (size_t)l * S.B.cap;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < st.n; i += (int64_t)gridDim.x * blockDim.x) {
    const float s = S.B.score[base + i], e = S.B.eps[base + i];
    if (score_bin(iv_lo(s, e)) == st.binL) {
      unsigned p = atomicAdd(&S.state[l].nL, 1u);
      S.colL[base + p] = lo_of(s, e);
    }
    if (score_bin(iv_hi(s, e)) == st.binH) {
      unsigned p = atomicAdd(&S.state[l].nH, 1u);
      S.colH[base + p] = hi_of(s, e);
    }
  }
}

// r-th largest (1-based) of n non-negative floats; block-wide radix select.
__device__ float kth_largest(const float *v, unsigned n, unsigned r, unsigned *hist) {
  __shared__ uint32_t sh_prefix, sh_mask;
  __shared__ unsigned sh_rem;
  if (threadIdx.x == 0) {
    sh_prefix = 0;
    sh_mask = 0;
    sh_rem = r;
  }
  __syncthreads();
  for (int shift = 24; shift >= 0; shift -= 8) {
    for (int b = threadIdx.x; b < 256; b += blockDim.x) hist[b] = 0;
    __syncthreads();
    const uint32_t prefix = sh_prefix, mask = sh_mask;
    // the collected values share one score bin, so most digits coincide:
    // lanes with equal digits add once per group (warp-aggregated atomics)
    const unsigned n_up = (n + 31u) & ~31u;
    for (unsigned i = threadIdx.x; i < n_up; i += blockDim.x) {
      int digit = -1;
      if (i < n) {
        const uint32_t key = __float_as_uint(v[i]);
        if ((key & mask) == prefix) digit = (int)((key >> shift) & 255u);
      }
      const unsigned peers = __match_any_sync(0xffffffffu, digit);
      if (digit >= 0 && (threadIdx.x & 31) == (unsigned)(__ffs(peers) - 1))
        atomicAdd(&hist[digit], (unsigned)__popc(peers));
    }
    __syncthreads();
    // warp 0: the digit d holding the rem-th largest, by a suffix scan of the
    // 256 counts (lane j owns digits 255-8j .. 248-8j, highest first)
    if (threadIdx.x < 32) {
      const int lane = threadIdx.x;
      const unsigned rem = sh_rem;
      unsigned c[8], tot = 0;
      for (int q = 0; q < 8; ++q) {
        c[q] = hist[255 - 8 * lane - q];
        tot += c[q];
      }
      unsigned incl = tot;  // inclusive prefix over lanes (higher digits first)
      for (int o = 1; o < 32; o <<= 1) {
        const unsigned t = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += t;
      }
      const unsigned excl = incl - tot;
      // the first lane whose inclusive count reaches rem holds the digit
      const unsigned hit = __ballot_sync(0xffffffffu, incl >= rem);
      const int owner = hit ? __ffs(hit) - 1 : 31;
      if (lane == owner) {
        unsigned cum = excl;
        int d = 255 - 8 * lane;
        for (int q = 0; q < 8; ++q, --d) {
          if (cum + c[q] >= rem || d == 0) break;
          cum += c[q];
        }
        sh_rem = rem - cum;
        sh_prefix = prefix | ((uint32_t)d << shift);
        sh_mask = mask | (255u << shift);
      }
    }
    __syncthreads();
  }
  return __uint_as_float(sh_prefix);
}

// 3) exact L and H from their bins (one block per list).
__global__ void __launch_bounds__(1024) k_sel_exact(const SelectArgs S) {
  __shared__ unsigned hist[256];
  const int l = blockIdx.x;
  SelState st = S.state[l];
  if (st.all_in) return;
  const size_t base = (size_t)l * S.B.cap;
  const float L = kth_largest(S.colL + base, st.nL, st.rankL, hist);
  const float H = kth_largest(S.colH + base, st.nH, st.rankH, hist);
  if (threadIdx.x == 0) {
    S.state[l].L = L;
    S.state[l].H = H;
  }
}

// Scores are non-negative, so the bit patterns of their doubles order like
// the values: ranks compare 64-bit integers (integer ALU), not doubles (FP64
// compares are slow on this part).
__device__ __forceinline__ uint64_t score_key(double s) { return (uint64_t)__double_as_longlong(s); }

// 4) classification into the retained set and the FP64 job list (all blocks).
__global__ void k_sel_classify(const SelectArgs S) {
  const int l = blockIdx.y;
  const SelState st = S.state[l];
  const size_t base = (size_t)l * S.B.cap;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < st.n; i += (int64_t)gridDim.x * blockDim.x) {
    const float s = S.B.score[base + i], e = S.B.eps[base + i];
    const bool in = st.all_in || lo_of(s, e) > st.H;
    const bool und = !in && hi_of(s, e) >= st.L;
    if (!(in || und)) continue;
    const unsigned pos = atomicAdd(&S.r_count[l], 1u);
    const size_t r = base + pos;
    S.r_rank[r] = 0u;
    S.r_id[r] = S.B.id[base + i];
    S.r_s32[r] = s;
    S.r_e32[r] = e;
    const bool need = S.all64 || und || e > kTol * s;
    S.r_need[r] = need ? 1 : 0;
    if (!need) S.r_key[r] = score_key((double)s);
    // with refit sums requested every retained entry is a job (the entries
    // that need no re-score keep their score and key: only their sums are
    // taken)
    if (S.r_x) S.r_x[r * 8 + 7] = 0.0;
    if (need && !und && S.rescore32) {
      // certainly in, bound wider than the tolerance: the FP32 re-score first
      unsigned j = atomicAdd(S.n_jobs + 1, 1u);
      S.job32[j] = pos;
      S.job32_list[j] = (uint32_t)l;
    } else if (need || S.r_x) {
      unsigned j = atomicAdd(S.n_jobs, 1u);
      S.job[j] = pos;
      S.job_list[j] = (uint32_t)l;
    }
  }
}

// 5) re-score.  Aggregated lists of several targets: FP64, one block of kRes
// threads per job (k_rescore_warp: one warp, for short sample ranges), one
// pass over the samples with sums shifted by the candidate's first value (so
// Sxx = S2 - S1^2/N keeps FP64 accuracy), at most 16 targets.  One-target
// lists: k_rescore1 below.
constexpr int kRes = 128;

// batch != nullptr: list l is problem l of a batched screen.  NT: 1 for
// per-target lists, 16 (the first nt used) for aggregated lists; a
// compile-time count keeps the accumulators in registers.
template <int NT>
__global__ void __launch_bounds__(kRes) k_rescore(const SelectArgs S, const ScreenArgs A0, const ScreenArgs *batch) {
  __shared__ double red[kRes / 32][2 + NT];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  const unsigned nj = *S.n_jobs;
  for (unsigned w = blockIdx.x; w < nj; w += gridDim.x) {
    const unsigned pos = S.job[w], l = S.job_list[w];
    const ScreenArgs &A = batch ? batch[l] : A0;
    const int64_t N = A.N;
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
    const int t_begin = A.mode == DSE_MODE_AGGREGATED ? 0 : (int)l;
    const int nt = A.mode == DSE_MODE_AGGREGATED ? (A.T < NT ? A.T : NT) : 1;
    const double c = eval_op64(op, xa[0], xb[0]);
    double acc[2 + NT];
#pragma unroll
    for (int i = 0; i < 2 + NT; ++i) acc[i] = 0.0;
    for (int64_t s = threadIdx.x; s < N; s += kRes) {
      const double v = eval_op64(op, xa[s], xb[s]) - c;
      acc[0] += v;
      acc[1] = fma(v, v, acc[1]);
#pragma unroll
      for (int t = 0; t < NT; ++t)
        if (t < nt) acc[2 + t] = fma(v, A.y64[(int64_t)(t_begin + t) * A.ldy + s], acc[2 + t]);
    }
#pragma unroll
    for (int i = 0; i < 2 + NT; ++i) {
      double v = warp_sum64(acc[i]);
      if (lane == 0) red[wid][i] = v;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
      double t1 = 0, t2 = 0;
      for (int q = 0; q < kRes / 32; ++q) {
        t1 += red[q][0];
        t2 += red[q][1];
      }
      const double mean = t1 / (double)N;
      const double sxx = t2 - t1 * mean;
      double agg = 0.0;
      for (int t = 0; t < nt; ++t) {
        double sy = 0;
        for (int q = 0; q < kRes / 32; ++q) sy += red[q][2 + t];
        // the targets are centred: sum (v - vbar) y = sum (v - c) y - (vbar - c) sum y, sum y = 0 up to rounding
        const double sc = fabs(sy) / sqrt(sxx);
        agg += sc * sc;
      }
      const double sc = A.mode == DSE_MODE_AGGREGATED ? sqrt(agg / (double)nt) : sqrt(agg);
      S.r_s64[r] = sc;
      S.r_e64[r] = (double)(N / kRes + 64) * 1.1102230246251565e-16 * 16.0 * (sc + 1e-3);
      S.r_key[r] = score_key(sc);
      atomicAdd(&A.stats[ST_RESCORED], 1ull);
    }
    __syncthreads();
  }
}

// The same re-score with one warp per job (lanes over samples, shuffle
// reductions, no block barriers): for short sample ranges, where a block per
// job would spend its time in barriers and reductions.
template <int NT>
__global__ void __launch_bounds__(256) k_rescore_warp(const SelectArgs S, const ScreenArgs A) {
  const int lane = threadIdx.x & 31;
  const unsigned nj = *S.n_jobs;
  const unsigned warps = (gridDim.x * blockDim.x) >> 5;
  const int64_t N = A.N;
  for (unsigned w = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; w < nj; w += warps) {
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
    const int t_begin = A.mode == DSE_MODE_AGGREGATED ? 0 : (int)l;
    const int nt = A.mode == DSE_MODE_AGGREGATED ? (A.T < NT ? A.T : NT) : 1;
    const double c = eval_op64(op, xa[0], xb[0]);
    double acc[2 + NT];
#pragma unroll
    for (int i = 0; i < 2 + NT; ++i) acc[i] = 0.0;
    for (int64_t s = lane; s < N; s += 32) {
      const double v = eval_op64(op, xa[s], xb[s]) - c;
      acc[0] += v;
      acc[1] = fma(v, v, acc[1]);
#pragma unroll
      for (int t = 0; t < NT; ++t)
        if (t < nt) acc[2 + t] = fma(v, A.y64[(int64_t)(t_begin + t) * A.ldy + s], acc[2 + t]);
    }
#pragma unroll
    for (int i = 0; i < 2 + NT; ++i) acc[i] = warp_sum64(acc[i]);
    const double eps = (double)(N / 32 + 64) * 1.7763568394002505e-15;
    if (lane == 0 && S.r_need[r]) {
      const double mean = acc[0] / (double)N;
      const double sxx = acc[1] - acc[0] * mean;
      double agg = 0.0;
#pragma unroll
      for (int t = 0; t < NT; ++t) {
        if (t >= nt) break;
        const double sc = fabs(acc[2 + t]) / sqrt(sxx);
        agg += sc * sc;
      }
      const double sc = A.mode == DSE_MODE_AGGREGATED ? sqrt(agg / (double)nt) : sqrt(agg);
      S.r_s64[r] = sc;
      S.r_e64[r] = eps * (sc + 1e-3);
      S.r_key[r] = score_key(sc);
      atomicAdd(&A.stats[ST_RESCORED], 1ull);
    }
  }
}

// 5a) FP32 re-score of entries that are certainly in the top k but whose
// screening bound is wider than the reporting tolerance (products,
// quotients, sums and differences from the Gram and tensor-core
// contractions): one warp per entry re-evaluates the candidate in FP32
// (r32_setup / r32_sums: the screen's evaluation forms, 8-sample FP32
// blocks added into FP32 pairs, gamma = kGamma32 u) and takes the interval
// from the screen's bound (realised test already decided).  The entry is
// taken when its bound is within the reporting tolerance; its reported
// score is the FP32 score clamped to the screening interval, which holds the
// FP64 score, so the clamp moves it towards that score (the bound stays
// valid) and keeps every certain entry above H, the list's (k+1)-th upper
// bound.  Entries it cannot take (other operators, operands outside the
// FP32-safe range, a wider bound) join the pair re-score's jobs.
__global__ void __launch_bounds__(256, 3) k_rescore32(const SelectArgs S, const ScreenArgs A) {
  const int lane = threadIdx.x & 31;
  const unsigned nj = S.n_jobs[1];
  const unsigned warps = (gridDim.x * blockDim.x) >> 5;
  const float u = 5.9604644775390625e-8f;
  const float Nf = (float)A.N, invN = (float)A.invN, sqrtN = sqrtf(Nf);
  const float gamma = kGamma32 * u;
  for (unsigned w = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; w < nj; w += warps) {
    const unsigned pos = S.job32[w], l = S.job32_list[w];
    const size_t r = (size_t)l * S.B.cap + pos;
    const uint64_t gid = S.r_id[r];
    int op = DSE_OP_PRIMARY;
    int64_t a = (int64_t)gid, b = -1;
    if (gid >= (uint64_t)A.n_stored) decode_flat(A.G, gid - (uint64_t)A.n_stored, &op, &a, &b);
    const int t = A.mode == DSE_MODE_AGGREGATED ? 0 : (int)l;
    R32Setup c;
    const bool ok = gid >= (uint64_t)A.n_stored && r32_setup(A, op, a, b, c);
    float Sm[3] = {0.f, 0.f, 0.f};
    if (ok) r32_sums<1, 4>(A, op, a, b, A.y32 + (int64_t)t * A.ldy, 1, c, Sm);
    if (lane == 0) {
      bool take = false;
      float s = 0.f, e = 1.f;
      if (ok) {
        const CandInterval<float> ci = cand_interval<float>(Sm[0], Sm[1], Nf, invN, sqrtN, c.cshift, c.ee, gamma, u,
                                                            -1.0f);
        if (ci.realised == 1) {
          cand_score<float>(ci, Sm[0], Sm[2], invN, A.ysum32[t], gamma, u, &s, &e);
          take = s > 0.f && e <= 0.99f * kTol * s;
        }
      }
      if (take) {
        const double lo = lo_of(S.r_s32[r], S.r_e32[r]), hi = hi_of(S.r_s32[r], S.r_e32[r]);
        double sc = (double)s;
        if (sc < lo) sc = lo;
        if (sc > hi) sc = hi;
        S.r_s64[r] = sc;
        S.r_e64[r] = (double)e;
        S.r_key[r] = score_key(sc);
        atomicAdd(&A.stats[ST_RESCORED], 1ull);
      } else {
        const unsigned j = atomicAdd(S.n_jobs, 1u);
        S.job[j] = pos;
        S.job_list[j] = l;
      }
    }
  }
}

// The re-score of one-target lists (per-target mode, or aggregated with one
// target; batched screens too): one block of kColThreads per job, the
// column's shifted sums against the list's target and the refit vectors (if
// any) by col_sums (FP32 pairs where they apply, else FP64); the score is
// |sum (v - c) y| / sqrt(Sxx) of the centred unit-norm target, its bound the
// sums' error scale times (s + 1e-3).  With S.r_x the record {c, S1, S2,
// E.., eps} of the entry is kept for the refit.
// ONE: every job is summed against its target alone (no refit vectors, a
// single screen): the one-vector column sums.
template <bool ONE>
__global__ void __launch_bounds__(kColThreads, ONE ? 6 : 1) k_rescore1(const SelectArgs S, const ScreenArgs A0,
                                                          const ScreenArgs *batch) {
  __shared__ ColShared sh;
  const unsigned nj = *S.n_jobs;
  for (unsigned w = blockIdx.x; w < nj; w += gridDim.x) {
    const unsigned pos = S.job[w], l = S.job_list[w];
    const ScreenArgs &A = batch ? batch[l] : A0;
    const int64_t N = A.N;
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
    if (!DSE_OPERANDS_OK(A.F, a, b, A0.err)) continue;
    const int t = A.mode == DSE_MODE_AGGREGATED ? 0 : (int)l;
    const int nx = batch ? 0 : S.nx;
    ColVecs V;
    V.nv = 1 + nx;
#pragma unroll
    for (int m = 0; m < kColVec; ++m) {
      V.v64[m] = m == 0 ? A.y64 + (int64_t)t * A.ldy : S.xv[m - 1];
      V.vdf[m] = m == 0 ? (A.ydf ? A.ydf + (int64_t)t * A.ldy : nullptr) : S.xdf[m - 1];
      V.e[m] = m == 0 || m >= V.nv ? 0 : S.xexp[m - 1];
    }
    ColSums cs;
    if (ONE)
      col_sums1(A.F, op, a, b, N, V, cs, sh);
    else
      col_sums(A.F, op, a, b, N, V, cs, sh);
    if (threadIdx.x == 0) {
      const double eps = col_err_scale(cs, N);
      if (S.r_x && !batch) {
        double *x = S.r_x + r * 8;
        x[0] = cs.c;
        x[1] = cs.acc[0];
        x[2] = cs.acc[1];
        for (int m = 0; m < 4; ++m) x[3 + m] = m < nx ? cs.acc[3 + m] : 0.0;
        x[7] = eps;
      }
      if (S.r_need[r]) {
        const double sc = cs.s0;
        S.r_s64[r] = sc;
        S.r_e64[r] = eps * (sc + 1e-3);
        S.r_key[r] = score_key(sc);
        atomicAdd(&A.stats[ST_RESCORED], 1ull);
      }
    }
  }
}

__device__ __forceinline__ bool before(uint64_t ka, uint64_t ia, uint64_t kb, uint64_t ib) {
  return ka > kb || (ka == kb && ia < ib);
}

__device__ __forceinline__ uint64_t retained_key(const SelectArgs &S, size_t r) { return S.r_key[r]; }

// 6) order of the retained set (score descending, id ascending) by counting:
// the rank of an entry is the number of entries ordered before it (ids are
// unique within a list, so the ranks are a permutation).  A block stages a
// tile's keys in shared memory and its warps count for their entries, lanes
// over the tile; partial counts meet in r_rank by atomic adds.  Spread over
// all blocks, so a list of a thousand entries costs a few microseconds
// instead of a single-block sort.
constexpr int kRankTile = 2048, kRankPer = 8, kRankGroup = 8 * kRankPer;

// Work items are (64 entries, a tile of kRankTile keys): each warp holds 8
// entries' keys in registers and its lanes run over the tile, so that every
// key read from shared memory serves 8 comparisons.
__global__ void __launch_bounds__(256) k_rank(const SelectArgs S) {
  __shared__ uint64_t tk[kRankTile], ti[kRankTile];
  const int l = blockIdx.y;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int64_t rn = S.r_count[l];
  const size_t base = (size_t)l * S.B.cap;
  const int64_t n_groups = (rn + kRankGroup - 1) / kRankGroup, n_tiles = (rn + kRankTile - 1) / kRankTile;
  int64_t loaded = -1;
  for (int64_t item = blockIdx.x; item < n_groups * n_tiles; item += gridDim.x) {
    const int64_t g = item / n_tiles, t = item % n_tiles;
    const int64_t t0 = t * kRankTile;
    const int nt = (int)(rn - t0 < kRankTile ? rn - t0 : kRankTile);
    if (t != loaded) {
      __syncthreads();
      for (int j = threadIdx.x; j < nt; j += blockDim.x) {
        tk[j] = retained_key(S, base + t0 + j);
        ti[j] = S.r_id[base + t0 + j];
      }
      __syncthreads();
      loaded = t;
    }
    const int64_t i0 = g * kRankGroup + (int64_t)warp * kRankPer;
    uint64_t ki[kRankPer], ii[kRankPer];
    unsigned c[kRankPer];
#pragma unroll
    for (int e = 0; e < kRankPer; ++e) {
      const int64_t i = i0 + e;
      ki[e] = i < rn ? retained_key(S, base + i) : 0ull;
      ii[e] = i < rn ? S.r_id[base + i] : 0ull;
      c[e] = 0;
    }
    for (int j = lane; j < nt; j += 32) {
      const uint64_t kj = tk[j], ij = ti[j];
#pragma unroll
      for (int e = 0; e < kRankPer; ++e) c[e] += before(kj, ij, ki[e], ii[e]) ? 1u : 0u;
    }
#pragma unroll
    for (int e = 0; e < kRankPer; ++e) {
      const unsigned v = __reduce_add_sync(0xffffffffu, c[e]);
      if (lane == 0 && v && i0 + e < rn) atomicAdd(&S.r_rank[base + i0 + e], v);
    }
  }
}

// 7) entries of rank < k to their output slots; the list's length and its
// largest returned bound (bounds are non-negative: their bit patterns order
// like the values).
__global__ void k_rank_write(const SelectArgs S) {
  const int l = blockIdx.y;
  const int64_t rn = S.r_count[l];
  const size_t base = (size_t)l * S.B.cap;
  const int64_t nout = rn < S.k ? rn : S.k;
  if (blockIdx.x == 0 && threadIdx.x == 0) S.out_n[l] = nout;
  double mx = 0.0;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < rn; i += (int64_t)gridDim.x * blockDim.x) {
    const size_t r = base + i;
    const unsigned rank = S.r_rank[r];
    if (rank >= nout) continue;
    const bool n64 = S.r_need[r] != 0;
    const size_t o = (size_t)l * S.k + rank;
    if (S.out_x) {
      const bool has = S.r_x[r * 8 + 7] != 0.0;
      for (int m = 0; m < 8; ++m) S.out_x[o * 8 + m] = has ? S.r_x[r * 8 + m] : 0.0;
    }
    S.out_id[o] = S.r_id[r];
    S.out_score[o] = n64 ? S.r_s64[r] : (double)S.r_s32[r];
    const double e = n64 ? S.r_e64[r] : (double)S.r_e32[r];
    S.out_eps[o] = e;
    mx = fmax(mx, e);
  }
  mx = warp_max64(mx);
  if ((threadIdx.x & 31) == 0 && mx > 0.0)
    atomicMax(reinterpret_cast<unsigned long long *>(&S.max_eps[l]), (unsigned long long)__double_as_longlong(mx));
}

dse_status launch_select(const SelectArgs &S0, const ScreenArgs &A, int sms, cudaStream_t st,
                         const ScreenArgs *batch) {
  note_launches(7);
  // the FP32 re-score serves one-target lists of a single FP32 screen
  // without refit sums
  SelectArgs S = S0;
  S.rescore32 = !batch && !S.all64 && S.nx == 0 && !S.r_x && S.job32 && S.job32_list && A.F.v32 && A.y32 &&
                A.ysum32 && (A.mode != DSE_MODE_AGGREGATED || A.T == 1);
  k_sel_bins<<<S.n_lists, 1024, 0, st>>>(S);
  const unsigned bx = (unsigned)std::max(1, std::min(256, (sms * 4 + S.n_lists - 1) / S.n_lists));
  dim3 g(bx, S.n_lists);
  k_sel_collect<<<g, 256, 0, st>>>(S);
  k_sel_exact<<<S.n_lists, 1024, 0, st>>>(S);
  k_sel_classify<<<g, 256, 0, st>>>(S);
  const bool one = batch || A.mode != DSE_MODE_AGGREGATED || A.T == 1;
  if (S.rescore32) {
    note_launches(1);
    k_rescore32<<<sms * 8, 256, 0, st>>>(S, A);
  }
  if (one && !batch && S.nx == 0)
    k_rescore1<true><<<sms * 16, kColThreads, 0, st>>>(S, A, batch);
  else if (one)
    k_rescore1<false><<<sms * 8, kColThreads, 0, st>>>(S, A, batch);
  else if (A.N <= 4096) k_rescore_warp<16><<<sms * 8, 256, 0, st>>>(S, A);
  else k_rescore<16><<<sms * 8, kRes, 0, st>>>(S, A, batch);
  const dim3 gr((unsigned)std::max(1, std::min(1024, (sms * 2 + S.n_lists - 1) / S.n_lists)), S.n_lists);
  k_rank<<<gr, 256, 0, st>>>(S);
  const dim3 gw((unsigned)std::max(1, std::min(64, (sms + S.n_lists - 1) / S.n_lists)), S.n_lists);
  k_rank_write<<<gw, 256, 0, st>>>(S);
  return DSE_OK;
}

}  // namespace dse
