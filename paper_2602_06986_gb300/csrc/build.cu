// build.cu -- dse_build_space: materialise rungs 0..max_rung-1 on the device.
//
// Follows the iterative generation of "Software Description" and the early
// exclusion of dimensionally invalid expressions of "Physics-Informed
// Constraints": rung r is generated from Phi_{r-1} (unary block over the
// newest rung, then every pair (i, j) with i in the newest rung and j < i, one
// slot per enabled binary op), every slot is tested (unit, complexity,
// domain, magnitude on FP64 summaries, then the realised test on the FP64
// values) and the valid ones are appended in flat order.  Everything runs in
// FP64 on the device; the host only sizes arrays between the passes.
#include <math.h>
#include <stdio.h>
#include <string.h>

#include <algorithm>
#include <numeric>

#include "dse_internal.cuh"
#include "eval64.cuh"
#include "util.cuh"

namespace dse {

// ---------------------------------------------------------------- kernels

__global__ void k_gather_rows(const double *X, int64_t ldx, const int64_t *idx, int64_t n0, int64_t N, int64_t ld,
                              double *out) {
  int64_t total = n0 * ld;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
    int64_t f = e / ld, s = e % ld;
    double v = 0.0;
    if (s < N) v = X[f * ldx + (idx ? idx[s] : s)];
    out[e] = v;
  }
}

// Order-preserving integer images of doubles (not NaN): signed for values,
// unsigned magnitude bits for absolute values.  Minima and maxima are taken
// on the integer pipe: on this part FP64 instructions issue at a small
// fraction of the integer rate, and the results are the same doubles.
__device__ __forceinline__ long long ord_key(double v) {
  const long long b = __double_as_longlong(v);
  return b ^ ((b >> 63) & 0x7FFFFFFFFFFFFFFFll);
}
__device__ __forceinline__ double ord_val(long long k) {
  return __longlong_as_double(k ^ ((k >> 63) & 0x7FFFFFFFFFFFFFFFll));
}

constexpr int kSumThreads = 128;

template <typename T, typename Op>
__device__ __forceinline__ T block_reduce_sum(T v, T *sm, Op op) {
  for (int o = 16; o > 0; o >>= 1) v = op(v, __shfl_xor_sync(0xffffffffu, v, o));
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  __syncthreads();
  if (lane == 0) sm[w] = v;
  __syncthreads();
  T t = sm[0];
  for (int i = 1; i < kSumThreads / 32; ++i) t = op(t, sm[i]);
  return t;
}

// Summaries of stored rows [f0, f1) (only the first *n_dev of them when n_dev
// is given): one block of kSumThreads per row.
// min, max, min|x|, max|x| and the smallest non-zero |x| on integer images;
// the FP64 sum for the mean, then the centred sum of squares and the sum of
// squares for the realised test (finite, std > fmin * rms) into ok[f - f0]
// when ok != nullptr.  rmean (the mean of 1/x, 0 if min|x| == 0) is only a
// shift constant of the quotient kernels, so it is accumulated in FP32
// (FP64 when a reciprocal leaves the FP32 range).
__global__ void __launch_bounds__(kSumThreads) k_summaries(double *v64, int64_t ld, int64_t N, int64_t f0,
                                                           int64_t f1, double *mean64, double *rmean64, double *min64,
                                                           double *max64, double *minabs64, double *maxabs64,
                                                           double *minabsnz64, double fmin_std_rel, uint8_t *ok,
                                                           const unsigned long long *n_dev) {
  __shared__ double smd[kSumThreads / 32];
  // the partials of the merged reductions: per warp {sum, min|x|} after the
  // first pass, then {min, max, max|x|, min nonzero |x|, finite, sxx, s2, rs}
  __shared__ unsigned long long sa[kSumThreads / 32][2], sb[kSumThreads / 32][8];
  const int64_t f = f0 + blockIdx.x;
  if (f >= f1 || (n_dev && (unsigned long long)(f - f0) >= *n_dev)) return;
  const double *x = v64 + f * ld;
  long long kmn = 0x7FFFFFFFFFFFFFFFll, kmx = (long long)0x8000000000000000ull;
  unsigned long long amn = ~0ull, amx = 0ull, anz = ~0ull;
  int fin = 1;
  double sum = 0.0;
  // four samples per thread per step, their loads issued together; each
  // thread takes its samples in increasing order
  constexpr int U = 4;
  for (int64_t s0 = threadIdx.x; s0 < N; s0 += U * kSumThreads) {
    double xv[U];
#pragma unroll
    for (int q = 0; q < U; ++q) xv[q] = s0 + q * kSumThreads < N ? x[s0 + q * kSumThreads] : 0.0;
#pragma unroll
    for (int q = 0; q < U; ++q) {
      if (s0 + q * kSumThreads >= N) break;
      const double v = xv[q];
      const unsigned long long b = (unsigned long long)__double_as_longlong(v);
      const unsigned long long a = b & 0x7FFFFFFFFFFFFFFFull;
      fin &= a < 0x7FF0000000000000ull;
      const long long k = ord_key(v);
      kmn = k < kmn ? k : kmn;
      kmx = k > kmx ? k : kmx;
      amn = a < amn ? a : amn;
      amx = a > amx ? a : amx;
      if (a != 0ull) anz = a < anz ? a : anz;
      sum = __dadd_rn(sum, v);
    }
  }
  // merged reduction 1 (every thread needs the sum and min|x|): one barrier
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  constexpr int NW = kSumThreads / 32;
  for (int o = 16; o > 0; o >>= 1) {
    sum += __shfl_xor_sync(0xffffffffu, sum, o);
    const unsigned long long q = __shfl_xor_sync(0xffffffffu, amn, o);
    amn = q < amn ? q : amn;
  }
  if (lane == 0) {
    sa[wid][0] = (unsigned long long)__double_as_longlong(sum);
    sa[wid][1] = amn;
  }
  __syncthreads();
  sum = 0.0;
  amn = ~0ull;
#pragma unroll
  for (int w = 0; w < NW; ++w) {
    sum += __longlong_as_double((long long)sa[w][0]);
    amn = sa[w][1] < amn ? sa[w][1] : amn;
  }
  const double mean = sum / (double)N;
  const double mna = __longlong_as_double((long long)amn);
  double sxx = 0.0, s2 = 0.0;
  float rs = 0.f;
  for (int64_t s0 = threadIdx.x; s0 < N; s0 += U * kSumThreads) {
    double xv[U];
#pragma unroll
    for (int q = 0; q < U; ++q) xv[q] = s0 + q * kSumThreads < N ? x[s0 + q * kSumThreads] : 0.0;
#pragma unroll
    for (int q = 0; q < U; ++q) {
      if (s0 + q * kSumThreads >= N) break;
      const double v = xv[q];
      const double d = __dsub_rn(v, mean);
      sxx = __fma_rn(d, d, sxx);
      s2 = __fma_rn(v, v, s2);
      if (mna > 0.0) rs += __frcp_rn(__double2float_rn(v));
    }
  }
  // merged reduction 2: the order statistics, the finite flag and the
  // second-pass sums, one barrier (every thread gets them)
  for (int o = 16; o > 0; o >>= 1) {
    const long long a = __shfl_xor_sync(0xffffffffu, kmn, o), b = __shfl_xor_sync(0xffffffffu, kmx, o);
    kmn = a < kmn ? a : kmn;
    kmx = b > kmx ? b : kmx;
    const unsigned long long c = __shfl_xor_sync(0xffffffffu, amx, o), e = __shfl_xor_sync(0xffffffffu, anz, o);
    amx = c > amx ? c : amx;
    anz = e < anz ? e : anz;
    sxx += __shfl_xor_sync(0xffffffffu, sxx, o);
    s2 += __shfl_xor_sync(0xffffffffu, s2, o);
    rs += __shfl_xor_sync(0xffffffffu, rs, o);
  }
  fin = __all_sync(0xffffffffu, fin);
  if (lane == 0) {
    sb[wid][0] = (unsigned long long)kmn;
    sb[wid][1] = (unsigned long long)kmx;
    sb[wid][2] = amx;
    sb[wid][3] = anz;
    sb[wid][4] = (unsigned long long)fin;
    sb[wid][5] = (unsigned long long)__double_as_longlong(sxx);
    sb[wid][6] = (unsigned long long)__double_as_longlong(s2);
    sb[wid][7] = (unsigned long long)__float_as_uint(rs);
  }
  __syncthreads();
  sxx = 0.0;
  s2 = 0.0;
  rs = 0.f;
  fin = 1;
#pragma unroll
  for (int w = 0; w < NW; ++w) {
    const long long a = (long long)sb[w][0], b = (long long)sb[w][1];
    kmn = a < kmn ? a : kmn;
    kmx = b > kmx ? b : kmx;
    amx = sb[w][2] > amx ? sb[w][2] : amx;
    anz = sb[w][3] < anz ? sb[w][3] : anz;
    fin &= (int)sb[w][4];
    sxx += __longlong_as_double((long long)sb[w][5]);
    s2 += __longlong_as_double((long long)sb[w][6]);
    rs += __uint_as_float((unsigned)sb[w][7]);
  }
  double rmean = 0.0;
  if (mna > 0.0) {
    rmean = (double)rs / (double)N;
    if (!isfinite(rmean)) {
      // a reciprocal outside the FP32 range: the FP64 mean of 1/x
      double r64 = 0.0;
      for (int64_t s = threadIdx.x; s < N; s += kSumThreads) r64 = __dadd_rn(r64, __drcp_rn(x[s]));
      rmean = block_reduce_sum(r64, smd, [](double p, double q) { return p + q; }) / (double)N;
    }
  }
  if (threadIdx.x == 0) {
    mean64[f] = mean;
    rmean64[f] = rmean;
    min64[f] = ord_val(kmn);
    max64[f] = ord_val(kmx);
    minabs64[f] = mna;
    maxabs64[f] = __longlong_as_double((long long)amx);
    minabsnz64[f] = anz == ~0ull ? INFINITY : __longlong_as_double((long long)anz);
    if (ok) {
      int good = fin;
      if (good && fmin_std_rel >= 0.0) {
        double sd = __dsqrt_rn(sxx / (double)N), rms = __dsqrt_rn(s2 / (double)N);
        good = sd > fmin_std_rel * rms;
      }
      ok[f - f0] = (uint8_t)(good ? 1 : 0);
    }
  }
}

// FP64 values of the listed slots (the first *n_dev of at most cap) into
// scratch rows: one block per slot, one evaluation per sample.
__global__ void __launch_bounds__(kSumThreads) k_eval_rows(FeatTable F, RungGeom g, const uint64_t *list, uint64_t cap,
                                                           const unsigned long long *n_dev, double *rows) {
  const uint64_t w = blockIdx.x;
  if (w >= cap || w >= *n_dev) return;
  int op;
  int64_t a, b;
  decode_flat(g, list[w], &op, &a, &b);
  const double *xa = F.v64 + a * F.ld;
  const double *xb = F.v64 + (b >= 0 ? b : a) * F.ld;
  double *out = rows + w * F.ld;
  // four samples per thread per step, their loads issued together
  constexpr int U = 4;
  for (int64_t s0 = threadIdx.x; s0 < F.ld; s0 += U * kSumThreads) {
    double va[U], vb[U];
#pragma unroll
    for (int q = 0; q < U; ++q) {
      const int64_t s = s0 + q * kSumThreads;
      va[q] = s < F.N ? xa[s] : 0.0;
      vb[q] = s < F.N ? xb[s] : 0.0;
    }
#pragma unroll
    for (int q = 0; q < U; ++q) {
      const int64_t s = s0 + q * kSumThreads;
      if (s < F.ld) out[s] = s < F.N ? eval_op64(op, va[q], vb[q]) : 0.0;
    }
  }
}

// Scratch summaries of one evaluated rung (per scratch row).
struct RowSummaries {
  double *mean64, *rmean64, *min64, *max64, *minabs64, *maxabs64, *minabsnz64;
};

// Kept rows: scratch row pos[w] (slot list[pos[w]]) becomes stored feature
// dst0 + w: values, summaries and the metadata of its expression (op,
// operands, complexity, units, rule masks).  One block per kept row.
__global__ void __launch_bounds__(kSumThreads) k_take_eval(FeatTable F, RungGeom g, AprioriParams P,
                                                           const uint64_t *list, const uint64_t *pos, uint64_t n_keep,
                                                           int64_t dst0, const double *rows, RowSummaries src,
                                                           double *v64, RowSummaries dst, int32_t *op_out,
                                                           int64_t *ca_out, int64_t *cb_out, int32_t *cplx_out,
                                                           int32_t *units_out, uint64_t *used_out,
                                                           uint64_t *dmask_out) {
  const uint64_t w = blockIdx.x;
  if (w >= n_keep) return;
  const uint64_t p = pos[w];
  const int64_t f = dst0 + (int64_t)w;
  for (int64_t s = threadIdx.x; s < F.ld; s += kSumThreads) v64[f * F.ld + s] = rows[p * F.ld + s];
  if (threadIdx.x == 0) {
    dst.mean64[f] = src.mean64[p];
    dst.rmean64[f] = src.rmean64[p];
    dst.min64[f] = src.min64[p];
    dst.max64[f] = src.max64[p];
    dst.minabs64[f] = src.minabs64[p];
    dst.maxabs64[f] = src.maxabs64[p];
    dst.minabsnz64[f] = src.minabsnz64[p];
    int op;
    int64_t a, b;
    decode_flat(g, list[p], &op, &a, &b);
    int32_t u[kMaxDims] = {0, 0, 0, 0, 0, 0, 0, 0}, cx = 0;
    int bad = 0;
    apriori64(F, P, op, a, b, u, &cx, &bad);
    op_out[f] = op;
    ca_out[f] = a;
    cb_out[f] = b;
    cplx_out[f] = cx;
    for (int d = 0; d < kMaxDims; ++d) units_out[f * kMaxDims + d] = u[d];
    if (F.used) {
      used_out[f] = F.used[a] | (b >= 0 ? F.used[b] : 0ull);
      dmask_out[f] = F.dmask[a] | (b >= 0 ? F.dmask[b] : 0ull);
    }
  }
}

// A-priori reason of every flat slot of rung r.
__global__ void k_apriori_rung(FeatTable F, RungGeom g, AprioriParams P, uint8_t *why, int *bad) {
  for (uint64_t p = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; p < g.slots;
       p += (uint64_t)gridDim.x * blockDim.x) {
    int op;
    int64_t a, b;
    decode_flat(g, p, &op, &a, &b);
    int32_t u[kMaxDims], cx;
    int b_ = 0;
    int r = apriori64(F, P, op, a, b, u, &cx, &b_);
    if (b_) atomicOr(bad, b_);
    why[p] = (uint8_t)r;
  }
}

// Rows keep[0..nk) of a table into rows 0..nk of another (values and
// summaries): one block per kept row.
__global__ void k_take_rows(const int64_t *keep, int64_t nk, int64_t ld, const double *v64, const double *mean64,
                            const double *rmean64, const double *min64, const double *max64, const double *minabs64,
                            const double *maxabs64, const double *minabsnz64, double *o_v64, double *o_mean64,
                            double *o_rmean64, double *o_min64, double *o_max64, double *o_minabs64,
                            double *o_maxabs64, double *o_minabsnz64) {
  const int64_t f = blockIdx.x;
  if (f >= nk) return;
  const int64_t p = keep[f];
  for (int64_t s = threadIdx.x; s < ld; s += blockDim.x) o_v64[f * ld + s] = v64[p * ld + s];
  if (threadIdx.x == 0) {
    o_mean64[f] = mean64[p];
    o_rmean64[f] = rmean64[p];
    o_min64[f] = min64[p];
    o_max64[f] = max64[p];
    o_minabs64[f] = minabs64[p];
    o_maxabs64[f] = maxabs64[p];
    o_minabsnz64[f] = minabsnz64[p];
  }
}

// FP32 rows and per-feature helpers: one block of kPrepThreads per feature
// (row conversion and the FP64 sum of squares for the norm bound over the
// block's threads: the conversions run on the FP64 pipe, and four warps per
// feature keep enough of them in flight), the feature's helpers by thread 0.
constexpr int kPrepThreads = 128;

__global__ void __launch_bounds__(kPrepThreads)
    k_fp32_prep(int64_t n, int64_t N, int64_t ld, int D, const double *v64, float *v32, float *v32lo,
                const double *mean64, const double *rmean64, const double *min64, const double *max64,
                const double *minabs64, const double *maxabs64, const double *minabsnz64, const int32_t *units,
                double exp_arg_max, float4 *fa, float2 *fr, uint32_t *flags, uint64_t *ukey, float *fnorm) {
  __shared__ double red[kPrepThreads / 32];
  const int lane = threadIdx.x & 31;
  for (int64_t f = blockIdx.x; f < n; f += gridDim.x) {
    double s2 = 0.0;
    for (int64_t s = threadIdx.x; s < ld; s += kPrepThreads) {
      const double v = s < N ? v64[f * ld + s] : 0.0;
      const float h = __double2float_rn(v);
      v32[f * ld + s] = h;
      v32lo[f * ld + s] = __double2float_rn(__dsub_rn(v, (double)h));
      s2 = __fma_rn(v, v, s2);
    }
    s2 = warp_sum64(s2);
    if (lane == 0) red[threadIdx.x >> 5] = s2;
    __syncthreads();
    if (threadIdx.x == 0) {
      s2 = 0.0;
      for (int w = 0; w < kPrepThreads / 32; ++w) s2 += red[w];
      double M = maxabs64[f], m = minabs64[f];
      fa[f] = make_float4(__double2float_rn(mean64[f]), __double2float_rn(rmean64[f]), __double2float_ru(M),
                          __double2float_rd(M));
      if (m > 0.0)
        fr[f] = make_float2(__double2float_ru(__ddiv_ru(1.0, m)), __double2float_rd(__ddiv_rd(1.0, m)));
      else
        fr[f] = make_float2(0.0f, 0.0f);
      uint32_t fl = 0;
      if (m > 0.0) fl |= F_MINABS_POS;
      if (min64[f] > 0.0) fl |= F_MIN_POS;
      if (min64[f] >= 0.0) fl |= F_MIN_NONNEG;
      if (max64[f] <= 80.0) fl |= F_EXP_DOMAIN;
      if (max64[f] <= exp_arg_max) fl |= F_EXP_MAG;
      const double lo = 8.673617379884035e-19, hi = 1.152921504606847e18;  // 2^-60, 2^60
      double nz = minabsnz64[f];
      if (M <= hi && (!(nz < INFINITY) || nz >= lo)) fl |= F_FP32_SAFE;
      uint64_t k0 = 0, k1 = 0;
      int dimless = 1;
      for (int d = 0; d < kMaxDims; ++d) {
        int32_t x = d < D ? units[f * kMaxDims + d] : 0;
        if (x) dimless = 0;
        uint64_t bits = (uint64_t)(uint16_t)(int16_t)x;
        if (d < 4) k0 |= bits << (16 * d);
        else k1 |= bits << (16 * (d - 4));
      }
      if (dimless) fl |= F_DIMLESS;
      flags[f] = fl;
      ukey[2 * f] = k0;
      ukey[2 * f + 1] = k1;
      // sum of non-negative terms: each thread's running sum of about N/128
      // FMAs, a 5-level tree, then 4 partials: relative error below
      // (N/128 + 10) u, inside the margin taken
      const double margin = 1.0 + ((double)(N / 32) + 8.0) * 2.3e-16;
      fnorm[f] = __double2float_ru(__dsqrt_ru(__dmul_ru(s2, margin)));
    }
    __syncthreads();  // red is reused by the next feature
  }
}

// ------------------------------------------------------------- host side

static unsigned grid_for(uint64_t work, int threads, unsigned cap = 65535u * 16) {
  uint64_t b = (work + threads - 1) / threads;
  if (b < 1) b = 1;
  if (b > cap) b = cap;
  return (unsigned)b;
}

struct TableArrays {
  double *v64 = nullptr, *mean64 = nullptr, *rmean64 = nullptr, *min64 = nullptr, *max64 = nullptr,
         *minabs64 = nullptr, *maxabs64 = nullptr, *minabsnz64 = nullptr;
  int32_t *op = nullptr, *cplx = nullptr, *units = nullptr;
  int64_t *ca = nullptr, *cb = nullptr;
  uint64_t *used = nullptr, *dmask = nullptr;  // only with user rules
  int64_t cap = 0;
  void release() {
    dfree(v64); dfree(mean64); dfree(rmean64); dfree(min64); dfree(max64); dfree(minabs64); dfree(maxabs64);
    dfree(minabsnz64); dfree(op); dfree(cplx); dfree(units); dfree(ca); dfree(cb); dfree(used); dfree(dmask);
    *this = TableArrays();
  }
};

static dse_status table_alloc(TableArrays &t, int64_t cap, int64_t ld, bool rules) {
  t.cap = cap;
  DSE_TRY(dalloc(&t.v64, (size_t)cap * ld, "FP64 feature rows"));
  DSE_TRY(dalloc(&t.mean64, cap, "summaries"));
  DSE_TRY(dalloc(&t.rmean64, cap, "summaries"));
  DSE_TRY(dalloc(&t.min64, cap, "summaries"));
  DSE_TRY(dalloc(&t.max64, cap, "summaries"));
  DSE_TRY(dalloc(&t.minabs64, cap, "summaries"));
  DSE_TRY(dalloc(&t.maxabs64, cap, "summaries"));
  DSE_TRY(dalloc(&t.minabsnz64, cap, "summaries"));
  DSE_TRY(dalloc(&t.op, cap, "table"));
  DSE_TRY(dalloc(&t.cplx, cap, "table"));
  DSE_TRY(dalloc(&t.units, (size_t)cap * kMaxDims, "table"));
  DSE_TRY(dalloc(&t.ca, cap, "table"));
  DSE_TRY(dalloc(&t.cb, cap, "table"));
  if (rules) {
    DSE_TRY(dalloc(&t.used, cap, "rule masks"));
    DSE_TRY(dalloc(&t.dmask, cap, "rule masks"));
  }
  return DSE_OK;
}

// The features ordered by unit key (two 64-bit words, high word first), ties
// by id (the host's stable sort of the same keys gives the same order), as
// row ids: row f goes to position rank(f) = #{g : key_g < key_f, or equal
// keys and g < f}; one_class: the identity.  rowid_ident gets 0..n-1.
// One warp per feature, lanes over the keys (staged in shared memory when
// they fit: 16 n bytes for n <= kClassStage).
constexpr int64_t kClassStage = 2048;

__global__ void k_class_rows(const uint64_t *ukey, int64_t n, int one_class, int32_t *class_rows,
                             int32_t *rowid_ident) {
  extern __shared__ uint64_t sk[];
  const bool staged = n <= kClassStage;
  if (staged && !one_class) {
    for (int64_t i = threadIdx.x; i < 2 * n; i += blockDim.x) sk[i] = ukey[i];
    __syncthreads();
  }
  const uint64_t *K = staged ? sk : ukey;
  const int lane = threadIdx.x & 31;
  const int64_t f = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  if (f >= n) return;
  if (lane == 0) rowid_ident[f] = (int32_t)f;
  if (one_class) {
    if (lane == 0) class_rows[f] = (int32_t)f;
    return;
  }
  const uint64_t k1 = K[2 * f + 1], k0 = K[2 * f];
  unsigned rank = 0;
  for (int64_t g = lane; g < n; g += 32) {
    const uint64_t g1 = K[2 * g + 1], g0 = K[2 * g];
    rank += (g1 < k1 || (g1 == k1 && (g0 < k0 || (g0 == k0 && g < f)))) ? 1u : 0u;
  }
  for (int o = 16; o > 0; o >>= 1) rank += __shfl_xor_sync(0xffffffffu, rank, o);
  if (lane == 0) class_rows[rank] = (int32_t)f;
}

// Up to 16 device-to-device copies in one launch (blockIdx.y: the copy;
// 4-byte words: every table array holds 4- or 8-byte elements).
struct CopySegs {
  uint32_t *dst[16];
  const uint32_t *src[16];
  uint64_t words[16];
  int n;
};

__global__ void k_copy_segments(const CopySegs c) {
  const int k = blockIdx.y;
  if (k >= c.n) return;
  for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < c.words[k];
       i += (uint64_t)gridDim.x * blockDim.x)
    c.dst[k][i] = c.src[k][i];
}

static dse_status table_copy(TableArrays &dst, const TableArrays &src, int64_t n, int64_t ld, cudaStream_t s) {
  if (n == 0) return DSE_OK;
  CopySegs c{};
  auto add = [&](void *d, const void *x, size_t bytes) {
    if (!d || !x) return;
    c.dst[c.n] = static_cast<uint32_t *>(d);
    c.src[c.n] = static_cast<const uint32_t *>(x);
    c.words[c.n] = bytes / 4;
    ++c.n;
  };
  add(dst.v64, src.v64, sizeof(double) * n * ld);
  add(dst.mean64, src.mean64, 8 * n);
  add(dst.rmean64, src.rmean64, 8 * n);
  add(dst.min64, src.min64, 8 * n);
  add(dst.max64, src.max64, 8 * n);
  add(dst.minabs64, src.minabs64, 8 * n);
  add(dst.maxabs64, src.maxabs64, 8 * n);
  add(dst.minabsnz64, src.minabsnz64, 8 * n);
  add(dst.op, src.op, 4 * n);
  add(dst.cplx, src.cplx, 4 * n);
  add(dst.units, src.units, 4 * n * kMaxDims);
  add(dst.ca, src.ca, 8 * n);
  add(dst.cb, src.cb, 8 * n);
  add(dst.used, src.used, 8 * n);
  add(dst.dmask, src.dmask, 8 * n);
  const uint64_t big = (uint64_t)2 * n * ld;  // the rows are the longest copy
  note_launches(1);
  k_copy_segments<<<dim3((unsigned)std::min<uint64_t>(1024, (big + 255) / 256), (unsigned)c.n), 256, 0, s>>>(c);
  DSE_CUDA(cudaGetLastError());
  return DSE_OK;
}

static FeatTable view(const TableArrays &t, int64_t n, int64_t N, int64_t ld, const uint64_t *op_deny) {
  FeatTable F{};
  if (t.used) {
    F.used = t.used;
    F.dmask = t.dmask;
    F.op_deny = op_deny;
  }
  F.n = n;
  F.N = N;
  F.ld = ld;
  F.v64 = t.v64;
  F.mean64 = t.mean64;
  F.rmean64 = t.rmean64;
  F.min64 = t.min64;
  F.max64 = t.max64;
  F.minabs64 = t.minabs64;
  F.maxabs64 = t.maxabs64;
  F.cplx = t.cplx;
  F.op = t.op;
  F.ca = t.ca;
  F.cb = t.cb;
  F.units = t.units;
  return F;
}

RungGeom make_geom(const dse_space *S, int r) {
  RungGeom g{};
  g.o = S->rung_begin[r - 1];
  g.n = S->rung_begin[r];
  g.nu = g.nb = 0;
  for (int c = 0; c <= 5; ++c)
    if (S->op_mask & (1u << c)) g.uops[g.nu++] = c;
  for (int c = 6; c <= 11; ++c)
    if (S->op_mask & (1u << c)) g.bops[g.nb++] = c;
  uint64_t m = (uint64_t)(g.n - g.o), o = (uint64_t)g.o;
  g.um = (uint64_t)g.nu * m;
  uint64_t pairs = m ? tri(m) + m * o : 0;
  g.slots = g.um + (uint64_t)g.nb * pairs;
  g.tri_o = o ? tri(o) : 0;
  return g;
}

dse_status space_release(dse_space *S);

static dse_status build_impl(const dse_space_desc *d, dse_space *S) {
  cudaStream_t st = (cudaStream_t)d->stream;
  const int64_t N = d->n_samples, n0 = d->n_primary;
  const int64_t ld = (N + 3) / 4 * 4;
  S->N = N;
  S->ld = ld;
  S->n_primary = n0;
  S->D = d->n_dims;
  S->max_rung = d->max_rung;
  S->op_mask = d->op_mask;
  S->max_complexity = d->max_complexity;
  S->unit_check_addsub = d->unit_check_addsub;
  S->explog_dimensionless = d->explog_dimensionless;
  S->fmax_max = d->fmax_max;
  S->fmin_std_rel = d->fmin_std_rel;
  S->exp_arg_max = log(d->fmax_max);
  DSE_CUDA(cudaGetDevice(&S->device));

  // user rules: the symmetric pair relation by primary, the op rows on the
  // device (the space keeps them for the screens)
  const bool rules = d->pair_deny || d->op_deny;
  std::vector<uint64_t> deny_sym(rules ? n0 : 0, 0ull);
  if (rules) {
    for (int64_t p = 0; p < n0; ++p)
      for (int64_t q = 0; q < n0; ++q)
        if (d->pair_deny && (((d->pair_deny[p] >> q) & 1ull) || ((d->pair_deny[q] >> p) & 1ull)))
          deny_sym[p] |= 1ull << q;
    uint64_t od[12];
    for (int o = 0; o < 12; ++o) od[o] = d->op_deny ? d->op_deny[o] : 0ull;
    DSE_TRY(dalloc(&S->op_deny, 12, "op rules"));
    DSE_CUDA(cudaMemcpyAsync(S->op_deny, od, sizeof(od), cudaMemcpyHostToDevice, st));
  }

  AprioriParams P{S->D, S->unit_check_addsub, S->explog_dimensionless, S->max_complexity, S->fmax_max,
                  S->exp_arg_max};

  // --- rung 0: gather the primaries on the device
  int64_t ldx = d->ld_x;
  const double *Xd = d->X;
  double *Xtmp = nullptr;
  int64_t *idx_d = nullptr;
  if (!d->x_on_device) {
    DSE_TRY(dalloc(&Xtmp, (size_t)n0 * ldx, "primary upload"));
    DSE_CUDA(cudaMemcpyAsync(Xtmp, d->X, sizeof(double) * n0 * ldx, cudaMemcpyHostToDevice, st));
    Xd = Xtmp;
  }
  if (d->sample_idx) {
    DSE_TRY(dalloc(&idx_d, N, "sample gather list"));
    DSE_CUDA(cudaMemcpyAsync(idx_d, d->sample_idx, sizeof(int64_t) * N, cudaMemcpyHostToDevice, st));
  }
  TableArrays T0;
  DSE_TRY(table_alloc(T0, n0, ld, false));
  k_gather_rows<<<grid_for(n0 * ld, 256), 256, 0, st>>>(Xd, ldx, idx_d, n0, N, ld, T0.v64);
  uint8_t *ok = nullptr;
  DSE_TRY(dalloc(&ok, n0, "primary flags"));
  k_summaries<<<(unsigned)n0, kSumThreads, 0, st>>>(T0.v64, ld, N, 0, n0, T0.mean64, T0.rmean64, T0.min64,
                                                       T0.max64, T0.minabs64, T0.maxabs64, T0.minabsnz64,
                                                       S->fmin_std_rel, ok, nullptr);
  std::vector<uint8_t> hok(n0);
  DSE_CUDA(cudaMemcpyAsync(hok.data(), ok, n0, cudaMemcpyDeviceToHost, st));
  DSE_CUDA(cudaStreamSynchronize(st));
  dfree(ok);
  dfree(Xtmp);
  dfree(idx_d);

  // keep the primaries that pass the realised test, in input order
  std::vector<int64_t> keep;
  for (int64_t p = 0; p < n0; ++p)
    if (hok[p]) keep.push_back(p);
  const int64_t nk = (int64_t)keep.size();
  S->slots[0] = (uint64_t)n0;
  memset(S->reasons, 0, sizeof(S->reasons));
  S->reasons[0][DSE_VALID] = nk;
  S->reasons[0][DSE_R_REALISED] = n0 - nk;
  S->have_counts[0] = true;
  if (nk == 0) {
    T0.release();
    set_error("no primary feature passes the realised test");
    return DSE_EINVAL;
  }
  TableArrays T;
  DSE_TRY(table_alloc(T, nk, ld, rules));
  {
    // host-assembled metadata of rung 0, rows copied device to device
    std::vector<int32_t> hop(nk, DSE_OP_PRIMARY), hcx(nk, 0), hun((size_t)nk * kMaxDims, 0);
    std::vector<int64_t> hca(nk), hcb(nk, -1);
    std::vector<uint64_t> hused(rules ? nk : 0), hdmask(rules ? nk : 0);
    const int64_t scale = (int64_t)1 << d->max_rung;
    for (int64_t f = 0; f < nk; ++f) {
      int64_t p = keep[f];
      hca[f] = p;
      if (rules) {
        hused[f] = 1ull << p;
        hdmask[f] = deny_sym[p];
      }
      for (int k = 0; k < S->D; ++k) {
        int64_t u = (int64_t)d->units[p * S->D + k] * scale;
        if (u > 32767 || u < -32767) {
          T0.release();
          T.release();
          set_error("unit exponent of primary %lld out of range", (long long)p);
          return DSE_EOVERFLOW;
        }
        hun[f * kMaxDims + k] = (int32_t)u;
      }
    }
    // the uploads go through the thread's pinned staging area (a copy from
    // pageable memory would synchronise the stream first); its next users
    // in this build write it only after a stream synchronisation, and the
    // device reads it in stream order before anything later lands there
    auto r256 = [](size_t b) { return (b + 255) / 256 * 256; };
    const size_t tot = r256(8 * nk) + 2 * r256(4 * nk) + r256((size_t)4 * nk * kMaxDims) + 2 * r256(8 * nk) +
                       (rules ? 2 * r256(8 * nk) : 0);
    char *hst = static_cast<char *>(pinned_staging(tot));
    if (!hst) return DSE_ENOMEM;
    int64_t *keep_d = nullptr;
    DSE_TRY(dalloc(&keep_d, nk, "kept primaries"));
    size_t off = 0;
    auto up = [&](void *dst, const void *src, size_t bytes) -> cudaError_t {
      if (!bytes) return cudaSuccess;
      memcpy(hst + off, src, bytes);
      const cudaError_t e = cudaMemcpyAsync(dst, hst + off, bytes, cudaMemcpyHostToDevice, st);
      off += r256(bytes);
      return e;
    };
    DSE_CUDA(up(keep_d, keep.data(), 8 * nk));
    note_launches(1);
    k_take_rows<<<(unsigned)nk, 128, 0, st>>>(keep_d, nk, ld, T0.v64, T0.mean64, T0.rmean64, T0.min64, T0.max64,
                                              T0.minabs64, T0.maxabs64, T0.minabsnz64, T.v64, T.mean64, T.rmean64,
                                              T.min64, T.max64, T.minabs64, T.maxabs64, T.minabsnz64);
    dfree(keep_d);
    DSE_CUDA(up(T.op, hop.data(), 4 * nk));
    DSE_CUDA(up(T.cplx, hcx.data(), 4 * nk));
    DSE_CUDA(up(T.units, hun.data(), (size_t)4 * nk * kMaxDims));
    DSE_CUDA(up(T.ca, hca.data(), 8 * nk));
    DSE_CUDA(up(T.cb, hcb.data(), 8 * nk));
    if (rules) {
      DSE_CUDA(up(T.used, hused.data(), 8 * nk));
      DSE_CUDA(up(T.dmask, hdmask.data(), 8 * nk));
    }
    T0.release();
  }
  int64_t n = nk;
  S->rung_begin[0] = 0;
  S->rung_begin[1] = n;
  S->h_rung.assign(n, 0);

  // per-rung counters on the device: 6 reason counts, a-priori valid count,
  // realised count, error flag -- read back with one copy and one sync
  unsigned long long *meta = nullptr;
  DSE_TRY(dalloc(&meta, 10, "rung counters"));
  unsigned long long *hmeta = static_cast<unsigned long long *>(pinned_staging(10 * sizeof(unsigned long long)));
  if (!hmeta) {
    dfree(meta);
    T.release();
    return DSE_ENOMEM;
  }

  // --- rungs 1 .. max_rung-1
  for (int r = 1; r < d->max_rung; ++r) {
    RungGeom g = make_geom(S, r);
    FeatTable F = view(T, n, N, ld, S->op_deny);
    S->slots[r] = g.slots;
    uint8_t *why = nullptr, *rw = nullptr;
    uint64_t *list = nullptr, *vlist = nullptr;
    // capacities: every slot (the counts are known only on the device)
    DSE_TRY(dalloc(&why, g.slots, "slot reasons"));
    DSE_TRY(dalloc(&list, g.slots, "a-priori list"));
    DSE_TRY(dalloc(&rw, g.slots, "realised flags"));
    DSE_TRY(dalloc(&vlist, g.slots, "valid list"));
    DSE_CUDA(cudaMemsetAsync(meta, 0, 10 * sizeof(unsigned long long), st));
    note_launches(1);
    if (g.slots) k_apriori_rung<<<grid_for(g.slots, 256), 256, 0, st>>>(F, g, P, why, (int *)(meta + 8));
    launch_count_reasons(why, g.slots, meta, st);
    DSE_TRY(compact_bytes_dev(why, g.slots, DSE_VALID, list, meta + 6, st));
    dfree(why);
    // every a-priori valid slot evaluated once into scratch rows and
    // summarised there (the summary carries the realised test); the kept
    // rows are then copied into the grown table.  The scratch has a row per
    // slot unless that passes 4 GiB, in which case the a-priori count is
    // read first.
    uint64_t cap_rows = g.slots;
    if ((double)g.slots * (double)ld * 8.0 > 4.0 * (double)(1ull << 30)) {
      DSE_CUDA(cudaMemcpyAsync(hmeta, meta + 6, sizeof(unsigned long long), cudaMemcpyDeviceToHost, st));
      DSE_CUDA(cudaStreamSynchronize(st));
      cap_rows = hmeta[0];
    }
    double *rows = nullptr;
    RowSummaries rsum{};
    DSE_TRY(dalloc(&rows, (size_t)std::max<uint64_t>(cap_rows, 1) * ld, "rung scratch rows"));
    double **rs_arr[7] = {&rsum.mean64, &rsum.rmean64, &rsum.min64, &rsum.max64, &rsum.minabs64, &rsum.maxabs64,
                          &rsum.minabsnz64};
    for (double **q : rs_arr) DSE_TRY(dalloc(q, std::max<uint64_t>(cap_rows, 1), "rung scratch summaries"));
    DSE_CUDA(cudaMemsetAsync(rw, 0, g.slots, st));
    note_launches(2);
    if (cap_rows) {
      k_eval_rows<<<(unsigned)cap_rows, kSumThreads, 0, st>>>(F, g, list, cap_rows, meta + 6, rows);
      k_summaries<<<(unsigned)cap_rows, kSumThreads, 0, st>>>(rows, ld, N, 0, (int64_t)cap_rows, rsum.mean64,
                                                             rsum.rmean64, rsum.min64, rsum.max64, rsum.minabs64,
                                                             rsum.maxabs64, rsum.minabsnz64, S->fmin_std_rel, rw,
                                                             meta + 6);
    }
    DSE_TRY(compact_bytes_dev(rw, cap_rows, 1, vlist, meta + 7, st));
    dfree(rw);
    DSE_CUDA(cudaMemcpyAsync(hmeta, meta, 10 * sizeof(unsigned long long), cudaMemcpyDeviceToHost, st));
    DSE_CUDA(cudaStreamSynchronize(st));
    const int hbad = (int)(hmeta[8] & 0xFFFFFFFFull);
    auto drop_scratch = [&]() {
      dfree(rows);
      for (double **q : rs_arr) dfree(*q);
      dfree(list);
      dfree(vlist);
    };
    if (hbad) {
      drop_scratch();
      dfree(meta);
      T.release();
      set_error(hbad == 1 ? "odd unit exponent under sqrt" : "unit exponent out of range");
      return DSE_EOVERFLOW;
    }
    const uint64_t n_ap = hmeta[6], n_new = hmeta[7];
    for (int c = 0; c < 6; ++c) S->reasons[r][c] = (int64_t)hmeta[c];
    S->reasons[r][DSE_VALID] = (int64_t)n_new;
    S->reasons[r][DSE_R_REALISED] = (int64_t)(n_ap - n_new);
    S->have_counts[r] = true;
    // grow the table and append
    TableArrays T2;
    dse_status s2 = table_alloc(T2, n + (int64_t)n_new, ld, rules);
    if (s2 != DSE_OK) {
      drop_scratch();
      dfree(meta);
      T.release();
      return s2;
    }
    DSE_TRY(table_copy(T2, T, n, ld, st));
    FeatTable Fold = view(T, n, N, ld, S->op_deny);
    RowSummaries dsum{T2.mean64, T2.rmean64, T2.min64, T2.max64, T2.minabs64, T2.maxabs64, T2.minabsnz64};
    note_launches(1);
    if (n_new)
      k_take_eval<<<(unsigned)n_new, kSumThreads, 0, st>>>(Fold, g, P, list, vlist, n_new, n, rows, rsum, T2.v64, dsum,
                                                           T2.op, T2.ca, T2.cb, T2.cplx, T2.units, T2.used, T2.dmask);
    drop_scratch();
    // stream-ordered frees: the old table and the scratch stay valid for
    // the kernels above
    T.release();
    T = T2;
    n += (int64_t)n_new;
    S->rung_begin[r + 1] = n;
    S->h_rung.resize(n, r);
  }
  dfree(meta);

  // --- FP32 rows and helpers
  S->n = n;
  S->v64 = T.v64;
  S->mean64 = T.mean64;
  S->rmean64 = T.rmean64;
  S->min64 = T.min64;
  S->max64 = T.max64;
  S->minabs64 = T.minabs64;
  S->maxabs64 = T.maxabs64;
  S->op = T.op;
  S->cplx = T.cplx;
  S->units = T.units;
  S->ca = T.ca;
  S->cb = T.cb;
  S->used = T.used;
  S->dmask = T.dmask;
  DSE_TRY(dalloc(&S->v32, (size_t)n * ld, "FP32 feature rows"));
  DSE_TRY(dalloc(&S->v32lo, (size_t)n * ld, "FP32 remainder rows"));
  DSE_TRY(dalloc(&S->fa, n, "helpers"));
  DSE_TRY(dalloc(&S->fr, n, "helpers"));
  DSE_TRY(dalloc(&S->fnorm, n, "helpers"));
  DSE_TRY(dalloc(&S->flags, n, "flags"));
  DSE_TRY(dalloc(&S->ukey, 2 * n, "unit keys"));
  k_fp32_prep<<<(unsigned)std::min<int64_t>(std::max<int64_t>(n, 1), 65535), kPrepThreads, 0, st>>>(n, N, ld, S->D, T.v64, S->v32, S->v32lo, T.mean64, T.rmean64, T.min64,
                                                     T.max64, T.minabs64, T.maxabs64, T.minabsnz64, T.units,
                                                     S->exp_arg_max, S->fa, S->fr, S->flags, S->ukey, S->fnorm);
  dfree(T.minabsnz64);

  // --- host copies for decoding and the unit classes
  S->h_op.resize(n);
  S->h_cplx.resize(n);
  S->h_ca.resize(n);
  S->h_cb.resize(n);
  S->h_ukey.resize(2 * n);
  {
    // one pinned staging area, five asynchronous copies, one sync
    char *hs = static_cast<char *>(pinned_staging((size_t)40 * n));
    if (!hs) return DSE_ENOMEM;
    DSE_CUDA(cudaMemcpyAsync(hs, S->op, 4 * n, cudaMemcpyDeviceToHost, st));
    DSE_CUDA(cudaMemcpyAsync(hs + 4 * n, S->cplx, 4 * n, cudaMemcpyDeviceToHost, st));
    DSE_CUDA(cudaMemcpyAsync(hs + 8 * n, S->ca, 8 * n, cudaMemcpyDeviceToHost, st));
    DSE_CUDA(cudaMemcpyAsync(hs + 16 * n, S->cb, 8 * n, cudaMemcpyDeviceToHost, st));
    DSE_CUDA(cudaMemcpyAsync(hs + 24 * n, S->ukey, 16 * n, cudaMemcpyDeviceToHost, st));
    DSE_CUDA(cudaStreamSynchronize(st));
    memcpy(S->h_op.data(), hs, 4 * n);
    memcpy(S->h_cplx.data(), hs + 4 * n, 4 * n);
    memcpy(S->h_ca.data(), hs + 8 * n, 8 * n);
    memcpy(S->h_cb.data(), hs + 16 * n, 8 * n);
    memcpy(S->h_ukey.data(), hs + 24 * n, 16 * n);
  }

  std::vector<int32_t> rows(n);
  std::iota(rows.begin(), rows.end(), 0);
  const bool one_class = !S->unit_check_addsub || S->D == 0;
  if (!one_class)
    std::stable_sort(rows.begin(), rows.end(), [&](int32_t x, int32_t y) {
      if (S->h_ukey[2 * x + 1] != S->h_ukey[2 * y + 1]) return S->h_ukey[2 * x + 1] < S->h_ukey[2 * y + 1];
      return S->h_ukey[2 * x] < S->h_ukey[2 * y];
    });
  S->h_class_rows = rows;
  S->h_class_begin.clear();
  for (int64_t f = 0; f < n; ++f)
    if (f == 0 || (!one_class && (S->h_ukey[2 * rows[f]] != S->h_ukey[2 * rows[f - 1]] ||
                                  S->h_ukey[2 * rows[f] + 1] != S->h_ukey[2 * rows[f - 1] + 1])))
      S->h_class_begin.push_back(f);
  S->h_class_begin.push_back(n);
  DSE_TRY(dalloc(&S->class_rows, n, "class rows"));
  DSE_TRY(dalloc(&S->rowid_ident, n, "row ids"));
  if (n <= 8192) {
    // the same order computed on the device (an upload from pageable memory
    // would synchronise the stream; the rank count is O(n^2))
    note_launches(1);
    const size_t shm = n <= kClassStage && !one_class ? (size_t)16 * n : 0;
    k_class_rows<<<(unsigned)((n + 7) / 8), 256, shm, st>>>(S->ukey, n, one_class ? 1 : 0, S->class_rows,
                                                           S->rowid_ident);
  } else {
    std::vector<int32_t> ident(n);
    std::iota(ident.begin(), ident.end(), 0);
    DSE_CUDA(cudaMemcpyAsync(S->class_rows, rows.data(), 4 * n, cudaMemcpyHostToDevice, st));
    DSE_CUDA(cudaMemcpyAsync(S->rowid_ident, ident.data(), 4 * n, cudaMemcpyHostToDevice, st));
  }

  S->geom = make_geom(S, d->max_rung);
  S->slots[d->max_rung] = S->geom.slots;
  return DSE_OK;
}

dse_status build_space(const dse_space_desc *d, dse_space **out) {
  dse_space *S = new (std::nothrow) dse_space();
  if (!S) {
    set_error("out of host memory");
    return DSE_ENOMEM;
  }
  for (int r = 0; r <= kMaxRung; ++r) S->have_counts[r] = false;
  dse_status s = build_impl(d, S);
  if (s != DSE_OK) {
    space_release(S);
    return s;
  }
  *out = S;
  return DSE_OK;
}

dse_status space_release(dse_space *S) {
  if (!S) return DSE_OK;
  dfree(S->v64); dfree(S->v32); dfree(S->v32lo); dfree(S->mean64); dfree(S->rmean64); dfree(S->min64); dfree(S->max64);
  dfree(S->minabs64); dfree(S->maxabs64); dfree(S->fa); dfree(S->fr); dfree(S->fnorm); dfree(S->flags); dfree(S->cplx);
  dfree(S->op); dfree(S->units); dfree(S->ca); dfree(S->cb); dfree(S->ukey); dfree(S->rowid_ident);
  dfree(S->used); dfree(S->dmask); dfree(S->op_deny); dfree(S->gram_buf); dfree(S->gmt_buf); dfree(S->v32_class); dfree(S->rcp32);
  dfree(S->class_rows);
  dfree(S->eq_pairs);
  delete S;
  return DSE_OK;
}

FeatTable table_of(const dse_space *S) {
  FeatTable F{};
  F.n = S->n;
  F.N = S->N;
  F.ld = S->ld;
  F.v64 = S->v64;
  F.v32 = S->v32;
  F.v32lo = S->v32lo;
  F.mean64 = S->mean64;
  F.rmean64 = S->rmean64;
  F.min64 = S->min64;
  F.max64 = S->max64;
  F.minabs64 = S->minabs64;
  F.maxabs64 = S->maxabs64;
  F.fa = S->fa;
  F.fr = S->fr;
  F.flags = S->flags;
  F.cplx = S->cplx;
  F.op = S->op;
  F.ca = S->ca;
  F.cb = S->cb;
  F.units = S->units;
  F.ukey = S->ukey;
  F.fnorm = S->fnorm;
  if (S->used) {
    F.used = S->used;
    F.dmask = S->dmask;
    F.op_deny = S->op_deny;
  }
  return F;
}

// A-priori reason counts of rung max_rung (no evaluation).
__global__ void k_count_apriori(FeatTable F, RungGeom g, AprioriParams P, unsigned long long *counts) {
  __shared__ unsigned int c[6];
  if (threadIdx.x < 6) c[threadIdx.x] = 0;
  __syncthreads();
  for (uint64_t p = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; p < g.slots;
       p += (uint64_t)gridDim.x * blockDim.x) {
    int op;
    int64_t a, b;
    decode_flat(g, p, &op, &a, &b);
    int32_t u[kMaxDims], cx;
    int bad = 0;
    atomicAdd(&c[apriori64(F, P, op, a, b, u, &cx, &bad)], 1u);
  }
  __syncthreads();
  if (threadIdx.x < 6 && c[threadIdx.x]) atomicAdd(&counts[threadIdx.x], (unsigned long long)c[threadIdx.x]);
}

dse_status count_last_rung(dse_space *S, cudaStream_t st) {
  int r = S->max_rung;
  if (S->have_counts[r]) return DSE_OK;
  unsigned long long *cnt = nullptr;
  DSE_TRY(dalloc(&cnt, 6, "counts"));
  DSE_CUDA(cudaMemsetAsync(cnt, 0, 6 * sizeof(unsigned long long), st));
  AprioriParams P{S->D, S->unit_check_addsub, S->explog_dimensionless, S->max_complexity, S->fmax_max,
                  S->exp_arg_max};
  if (S->geom.slots) k_count_apriori<<<grid_for(S->geom.slots, 256, 152 * 32), 256, 0, st>>>(table_of(S), S->geom, P, cnt);
  unsigned long long hc[6];
  DSE_CUDA(cudaMemcpyAsync(hc, cnt, sizeof(hc), cudaMemcpyDeviceToHost, st));
  DSE_CUDA(cudaStreamSynchronize(st));
  dfree(cnt);
  for (int c = 0; c < 6; ++c) S->reasons[r][c] = (int64_t)hc[c];
  S->reasons[r][DSE_R_REALISED] = -1;
  S->have_counts[r] = true;
  return DSE_OK;
}

}  // namespace dse
