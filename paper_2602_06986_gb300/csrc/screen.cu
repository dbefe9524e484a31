// screen.cu -- the SIS screening kernels (CUDA cores, FP32 with error bounds or
// plain FP64).
//
// The screened set is Phi_k = the stored features (rungs < k) plus rung k,
// which is generated on the fly and never written to memory ("Software
// Description": candidates generated from features and operators, evaluated
// against the target; "Physics-Informed Constraints": dimensionally invalid
// ones excluded).  Three kernels cover it:
//   k_feature  one warp per candidate, lanes over samples, warp-shuffle
//              reduction: the stored features themselves and the unary block
//              of rung k;
//   k_pair     the binary block of rung k: a CTA owns a tile of 16*MI x 16*MJ
//              operand rows, streams their samples through shared memory in
//              chunks with 1-D bulk async copies (double-buffered on
//              mbarriers), and every lane owns MI x MJ pairs (all three slots
//              of its kind) for the whole sample range, so no cross-lane
//              reduction is needed;  KIND_MUL covers a*b, a/b, b/a over every
//              pair, KIND_ADD covers a+b, a-b, |a-b| over pairs of equal
//              units only (tiles built per unit class);
//   k_escalate FP64 evaluation of candidates whose FP32 realised test could
//              not be decided, or whose operands are outside the FP32-safe
//              range.
// Candidates whose score interval reaches a list's threshold are appended to
// that list's buffer; the threshold rises monotonically from a histogram of
// the buffered lower bounds (the k-th best lower bound is never below it).
#include <math.h>

#include "dse_internal.cuh"
#include "eval64.cuh"
#include "screen_common.cuh"
#include "screen_kernels.cuh"
#include "util.cuh"

namespace dse {

constexpr uint32_t kWaitLimit = 1u << 22;

// ----------------------------------------------------------- target prep

// Centre and normalise each target in FP64 (one block per target).
__global__ void k_targets(const double *Y, int64_t ldY, int T, int64_t N, int32_t ldy, double *y64, float *y32,
                          float *ysum32, int *err) {
  __shared__ double red[32];
  const int t = blockIdx.x;
  if (t >= T) return;
  const double *y = Y + (int64_t)t * ldY;
  auto block_sum = [&](double v) {
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
    __syncthreads();
    double tot = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) tot += red[w];
    __syncthreads();
    return tot;
  };
  double s = 0.0;
  for (int64_t i = threadIdx.x; i < N; i += blockDim.x) s += y[i];
  const double mean = block_sum(s) / (double)N;
  double q = 0.0;
  for (int64_t i = threadIdx.x; i < N; i += blockDim.x) {
    double d = y[i] - mean;
    q = fma(d, d, q);
  }
  const double syy = block_sum(q);
  if (!(syy > 0.0) || !isfinite(syy)) {
    if (threadIdx.x == 0) atomicExch(err, DSE_EINVAL);
    return;
  }
  const double inv = 1.0 / sqrt(syy);
  double fs = 0.0;
  for (int64_t i = threadIdx.x; i < ldy; i += blockDim.x) {
    double v = i < N ? (y[i] - mean) * inv : 0.0;
    float f = __double2float_rn(v);
    y64[(int64_t)t * ldy + i] = v;
    y32[(int64_t)t * ldy + i] = f;
    fs += (double)f;
  }
  fs = block_sum(fs);
  if (threadIdx.x == 0) ysum32[t] = (float)fs;
}

// ------------------------------------------------------ shared epilogue

struct LaneStats {
  unsigned r[6];
  unsigned evaluated, escalated, seen;
  __device__ void zero() {
    for (int i = 0; i < 6; ++i) r[i] = 0;
    evaluated = escalated = seen = 0;
  }
};

__device__ __forceinline__ void flush_stats(const ScreenArgs &A, LaneStats &ls) {
  if (!A.first_pass) {
    ls.zero();
    return;
  }
  {
    unsigned v = ls.seen;
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    if ((threadIdx.x & 31) == 0 && v) atomicAdd(&A.stats[ST_ADD_SEEN], (unsigned long long)v);
  }
  for (int i = 0; i < 6; ++i) {
    unsigned v = ls.r[i];
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    if ((threadIdx.x & 31) == 0 && v) atomicAdd(&A.stats[ST_REASON0 + i], (unsigned long long)v);
  }
  {
    unsigned v = ls.r[DSE_VALID];
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    if ((threadIdx.x & 31) == 0 && v) atomicAdd(&A.stats[ST_VALID_G0 + A.group], (unsigned long long)v);
  }
  unsigned e = ls.evaluated, x = ls.escalated;
  for (int o = 16; o > 0; o >>= 1) {
    e += __shfl_xor_sync(0xffffffffu, e, o);
    x += __shfl_xor_sync(0xffffffffu, x, o);
  }
  if ((threadIdx.x & 31) == 0) {
    if (e) atomicAdd(&A.stats[ST_EVALUATED], (unsigned long long)e);
    if (x) atomicAdd(&A.stats[ST_ESCALATED], (unsigned long long)x);
  }
  ls.zero();
}

__device__ __forceinline__ void escalate(const ScreenArgs &A, uint64_t gid) {
  if (!A.first_pass) return;
  unsigned pos = atomicAdd(A.esc_count, 1u);
  if ((int64_t)pos < A.esc_cap)
    A.esc_id[pos] = gid;
  else
    atomicAdd(&A.stats[ST_ESC_OVERFLOW], 1ull);
}

// Score a candidate's statistics against the pass's targets and push.
// Warp-cooperative: all lanes call with the same loop structure.
template <typename R, int NT>
__device__ __forceinline__ unsigned score_and_push(const ScreenArgs &A, bool want, uint64_t gid,
                                                   const CandInterval<R> &ci, R S1, const R *Sy, R invN, R gamma,
                                                   R u, const R *ysum) {
  unsigned pushed = 0;
  if (A.mode == DSE_MODE_AGGREGATED) {
    R a = 0, alo = 0, ahi = 0;
    for (int t = 0; t < NT; ++t) {
      if (t < A.T) {
        R s, e;
        cand_score<R>(ci, S1, Sy[t], invN, ysum[t], gamma, u, &s, &e);
        R lo = s - e > R(0) ? s - e : R(0), hi = s + e < R(1) ? s + e : R(1);
        a += s * s;
        alo += lo * lo;
        ahi += hi * hi;
      }
    }
    R invT = R(1) / R(A.T);
    R s = Num<R>::sqrt_(a * invT);
    R lo = Num<R>::sqrt_(alo * invT), hi = Num<R>::sqrt_(ahi * invT);
    R e = (s - lo > hi - s ? s - lo : hi - s) * (R(1) + R(8) * u);
    float sf = (float)s;
    float ef = (float)e + fabsf((float)(s - (R)sf)) + 1e-30f;
    ef = ef * (1.0f + 2.4e-7f);
    if (push_warp(A.B, 0, want, gid, sf, ef)) pushed |= 1u;
    if (__any_sync(0xffffffffu, pushed)) pushed = 1u;
    return pushed;
  }
  for (int t = 0; t < NT; ++t) {
    bool w = want && t < A.T;
    R s = 0, e = 1;
    if (w) cand_score<R>(ci, S1, Sy[t], invN, ysum[t], gamma, u, &s, &e);
    float sf = (float)s;
    float ef = (float)e + fabsf((float)(s - (R)sf));
    ef = ef * (1.0f + 2.4e-7f);
    if (__any_sync(0xffffffffu, w)) {
      bool p = push_warp(A.B, A.t0 + t, w, gid, sf, ef);
      if (__any_sync(0xffffffffu, p)) pushed |= 1u << t;
    }
  }
  return pushed;
}

template <int NT>
__device__ __forceinline__ void refresh_pushed(const ScreenArgs &A, unsigned pushed) {
  if (A.mode == DSE_MODE_AGGREGATED) {
    if (pushed) refresh_theta(A.B, 0, A.k);
    return;
  }
  for (int t = 0; t < NT; ++t)
    if (pushed & (1u << t)) refresh_theta(A.B, A.t0 + t, A.k);
}

// ------------------------------------------------------- feature kernel

template <typename R>
__device__ __forceinline__ R unary_eval(int op, R a, R c);
template <>
__device__ __forceinline__ float unary_eval<float>(int op, float a, float c) {
  switch (op) {
    case DSE_OP_SQUARE: return fmaf(a, a, -c);
    case DSE_OP_CUBE: return fmaf(a * a, a, -c);
    case DSE_OP_INV: return rcp_approx(a) - c;
    case DSE_OP_SQRT: return sqrtf(a) - c;
    case DSE_OP_EXP: return expf(a) - c;
    case DSE_OP_LOG: return logf(a) - c;
    default: return a - c;
  }
}
template <>
__device__ __forceinline__ double unary_eval<double>(int op, double a, double c) {
  switch (op) {
    case DSE_OP_SQUARE: return fma(a, a, -c);
    case DSE_OP_CUBE: return fma(a * a, a, -c);
    case DSE_OP_INV: return __drcp_rn(a) - c;
    case DSE_OP_SQRT: return sqrt(a) - c;
    case DSE_OP_EXP: return exp(a) - c;
    case DSE_OP_LOG: return log(a) - c;
    default: return a - c;
  }
}

// W (per-sample evaluation error / u) of a unary op on feature f with shift c.
__device__ __forceinline__ double unary_W(const FeatTable &F, int op, int64_t f, double c) {
  const double M = F.maxabs64[f], m = F.minabs64[f], ac = fabs(c);
  switch (op) {
    case DSE_OP_SQUARE: return 1.01 * (3.0 * M * M + ac);
    case DSE_OP_CUBE: return 1.01 * (5.0 * M * M * M + ac);
    case DSE_OP_INV: return 1.01 * (4.0 / m + ac);
    case DSE_OP_SQRT: return 1.01 * (2.5 * sqrt(M) + ac);
    case DSE_OP_EXP: {
      double E = exp(F.max64[f]) * 1.0000001;
      return 1.01 * ((5.0 + M) * E + ac);
    }
    case DSE_OP_LOG: {
      double L = fmax(fabs(log(F.min64[f])), fabs(log(F.max64[f])));
      return 1.01 * (3.0 * L + 1.0 + ac);
    }
    default: return 1.01 * (2.0 * M + ac);
  }
}

// Candidates: stored ids [id0, id1) then unary flat indices [p0, p1).
template <typename R, int NT>
__global__ void __launch_bounds__(256) k_feature(const ScreenArgs A, uint64_t id0, uint64_t id1, uint64_t p0,
                                                 uint64_t p1, float gamma_lane) {
  const int lane = threadIdx.x & 31;
  const uint64_t nid = id1 - id0, ncand = nid + (p1 - p0);
  const uint64_t warps = (uint64_t)gridDim.x * (blockDim.x >> 5);
  const R u = sizeof(R) == 4 ? R(5.9604644775390625e-8) : R(1.1102230246251565e-16);
  const R gamma = (R)gamma_lane;
  const R N = (R)A.N, invN = (R)A.invN, sqrtN = Num<R>::sqrt_(N);
  const R fmin = (R)A.fmin_std_rel64;
  const R *Y = sizeof(R) == 4 ? (const R *)A.y32 : (const R *)A.y64;
  R ysum[NT];
  for (int t = 0; t < NT; ++t) ysum[t] = 0;
  if (sizeof(R) == 4) {
    for (int t = 0; t < NT; ++t)
      if (t < A.T) ysum[t] = (R)A.ysum32[A.t0 + t];
  }
  LaneStats ls;
  ls.zero();
  for (uint64_t w = ((uint64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; w < ncand; w += warps) {
    int op;
    int64_t f;
    uint64_t gid;
    int reason = DSE_VALID;
    if (w < nid) {
      gid = id0 + w;
      f = (int64_t)gid;
      op = DSE_OP_PRIMARY;
    } else {
      uint64_t p = p0 + (w - nid);
      gid = (uint64_t)A.n_stored + p;
      int64_t b;
      decode_flat(A.G, p, &op, &f, &b);
      // unit (exp/log need a dimensionless operand), complexity, domain, magnitude
      if ((op == DSE_OP_EXP || op == DSE_OP_LOG) && A.explog_dimensionless && !(A.F.flags[f] & F_DIMLESS))
        reason = DSE_R_UNIT;
      else if (A.max_complexity > 0 && A.F.cplx[f] + 1 > A.max_complexity)
        reason = DSE_R_COMPLEXITY;
      else {
        double ea = (op == DSE_OP_EXP && (A.F.flags[f] & F_EXP_MAG)) ? INFINITY : -INFINITY;
        reason = domain_magnitude64(op, A.F.min64[f], A.F.max64[f], A.F.minabs64[f], A.F.maxabs64[f], 0.0, 0.0,
                                    A.fmax64, ea);
      }
    }
    if (reason != DSE_VALID) {
      if (lane == 0) ls.r[reason]++;
      continue;
    }
    if (sizeof(R) == 4 && !(A.F.flags[f] & F_FP32_SAFE)) {
      if (lane == 0) {
        escalate(A, gid);
        ls.escalated++;
      }
      continue;
    }
    const R *x = sizeof(R) == 4 ? (const R *)(A.F.v32 + f * A.F.ld) : (const R *)(A.F.v64 + f * A.F.ld);
    const R c = unary_eval<R>(op, x[0], R(0));
    const R W = (R)unary_W(A.F, op, f, (double)c);
    R S1 = 0, S2 = 0, Sy[NT];
    R o1 = 0, o2 = 0, oy[NT];
    for (int t = 0; t < NT; ++t) Sy[t] = oy[t] = 0;
    int blk = 0;
    for (int64_t s = lane; s < A.N; s += 32) {
      R v = unary_eval<R>(op, x[s], c);
      S1 += v;
      S2 = Num<R>::fma_(v, v, S2);
      for (int t = 0; t < NT; ++t)
        if (t < A.T) Sy[t] = Num<R>::fma_(v, Y[(int64_t)(A.t0 + t) * A.ldy + s], Sy[t]);
      if (sizeof(R) == 4 && ++blk == 16) {
        blk = 0;
        o1 += S1; o2 += S2; S1 = 0; S2 = 0;
        for (int t = 0; t < NT; ++t) { oy[t] += Sy[t]; Sy[t] = 0; }
      }
    }
    S1 += o1;
    S2 += o2;
    for (int t = 0; t < NT; ++t) Sy[t] += oy[t];
    for (int o = 16; o > 0; o >>= 1) {
      S1 += __shfl_xor_sync(0xffffffffu, S1, o);
      S2 += __shfl_xor_sync(0xffffffffu, S2, o);
      for (int t = 0; t < NT; ++t) Sy[t] += __shfl_xor_sync(0xffffffffu, Sy[t], o);
    }
    CandInterval<R> ci = cand_interval<R>(S1, S2, N, invN, sqrtN, c, W, gamma, u, fmin);
    if (ci.realised == 0) {
      if (lane == 0) ls.r[DSE_R_REALISED]++;
      continue;
    }
    if (ci.realised == 2) {
      if (lane == 0) {
        escalate(A, gid);
        ls.escalated++;
      }
      continue;
    }
    if (lane == 0) {
      ls.r[DSE_VALID]++;
      ls.evaluated++;
    }
    unsigned pushed = score_and_push<R, NT>(A, lane == 0, gid, ci, S1, Sy, invN, gamma, u, ysum);
    refresh_pushed<NT>(A, pushed);
  }
  flush_stats(A, ls);
}

// ----------------------------------------------------------- pair kernel

template <typename R, int KIND, int NT, int MI, int MJ>
struct PairCfg {
  static constexpr int BI = 16 * MI, BJ = 16 * MJ, ROWS = BI + BJ;
  static constexpr int CH = sizeof(R) == 4 ? 128 : 64;
  static constexpr int STR = CH + (sizeof(R) == 4 ? 4 : 2);
  static constexpr int STAGE = ROWS * STR + NT * CH;  // elements
  static constexpr size_t SMEM = 2 * (size_t)STAGE * sizeof(R) + 64;
};

template <typename R>
struct Vec2;
template <>
struct Vec2<float> {
  using T = float2;
};
template <>
struct Vec2<double> {
  using T = double2;
};

template <typename R>
__device__ __forceinline__ R rcp_of(R x);
template <>
__device__ __forceinline__ float rcp_of<float>(float x) { return rcp_approx(x); }
template <>
__device__ __forceinline__ double rcp_of<double>(double x) { return __drcp_rn(x); }

template <typename R, int KIND, int NT, int MI, int MJ>
__device__ __forceinline__ void pair_update(const R (&a)[MI], const R (&b)[MJ], const R (&y)[NT],
                                            const R (&k0)[MI][MJ], const R (&k1)[MI][MJ], const R (&k2)[MI][MJ],
                                            const R (&mi)[MI], const R (&mj)[MJ], R (&acc)[MI][MJ][3][2 + NT]) {
  if (KIND == KIND_MUL) {
    R ra[MI], rb[MJ];
#pragma unroll
    for (int r = 0; r < MI; ++r) ra[r] = rcp_of<R>(a[r]);
#pragma unroll
    for (int c = 0; c < MJ; ++c) rb[c] = rcp_of<R>(b[c]);
#pragma unroll
    for (int r = 0; r < MI; ++r)
#pragma unroll
      for (int c = 0; c < MJ; ++c) {
        R w[3];
        w[0] = Num<R>::fma_(a[r], b[c], -k0[r][c]);
        w[1] = Num<R>::fma_(a[r], rb[c], -k1[r][c]);
        w[2] = Num<R>::fma_(b[c], ra[r], -k2[r][c]);
#pragma unroll
        for (int k = 0; k < 3; ++k) {
          acc[r][c][k][0] += w[k];
          acc[r][c][k][1] = Num<R>::fma_(w[k], w[k], acc[r][c][k][1]);
#pragma unroll
          for (int t = 0; t < NT; ++t) acc[r][c][k][2 + t] = Num<R>::fma_(w[k], y[t], acc[r][c][k][2 + t]);
        }
      }
  } else {
    R ac[MI], bc[MJ];
#pragma unroll
    for (int r = 0; r < MI; ++r) ac[r] = a[r] - mi[r];
#pragma unroll
    for (int c = 0; c < MJ; ++c) bc[c] = b[c] - mj[c];
#pragma unroll
    for (int r = 0; r < MI; ++r)
#pragma unroll
      for (int c = 0; c < MJ; ++c) {
        R w[3];
        w[0] = ac[r] + bc[c];
        w[1] = ac[r] - bc[c];
        R d = a[r] - b[c];
        w[2] = (d < R(0) ? -d : d) - k2[r][c];
#pragma unroll
        for (int k = 0; k < 3; ++k) {
          acc[r][c][k][0] += w[k];
          acc[r][c][k][1] = Num<R>::fma_(w[k], w[k], acc[r][c][k][1]);
#pragma unroll
          for (int t = 0; t < NT; ++t) acc[r][c][k][2 + t] = Num<R>::fma_(w[k], y[t], acc[r][c][k][2 + t]);
        }
      }
  }
}

template <typename R, int KIND, int NT, int MI, int MJ>
__global__ void __launch_bounds__(256) k_pair(const ScreenArgs A, int block_len) {
  using C = PairCfg<R, KIND, NT, MI, MJ>;
  using V2 = typename Vec2<R>::T;
  extern __shared__ __align__(128) unsigned char smem_raw[];
  R *stage_base = reinterpret_cast<R *>(smem_raw);
  uint64_t *bar = reinterpret_cast<uint64_t *>(smem_raw + 2 * (size_t)C::STAGE * sizeof(R));
  __shared__ int s_tile, s_abort;
  __shared__ int32_t s_row[C::ROWS];

  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int wi = warp >> 2, wj = warp & 3, li = lane >> 2, lj = lane & 3;
  const R u = sizeof(R) == 4 ? R(5.9604644775390625e-8) : R(1.1102230246251565e-16);
  const R gamma = (R)A.gamma;
  const R N = (R)A.N, invN = (R)A.invN, sqrtN = Num<R>::sqrt_(N);
  const R fmin = (R)A.fmin_std_rel64;
  const int nchunks = (A.N + C::CH - 1) / C::CH;
  const int64_t ld = A.F.ld;
  const R *rows_src = sizeof(R) == 4 ? (const R *)A.F.v32 : (const R *)A.F.v64;
  const R *y_src = sizeof(R) == 4 ? (const R *)A.y32 : (const R *)A.y64;
  R ysum[NT];
#pragma unroll
  for (int t = 0; t < NT; ++t) ysum[t] = (sizeof(R) == 4 && t < A.T) ? (R)A.ysum32[A.t0 + t] : R(0);

  if (tid == 0) {
    mbar_init(&bar[0], 1);
    mbar_init(&bar[1], 1);
    mbar_fence_init();
    s_abort = 0;
  }
  __syncthreads();
  uint32_t gchunk = 0;
  LaneStats ls;
  ls.zero();

  for (;;) {
    if (tid == 0) s_tile = (int)atomicAdd(A.tile_counter, 1u);
    __syncthreads();
    const int tile = s_tile;
    if (tile >= A.n_tiles || s_abort) break;
    const Tile tl = A.tiles[tile];
    if (tid < C::ROWS) {
      int id = -1;
      if (tid < C::BI) {
        if (tid < tl.ni) id = A.rowid[tl.ibase + tid];
      } else if (tid - C::BI < tl.nj) {
        id = A.rowid[tl.jbase + tid - C::BI];
      }
      s_row[tid] = id;
    }
    __syncthreads();

    int ri[MI], rj[MJ];
    int64_t fi[MI], fj[MJ];
#pragma unroll
    for (int r = 0; r < MI; ++r) {
      ri[r] = wi * 8 * MI + li + 8 * r;
      fi[r] = s_row[ri[r]];
    }
#pragma unroll
    for (int c = 0; c < MJ; ++c) {
      rj[c] = wj * 4 * MJ + lj + 4 * c;
      fj[c] = s_row[C::BI + rj[c]];
    }
    // per-pair shift constants and per-operand centring
    R k0[MI][MJ], k1[MI][MJ], k2[MI][MJ], mi[MI], mj[MJ];
    float4 fai[MI], faj[MJ];
#pragma unroll
    for (int r = 0; r < MI; ++r) {
      fai[r] = fi[r] >= 0 ? A.F.fa[fi[r]] : make_float4(0.f, 0.f, 0.f, 0.f);
      mi[r] = sizeof(R) == 4 ? (R)fai[r].x : (fi[r] >= 0 ? (R)A.F.mean64[fi[r]] : R(0));
    }
#pragma unroll
    for (int c = 0; c < MJ; ++c) {
      faj[c] = fj[c] >= 0 ? A.F.fa[fj[c]] : make_float4(0.f, 0.f, 0.f, 0.f);
      mj[c] = sizeof(R) == 4 ? (R)faj[c].x : (fj[c] >= 0 ? (R)A.F.mean64[fj[c]] : R(0));
    }
#pragma unroll
    for (int r = 0; r < MI; ++r)
#pragma unroll
      for (int c = 0; c < MJ; ++c) {
        R rmi = sizeof(R) == 4 ? (R)fai[r].y : (fi[r] >= 0 ? (R)A.F.rmean64[fi[r]] : R(0));
        R rmj = sizeof(R) == 4 ? (R)faj[c].y : (fj[c] >= 0 ? (R)A.F.rmean64[fj[c]] : R(0));
        k0[r][c] = mi[r] * mj[c];
        k1[r][c] = mi[r] * rmj;
        k2[r][c] = KIND == KIND_MUL ? mj[c] * rmi : (mi[r] - mj[c] < R(0) ? mj[c] - mi[r] : mi[r] - mj[c]);
      }

    R acc[MI][MJ][3][2 + NT], tot[MI][MJ][3][2 + NT];
#pragma unroll
    for (int r = 0; r < MI; ++r)
#pragma unroll
      for (int c = 0; c < MJ; ++c)
#pragma unroll
        for (int k = 0; k < 3; ++k)
#pragma unroll
          for (int e = 0; e < 2 + NT; ++e) acc[r][c][k][e] = tot[r][c][k][e] = R(0);

    auto issue = [&](int chunk) {
      const int st = (gchunk + chunk) & 1;
      R *dst = stage_base + (size_t)st * C::STAGE;
      const int64_t s0 = (int64_t)chunk * C::CH;
      int64_t cnt = ld - s0;
      if (cnt > C::CH) cnt = C::CH;
      const uint32_t rb = (uint32_t)(cnt * sizeof(R));
      uint32_t bytes = 0;
      for (int r = 0; r < C::ROWS; ++r)
        if (s_row[r] >= 0) bytes += rb;
      int64_t ycnt = (int64_t)A.ldy - s0;
      if (ycnt > C::CH) ycnt = C::CH;
      const uint32_t yb = (uint32_t)(ycnt * sizeof(R));
      for (int t = 0; t < NT; ++t)
        if (t < A.T) bytes += yb;
      mbar_arrive_expect_tx(&bar[st], bytes);
      for (int r = 0; r < C::ROWS; ++r)
        if (s_row[r] >= 0) bulk_g2s(dst + r * C::STR, rows_src + (int64_t)s_row[r] * ld + s0, rb, &bar[st]);
      for (int t = 0; t < NT; ++t)
        if (t < A.T)
          bulk_g2s(dst + C::ROWS * C::STR + t * C::CH, y_src + (int64_t)(A.t0 + t) * A.ldy + s0, yb, &bar[st]);
    };

    if (tid == 0) issue(0);
    int blk = 0;
    for (int ch = 0; ch < nchunks; ++ch) {
      if (tid == 0 && ch + 1 < nchunks) issue(ch + 1);
      const uint32_t g = gchunk + ch;
      const int st = g & 1;
      if (!mbar_wait_bounded(&bar[st], (g >> 1) & 1, kWaitLimit)) {
        atomicExch(A.err, DSE_ETIMEOUT);
        s_abort = 1;
      }
      __syncthreads();
      if (s_abort) break;
      const R *S = stage_base + (size_t)st * C::STAGE;
      const R *Si = S, *Sj = S + C::BI * C::STR, *Sy = S + C::ROWS * C::STR;
      int ns = A.N - ch * C::CH;
      if (ns > C::CH) ns = C::CH;
      int s = 0;
      for (; s + 2 <= ns; s += 2) {
        V2 av[MI], bv[MJ], yv[NT];
#pragma unroll
        for (int r = 0; r < MI; ++r) av[r] = *reinterpret_cast<const V2 *>(Si + ri[r] * C::STR + s);
#pragma unroll
        for (int c = 0; c < MJ; ++c) bv[c] = *reinterpret_cast<const V2 *>(Sj + rj[c] * C::STR + s);
#pragma unroll
        for (int t = 0; t < NT; ++t) yv[t] = *reinterpret_cast<const V2 *>(Sy + t * C::CH + s);
        {
          R a[MI], b[MJ], y[NT];
#pragma unroll
          for (int r = 0; r < MI; ++r) a[r] = av[r].x;
#pragma unroll
          for (int c = 0; c < MJ; ++c) b[c] = bv[c].x;
#pragma unroll
          for (int t = 0; t < NT; ++t) y[t] = yv[t].x;
          pair_update<R, KIND, NT, MI, MJ>(a, b, y, k0, k1, k2, mi, mj, acc);
        }
        {
          R a[MI], b[MJ], y[NT];
#pragma unroll
          for (int r = 0; r < MI; ++r) a[r] = av[r].y;
#pragma unroll
          for (int c = 0; c < MJ; ++c) b[c] = bv[c].y;
#pragma unroll
          for (int t = 0; t < NT; ++t) y[t] = yv[t].y;
          pair_update<R, KIND, NT, MI, MJ>(a, b, y, k0, k1, k2, mi, mj, acc);
        }
        if (sizeof(R) == 4) {
          blk += 2;
          if (blk >= block_len) {
            blk = 0;
#pragma unroll
            for (int r = 0; r < MI; ++r)
#pragma unroll
              for (int c = 0; c < MJ; ++c)
#pragma unroll
                for (int k = 0; k < 3; ++k)
#pragma unroll
                  for (int e = 0; e < 2 + NT; ++e) {
                    tot[r][c][k][e] += acc[r][c][k][e];
                    acc[r][c][k][e] = R(0);
                  }
          }
        }
      }
      if (s < ns) {
        R a[MI], b[MJ], y[NT];
#pragma unroll
        for (int r = 0; r < MI; ++r) a[r] = Si[ri[r] * C::STR + s];
#pragma unroll
        for (int c = 0; c < MJ; ++c) b[c] = Sj[rj[c] * C::STR + s];
#pragma unroll
        for (int t = 0; t < NT; ++t) y[t] = Sy[t * C::CH + s];
        pair_update<R, KIND, NT, MI, MJ>(a, b, y, k0, k1, k2, mi, mj, acc);
      }
      __syncthreads();
    }
    gchunk += nchunks;
    if (s_abort) break;
#pragma unroll
    for (int r = 0; r < MI; ++r)
#pragma unroll
      for (int c = 0; c < MJ; ++c)
#pragma unroll
        for (int k = 0; k < 3; ++k)
#pragma unroll
          for (int e = 0; e < 2 + NT; ++e) tot[r][c][k][e] += acc[r][c][k][e];

    // ---------------------------------------------------------- epilogue
    unsigned pushed = 0;
#pragma unroll
    for (int r = 0; r < MI; ++r)
#pragma unroll
      for (int c = 0; c < MJ; ++c) {
        const int64_t x = fi[r], y = fj[c];
        bool pv = x >= 0 && y >= 0 && (tl.ibase + ri[r]) > (tl.jbase + rj[c]);
        const int64_t ia = x > y ? x : y, ib = x > y ? y : x;
        pv = pv && ia >= A.G.o;
        uint64_t pbase = 0;
        if (pv) pbase = A.G.um + (tri((uint64_t)ia) + (uint64_t)ib - A.G.tri_o) * (uint64_t)A.G.nb;
        const float4 fa_a = x > y ? fai[r] : faj[c];
        const float4 fa_b = x > y ? faj[c] : fai[r];
#pragma unroll
        for (int k = 0; k < 3; ++k) {
          const int opc = KIND == KIND_MUL ? (k == 0 ? DSE_OP_MUL : k == 1 ? DSE_OP_DIV : DSE_OP_RDIV)
                                           : (k == 0 ? DSE_OP_ADD : k == 1 ? DSE_OP_SUB : DSE_OP_ABSDIFF);
          const int pos = A.slot_pos[opc - 6];
          const uint64_t gid = (uint64_t)A.n_stored + pbase + (uint64_t)(pos < 0 ? 0 : pos);
          bool cand = pv && pos >= 0 && gid >= A.id_begin && gid < A.id_end;
          int reason = DSE_VALID;
          R W = 0;
          if (cand) {
            // a-priori tests (exact: integer, flags, FP32 directed-rounding
            // intervals with an FP64 fall-back when the interval straddles)
            if (KIND == KIND_ADD && A.unit_check_addsub &&
                (A.F.ukey[2 * ia] != A.F.ukey[2 * ib] || A.F.ukey[2 * ia + 1] != A.F.ukey[2 * ib + 1]))
              reason = DSE_R_UNIT;
            else if (A.max_complexity > 0 && A.F.cplx[ia] + A.F.cplx[ib] + 1 > A.max_complexity)
              reason = DSE_R_COMPLEXITY;
            else if (opc == DSE_OP_DIV && !(A.F.flags[ib] & F_MINABS_POS))
              reason = DSE_R_DOMAIN;
            else if (opc == DSE_OP_RDIV && !(A.F.flags[ia] & F_MINABS_POS))
              reason = DSE_R_DOMAIN;
            else {
              float lo, hi;
              if (opc == DSE_OP_MUL) {
                lo = __fmul_rd(fa_a.w, fa_b.w);
                hi = __fmul_ru(fa_a.z, fa_b.z);
              } else if (opc == DSE_OP_DIV) {
                float2 rr = A.F.fr[ib];
                lo = __fmul_rd(fa_a.w, rr.y);
                hi = __fmul_ru(fa_a.z, rr.x);
              } else if (opc == DSE_OP_RDIV) {
                float2 rr = A.F.fr[ia];
                lo = __fmul_rd(fa_b.w, rr.y);
                hi = __fmul_ru(fa_b.z, rr.x);
              } else {
                lo = __fadd_rd(fa_a.w, fa_b.w);
                hi = __fadd_ru(fa_a.z, fa_b.z);
              }
              if (hi <= A.fmax32_dn) {
              } else if (lo > A.fmax32_up) {
                reason = DSE_R_MAGNITUDE;
              } else {
                reason = domain_magnitude64(opc, A.F.min64[ia], A.F.max64[ia], A.F.minabs64[ia], A.F.maxabs64[ia],
                                            A.F.minabs64[ib], A.F.maxabs64[ib], A.fmax64, 0.0);
              }
              // evaluation error constant W (upper bounds of the magnitudes)
              const R Ma = (R)fa_a.z, Mb = (R)fa_b.z;
              const R kk = (k == 0 ? k0[r][c] : k == 1 ? k1[r][c] : k2[r][c]);
              const R akk = kk < R(0) ? -kk : kk;
              if (opc == DSE_OP_MUL) {
                W = R(2.01) * Ma * Mb + R(1.01) * (Ma * Mb + akk);
              } else if (opc == DSE_OP_DIV) {
                R q = Ma * (R)A.F.fr[ib].x;
                W = R(4.02) * q + R(1.01) * (q + akk);
              } else if (opc == DSE_OP_RDIV) {
                R q = Mb * (R)A.F.fr[ia].x;
                W = R(4.02) * q + R(1.01) * (q + akk);
              } else if (opc == DSE_OP_ABSDIFF) {
                W = R(1.01) * (R(3) * (Ma + Mb) + akk);
              } else {
                const R am = mi[r] < R(0) ? -mi[r] : mi[r], bm = mj[c] < R(0) ? -mj[c] : mj[c];
                W = R(1.01) * (R(3) * (Ma + Mb) + R(2) * (am + bm));
              }
            }
          }
          if (cand && KIND == KIND_ADD) ls.seen++;
          if (cand && reason != DSE_VALID) ls.r[reason]++;
          bool ok = cand && reason == DSE_VALID;
          if (ok && sizeof(R) == 4 && !((A.F.flags[ia] & A.F.flags[ib]) & F_FP32_SAFE)) {
            escalate(A, gid);
            ls.escalated++;
            ok = false;
          }
          const R S1 = tot[r][c][k][0], S2 = tot[r][c][k][1];
          const R shift = (KIND == KIND_MUL) ? (k == 0 ? k0[r][c] : k == 1 ? k1[r][c] : k2[r][c])
                                             : (k == 2 ? k2[r][c] : R(0));
          CandInterval<R> ci{};
          if (ok) {
            // w = V - c: c = k0/k1/k2 for the products, mi +- mj for the
            // centred sum and difference, k2 for |a-b|
            const R cshift = (KIND == KIND_ADD && k < 2) ? (k == 0 ? mi[r] + mj[c] : mi[r] - mj[c]) : shift;
            ci = cand_interval<R>(S1, S2, N, invN, sqrtN, cshift, W, gamma, u, fmin);
            if (ci.realised == 0) {
              ls.r[DSE_R_REALISED]++;
              ok = false;
            } else if (ci.realised == 2) {
              escalate(A, gid);
              ls.escalated++;
              ok = false;
            } else {
              ls.r[DSE_VALID]++;
              ls.evaluated++;
            }
          }
          R Sy[NT];
#pragma unroll
          for (int t = 0; t < NT; ++t) Sy[t] = tot[r][c][k][2 + t];
          pushed |= score_and_push<R, NT>(A, ok, gid, ci, S1, Sy, invN, gamma, u, ysum);
        }
      }
    refresh_pushed<NT>(A, pushed);
  }
  flush_stats(A, ls);
}

// --------------------------------------------------- FP64 escalation

// FP64 two-pass evaluation of one candidate (whole warp); returns the
// realised decision and fills Sxx, mean, and Sxy for targets [t0, t0+T).
__device__ double cand_value64(const FeatTable &F, const RungGeom &G, int64_t n_stored, uint64_t gid, int64_t s,
                               int op, int64_t a, int64_t b) {
  (void)G;
  (void)n_stored;
  (void)gid;
  const double xa = F.v64[a * F.ld + s];
  const double xb = b >= 0 ? F.v64[b * F.ld + s] : 0.0;
  return eval_op64(op, xa, xb);
}

__device__ __forceinline__ void decode_gid(const ScreenArgs &A, uint64_t gid, int *op, int64_t *a, int64_t *b) {
  if (gid < (uint64_t)A.n_stored) {
    *op = DSE_OP_PRIMARY;
    *a = (int64_t)gid;
    *b = -1;
  } else {
    decode_flat(A.G, gid - (uint64_t)A.n_stored, op, a, b);
  }
}

// Escalated candidates: decide the realised test in FP64 and, if valid,
// push FP64 scores for every target.  One warp per candidate.
__global__ void k_escalate(const ScreenArgs A) {
  const int lane = threadIdx.x & 31;
  const unsigned n = min(*A.esc_count, (unsigned)A.esc_cap);
  const uint64_t warps = (uint64_t)gridDim.x * (blockDim.x >> 5);
  for (uint64_t w = ((uint64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; w < n; w += warps) {
    const uint64_t gid = A.esc_id[w];
    int op;
    int64_t a, b;
    decode_gid(A, gid, &op, &a, &b);
    const int64_t N = A.N;
    double sum = 0.0;
    int fin = 1;
    for (int64_t s = lane; s < N; s += 32) {
      double v = cand_value64(A.F, A.G, A.n_stored, gid, s, op, a, b);
      if (!isfinite(v)) fin = 0;
      sum += v;
    }
    fin = !__any_sync(0xffffffffu, !fin);
    sum = warp_sum64(sum);
    const double mean = sum / (double)N;
    double sxx = 0.0, s2 = 0.0;
    for (int64_t s = lane; s < N; s += 32) {
      double v = cand_value64(A.F, A.G, A.n_stored, gid, s, op, a, b);
      double d = v - mean;
      sxx = fma(d, d, sxx);
      s2 = fma(v, v, s2);
    }
    sxx = warp_sum64(sxx);
    s2 = warp_sum64(s2);
    int good = fin;
    if (good && A.fmin_std_rel64 >= 0.0)
      good = __dsqrt_rn(sxx / (double)N) > A.fmin_std_rel64 * __dsqrt_rn(s2 / (double)N);
    if (lane == 0) atomicAdd(&A.stats[good ? ST_REASON0 + DSE_VALID : ST_REASON0 + DSE_R_REALISED], 1ull);
    if (!good) continue;
    if (lane == 0) atomicAdd(&A.stats[ST_EVALUATED], 1ull);
    // scores against every target of the screen (FP64 two-pass)
    const double err = (double)(N / 32 + 40) * 1.1102230246251565e-16 * 8.0;
    double agg = 0.0;
    for (int t = 0; t < A.T; ++t) {
      const double *y = A.y64 + (int64_t)t * A.ldy;
      double sxy = 0.0;
      for (int64_t s = lane; s < N; s += 32) {
        double v = cand_value64(A.F, A.G, A.n_stored, gid, s, op, a, b);
        sxy = fma(v - mean, y[s], sxy);
      }
      sxy = warp_sum64(sxy);
      double sc = fabs(sxy) / sqrt(sxx);
      if (A.mode == DSE_MODE_AGGREGATED) {
        agg += sc * sc;
      } else if (lane == 0) {
        float sf = (float)sc;
        float ef = (float)(err * (sc + 1e-3)) + fabsf((float)(sc - (double)sf)) * 1.0001f + 1e-30f;
        push_one(A.B, t, gid, sf, ef);
      }
    }
    if (A.mode == DSE_MODE_AGGREGATED && lane == 0) {
      double sc = sqrt(agg / (double)A.T);
      float sf = (float)sc;
      float ef = (float)(err * (sc + 1e-3)) + fabsf((float)(sc - (double)sf)) * 1.0001f + 1e-30f;
      push_one(A.B, 0, gid, sf, ef);
    }
  }
}

// ------------------------------------------------------------ launchers

template <typename R, int NT>
void launch_feature_t(const ScreenArgs &A, uint64_t id0, uint64_t id1, uint64_t p0, uint64_t p1, float gamma,
                      int sms, cudaStream_t st) {
  uint64_t ncand = (id1 - id0) + (p1 - p0);
  if (!ncand) return;
  uint64_t blocks = (ncand + 7) / 8;
  uint64_t cap = (uint64_t)sms * 8;
  if (blocks > cap) blocks = cap;
  note_launches(1);
  ScreenArgs B = A;
  B.group = 0;
  k_feature<R, NT><<<(unsigned)blocks, 256, 0, st>>>(B, id0, id1, p0, p1, gamma);
}

template <typename R, int KIND, int NT, int MI, int MJ>
dse_status launch_pair_t(const ScreenArgs &A, int block_len, int sms, cudaStream_t st) {
  using C = PairCfg<R, KIND, NT, MI, MJ>;
  if (A.n_tiles <= 0) return DSE_OK;
  static bool attr_set[64] = {false};
  int dev = 0;
  cudaGetDevice(&dev);
  if (!attr_set[dev & 63]) {
    DSE_CUDA(cudaFuncSetAttribute(k_pair<R, KIND, NT, MI, MJ>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  (int)C::SMEM));
    attr_set[dev & 63] = true;
  }
  int per_sm = 0;
  DSE_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_pair<R, KIND, NT, MI, MJ>, 256, C::SMEM));
  if (per_sm < 1) per_sm = 1;
  int grid = sms * per_sm;
  if (grid > A.n_tiles) grid = A.n_tiles;
  note_launches(1);
  ScreenArgs B = A;
  B.group = KIND == KIND_MUL ? 1 : 2;
  k_pair<R, KIND, NT, MI, MJ><<<grid, 256, C::SMEM, st>>>(B, block_len);
  return DSE_OK;
}

void launch_feature(int prec64, int nt, const ScreenArgs &A, uint64_t id0, uint64_t id1, uint64_t p0, uint64_t p1,
                    float gamma, int sms, cudaStream_t st) {
  if (prec64) {
    if (nt == 1) launch_feature_t<double, 1>(A, id0, id1, p0, p1, gamma, sms, st);
    else launch_feature_t<double, 16>(A, id0, id1, p0, p1, gamma, sms, st);
  } else {
    if (nt == 1) launch_feature_t<float, 1>(A, id0, id1, p0, p1, gamma, sms, st);
    else launch_feature_t<float, 16>(A, id0, id1, p0, p1, gamma, sms, st);
  }
}

dse_status launch_pair(int prec64, int kind, int nt, const ScreenArgs &A, int block_len, int sms, cudaStream_t st) {
  if (prec64) {
    if (nt == 1)
      return kind == KIND_MUL ? launch_pair_t<double, KIND_MUL, 1, 2, 2>(A, block_len, sms, st)
                              : launch_pair_t<double, KIND_ADD, 1, 2, 2>(A, block_len, sms, st);
    return kind == KIND_MUL ? launch_pair_t<double, KIND_MUL, 16, 1, 1>(A, block_len, sms, st)
                            : launch_pair_t<double, KIND_ADD, 16, 1, 1>(A, block_len, sms, st);
  }
  if (nt == 1)
    return kind == KIND_MUL ? launch_pair_t<float, KIND_MUL, 1, 2, 2>(A, block_len, sms, st)
                            : launch_pair_t<float, KIND_ADD, 1, 2, 2>(A, block_len, sms, st);
  return kind == KIND_MUL ? launch_pair_t<float, KIND_MUL, 16, 1, 1>(A, block_len, sms, st)
                          : launch_pair_t<float, KIND_ADD, 16, 1, 1>(A, block_len, sms, st);
}

void launch_escalate(const ScreenArgs &A, int sms, cudaStream_t st) {
  note_launches(1);
  k_escalate<<<sms * 4, 256, 0, st>>>(A);
}

void launch_targets(const double *Y, int64_t ldY, int T, int64_t N, int32_t ldy, double *y64, float *y32,
                    float *ysum32, int *err, cudaStream_t st) {
  note_launches(1);
  k_targets<<<T, 256, 0, st>>>(Y, ldY, T, N, ldy, y64, y32, ysum32, err);
}

}  // namespace dse
