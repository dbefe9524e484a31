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

#include <algorithm>

#include "dse_internal.cuh"
#include "eval64.cuh"
#include "screen_common.cuh"
#include "screen_kernels.cuh"
#include "util.cuh"

namespace dse {

constexpr uint32_t kWaitLimit = 1u << 22;

// ----------------------------------------------------------- target prep

// Centre and normalise one target in FP64 (whole block): row y of N values
// into rows y64 / y32 of ldy (zero beyond N) and the sum of the FP32 row.
__device__ void target_prep(const double *y, int64_t N, int32_t ldy, double *y64, float *y32, float2 *ydf,
                            float *ysum32, int *err) {
  // warp partials, then thread 0 finishes each reduction and broadcasts what
  // the block needs (FP64 work in every thread is slow on this part)
  __shared__ double red[32], bc[2];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = (int)(blockDim.x >> 5);
  auto partial = [&](double v) {
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    if (lane == 0) red[w] = v;
    __syncthreads();
  };
  auto total = [&]() {
    double t = 0.0;
    for (int k = 0; k < nw; ++k) t += red[k];
    return t;
  };
  double s = 0.0;
  for (int64_t i = threadIdx.x; i < N; i += blockDim.x) s += y[i];
  partial(s);
  if (threadIdx.x == 0) bc[0] = total() / (double)N;
  __syncthreads();
  const double mean = bc[0];
  double q = 0.0;
  for (int64_t i = threadIdx.x; i < N; i += blockDim.x) {
    double d = y[i] - mean;
    q = fma(d, d, q);
  }
  partial(q);
  if (threadIdx.x == 0) {
    const double syy = total();
    bc[1] = (syy > 0.0 && isfinite(syy)) ? 1.0 / sqrt(syy) : 0.0;
  }
  __syncthreads();
  const double inv = bc[1];
  if (!(inv > 0.0)) {
    if (threadIdx.x == 0) atomicExch(err, DSE_EINVAL);
    return;
  }
  double fs = 0.0;
  for (int64_t i = threadIdx.x; i < ldy; i += blockDim.x) {
    double v = i < N ? (y[i] - mean) * inv : 0.0;
    float f = __double2float_rn(v);
    y64[i] = v;
    y32[i] = f;
    if (ydf) ydf[i] = make_float2(f, __double2float_rn(__dsub_rn(v, (double)f)));
    fs += (double)f;
  }
  partial(fs);
  if (threadIdx.x == 0) *ysum32 = (float)total();
}

// One block per target.
__global__ void k_targets(const double *Y, int64_t ldY, int T, int64_t N, int32_t ldy, double *y64, float *y32,
                          float2 *ydf, float *ysum32, int *err) {
  const int t = blockIdx.x;
  if (t >= T) return;
  target_prep(Y + (int64_t)t * ldY, N, ldy, y64 + (int64_t)t * ldy, y32 + (int64_t)t * ldy,
              ydf ? ydf + (int64_t)t * ldy : nullptr, ysum32 + t, err);
}

// Batched screens: one block per problem, its target at Y + yoff[p] with the
// problem's own sample count, into row p.
__global__ void k_targets_batched(const double *Y, const int64_t *yoff, const ScreenArgs *args, int n,
                                  int32_t ldy, double *y64, float *y32, float *ysum32, int *err) {
  const int p = blockIdx.x;
  if (p >= n) return;
  target_prep(Y + yoff[p], args[p].N, ldy, y64 + (int64_t)p * ldy, y32 + (int64_t)p * ldy, nullptr, ysum32 + p, err);
}

// ------------------------------------------------------ shared epilogue

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
        // edges rounded outwards (see iv_lo / iv_hi)
        R lo = Num<R>::sub_rd(s, e), hi = Num<R>::add_ru(s, e);
        lo = lo > R(0) ? lo : R(0);
        hi = hi < R(1) ? hi : R(1);
        a += s * s;
        alo += lo * lo;
        ahi += hi * hi;
      }
    }
    R invT = R(1) / R(A.T);
    R s = Num<R>::sqrt_(a * invT);
    R lo = Num<R>::sqrt_(alo * invT), hi = Num<R>::sqrt_(ahi * invT);
    // the sums of T squares and the square roots carry relative errors of
    // at most (T + 2) u of hi, which the last term covers
    R e = (s - lo > hi - s ? s - lo : hi - s) * (R(1) + R(8) * u) + R(A.T + 8) * u * hi;
    float sf = (float)s;
    float ef = (float)e + fabsf((float)(s - (R)sf)) + 1e-30f;
    ef = ef * (1.0f + 2.4e-7f);
    if (want) note_ivl(A, gid, 0, sf, ef);
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
    if (w) note_ivl(A, gid, A.t0 + t, sf, ef);
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

// Evaluation-error coefficients (E = u (kappa ||V|| + lambda)) of a unary op
// on feature f with shift c: per sample the operand's rounding, the op's own
// bound (x^2 and x^3: exact products then the FMA; rcp.approx 1 ulp; sqrtf
// correctly rounded; expf 2 ulp plus the input perturbation |A| u; logf 1 ulp
// plus an absolute u from the input) and the rounding of the shift.
template <typename R>
__device__ __forceinline__ EvalErr<R> unary_err(const FeatTable &F, int op, int64_t f, R c, R sqrtN) {
  const R ac = c < R(0) ? -c : c;
  R kappa;
  R lam = ac * sqrtN;
  switch (op) {
    case DSE_OP_SQUARE: kappa = R(3.01); break;
    case DSE_OP_CUBE: kappa = R(5.01); break;
    case DSE_OP_INV: kappa = R(4.01); break;
    case DSE_OP_SQRT: kappa = R(2.51); break;
    case DSE_OP_EXP: kappa = R(5.01) + (R)F.fa[f].z; break;
    case DSE_OP_LOG:
      kappa = R(3.01);
      lam += R(1.01) * sqrtN;
      break;
    default: kappa = R(2.01); break;
  }
  return EvalErr<R>{kappa, lam};
}

// One candidate of the stored/unary group (whole warp, lanes over samples):
// index w < nid is stored id id0 + w, otherwise unary flat index
// p0 + (w - nid) of rung k.
// Candidate w of the stored/unary group (stored ids [id0, id0 + nid), then
// unary flat indices from p0): its id, op and operand, and its a-priori
// reason (unit: exp/log need a dimensionless operand; complexity; rules;
// domain; magnitude).
__device__ __forceinline__ int feature_setup(const ScreenArgs &A, uint64_t w, uint64_t id0, uint64_t nid,
                                             uint64_t p0, uint64_t *gid_out, int *op_out, int64_t *f_out) {
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
    if (!DSE_IN_BOUNDS(f, A.F.n, A.err)) f = 0;  // (the error stands; the candidate is scored on row 0)
    if ((op == DSE_OP_EXP || op == DSE_OP_LOG) && A.explog_dimensionless && !(A.F.flags[f] & F_DIMLESS))
      reason = DSE_R_UNIT;
    else if (A.max_complexity > 0 && A.F.cplx[f] + 1 > A.max_complexity)
      reason = DSE_R_COMPLEXITY;
    else if (rule_fails(A.F, op, f, -1))
      reason = DSE_R_COMPLEXITY;
    else {
      double ea = (op == DSE_OP_EXP && (A.F.flags[f] & F_EXP_MAG)) ? INFINITY : -INFINITY;
      reason = domain_magnitude64(op, A.F.min64[f], A.F.max64[f], A.F.minabs64[f], A.F.maxabs64[f], 0.0, 0.0,
                                  A.fmax64, ea);
    }
  }
  *gid_out = gid;
  *op_out = op;
  *f_out = f;
  return reason;
}

template <typename R, int NT>
__device__ __forceinline__ void feature_cand(const ScreenArgs &A, uint64_t w, uint64_t id0, uint64_t nid,
                                             uint64_t p0, R gamma, const R *ysum, LaneStats &ls) {
  const int lane = threadIdx.x & 31;
  const R u = sizeof(R) == 4 ? R(5.9604644775390625e-8) : R(1.1102230246251565e-16);
  const int64_t Ns = A.N;
  const int T = A.T, t0 = A.t0;
  const int64_t ldy = A.ldy;
  const R N = (R)Ns, invN = (R)A.invN, sqrtN = Num<R>::sqrt_(N);
  const R fmin = (R)A.fmin_std_rel64;
  const R *Y = sizeof(R) == 4 ? (const R *)A.y32 : (const R *)A.y64;
  int op;
  int64_t f;
  uint64_t gid;
  const int reason = feature_setup(A, w, id0, nid, p0, &gid, &op, &f);
  if (reason != DSE_VALID) {
    if (lane == 0) {
      ls.r[reason]++;
      note_why(A, gid, reason);
    }
    return;
  }
  if (sizeof(R) == 4 && !(A.F.flags[f] & F_FP32_SAFE)) {
    if (lane == 0) {
      escalate(A, gid);
      ls.escalated++;
    }
    return;
  }
  const R *x = sizeof(R) == 4 ? (const R *)(A.F.v32 + f * A.F.ld) : (const R *)(A.F.v64 + f * A.F.ld);
  const R c = unary_eval<R>(op, x[0], R(0));
  const EvalErr<R> ee = unary_err<R>(A.F, op, f, c, sqrtN);
  R S1 = 0, S2 = 0, Sy[NT];
  R o1 = 0, o2 = 0, oy[NT];
  for (int t = 0; t < NT; ++t) Sy[t] = oy[t] = 0;
  int blk = 0;
  // one target: four samples per lane per step, their loads issued
  // together (the loop is bound by load latency otherwise); the sums take
  // them in sample order
  constexpr int U = NT == 1 ? 4 : 1;
  for (int64_t s0 = lane; s0 < Ns; s0 += 32 * U) {
    R xs[U], ys[U][NT];
#pragma unroll
    for (int k = 0; k < U; ++k) {
      const int64_t s = s0 + 32 * k;
      xs[k] = s < Ns ? x[s] : R(0);
#pragma unroll
      for (int t = 0; t < NT; ++t) ys[k][t] = (s < Ns && t < T) ? Y[(int64_t)(t0 + t) * ldy + s] : R(0);
    }
#pragma unroll
    for (int k = 0; k < U; ++k) {
      if (s0 + 32 * k >= Ns) break;
      R v = unary_eval<R>(op, xs[k], c);
      S1 += v;
      S2 = Num<R>::fma_(v, v, S2);
      for (int t = 0; t < NT; ++t)
        if (t < T) Sy[t] = Num<R>::fma_(v, ys[k][t], Sy[t]);
      if (sizeof(R) == 4 && ++blk == 16) {
        blk = 0;
        o1 += S1; o2 += S2; S1 = 0; S2 = 0;
        for (int t = 0; t < NT; ++t) { oy[t] += Sy[t]; Sy[t] = 0; }
      }
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
  CandInterval<R> ci = cand_interval<R>(S1, S2, N, invN, sqrtN, c, ee, gamma, u, fmin);
  if (ci.realised == 0) {
    if (lane == 0) {
      ls.r[DSE_R_REALISED]++;
      note_why(A, gid, DSE_R_REALISED);
    }
    return;
  }
  if (ci.realised == 2) {
    if (lane == 0) {
      escalate(A, gid);
      ls.escalated++;
    }
    return;
  }
  if (lane == 0) {
    ls.r[DSE_VALID]++;
    ls.evaluated++;
    note_why(A, gid, DSE_VALID);
  }
  unsigned pushed = score_and_push<R, NT>(A, lane == 0, gid, ci, S1, Sy, invN, gamma, u, ysum);
  refresh_pushed<NT>(A, pushed);
}

template <typename R, int NT>
__device__ __forceinline__ void load_ysum(const ScreenArgs &A, R (&ysum)[NT]) {
#pragma unroll
  for (int t = 0; t < NT; ++t) ysum[t] = (sizeof(R) == 4 && t < A.T) ? (R)A.ysum32[A.t0 + t] : R(0);
}

// Candidates: stored ids [id0, id1) then unary flat indices [p0, p1).
template <typename R, int NT>
__global__ void __launch_bounds__(256) k_feature(const ScreenArgs A, uint64_t id0, uint64_t id1, uint64_t p0,
                                                 uint64_t p1, float gamma_lane) {
  const uint64_t nid = id1 - id0, ncand = nid + (p1 - p0);
  const uint64_t warps = (uint64_t)gridDim.x * (blockDim.x >> 5);
  R ysum[NT];
  load_ysum<R, NT>(A, ysum);
  LaneStats ls;
  ls.zero();
  for (uint64_t w = ((uint64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; w < ncand; w += warps)
    feature_cand<R, NT>(A, w, id0, nid, p0, (R)gamma_lane, ysum, ls);
  flush_stats(A, ls);
}

// Stored and unary candidates against 16 targets in FP32.  One warp per
// candidate would read all 16 target rows from L2 for every candidate; here
// a warp scores CW candidates at once and the block's 8 warps move through
// the samples together: each 256-sample chunk of the targets (sample-major,
// [s][8], read with 16-byte loads) and of the block's 32 operand rows is
// staged in shared memory by asynchronous copies (cp.async, zero-filled past
// N), double-buffered, so the scoring loop reads shared memory only.  The
// samples are taken twice, for targets 0..7 (with S1 and S2) and 8..15, so
// that the running sums of one half fit in registers at two blocks per SM
// (one pass over all 16 needed 233 registers: one block, 8 warps per SM);
// the reduced sums of the first half wait in shared memory.  Each lane takes
// samples lane, lane + 32, ... in order with the same blocking as
// k_feature, so the sums, bounds and decisions are those of
// k_feature<float, 16>.
constexpr int kF16Chunk = 256, kF16CW = 4, kF16Half = 8;

__device__ __forceinline__ void cp_async4(void *dst, const void *src, bool valid) {
  asm volatile("cp.async.ca.shared.global [%0], [%1], 4, %2;" ::"r"(smem_u32(dst)), "l"(src),
               "r"(valid ? 4 : 0)
               : "memory");
}

template <int CW>
__global__ void __launch_bounds__(256, 2) k_feature16(const ScreenArgs A, uint64_t id0, uint64_t id1, uint64_t p0,
                                                      uint64_t p1, float gamma_lane) {
  constexpr int NT = 16, TH = kF16Half, KS = kF16Chunk, WARPS = 8, NC = WARPS * CW;
  extern __shared__ __align__(16) float f16sm[];
  float(*ys)[KS][TH] = reinterpret_cast<float(*)[KS][TH]>(f16sm);                  // [2][KS][TH]
  float(*xs)[NC][KS] = reinterpret_cast<float(*)[NC][KS]>(f16sm + 2 * KS * TH);     // [2][NC][KS]
  __shared__ const float *rows[NC];
  __shared__ int ract[NC];
  __shared__ float sres[NC][2 + NT];  // reduced S1, S2, Sy of the first half
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const uint64_t nid = id1 - id0, ncand = nid + (p1 - p0);
  const uint64_t per_tile = (uint64_t)NC;
  const uint64_t n_tiles = (ncand + per_tile - 1) / per_tile;
  const float u = 5.9604644775390625e-8f;
  const int64_t Ns = A.N;
  const int T = A.T, t0 = A.t0;
  const int64_t ldy = A.ldy;
  const float N = (float)Ns, invN = (float)A.invN, sqrtN = sqrtf(N);
  const float fmin = (float)A.fmin_std_rel64, gamma = gamma_lane;
  float ysum[NT];
  load_ysum<float, NT>(A, ysum);
  LaneStats ls;
  ls.zero();
  const int nchunk = (int)((Ns + KS - 1) / KS);
  // thread i stages sample i of a chunk: the half's 8 targets and the 32 rows
  auto stage = [&](int ch, int buf, int th0) {
    const int64_t s = (int64_t)ch * KS + threadIdx.x;
    const bool in = s < Ns;
#pragma unroll
    for (int t = 0; t < TH; ++t) {
      const bool v = in && th0 + t < T;
      cp_async4(&ys[buf][threadIdx.x][t], A.y32 + (v ? (int64_t)(t0 + th0 + t) * ldy + s : 0), v);
    }
#pragma unroll 8
    for (int k = 0; k < NC; ++k) {
      const bool v = in && ract[k];
      cp_async4(&xs[buf][k][threadIdx.x], rows[k] + (v ? s : 0), v);
    }
    asm volatile("cp.async.commit_group;" ::: "memory");
  };
  for (uint64_t tile = blockIdx.x; tile < n_tiles; tile += gridDim.x) {
    uint64_t gid[CW];
    int op[CW];
    float c[CW];
    bool act[CW];
    EvalErr<float> ee[CW];
#pragma unroll
    for (int k = 0; k < CW; ++k) {
      const uint64_t w = tile * per_tile + (uint64_t)warp * CW + k;
      act[k] = false;
      gid[k] = 0;
      op[k] = DSE_OP_PRIMARY;
      c[k] = 0.f;
      ee[k] = EvalErr<float>{0.f, 0.f};
      const float *xr = A.F.v32;
      if (w < ncand) {
        int64_t f;
        const int reason = feature_setup(A, w, id0, nid, p0, &gid[k], &op[k], &f);
        if (reason != DSE_VALID) {
          if (lane == 0) {
            ls.r[reason]++;
            note_why(A, gid[k], reason);
          }
        } else if (!(A.F.flags[f] & F_FP32_SAFE)) {
          if (lane == 0) {
            escalate(A, gid[k]);
            ls.escalated++;
          }
        } else {
          act[k] = true;
          xr = A.F.v32 + f * A.F.ld;
          c[k] = unary_eval<float>(op[k], xr[0], 0.f);
          ee[k] = unary_err<float>(A.F, op[k], f, c[k], sqrtN);
        }
      }
      if (lane == 0) {
        rows[warp * CW + k] = xr;
        ract[warp * CW + k] = act[k] ? 1 : 0;
      }
    }
    for (int half = 0; half < 2; ++half) {
      const int th0 = half * TH;
      const bool first = half == 0;
      float S1[CW], S2[CW], o1[CW], o2[CW], Sy[CW][TH], oy[CW][TH];
#pragma unroll
      for (int k = 0; k < CW; ++k) {
        S1[k] = S2[k] = o1[k] = o2[k] = 0.f;
#pragma unroll
        for (int t = 0; t < TH; ++t) Sy[k][t] = oy[k][t] = 0.f;
      }
      int blk = 0;
      __syncthreads();  // (rows of this tile; the previous pass's last chunk is no longer read)
      stage(0, 0, th0);
      for (int ch = 0; ch < nchunk; ++ch) {
        const int buf = ch & 1;
        if (ch + 1 < nchunk) {
          stage(ch + 1, buf ^ 1, th0);
          asm volatile("cp.async.wait_group 1;" ::: "memory");
        } else {
          asm volatile("cp.async.wait_group 0;" ::: "memory");
        }
        __syncthreads();
#pragma unroll 1
        for (int j = 0; j < KS / 32; ++j) {
          const int64_t s = (int64_t)ch * KS + lane + 32 * j;
          if (s >= Ns) break;
          float xv[CW];
#pragma unroll
          for (int k = 0; k < CW; ++k) xv[k] = xs[buf][warp * CW + k][lane + 32 * j];
          float yv[TH];
          const float4 *yp = reinterpret_cast<const float4 *>(&ys[buf][lane + 32 * j][0]);
#pragma unroll
          for (int q = 0; q < TH / 4; ++q) {
            const float4 y4 = yp[q];
            yv[4 * q] = y4.x, yv[4 * q + 1] = y4.y, yv[4 * q + 2] = y4.z, yv[4 * q + 3] = y4.w;
          }
#pragma unroll
          for (int k = 0; k < CW; ++k) {
            if (!act[k]) continue;
            const float v = unary_eval<float>(op[k], xv[k], c[k]);
            if (first) {
              S1[k] += v;
              S2[k] = fmaf(v, v, S2[k]);
            }
#pragma unroll
            for (int t = 0; t < TH; ++t)
              if (th0 + t < T) Sy[k][t] = fmaf(v, yv[t], Sy[k][t]);
          }
          if (++blk == 16) {
            blk = 0;
#pragma unroll
            for (int k = 0; k < CW; ++k) {
              o1[k] += S1[k];
              o2[k] += S2[k];
              S1[k] = 0.f;
              S2[k] = 0.f;
#pragma unroll
              for (int t = 0; t < TH; ++t) {
                oy[k][t] += Sy[k][t];
                Sy[k][t] = 0.f;
              }
            }
          }
        }
        __syncthreads();  // (the buffer is staged again two chunks later)
      }
      // the half's sums, reduced over the warp, wait in shared memory
#pragma unroll
      for (int k = 0; k < CW; ++k) {
        if (!act[k]) continue;  // (warp-uniform)
        float s1 = S1[k] + o1[k], s2 = S2[k] + o2[k], sy[TH];
#pragma unroll
        for (int t = 0; t < TH; ++t) sy[t] = Sy[k][t] + oy[k][t];
        for (int o = 16; o > 0; o >>= 1) {
          s1 += __shfl_xor_sync(0xffffffffu, s1, o);
          s2 += __shfl_xor_sync(0xffffffffu, s2, o);
#pragma unroll
          for (int t = 0; t < TH; ++t) sy[t] += __shfl_xor_sync(0xffffffffu, sy[t], o);
        }
        if (lane == 0) {
          float *r = sres[warp * CW + k];
          if (first) {
            r[0] = s1;
            r[1] = s2;
          }
#pragma unroll
          for (int t = 0; t < TH; ++t) r[2 + th0 + t] = sy[t];
        }
      }
      __syncwarp();
    }
#pragma unroll 1
    for (int k = 0; k < CW; ++k) {
      if (!act[k]) continue;  // (warp-uniform)
      const float *r = sres[warp * CW + k];
      const float s1 = r[0], s2 = r[1];
      float sy[NT];
#pragma unroll
      for (int t = 0; t < NT; ++t) sy[t] = r[2 + t];
      const CandInterval<float> ci = cand_interval<float>(s1, s2, N, invN, sqrtN, c[k], ee[k], gamma, u, fmin);
      if (ci.realised == 0) {
        if (lane == 0) {
          ls.r[DSE_R_REALISED]++;
          note_why(A, gid[k], DSE_R_REALISED);
        }
        continue;
      }
      if (ci.realised == 2) {
        if (lane == 0) {
          escalate(A, gid[k]);
          ls.escalated++;
        }
        continue;
      }
      if (lane == 0) {
        ls.r[DSE_VALID]++;
        ls.evaluated++;
        note_why(A, gid[k], DSE_VALID);
      }
      const unsigned pushed = score_and_push<float, NT>(A, lane == 0, gid[k], ci, s1, sy, invN, gamma, u, ysum);
      refresh_pushed<NT>(A, pushed);
    }
  }
  flush_stats(A, ls);
}

constexpr size_t kF16Smem =
    (size_t)2 * kF16Chunk * kF16Half * sizeof(float) + (size_t)2 * 8 * kF16CW * kF16Chunk * sizeof(float);

// Batched screens: warps take jobs (runs of one problem's stored/unary
// candidates, the whole group of every problem) from a shared counter.
__device__ __forceinline__ bool next_job(unsigned int *counter, int n_jobs, int *j) {
  unsigned v = 0;
  if ((threadIdx.x & 31) == 0) v = atomicAdd(counter, 1u);
  v = __shfl_sync(0xffffffffu, v, 0);
  *j = (int)v;
  return (int)v < n_jobs;
}

template <typename R>
__global__ void __launch_bounds__(256) k_feature_batched(const ScreenArgs *args, const Job *jobs, int n_jobs,
                                                         unsigned int *counter) {
  int j;
  while (next_job(counter, n_jobs, &j)) {
    const Job jb = jobs[j];
    const ScreenArgs &A = args[jb.prob];
    R ysum[1];
    load_ysum<R, 1>(A, ysum);
    LaneStats ls;
    ls.zero();
    const uint64_t nid = (uint64_t)A.n_stored;
    for (int64_t w = jb.first; w < jb.first + jb.count; ++w)
      feature_cand<R, 1>(A, (uint64_t)w, 0, nid, 0, (R)A.gamma_lane, ysum, ls);
    flush_stats(A, ls, 0);
  }
}

// ----------------------------------------------------------- pair kernel

template <typename R, int KIND, int NT, int MI, int MJ>
struct PairCfg {
  static constexpr int BI = 16 * MI, BJ = 16 * MJ, ROWS = BI + BJ;
  static constexpr int CH = sizeof(R) == 4 ? 128 : 64;
  static constexpr int STR = CH + (sizeof(R) == 4 ? 4 : 2);
  static constexpr int STAGE = ROWS * STR + NT * CH;  // elements
  static constexpr int NS = 3;                        // ring stages
  static constexpr size_t SMEM = NS * (size_t)STAGE * sizeof(R) + 128;
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

// One binary candidate (pair ia > ib, op opc) from its accumulated sums:
// a-priori tests, evaluation-error constant W, score interval, realised
// decision, escalation and threshold push.  Every lane of the warp calls it
// (the push is warp-cooperative); only lanes with `active` count and push.
// kk: the shift constant of the evaluation (a*b, a/b, b/a: the FMA constant;
// |a-b|: the constant subtracted); mi, mj: the centring means of the two
// operands in evaluation order (a+b, a-b shift by mi +- mj).
template <typename R, int NT>
__device__ __forceinline__ unsigned binary_candidate(const ScreenArgs &A, LaneStats &ls, bool active, bool pv,
                                                     int64_t ia, int64_t ib, int opc, uint64_t pbase,
                                                     const float4 &fa_a, const float4 &fa_b, R kk, R mi, R mj,
                                                     R S1, R S2, const R *Sy, R N, R invN, R sqrtN, R gamma, R u,
                                                     R fmin, const R *ysum) {
  const bool additive = opc == DSE_OP_ADD || opc == DSE_OP_SUB || opc == DSE_OP_ABSDIFF;
  const int pos = A.slot_pos[opc - 6];
  const uint64_t gid = (uint64_t)A.n_stored + pbase + (uint64_t)(pos < 0 ? 0 : pos);
  // (a+b and a-b of every pair are the Gram kernel's when it runs)
  const bool gram_taken = A.gram_addsub && (opc == DSE_OP_ADD || opc == DSE_OP_SUB);
  const bool cand = active && pv && pos >= 0 && !gram_taken && gid >= A.id_begin && gid < A.id_end;
  int reason = DSE_VALID;
  EvalErr<R> ee{R(0), R(0)};
  if (cand) reason = binary_apriori_W<R>(A, opc, ia, ib, fa_a, fa_b, kk, mi, mj, &ee);
  if (cand && additive) ls.seen++;
  if (cand && reason != DSE_VALID) {
    ls.r[reason]++;
    note_why(A, gid, reason);
  }
  bool ok = cand && reason == DSE_VALID;
  if (ok && sizeof(R) == 4 && !((A.F.flags[ia] & A.F.flags[ib]) & F_FP32_SAFE)) {
    escalate(A, gid);
    ls.escalated++;
    ok = false;
  }
  CandInterval<R> ci{};
  if (ok) {
    // w = V - c: c = kk for the products and |a-b|, mi +- mj for the centred
    // sum and difference
    const R cshift = opc == DSE_OP_ADD ? mi + mj : opc == DSE_OP_SUB ? mi - mj : kk;
    ci = cand_interval<R>(S1, S2, N, invN, sqrtN, cshift, ee, gamma, u, fmin);
    if (ci.realised == 0) {
      ls.r[DSE_R_REALISED]++;
      note_why(A, gid, DSE_R_REALISED);
      ok = false;
    } else if (ci.realised == 2) {
      escalate(A, gid);
      ls.escalated++;
      ok = false;
    } else {
      ls.r[DSE_VALID]++;
      ls.evaluated++;
      note_why(A, gid, DSE_VALID);
    }
  }
  return score_and_push<R, NT>(A, ok, gid, ci, S1, Sy, invN, gamma, u, ysum);
}

// Shared-memory ring of the pair kernel (after its stage buffers): a stage
// is refilled by the last warp to finish with it (no block-wide barrier), in
// the CTA's chunk order kept by the issue cursor.
struct PairRing {
  uint64_t full[4];    // stage holds its chunk (one arrival + transaction bytes)
  unsigned done[4];    // warps finished with the stage's current chunk
  unsigned issued[4];  // chunks issued into the stage
  int cur_i, cur_c;    // next chunk to issue: chunk cur_c of the CTA's cur_i-th tile
  int pad[2];
};

// A CTA takes tiles blockIdx.x, blockIdx.x + gridDim.x, ... (a static
// schedule, so that any warp can name the tile of any later chunk).  Each of
// its 8 warps owns a 2-D slice of the tile's pairs and runs through the
// tile's sample chunks on its own; the chunks stream through NS stages.
// BATCH: the tiles of every problem of a batched screen in one launch; each
// tile names its problem, whose arguments are read from `batch` (A0 then
// carries only the tile list and the error flag).
template <typename R, int KIND, int NT, int MI, int MJ, bool BATCH>
__global__ void __launch_bounds__(256, (sizeof(R) == 4 && NT == 1) ? 2 : 1)
    k_pair(const ScreenArgs A0, const ScreenArgs *batch, int block_len0) {
  using C = PairCfg<R, KIND, NT, MI, MJ>;
  using V2 = typename Vec2<R>::T;
  constexpr int NS = C::NS, WARPS = 8;
  extern __shared__ __align__(128) unsigned char smem_raw[];
  R *stage_base = reinterpret_cast<R *>(smem_raw);
  PairRing *ring = reinterpret_cast<PairRing *>(smem_raw + (size_t)NS * C::STAGE * sizeof(R));

  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int wi = warp >> 2, wj = warp & 3, li = lane >> 2, lj = lane & 3;
  const R u = sizeof(R) == 4 ? R(5.9604644775390625e-8) : R(1.1102230246251565e-16);
  constexpr int kGroup = KIND == KIND_MUL ? 1 : 2;
  const int n_tiles = A0.n_tiles;

  auto tile_of = [&](int i) { return (int)blockIdx.x + i * (int)gridDim.x; };
  auto row_id = [&](const ScreenArgs &A, const Tile &tl, int r) -> int {
    if (r < C::BI) return r < tl.ni ? A.rowid[tl.ibase + r] : -1;
    return (r - C::BI) < tl.nj ? A.rowid[tl.jbase + r - C::BI] : -1;
  };
  // whole warp: the bulk copies of chunk c of tile t into stage st
  auto issue = [&](int t, int c, int st) {
    const Tile tl = A0.tiles[t];
    const ScreenArgs &A = BATCH ? batch[tl.prob] : A0;
    const int64_t ld = A.F.ld;
    const R *rows_src = sizeof(R) == 4 ? (const R *)A.F.v32 : (const R *)A.F.v64;
    const R *y_src = sizeof(R) == 4 ? (const R *)A.y32 : (const R *)A.y64;
    const int64_t s0 = (int64_t)c * C::CH;
    int64_t cnt = ld - s0;
    if (cnt > C::CH) cnt = C::CH;
    const uint32_t rb = (uint32_t)(cnt * sizeof(R));
    int64_t ycnt = (int64_t)A.ldy - s0;
    if (ycnt > C::CH) ycnt = C::CH;
    const uint32_t yb = (uint32_t)(ycnt * sizeof(R));
    constexpr int RPL = (C::ROWS + 31) / 32;  // rows per lane
    int ids[RPL];
    unsigned mine = 0;
#pragma unroll
    for (int q = 0; q < RPL; ++q) {
      const int r = lane + 32 * q;
      ids[q] = r < C::ROWS ? row_id(A, tl, r) : -1;
      if (ids[q] >= 0) mine += rb;
    }
    const bool ylane = lane < NT && lane < A.T;
    if (ylane) mine += yb;
    const unsigned bytes = __reduce_add_sync(0xffffffffu, mine);
    R *dst = stage_base + (size_t)st * C::STAGE;
    if (lane == 0) {
      mbar_arrive_expect_tx(&ring->full[st], bytes);
      ring->issued[st] += 1;
    }
    __syncwarp();
#pragma unroll
    for (int q = 0; q < RPL; ++q)
      if (ids[q] >= 0)
        bulk_g2s(dst + (lane + 32 * q) * C::STR, rows_src + (int64_t)ids[q] * ld + s0, rb, &ring->full[st]);
    if (ylane)
      bulk_g2s(dst + C::ROWS * C::STR + lane * C::CH, y_src + (int64_t)(A.t0 + lane) * A.ldy + s0, yb,
               &ring->full[st]);
  };
  // whole warp: issue the chunk the cursor names (if any) into stage st
  auto issue_next = [&](int st) {
    int i = ring->cur_i, c = ring->cur_c;
    const int t = tile_of(i);
    if (t < n_tiles) {
      issue(t, c, st);
      const Tile tl = A0.tiles[t];
      const int nch = ((BATCH ? batch[tl.prob].N : A0.N) + C::CH - 1) / C::CH;
      if (++c == nch) {
        c = 0;
        ++i;
      }
    }
    __syncwarp();
    if (lane == 0) {
      ring->cur_i = i;
      ring->cur_c = c;
    }
    __syncwarp();
  };

  if (warp == 0) {
    if (lane == 0) {
      for (int st = 0; st < NS; ++st) {
        mbar_init(&ring->full[st], 1);
        ring->done[st] = 0;
        ring->issued[st] = 0;
      }
      ring->cur_i = 0;
      ring->cur_c = 0;
      mbar_fence_init();
    }
    __syncwarp();
    for (int st = 0; st < NS; ++st) issue_next(st);
  }
  __syncthreads();

  uint32_t g = 0;  // the CTA's chunk counter (same sequence in every warp)
  bool aborted = false;
  LaneStats ls;
  ls.zero();
  int cur = BATCH ? -1 : 0;  // problem whose statistics ls holds

  for (int ti = 0;; ++ti) {
    const int tile = tile_of(ti);
    if (tile >= n_tiles) break;
    const Tile tl = A0.tiles[tile];
    if (BATCH && tl.prob != cur) {
      if (cur >= 0) flush_stats(batch[cur], ls, kGroup);
      cur = tl.prob;
    }
    const ScreenArgs &A = BATCH ? batch[tl.prob] : A0;
    const int block_len = BATCH ? A.block_len : block_len0;
    const R gamma = (R)A.gamma;
    const R N = (R)A.N, invN = (R)A.invN, sqrtN = Num<R>::sqrt_(N);
    const R fmin = (R)A.fmin_std_rel64;
    const int nchunks = (A.N + C::CH - 1) / C::CH;
    R ysum[NT];
    load_ysum<R, NT>(A, ysum);

    int ri[MI], rj[MJ];
    int64_t fi[MI], fj[MJ];
#pragma unroll
    for (int r = 0; r < MI; ++r) {
      ri[r] = wi * 8 * MI + li + 8 * r;
      fi[r] = row_id(A, tl, ri[r]);
    }
#pragma unroll
    for (int c = 0; c < MJ; ++c) {
      rj[c] = wj * 4 * MJ + lj + 4 * c;
      fj[c] = row_id(A, tl, C::BI + rj[c]);
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

    int blk = 0;
    for (int ch = 0; ch < nchunks; ++ch, ++g) {
      const int st = (int)(g % NS);
      if (!__all_sync(0xffffffffu, mbar_wait_bounded(&ring->full[st], (g / NS) & 1u, kWaitLimit))) {
        if (lane == 0) atomicExch(A0.err, DSE_ETIMEOUT);
        aborted = true;
        break;
      }
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
      // release the stage; the last warp to do so refills it
      __syncwarp();
      unsigned last = 0;
      if (lane == 0) {
        __threadfence_block();
        last = atomicAdd(&ring->done[st], 1u) == WARPS - 1 ? 1u : 0u;
        if (last) ring->done[st] = 0;
        __threadfence_block();
      }
      if (__shfl_sync(0xffffffffu, last, 0)) {
        __syncwarp();  // the cursor lane 0 acquired is visible to every lane
        issue_next(st);
      }
    }
    if (aborted) break;
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
          const R kk = (k == 0 ? k0[r][c] : k == 1 ? k1[r][c] : k2[r][c]);
          R Sy[NT];
#pragma unroll
          for (int t = 0; t < NT; ++t) Sy[t] = tot[r][c][k][2 + t];
          pushed |= binary_candidate<R, NT>(A, ls, true, pv, ia, ib, opc, pbase, fa_a, fa_b, kk, mi[r], mj[c],
                                            tot[r][c][k][0], tot[r][c][k][1], Sy, N, invN, sqrtN, gamma, u, fmin,
                                            ysum);
        }
      }
    refresh_pushed<NT>(A, pushed);
  }
  if (aborted) {
    // no copy may still be landing when the CTA exits
    if (lane == 0)
      for (int st = 0; st < NS; ++st) {
        const unsigned n = ((volatile unsigned *)ring->issued)[st];
        if (n) mbar_wait_bounded(&ring->full[st], (n - 1) & 1u, kWaitLimit);
      }
    return;
  }
  if (cur >= 0) flush_stats(BATCH ? batch[cur] : A0, ls, kGroup);
}

// ------------------------------------------------ explicit pair lists

// The additive slots (a+b, a-b, |a-b|) of an explicit list of pairs (i > j,
// equal units): one warp per pair, lanes over samples, warp-shuffle
// reduction.  Used when equal-unit pairs are a small fraction of all pairs,
// where tiles over unit classes would be mostly empty.
template <typename R, int NT>
__device__ __forceinline__ void pairlist_one(const ScreenArgs &A, int64_t ia, int64_t ib, R gamma, const R *ysum,
                                             LaneStats &ls) {
  const int lane = threadIdx.x & 31;
  const R u = sizeof(R) == 4 ? R(5.9604644775390625e-8) : R(1.1102230246251565e-16);
  const int64_t Ns = A.N;
  const int T = A.T, t0 = A.t0;
  const int64_t ldy = A.ldy;
  const R N = (R)Ns, invN = (R)A.invN, sqrtN = Num<R>::sqrt_(N);
  const R fmin = (R)A.fmin_std_rel64;
  const R *Y = sizeof(R) == 4 ? (const R *)A.y32 : (const R *)A.y64;
  const R *rows = sizeof(R) == 4 ? (const R *)A.F.v32 : (const R *)A.F.v64;
  const uint64_t pbase = A.G.um + (tri((uint64_t)ia) + (uint64_t)ib - A.G.tri_o) * (uint64_t)A.G.nb;
  const float4 fa_a = A.F.fa[ia], fa_b = A.F.fa[ib];
  const R mi = sizeof(R) == 4 ? (R)fa_a.x : (R)A.F.mean64[ia];
  const R mj = sizeof(R) == 4 ? (R)fa_b.x : (R)A.F.mean64[ib];
  const R cabs = mi - mj < R(0) ? mj - mi : mi - mj;
  const R *xa = rows + ia * A.F.ld, *xb = rows + ib * A.F.ld;
  R acc[3][2 + NT], tot[3][2 + NT];
#pragma unroll
  for (int k = 0; k < 3; ++k)
#pragma unroll
    for (int e = 0; e < 2 + NT; ++e) acc[k][e] = tot[k][e] = R(0);
  int blk = 0;
  // one target: four samples per lane per step, their loads issued together
  // (the loop is bound by load latency otherwise), taken in sample order
  constexpr int U = NT == 1 ? 4 : 1;
  for (int64_t s0 = lane; s0 < Ns; s0 += 32 * U) {
    R av[U], bv[U], yv[U][NT];
#pragma unroll
    for (int q = 0; q < U; ++q) {
      const int64_t s = s0 + 32 * q;
      const bool in = s < Ns;
      av[q] = in ? xa[s] : R(0);
      bv[q] = in ? xb[s] : R(0);
#pragma unroll
      for (int t = 0; t < NT; ++t) yv[q][t] = (in && t < T) ? Y[(int64_t)(t0 + t) * ldy + s] : R(0);
    }
#pragma unroll
    for (int q = 0; q < U; ++q) {
      if (s0 + 32 * q >= Ns) break;
      const R a = av[q], b = bv[q];
      const R ac = a - mi, bc = b - mj, d = a - b;
      R w3[3];
      w3[0] = ac + bc;
      w3[1] = ac - bc;
      w3[2] = (d < R(0) ? -d : d) - cabs;
#pragma unroll
      for (int k = 0; k < 3; ++k) {
        acc[k][0] += w3[k];
        acc[k][1] = Num<R>::fma_(w3[k], w3[k], acc[k][1]);
#pragma unroll
        for (int t = 0; t < NT; ++t) acc[k][2 + t] = Num<R>::fma_(w3[k], yv[q][t], acc[k][2 + t]);
      }
      if (sizeof(R) == 4 && ++blk == 16) {
        blk = 0;
#pragma unroll
        for (int k = 0; k < 3; ++k)
#pragma unroll
          for (int e = 0; e < 2 + NT; ++e) {
            tot[k][e] += acc[k][e];
            acc[k][e] = R(0);
          }
      }
    }
  }
#pragma unroll
  for (int k = 0; k < 3; ++k)
#pragma unroll
    for (int e = 0; e < 2 + NT; ++e) {
      R v = tot[k][e] + acc[k][e];
      for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
      tot[k][e] = v;
    }
  unsigned pushed = 0;
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    const int opc = k == 0 ? DSE_OP_ADD : k == 1 ? DSE_OP_SUB : DSE_OP_ABSDIFF;
    R Sy[NT];
#pragma unroll
    for (int t = 0; t < NT; ++t) Sy[t] = tot[k][2 + t];
    pushed |= binary_candidate<R, NT>(A, ls, lane == 0, true, ia, ib, opc, pbase, fa_a, fa_b, cabs, mi, mj,
                                      tot[k][0], tot[k][1], Sy, N, invN, sqrtN, gamma, u, fmin, ysum);
  }
  refresh_pushed<NT>(A, pushed);
}

template <typename R, int NT>
__global__ void __launch_bounds__(256) k_pairlist(const ScreenArgs A, const int2 *pairs, int64_t n_pairs,
                                                  float gamma_lane) {
  const uint64_t warps = (uint64_t)gridDim.x * (blockDim.x >> 5);
  R ysum[NT];
  load_ysum<R, NT>(A, ysum);
  LaneStats ls;
  ls.zero();
  for (uint64_t w = ((uint64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; w < (uint64_t)n_pairs; w += warps) {
    const int2 pr = pairs[w];
    pairlist_one<R, NT>(A, pr.x, pr.y, (R)gamma_lane, ysum, ls);
  }
  flush_stats(A, ls);
}

// Batched screens: the equal-unit pair lists of every problem, concatenated;
// warps take jobs (runs of one problem's pairs) from a shared counter.
template <typename R>
__global__ void __launch_bounds__(256) k_pairlist_batched(const ScreenArgs *args, const int2 *pairs,
                                                          const Job *jobs, int n_jobs, unsigned int *counter) {
  int j;
  while (next_job(counter, n_jobs, &j)) {
    const Job jb = jobs[j];
    const ScreenArgs &A = args[jb.prob];
    R ysum[1];
    load_ysum<R, 1>(A, ysum);
    LaneStats ls;
    ls.zero();
    for (int64_t w = jb.first; w < jb.first + jb.count; ++w) {
      const int2 pr = pairs[w];
      pairlist_one<R, 1>(A, pr.x, pr.y, (R)A.gamma_lane, ysum, ls);
    }
    flush_stats(A, ls, 2);
  }
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
// push FP64 scores for every target.  One block of kEsc threads per
// candidate; one pass for the statistics (sums shifted by the first value, so
// Sxx = S2 - S1^2/N keeps FP64 accuracy even for a near-constant candidate),
// then one pass per group of 16 targets.
constexpr int kEsc = 128;

// Block sums of v: in every thread, or (ALL = false) in thread 0 only (the
// FP64 adds then leave the SM's FP64 units to the other blocks).
template <int NV, bool ALL = true, int THREADS = kEsc>
__device__ __forceinline__ void block_sum64(double (&v)[NV], double *sm) {
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
#pragma unroll
  for (int i = 0; i < NV; ++i) v[i] = warp_sum64(v[i]);
  if (lane == 0)
#pragma unroll
    for (int i = 0; i < NV; ++i) sm[w * NV + i] = v[i];
  __syncthreads();
  if (ALL || threadIdx.x == 0) {
#pragma unroll
    for (int i = 0; i < NV; ++i) {
      double t = 0.0;
      for (int ww = 0; ww < THREADS / 32; ++ww) t += sm[ww * NV + i];
      v[i] = t;
    }
  }
  __syncthreads();
}

// The FP64 passes of the escalation kernels, instantiated per operator (the
// operator is then not a branch inside the sample loop).
template <int OP>
__device__ __forceinline__ bool esc_binary() {
  return OP == DSE_OP_ADD || OP == DSE_OP_SUB || OP == DSE_OP_MUL || OP == DSE_OP_DIV || OP == DSE_OP_RDIV ||
         OP == DSE_OP_ABSDIFF;
}

// k_escalate_stash: sum (v-c), sum (v-c)^2, sum v^2, non-finite count, and
// fl32(v - c) of every sample into w (THREADS threads over the samples).
template <int OP, int THREADS>
__device__ __forceinline__ void esc_pass_stash(const double *xa, const double *xb, int64_t N, double c,
                                               double (&st)[4], float *w) {
  for (int64_t s = threadIdx.x; s < N; s += THREADS) {
    const double v = eval_op64(OP, xa[s], esc_binary<OP>() ? xb[s] : 0.0);
    if (!isfinite(v)) st[3] += 1.0;
    const double d = v - c;
    st[0] += d;
    st[1] = fma(d, d, st[1]);
    st[2] = fma(v, v, st[2]);
    w[s] = (float)d;
  }
}

// k_escalate1: sum (v-c), sum (v-c)^2, sum v^2, non-finite count, sum (v-c)
// y, sum y; four samples per thread per step, their loads issued together,
// each thread taking its samples in increasing order.
template <int OP, int THREADS>
__device__ __forceinline__ void esc_pass1(const double *xa, const double *xb, const double *y, int64_t N, double c,
                                          double (&st)[6]) {
  constexpr int U = 4;
  for (int64_t s0 = threadIdx.x; s0 < N; s0 += U * THREADS) {
    double va[U], vb[U], yv[U];
#pragma unroll
    for (int k = 0; k < U; ++k) {
      const int64_t s = s0 + (int64_t)k * THREADS;
      const bool in = s < N;
      va[k] = in ? xa[s] : 0.0;
      vb[k] = in && esc_binary<OP>() ? xb[s] : 0.0;
      yv[k] = in ? y[s] : 0.0;
    }
#pragma unroll
    for (int k = 0; k < U; ++k) {
      if (s0 + (int64_t)k * THREADS >= N) break;
      const double v = eval_op64(OP, va[k], vb[k]);
      if (!isfinite(v)) st[3] += 1.0;
      const double d = v - c;
      st[0] += d;
      st[1] = fma(d, d, st[1]);
      st[2] = fma(v, v, st[2]);
      st[4] = fma(d, yv[k], st[4]);
      st[5] += yv[k];
    }
  }
}

// switch over the operator codes, CALL(OPC) for each (the primary /
// identity code as the default)
#define DSE_OP_SWITCH(op, CALL)  \
  switch (op) {                  \
    case DSE_OP_SQUARE: CALL(DSE_OP_SQUARE); break; \
    case DSE_OP_CUBE: CALL(DSE_OP_CUBE); break;     \
    case DSE_OP_INV: CALL(DSE_OP_INV); break;       \
    case DSE_OP_SQRT: CALL(DSE_OP_SQRT); break;     \
    case DSE_OP_EXP: CALL(DSE_OP_EXP); break;       \
    case DSE_OP_LOG: CALL(DSE_OP_LOG); break;       \
    case DSE_OP_ADD: CALL(DSE_OP_ADD); break;       \
    case DSE_OP_SUB: CALL(DSE_OP_SUB); break;       \
    case DSE_OP_MUL: CALL(DSE_OP_MUL); break;       \
    case DSE_OP_DIV: CALL(DSE_OP_DIV); break;       \
    case DSE_OP_RDIV: CALL(DSE_OP_RDIV); break;     \
    case DSE_OP_ABSDIFF: CALL(DSE_OP_ABSDIFF); break; \
    default: CALL(DSE_OP_PRIMARY); break;           \
  }

// batch != nullptr: entries of a batched screen, each with its problem.
__global__ void __launch_bounds__(kEsc) k_escalate(const ScreenArgs A0, const ScreenArgs *batch) {
  __shared__ double sm[(kEsc / 32) * 16];
  const unsigned n = min(*A0.esc_count, (unsigned)A0.esc_cap);
  for (unsigned w = blockIdx.x; w < n; w += gridDim.x) {
    const ScreenArgs &A = batch ? batch[A0.esc_prob[w]] : A0;
    const int64_t N = A.N;
    const uint64_t gid = A0.esc_id[w];
    int op;
    int64_t a, b;
    decode_gid(A, gid, &op, &a, &b);
    if (!DSE_OPERANDS_OK(A.F, a, b, A0.err)) continue;
    const double c = cand_value64(A.F, A.G, A.n_stored, gid, 0, op, a, b);
    // sum (v-c), sum (v-c)^2, sum v^2, number of non-finite values
    double st[4] = {0.0, 0.0, 0.0, 0.0};
    for (int64_t s = threadIdx.x; s < N; s += kEsc) {
      const double v = cand_value64(A.F, A.G, A.n_stored, gid, s, op, a, b);
      if (!isfinite(v)) st[3] += 1.0;
      const double d = v - c;
      st[0] += d;
      st[1] = fma(d, d, st[1]);
      st[2] = fma(v, v, st[2]);
    }
    block_sum64<4>(st, sm);
    const double sxx = st[1] - st[0] * (st[0] / (double)N);
    int good = st[3] == 0.0 && isfinite(sxx);
    if (good && A.fmin_std_rel64 >= 0.0)
      good = __dsqrt_rn(fmax(sxx, 0.0) / (double)N) > A.fmin_std_rel64 * __dsqrt_rn(st[2] / (double)N);
    if (threadIdx.x == 0) {
      atomicAdd(&A.stats[good ? ST_REASON0 + DSE_VALID : ST_REASON0 + DSE_R_REALISED], 1ull);
      if (good) atomicAdd(&A.stats[ST_EVALUATED], 1ull);
      if (A.why) A.why[gid - A.id_begin] = (int8_t)(good ? DSE_VALID : DSE_R_REALISED);
    }
    if (!good || !(sxx > 0.0)) continue;
    const double err = (double)(N / kEsc + 64) * 1.1102230246251565e-16 * 16.0;
    const double dm = st[0] / (double)N;  // vbar - c
    double agg = 0.0;
    for (int t0 = 0; t0 < A.T; t0 += 16) {
      double sy[16];
#pragma unroll
      for (int t = 0; t < 16; ++t) sy[t] = 0.0;
      for (int64_t s = threadIdx.x; s < N; s += kEsc) {
        const double d = (cand_value64(A.F, A.G, A.n_stored, gid, s, op, a, b) - c) - dm;
#pragma unroll
        for (int t = 0; t < 16; ++t)
          if (t0 + t < A.T) sy[t] = fma(d, A.y64[(int64_t)(A.t0 + t0 + t) * A.ldy + s], sy[t]);
      }
      block_sum64<16>(sy, sm);
      if (threadIdx.x == 0) {
        for (int t = 0; t < 16 && t0 + t < A.T; ++t) {
          const double sc = fabs(sy[t]) / sqrt(sxx);
          if (A.mode == DSE_MODE_AGGREGATED) {
            agg += sc * sc;
          } else {
            const float sf = (float)sc;
            const float ef = (float)(err * (sc + 1e-3)) + fabsf((float)(sc - (double)sf)) * 1.0001f + 1e-30f;
            note_ivl(A, gid, A.t0 + t0 + t, sf, ef);
            push_one(A.B, A.t0 + t0 + t, gid, sf, ef);
          }
        }
      }
    }
    if (A.mode == DSE_MODE_AGGREGATED && threadIdx.x == 0) {
      const double sc = sqrt(agg / (double)A.T);
      const float sf = (float)sc;
      const float ef = (float)(err * (sc + 1e-3)) + fabsf((float)(sc - (double)sf)) * 1.0001f + 1e-30f;
      note_ivl(A, gid, A.t0, sf, ef);
      push_one(A.B, A.t0, gid, sf, ef);
    }
  }
}

// Many targets, 8192 <= N <= 40960 (single screens): the FP64 pass of
// k_escalate also keeps w_s = fl32(v_s - c) in
// shared memory, and the numerators come from it in FP32 (blocks of 16
// samples per thread, then warp shuffles and the warps in FP64), without a
// second FP64 evaluation of every sample.  Numerator error for target t,
// with e_s = fl32(w_s - fl32(vbar - c)) and the FP32 target y32 (within u of
// the FP64 one per sample), by Cauchy-Schwarz (|y| = 1):
//   u (2 |v - c| + 2 |vbar - c| sqrt(N)) + (u + gamma) |e|,
//   gamma = (16 + m / 16 + 8) u, m = N / kEscS terms per thread,
// |e| <= sqrt(Sxx) + 2u of the above; the score's bound is that / sqrt(Sxx)
// plus the FP64 part's.  Columns outside [2^-60, 2^60] take k_escalate.
constexpr int64_t kEscStashMax = 40960;  // samples kept in shared memory (160 KB)
constexpr int kEscS = 512;                // threads per candidate (FP64 latency wants many warps)

__global__ void __launch_bounds__(kEscS, 2) k_escalate_stash(const ScreenArgs A) {
  extern __shared__ float wsm[];
  __shared__ double sm[(kEscS / 32) * 16];
  const unsigned n = min(*A.esc_count, (unsigned)A.esc_cap);
  const int64_t N = A.N;
  const float u = 5.9604644775390625e-8f;
  for (unsigned w = blockIdx.x; w < n; w += gridDim.x) {
    const uint64_t gid = A.esc_id[w];
    int op;
    int64_t a, b;
    decode_gid(A, gid, &op, &a, &b);
    if (!DSE_OPERANDS_OK(A.F, a, b, A.err)) continue;
    const double c = cand_value64(A.F, A.G, A.n_stored, gid, 0, op, a, b);
    double st[4] = {0.0, 0.0, 0.0, 0.0};
    const double *xa = A.F.v64 + a * A.F.ld, *xb = A.F.v64 + (b >= 0 ? b : a) * A.F.ld;
#define DSE_ESC_STASH(OPC) esc_pass_stash<OPC, kEscS>(xa, xb, N, c, st, wsm)
    DSE_OP_SWITCH(op, DSE_ESC_STASH)
#undef DSE_ESC_STASH
    block_sum64<4, true, kEscS>(st, sm);
    const double sxx = st[1] - st[0] * (st[0] / (double)N);
    int good = st[3] == 0.0 && isfinite(sxx);
    if (good && A.fmin_std_rel64 >= 0.0)
      good = __dsqrt_rn(fmax(sxx, 0.0) / (double)N) > A.fmin_std_rel64 * __dsqrt_rn(st[2] / (double)N);
    if (threadIdx.x == 0) {
      atomicAdd(&A.stats[good ? ST_REASON0 + DSE_VALID : ST_REASON0 + DSE_R_REALISED], 1ull);
      if (good) atomicAdd(&A.stats[ST_EVALUATED], 1ull);
      if (A.why && DSE_IN_BOUNDS(gid - A.id_begin, A.id_end - A.id_begin, A.err))
        A.why[gid - A.id_begin] = (int8_t)(good ? DSE_VALID : DSE_R_REALISED);
    }
    if (!good || !(sxx > 0.0)) continue;
    const double err = (double)(N / kEscS + 64) * 1.1102230246251565e-16 * 16.0;
    const double dm = st[0] / (double)N;  // vbar - c
    const double q = sqrt(sxx), nvc = sqrt(st[1]), dmn = fabs(dm) * sqrt((double)N);
    const bool fp32 = q > 8.67e-19 && nvc < 1.15e18 && dmn < 1.15e18;  // 2^-60 .. 2^60
    const float dm32 = (float)dm;
    const double m = (double)((N + kEscS - 1) / kEscS);
    const double gamma = (16.0 + m / 16.0 + 8.0) * (double)u;
    const double esx = q + 2.0 * (double)u * (2.0 * nvc + 2.0 * dmn);
    const double dnum = ((double)u * (2.0 * nvc + 2.0 * dmn) + ((double)u + gamma) * esx) * 1.01;
    double agg = 0.0;
    constexpr int TG = 8;  // targets per pass over the kept values
    for (int t0 = 0; t0 < A.T; t0 += TG) {
      double sy[TG];
#pragma unroll
      for (int t = 0; t < TG; ++t) sy[t] = 0.0;
      if (fp32) {
        float acc[TG], blk[TG];
#pragma unroll
        for (int t = 0; t < TG; ++t) acc[t] = blk[t] = 0.f;
        int nb = 0;
        for (int64_t s = threadIdx.x; s < N; s += kEscS) {
          const float e = wsm[s] - dm32;
#pragma unroll
          for (int t = 0; t < TG; ++t)
            if (t0 + t < A.T) blk[t] = fmaf(e, A.y32[(int64_t)(A.t0 + t0 + t) * A.ldy + s], blk[t]);
          if (++nb == 16) {
            nb = 0;
#pragma unroll
            for (int t = 0; t < TG; ++t) {
              acc[t] += blk[t];
              blk[t] = 0.f;
            }
          }
        }
#pragma unroll
        for (int t = 0; t < TG; ++t) sy[t] = (double)(acc[t] + blk[t]);
      } else {
        for (int64_t s = threadIdx.x; s < N; s += kEscS) {
          const double d = (cand_value64(A.F, A.G, A.n_stored, gid, s, op, a, b) - c) - dm;
#pragma unroll
          for (int t = 0; t < TG; ++t)
            if (t0 + t < A.T) sy[t] = fma(d, A.y64[(int64_t)(A.t0 + t0 + t) * A.ldy + s], sy[t]);
        }
      }
      block_sum64<TG, true, kEscS>(sy, sm);
      if (threadIdx.x == 0) {
        for (int t = 0; t < TG && t0 + t < A.T; ++t) {
          const double sc = fabs(sy[t]) / q;
          // (the FP32 numerators add dnum / q; the FP64 ones the err term)
          const double eb = err * (sc + 1e-3) + (fp32 ? dnum / q * 1.01 : 0.0);
          if (A.mode == DSE_MODE_AGGREGATED) {
            agg += sc * sc;
          } else {
            const float sf = (float)(sc < 1.0 ? sc : 1.0);
            const float ef = (float)eb + fabsf((float)(sc - (double)sf)) * 1.0001f + 1e-30f;
            note_ivl(A, gid, A.t0 + t0 + t, sf, ef);
            push_one(A.B, A.t0 + t0 + t, gid, sf, ef);
          }
        }
      }
    }
    if (A.mode == DSE_MODE_AGGREGATED && threadIdx.x == 0) {
      // sqrt(mean sc^2) moves by at most the largest target's bound
      const double sc = sqrt(agg / (double)A.T);
      const float sf = (float)sc;
      const double eb = err * (sc + 1e-3) + (fp32 ? dnum / q * 1.01 : 0.0);
      const float ef = (float)eb + fabsf((float)(sc - (double)sf)) * 1.0001f + 1e-30f;
      note_ivl(A, gid, A.t0, sf, ef);
      push_one(A.B, A.t0, gid, sf, ef);
    }
  }
}

// FP32 stage of the escalation (single screens, at most 16 targets): one
// warp per escalated binary candidate evaluates it again in FP32 with the
// tight accumulation of r32_sums (8-sample FP32 blocks into FP32 pairs,
// gamma = kGamma32 u instead of the screening kernel's wider bound: the Gram
// contractions escalate candidates whose BF16x3 interval of the centred sum
// of squares reaches zero, most of which are far from degenerate) and
// decides the realised test on the screen's interval.  Decided candidates
// take their reason code, statistics and every target's score and push here,
// exactly as in the FP32 screen; the others (near-constant columns such as
// x * (1/x), other operators, operands outside the FP32-safe range) go to
// the undecided list that the FP64 kernels then take.
__global__ void __launch_bounds__(256, 2) k_escalate32(const ScreenArgs A) {
  const int lane = threadIdx.x & 31;
  const unsigned n = min(*A.esc_count, (unsigned)A.esc_cap);
  const unsigned warps = (gridDim.x * blockDim.x) >> 5;
  const float u = 5.9604644775390625e-8f;
  const float Nf = (float)A.N, invN = (float)A.invN, sqrtN = sqrtf(Nf);
  const float gamma = kGamma32 * u, fmin = (float)A.fmin_std_rel64;
  float ysum[16];
  load_ysum<float, 16>(A, ysum);
  LaneStats ls;
  ls.zero();
  for (unsigned w = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; w < n; w += warps) {
    const uint64_t gid = A.esc_id[w];
    int op;
    int64_t a, b;
    decode_gid(A, gid, &op, &a, &b);
    R32Setup c;
    const bool ok = gid >= (uint64_t)A.n_stored && r32_setup(A, op, a, b, c);
    // two passes over the samples, targets 0..7 with the realised decision,
    // then (valid candidates only) targets 8..15: half the running sums, so
    // that two blocks fit on an SM; the sums are those of one pass over all
    float Sm[18], Sh[10];
#pragma unroll
    for (int k = 0; k < 18; ++k) Sm[k] = 0.f;
    if (ok) {
      r32_sums<8, 1>(A, op, a, b, A.y32 + (int64_t)A.t0 * A.ldy, A.T < 8 ? A.T : 8, c, Sh);
#pragma unroll
      for (int k = 0; k < 10; ++k) Sm[k] = Sh[k];
    }
    CandInterval<float> ci{};
    int decided = 0;  // 1 valid, 2 degenerate
    if (ok) {
      ci = cand_interval<float>(Sm[0], Sm[1], Nf, invN, sqrtN, c.cshift, c.ee, gamma, u, fmin);
      decided = ci.realised == 1 ? 1 : ci.realised == 0 ? 2 : 0;
    }
    if (decided == 1 && A.T > 8) {
      r32_sums<8, 1>(A, op, a, b, A.y32 + (int64_t)(A.t0 + 8) * A.ldy, A.T - 8, c, Sh);
#pragma unroll
      for (int k = 0; k < 8; ++k) Sm[10 + k] = Sh[2 + k];
    }
    if (lane == 0) {
      if (decided == 1) {
        ls.r[DSE_VALID]++;
        ls.evaluated++;
        note_why(A, gid, DSE_VALID);
      } else if (decided == 2) {
        ls.r[DSE_R_REALISED]++;
        note_why(A, gid, DSE_R_REALISED);
      } else {
        const unsigned pos = atomicAdd(A.esc2_count, 1u);
        A.esc2_id[pos] = gid;
      }
    }
    float Sy[16];
#pragma unroll
    for (int t = 0; t < 16; ++t) Sy[t] = Sm[2 + t];
    const unsigned pushed =
        score_and_push<float, 16>(A, lane == 0 && decided == 1, gid, ci, Sm[0], Sy, invN, gamma, u, ysum);
    refresh_pushed<16>(A, pushed);
  }
  flush_stats(A, ls);
}

// The same decision and score for screens with one target (every problem of
// a batched screen too), in one pass over the samples: the centred numerator
// follows from the shifted sums, sum (v - vbar) y = sum (v - c) y -
// (vbar - c) sum y, with sum y accumulated alongside.
__global__ void __launch_bounds__(kEsc) k_escalate1(const ScreenArgs A0, const ScreenArgs *batch) {
  __shared__ double sm[(kEsc / 32) * 6];
  const unsigned n = min(*A0.esc_count, (unsigned)A0.esc_cap);
  for (unsigned w = blockIdx.x; w < n; w += gridDim.x) {
    const ScreenArgs &A = batch ? batch[A0.esc_prob[w]] : A0;
    const int64_t N = A.N;
    const uint64_t gid = A0.esc_id[w];
    int op;
    int64_t a, b;
    decode_gid(A, gid, &op, &a, &b);
    if (!DSE_OPERANDS_OK(A.F, a, b, A0.err)) continue;
    const double c = cand_value64(A.F, A.G, A.n_stored, gid, 0, op, a, b);
    const double *y = A.y64 + (int64_t)A.t0 * A.ldy;
    // sum (v-c), sum (v-c)^2, sum v^2, non-finite count, sum (v-c) y, sum y;
    // four samples per thread per step, their loads issued together, each
    // thread taking its samples in increasing order
    double st[6] = {0.0, 0.0, 0.0, 0.0, 0.0, 0.0};
    const double *xa = A.F.v64 + a * A.F.ld, *xb = A.F.v64 + (b >= 0 ? b : a) * A.F.ld;
#define DSE_ESC1(OPC) esc_pass1<OPC, kEsc>(xa, xb, y, N, c, st)
    DSE_OP_SWITCH(op, DSE_ESC1)
#undef DSE_ESC1
    block_sum64<6, false>(st, sm);
    if (threadIdx.x == 0) {  // (FP64 work is slow on this part: one thread decides)
      const double sxx = st[1] - st[0] * (st[0] / (double)N);
      int good = st[3] == 0.0 && isfinite(sxx);
      if (good && A.fmin_std_rel64 >= 0.0)
        good = __dsqrt_rn(fmax(sxx, 0.0) / (double)N) > A.fmin_std_rel64 * __dsqrt_rn(st[2] / (double)N);
      atomicAdd(&A.stats[good ? ST_REASON0 + DSE_VALID : ST_REASON0 + DSE_R_REALISED], 1ull);
      if (good) atomicAdd(&A.stats[ST_EVALUATED], 1ull);
      if (A.why) A.why[gid - A.id_begin] = (int8_t)(good ? DSE_VALID : DSE_R_REALISED);
      if (good && sxx > 0.0) {
        const double err = (double)(N / kEsc + 64) * 1.1102230246251565e-16 * 16.0;
        const double dm = st[0] / (double)N;  // vbar - c
        const double sc = fabs(st[4] - dm * st[5]) / sqrt(sxx);
        const float sf = (float)sc;
        const float ef = (float)(err * (sc + 1e-3)) + fabsf((float)(sc - (double)sf)) * 1.0001f + 1e-30f;
        note_ivl(A, gid, A.t0, sf, ef);
        push_one(A.B, A.t0, gid, sf, ef);
      }
    }
    __syncthreads();
  }
}

// Candidates no kernel visits: the additive slots of pairs whose units
// differ (the additive kernels run over equal-unit pairs only).  Every other
// entry of the range was written by the kernel that decided it; an entry
// still at -1 afterwards would be a candidate no kernel looked at.
__global__ void k_why_fixup(const ScreenArgs A) {
  const uint64_t n = A.id_end - A.id_begin;
  for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (uint64_t)gridDim.x * blockDim.x) {
    if (A.why[i] != -1) continue;
    const uint64_t gid = A.id_begin + i;
    if (gid < (uint64_t)A.n_stored) continue;
    int op;
    int64_t a, b;
    decode_gid(A, gid, &op, &a, &b);
    const bool additive = op == DSE_OP_ADD || op == DSE_OP_SUB || op == DSE_OP_ABSDIFF;
    if (additive && A.unit_check_addsub &&
        (A.F.ukey[2 * a] != A.F.ukey[2 * b] || A.F.ukey[2 * a + 1] != A.F.ukey[2 * b + 1]))
      A.why[i] = (int8_t)DSE_R_UNIT;
  }
}

void launch_why_fixup(const ScreenArgs &A, int sms, cudaStream_t st) {
  const uint64_t n = A.id_end - A.id_begin;
  if (!A.why || n == 0) return;
  uint64_t blocks = (n + 255) / 256;
  if (blocks > (uint64_t)sms * 8) blocks = (uint64_t)sms * 8;
  note_launches(1);
  k_why_fixup<<<(unsigned)blocks, 256, 0, st>>>(A);
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
  if (sizeof(R) == 4 && NT == 16) {
    // 32 candidates per block, two blocks per SM at a time
    uint64_t tiles = (ncand + 8 * kF16CW - 1) / (8 * kF16CW);
    if (tiles > (uint64_t)sms * 2) tiles = (uint64_t)sms * 2;
    static bool attr[64] = {false};
    int dev = 0;
    cudaGetDevice(&dev);
    if (!attr[dev & 63]) {
      cudaFuncSetAttribute(k_feature16<kF16CW>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kF16Smem);
      attr[dev & 63] = true;
    }
    k_feature16<kF16CW><<<(unsigned)tiles, 256, kF16Smem, st>>>(B, id0, id1, p0, p1, gamma);
    return;
  }
  k_feature<R, NT><<<(unsigned)blocks, 256, 0, st>>>(B, id0, id1, p0, p1, gamma);
}

template <typename R, int KIND, int NT, int MI, int MJ, bool BATCH = false>
dse_status launch_pair_t(const ScreenArgs &A, int block_len, int sms, cudaStream_t st,
                         const ScreenArgs *batch = nullptr) {
  using C = PairCfg<R, KIND, NT, MI, MJ>;
  if (A.n_tiles <= 0) return DSE_OK;
  static bool attr_set[64] = {false};
  static int per_sm_of[64] = {0};
  int dev = 0;
  cudaGetDevice(&dev);
  if (!attr_set[dev & 63]) {
    DSE_CUDA(cudaFuncSetAttribute(k_pair<R, KIND, NT, MI, MJ, BATCH>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  (int)C::SMEM));
    int per_sm = 0;
    DSE_CUDA(
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_pair<R, KIND, NT, MI, MJ, BATCH>, 256, C::SMEM));
    per_sm_of[dev & 63] = per_sm < 1 ? 1 : per_sm;
    attr_set[dev & 63] = true;
  }
  int grid = sms * per_sm_of[dev & 63];
  if (grid > A.n_tiles) grid = A.n_tiles;
  note_launches(1);
  ScreenArgs B = A;
  B.group = KIND == KIND_MUL ? 1 : 2;
  k_pair<R, KIND, NT, MI, MJ, BATCH><<<grid, 256, C::SMEM, st>>>(B, batch, block_len);
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

void launch_pairlist(int prec64, int nt, const ScreenArgs &A, const int2 *pairs, int64_t n_pairs, float gamma,
                     int sms, cudaStream_t st) {
  if (n_pairs <= 0) return;
  uint64_t blocks = ((uint64_t)n_pairs + 7) / 8;
  if (blocks > (uint64_t)sms * 16) blocks = (uint64_t)sms * 16;
  note_launches(1);
  ScreenArgs B = A;
  B.group = 2;
  if (prec64) {
    if (nt == 1) k_pairlist<double, 1><<<(unsigned)blocks, 256, 0, st>>>(B, pairs, n_pairs, gamma);
    else k_pairlist<double, 16><<<(unsigned)blocks, 256, 0, st>>>(B, pairs, n_pairs, gamma);
  } else {
    if (nt == 1) k_pairlist<float, 1><<<(unsigned)blocks, 256, 0, st>>>(B, pairs, n_pairs, gamma);
    else k_pairlist<float, 16><<<(unsigned)blocks, 256, 0, st>>>(B, pairs, n_pairs, gamma);
  }
}

// ---------------------------------------------------- batched launchers

void launch_targets_batched(const double *Y, const int64_t *yoff, const ScreenArgs *args, int n, int32_t ldy,
                            double *y64, float *y32, float *ysum32, int *err, cudaStream_t st) {
  if (n <= 0) return;
  note_launches(1);
  k_targets_batched<<<n, 256, 0, st>>>(Y, yoff, args, n, ldy, y64, y32, ysum32, err);
}

void launch_feature_batched(int prec64, const ScreenArgs *args, const Job *jobs, int n_jobs, unsigned int *counter,
                            int sms, cudaStream_t st) {
  if (n_jobs <= 0) return;
  const int blocks = std::min(sms * 8, (n_jobs + 7) / 8);
  note_launches(1);
  if (prec64) k_feature_batched<double><<<blocks, 256, 0, st>>>(args, jobs, n_jobs, counter);
  else k_feature_batched<float><<<blocks, 256, 0, st>>>(args, jobs, n_jobs, counter);
}

dse_status launch_pair_batched(int prec64, int kind, const ScreenArgs &A0, const ScreenArgs *args, int sms,
                               cudaStream_t st) {
  if (prec64)
    return kind == KIND_MUL ? launch_pair_t<double, KIND_MUL, 1, 2, 2, true>(A0, 0, sms, st, args)
                            : launch_pair_t<double, KIND_ADD, 1, 2, 2, true>(A0, 0, sms, st, args);
  return kind == KIND_MUL ? launch_pair_t<float, KIND_MUL, 1, 2, 2, true>(A0, 0, sms, st, args)
                          : launch_pair_t<float, KIND_ADD, 1, 2, 2, true>(A0, 0, sms, st, args);
}

void launch_pairlist_batched(int prec64, const ScreenArgs *args, const int2 *pairs, const Job *jobs, int n_jobs,
                             unsigned int *counter, int sms, cudaStream_t st) {
  if (n_jobs <= 0) return;
  const int blocks = std::min(sms * 8, (n_jobs + 7) / 8);
  note_launches(1);
  if (prec64) k_pairlist_batched<double><<<blocks, 256, 0, st>>>(args, pairs, jobs, n_jobs, counter);
  else k_pairlist_batched<float><<<blocks, 256, 0, st>>>(args, pairs, jobs, n_jobs, counter);
}

void launch_escalate(const ScreenArgs &A0, int sms, cudaStream_t st, const ScreenArgs *batch) {
  ScreenArgs A = A0;
  if (!batch && A.esc2_id && A.esc2_count && A.T <= 16 && A.N >= 4096 && A.F.v32 && A.y32 && A.ysum32 &&
      A.u > 1e-10f) {
    // (FP32 screens) the FP32 stage first; the FP64 kernels below take what
    // it left undecided (below 4096 samples the FP64 pass of a few hundred
    // candidates costs less than the stage's extra launches)
    if (cudaMemsetAsync(A.esc2_count, 0, sizeof(unsigned), st) == cudaSuccess) {
      note_launches(1);
      k_escalate32<<<sms * 4, 256, 0, st>>>(A0);
      A.esc_id = A.esc2_id;
      A.esc_count = A.esc2_count;
    } else {
      cudaGetLastError();  // (the FP64 kernels then take the whole list)
    }
  }
  note_launches(1);
  if (batch || A.T == 1) {
    k_escalate1<<<sms * 8, kEsc, 0, st>>>(A, batch);
  } else if (A.N >= 8192 && A.N <= kEscStashMax) {
    // (below 8192 samples the 128-thread blocks of k_escalate keep more
    // candidates in flight and win)
    static bool attr[64] = {false};
    int dev = 0;
    cudaGetDevice(&dev);
    if (!attr[dev & 63]) {
      cudaFuncSetAttribute(k_escalate_stash, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           (int)(kEscStashMax * sizeof(float)));
      attr[dev & 63] = true;
    }
    k_escalate_stash<<<sms * 2, kEscS, (size_t)A.N * sizeof(float), st>>>(A);
  } else {
    k_escalate<<<sms * 8, kEsc, 0, st>>>(A, batch);
  }
}

void launch_targets(const double *Y, int64_t ldY, int T, int64_t N, int32_t ldy, double *y64, float *y32,
                    float2 *ydf, float *ysum32, int *err, cudaStream_t st) {
  note_launches(1);
  k_targets<<<T, 256, 0, st>>>(Y, ldY, T, N, ldy, y64, y32, ydf, ysum32, err);
}

}  // namespace dse
