// screen_common.cuh -- statistics, error bounds and the threshold filter shared
// by the screening kernels.
//
// SIS score of a candidate v against a centred, unit-norm target y:
//   r = |sum (v - vbar) y| / sqrt(sum (v - vbar)^2)
// (SISSO screening, the method the paper builds on; "Summary").  The kernels
// accumulate, over samples, S1 = sum w, S2 = sum w^2 and Sy_t = sum w y_t of a
// shifted value w = v - c (c a per-candidate constant near the mean, so that
// S2 - S1^2/N does not cancel), in the evaluation type R (float or double).
//
// Error bound (float path).  With u the unit roundoff of R:
//   * evaluation: every sample's w differs from the exact op(A, B) - c (A, B
//     the FP64 operands) by at most u * (kappa |V_s| + lambda_s), where kappa
//     counts the roundings of the operation (operand rounding, the op's own
//     documented ulp bound, the shifted FMA) and lambda_s collects the shift
//     and, for sums and differences, the operands' magnitudes; by Minkowski
//     the 2-norm of the error vector is at most E = u (kappa ||V|| + Lambda)
//     with ||V|| from the accumulated sums and Lambda from per-feature norms,
//     which bounds the error of sqrt(Sxx) directly (triangle inequality) and
//     of the numerator (Cauchy-Schwarz).
//   * accumulation: each sum is a sum of n terms in a fixed order with at most
//     `gamma` relative error on the sum of absolute terms (blocked summation,
//     gamma from the block structure); sum |w| <= sqrt(N S2), sum |w y| <=
//     sqrt(S2) ||y||.
// The score interval [r_lo, r_hi] (clamped to [0, 1]) follows, and
// eps = max(s - r_lo, r_hi - s) bounds the reported score's error against the
// FP64 value.  The realised test (std > fmin * rms) is decided on intervals
// of both sides; an undecidable case is escalated to FP64.
#pragma once

#include "dse_internal.cuh"
#include "eval64.cuh"

namespace dse {

template <typename R>
struct Num;
template <>
struct Num<float> {
  __device__ static float sqrt_(float x) { return sqrtf(x); }
  __device__ static float fma_(float a, float b, float c) { return fmaf(a, b, c); }
  __device__ static float sub_rd(float a, float b) { return __fsub_rd(a, b); }
  __device__ static float add_ru(float a, float b) { return __fadd_ru(a, b); }
  // 2^-90: a shifted sum of squares below N times this is within 2^36 of
  // the underflow threshold, where products that flushed (absolute error up
  // to 2^-126 each) are no longer negligible against the relative model
  __device__ static float tiny() { return 8.077935669463161e-28f; }
};
template <>
struct Num<double> {
  __device__ static double sqrt_(double x) { return sqrt(x); }
  __device__ static double fma_(double a, double b, double c) { return fma(a, b, c); }
  __device__ static double sub_rd(double a, double b) { return __dsub_rd(a, b); }
  __device__ static double add_ru(double a, double b) { return __dadd_ru(a, b); }
  __device__ static double tiny() { return 1.1754943508222875e-271; }  // 2^-900
};

// Centred-norm interval and realised decision of one candidate.
template <typename R>
struct CandInterval {
  R q;        // computed sqrt(Sxx)
  R q_lo, q_hi;
  R sqS2;     // sqrt(S2)
  R E;        // bound of the evaluation error vector's 2-norm
  int realised;  // 1 valid, 0 degenerate, 2 undecided
};

// Per-candidate evaluation-error coefficients: E = u (kappa ||V|| + lambda).
template <typename R>
struct EvalErr {
  R kappa, lambda;
};

template <typename R>
__device__ __forceinline__ CandInterval<R> cand_interval(R S1, R S2, R N, R invN, R sqrtN, R c, EvalErr<R> ee,
                                                         R gamma, R u, R fmin) {
  CandInterval<R> o;
  const R mean = S1 * invN;
  const R Sxx = Num<R>::fma_(-S1, mean, S2);
  const R dSxx = (R(3) * gamma + R(6) * u) * S2 * R(1.01);
  o.sqS2 = Num<R>::sqrt_(S2);
  // ||V||^2 = sum (w + c)^2 = S2 + 2 c S1 + N c^2 (of the computed values)
  const R ac = c < R(0) ? -c : c;
  const R Z = S2 + R(2) * c * S1 + N * c * c;
  const R dZ = (gamma + R(8) * u) * (S2 + R(2) * ac * sqrtN * o.sqS2 + N * c * c) * R(1.01);
  const R Vc_hi = Num<R>::sqrt_(Z + dZ) * (R(1) + R(4) * u);
  o.E = u * (ee.kappa * Vc_hi + ee.lambda) * R(1.02);
  o.q = Num<R>::sqrt_(Sxx > R(0) ? Sxx : R(0));
  const R lo2 = Sxx - dSxx;
  o.q_lo = Num<R>::sqrt_(lo2 > R(0) ? lo2 : R(0)) * (R(1) - R(4) * u) - o.E;
  o.q_hi = Num<R>::sqrt_(Sxx + dSxx) * (R(1) + R(4) * u) + o.E;
  // non-finite sums, or a column so small that underflow could hide in it:
  // undecided (the FP64 escalation decides)
  bool finite = isfinite(S1) && isfinite(S2) && isfinite(o.E) && S2 > N * Num<R>::tiny();
  if (!finite) {
    o.realised = 2;
    return o;
  }
  if (fmin < R(0)) {
    o.realised = 1;
    return o;
  }
  const R vlo2 = Z - dZ;
  const R V_lo = Num<R>::sqrt_(vlo2 > R(0) ? vlo2 : R(0)) * (R(1) - R(4) * u) - o.E;
  const R V_hi = Vc_hi + o.E;
  if (o.q_lo > fmin * V_hi * (R(1) + R(8) * u))
    o.realised = 1;
  else if (o.q_hi < fmin * (V_lo > R(0) ? V_lo : R(0)) * (R(1) - R(8) * u))
    o.realised = 0;
  else
    o.realised = 2;
  return o;
}

// Score and bound against one target.  ysum: sum of the target values used;
// ynorm: their 2-norm (1 up to rounding).
template <typename R>
__device__ __forceinline__ void cand_score(const CandInterval<R> &ci, R S1, R Sy, R invN, R ysum, R gamma, R u,
                                           R *s_out, R *eps_out) {
  const R P = Num<R>::fma_(-S1, ysum * invN, Sy);
  const R aP = P < R(0) ? -P : P;
  const R aS1 = S1 < R(0) ? -S1 : S1;
  const R ays = ysum < R(0) ? -ysum : ysum;
  const R dP = (gamma * ci.sqS2 * (R(1) + R(2) * u) + aS1 * invN * ays * (gamma + R(4) * u) + u * aP +
                ci.E * (R(1) + R(2) * u) + R(2) * u * ci.q_hi) *
               R(1.01);
  R s, eps;
  if (!(ci.q > R(0))) {
    s = R(0);
    eps = R(1);
  } else {
    s = aP / ci.q;
    R rlo = (aP - dP) / ci.q_hi;
    if (!(rlo > R(0))) rlo = R(0);
    R rhi = ci.q_lo > R(0) ? (aP + dP) / ci.q_lo : R(1);
    if (!(rhi < R(1))) rhi = R(1);
    if (s > R(1)) s = R(1);
    R e1 = s - rlo, e2 = rhi - s;
    eps = (e1 > e2 ? e1 : e2) * (R(1) + R(16) * u) + R(4e-12) * s;
    if (!(eps >= R(0))) eps = R(1);
  }
  *s_out = s;
  *eps_out = eps;
}

// Score interval against one target with a separate relative error factor
// for the numerator accumulation (the tensor-core path's contraction error);
// otherwise as cand_score.
template <typename R>
__device__ __forceinline__ void cand_score_num(const CandInterval<R> &ci, R S1, R Sy, R invN, R ysum, R gamma,
                                               R gamma_num, R u, R *s_out, R *eps_out) {
  const R P = Num<R>::fma_(-S1, ysum * invN, Sy);
  const R aP = P < R(0) ? -P : P;
  const R aS1 = S1 < R(0) ? -S1 : S1;
  const R ays = ysum < R(0) ? -ysum : ysum;
  const R dP = (gamma_num * ci.sqS2 * (R(1) + R(2) * u) + aS1 * invN * ays * (gamma + R(4) * u) + u * aP +
                ci.E * (R(1) + R(2) * u) + R(2) * u * ci.q_hi) *
               R(1.01);
  R s, eps;
  if (!(ci.q > R(0))) {
    s = R(0);
    eps = R(1);
  } else {
    s = aP / ci.q;
    R rlo = (aP - dP) / ci.q_hi;
    if (!(rlo > R(0))) rlo = R(0);
    R rhi = ci.q_lo > R(0) ? (aP + dP) / ci.q_lo : R(1);
    if (!(rhi < R(1))) rhi = R(1);
    if (s > R(1)) s = R(1);
    R e1 = s - rlo, e2 = rhi - s;
    eps = (e1 > e2 ? e1 : e2) * (R(1) + R(16) * u) + R(4e-12) * s;
    if (!(eps >= R(0))) eps = R(1);
  }
  *s_out = s;
  *eps_out = eps;
}

// Record the reason code a kernel assigned to candidate gid (in the first
// target pass; a screen re-run writes the same codes again).
__device__ __forceinline__ void note_why(const ScreenArgs &A, uint64_t gid, int reason) {
  if (A.why && A.first_pass && DSE_IN_BOUNDS(gid - A.id_begin, A.id_end - A.id_begin, A.err))
    A.why[gid - A.id_begin] = (int8_t)reason;
}

// Record the score interval a kernel computed for candidate gid in list l.
__device__ __forceinline__ void note_ivl(const ScreenArgs &A, uint64_t gid, int l, float s, float e) {
  if (A.ivl && DSE_IN_BOUNDS(gid - A.id_begin, A.id_end - A.id_begin, A.err) && DSE_IN_BOUNDS(l, A.n_lists, A.err))
    A.ivl[(gid - A.id_begin) * (uint64_t)A.n_lists + (uint64_t)l] = make_float2(s, e);
}

// ----------------------------------------------------- per-lane statistics

struct LaneStats {
  unsigned r[6];
  unsigned evaluated, escalated, seen;
  __device__ void zero() {
    for (int i = 0; i < 6; ++i) r[i] = 0;
    evaluated = escalated = seen = 0;
  }
};

// Warp-reduce the lane counters into the screen's statistics (whole warp).
__device__ __forceinline__ void flush_stats(const ScreenArgs &A, LaneStats &ls, int group = -1) {
  if (group < 0) group = A.group;
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
    if ((threadIdx.x & 31) == 0 && v) atomicAdd(&A.stats[ST_VALID_G0 + group], (unsigned long long)v);
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

// Queue a candidate for the FP64 decision of its realised test.
__device__ __forceinline__ void escalate(const ScreenArgs &A, uint64_t gid) {
  if (!A.first_pass) return;
  unsigned pos = atomicAdd(A.esc_count, 1u);
  if ((int64_t)pos < A.esc_cap) {
    A.esc_id[pos] = gid;
    if (A.esc_prob) A.esc_prob[pos] = (uint32_t)A.prob;
  } else
    atomicAdd(&A.stats[ST_ESC_OVERFLOW], 1ull);
}

// A-priori tests (unit, complexity, domain, magnitude) of the binary
// candidate op(ia, ib), exact: integer keys, flags, FP32 directed-rounding
// intervals with an FP64 fall-back when the interval straddles the limit.
// Also the evaluation-error coefficients of the evaluation with shift kk
// (a*b, a/b, b/a: the FMA constant; |a-b|: the subtracted constant) or, for
// a+b and a-b, centring means mi, mj:
//   a*b   fma(a, b, -c): operands rounded (2u |V|) and one rounding of the
//         shifted result (u (|V| + |c|))                 kappa 3, lambda |c| sqrt(N)
//   a/b   fma(a, rcp(b), -c): operands (2u), rcp.approx (2u), FMA rounding
//                                                         kappa 5, lambda |c| sqrt(N)
//   |a-b| rounded operands and difference (3u (|A|+|B|)), shift rounding
//                                                         kappa 0, lambda 3(||A||+||B||) + |c| sqrt(N)
//   a+-b  centred operands (2u|A| + u|mean|, likewise B) and the sum
//                                                         kappa 0, lambda 3(||A||+||B||) + 2(|mi|+|mj|) sqrt(N)
template <typename R>
__device__ __forceinline__ int binary_apriori_W(const ScreenArgs &A, int opc, int64_t ia, int64_t ib,
                                                const float4 &fa_a, const float4 &fa_b, R kk, R mi, R mj,
                                                EvalErr<R> *err_out) {
  const bool additive = opc == DSE_OP_ADD || opc == DSE_OP_SUB || opc == DSE_OP_ABSDIFF;
  int reason = DSE_VALID;
  EvalErr<R> ee{R(0), R(0)};
  if (additive && A.unit_check_addsub &&
      (A.F.ukey[2 * ia] != A.F.ukey[2 * ib] || A.F.ukey[2 * ia + 1] != A.F.ukey[2 * ib + 1]))
    reason = DSE_R_UNIT;
  else if (A.max_complexity > 0 && A.F.cplx[ia] + A.F.cplx[ib] + 1 > A.max_complexity)
    reason = DSE_R_COMPLEXITY;
  else if (rule_fails(A.F, opc, ia, ib))
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
    const R akk = kk < R(0) ? -kk : kk;
    const R sqrtN = Num<R>::sqrt_((R)A.N);
    const R na = (R)A.F.fnorm[ia], nb = (R)A.F.fnorm[ib];
    if (opc == DSE_OP_MUL) {
      ee.kappa = R(3.01);
      ee.lambda = akk * sqrtN;
    } else if (opc == DSE_OP_DIV || opc == DSE_OP_RDIV) {
      ee.kappa = R(5.01);
      ee.lambda = akk * sqrtN;
    } else if (opc == DSE_OP_ABSDIFF) {
      ee.kappa = R(0);
      ee.lambda = R(3.01) * (na + nb) + akk * sqrtN;
    } else {
      const R am = mi < R(0) ? -mi : mi, bm = mj < R(0) ? -mj : mj;
      ee.kappa = R(0);
      ee.lambda = R(3.01) * (na + nb) + R(2.01) * (am + bm) * sqrtN;
    }
  }
  *err_out = ee;
  return reason;
}

// ------------------------------------------- FP32 re-evaluation (one warp)
//
// The selection's FP32 re-score and the FP32 stage of the escalation
// evaluate a binary candidate again, one warp per candidate, in the screen's
// own FP32 evaluation forms (so binary_apriori_W's evaluation-error
// coefficients apply): float4 groups lane, lane + 32, ... of the operand rows
// and the targets; every kR32Block of a lane's samples form one FP32
// summation block whose totals are added into FP32 pairs (hi, lo); the lane
// totals meet in FP64 and are rounded to FP32 once.  The accumulation error
// on the sum of absolute terms is then at most (kR32Block - 1) u (the
// blocks), u (the pairs' residual, which gathers rounding errors of size u^2)
// and u (the final rounding), plus 2^-48 for the FP64 lane tree: gamma takes
// (kR32Block + 2) u with 5% to spare.
constexpr int kR32Block = 8;  // samples per summation block (two float4 groups)
constexpr float kGamma32 = (float)(kR32Block + 2) * 1.05f;  // units of u

// (hi, lo) += x, Knuth's two-sum with the error term gathered in lo
__device__ __forceinline__ void pair_acc(float &hi, float &lo, float x) {
  const float t = __fadd_rn(hi, x);
  const float z = __fsub_rn(t, hi);
  lo = __fadd_rn(lo, __fadd_rn(__fsub_rn(hi, __fsub_rn(t, z)), __fsub_rn(x, z)));
  hi = t;
}

// The screen's FP32 evaluation forms of the binary operators (shift kk for
// the products, quotients and |a-b|; centring means mi, mj for a+b, a-b).
template <int OP>
__device__ __forceinline__ float r32_value(float a, float b, float kk, float mi, float mj) {
  if (OP == DSE_OP_MUL) return __fmaf_rn(a, b, -kk);
  if (OP == DSE_OP_DIV) return __fmaf_rn(a, rcp_approx(b), -kk);
  if (OP == DSE_OP_RDIV) return __fmaf_rn(b, rcp_approx(a), -kk);
  if (OP == DSE_OP_ADD) return __fadd_rn(__fsub_rn(a, mi), __fsub_rn(b, mj));
  if (OP == DSE_OP_SUB) return __fsub_rn(__fsub_rn(a, mi), __fsub_rn(b, mj));
  return __fsub_rn(fabsf(__fsub_rn(a, b)), kk);  // |a-b|
}

// the unshifted value (for the shift estimate)
__device__ __forceinline__ float r32_plain(int op, float a, float b) {
  switch (op) {
    case DSE_OP_MUL: return __fmul_rn(a, b);
    case DSE_OP_DIV: return __fmul_rn(a, rcp_approx(b));
    case DSE_OP_RDIV: return __fmul_rn(b, rcp_approx(a));
    default: return fabsf(__fsub_rn(a, b));
  }
}

// the samples of a row's last float4 group past N read as zero
__device__ __forceinline__ void r32_zero_tail(float4 &v, int64_t i, int64_t n4, int rem) {
  if (rem == 0 || i != n4 - 1) return;
  if (rem == 1) v.y = 0.f;
  if (rem <= 2) v.z = 0.f;
  v.w = 0.f;
}

// One lane's samples: s[0] = sum w, s[1] = sum w^2, s[2 + t] = sum w y_t for
// the nt (<= NT) target rows y + t ldy; U float4 groups per step.
template <int OP, int NT, int U>
__device__ __forceinline__ void r32_pass(const float *ra, const float *rb, const float *y, int64_t ldy, int nt,
                                         int64_t N, float kk, float mi, float mj, float (&hi)[2 + NT],
                                         float (&lo)[2 + NT]) {
  constexpr int BQ = kR32Block / 4;  // float4 groups per block
  static_assert(kR32Block % 4 == 0 && (U % BQ == 0 || BQ % U == 0), "blocks of whole groups and steps");
  constexpr int STEPS = BQ > U ? BQ / U : 1;  // steps per block (blocks of several steps)
  const int lane = threadIdx.x & 31;
  const int64_t n4 = (N + 3) >> 2;
  const int rem = (int)(N & 3);
  const float4 *xa = reinterpret_cast<const float4 *>(ra), *xb = reinterpret_cast<const float4 *>(rb);
  float acc[2 + NT];
#pragma unroll
  for (int k = 0; k < 2 + NT; ++k) acc[k] = 0.f;
  int nb = 0;
  for (int64_t i0 = lane; i0 < n4; i0 += 32 * U) {
    float4 av[U], bv[U], yv[U][NT];
#pragma unroll
    for (int q = 0; q < U; ++q) {
      const int64_t i = i0 + 32 * q;
      const bool in = i < n4;
      av[q] = in ? __ldg(xa + i) : make_float4(0.f, 0.f, 0.f, 0.f);
      bv[q] = in ? __ldg(xb + i) : make_float4(0.f, 0.f, 0.f, 0.f);
#pragma unroll
      for (int t = 0; t < NT; ++t) {
        yv[q][t] = in && t < nt ? __ldg(reinterpret_cast<const float4 *>(y + (int64_t)t * ldy) + i)
                                : make_float4(0.f, 0.f, 0.f, 0.f);
        r32_zero_tail(yv[q][t], i, n4, rem);
      }
    }
#pragma unroll
    for (int q = 0; q < U; ++q) {
      const int64_t s = (i0 + 32 * q) * 4;
      const float ae[4] = {av[q].x, av[q].y, av[q].z, av[q].w};
      const float be[4] = {bv[q].x, bv[q].y, bv[q].z, bv[q].w};
#pragma unroll
      for (int e = 0; e < 4; ++e) {
        float w = r32_value<OP>(ae[e], be[e], kk, mi, mj);
        w = s + e < N ? w : 0.f;  // padding and groups past the row: no term
        acc[0] = __fadd_rn(acc[0], w);
        acc[1] = __fmaf_rn(w, w, acc[1]);
#pragma unroll
        for (int t = 0; t < NT; ++t) {
          const float yy = e == 0 ? yv[q][t].x : e == 1 ? yv[q][t].y : e == 2 ? yv[q][t].z : yv[q][t].w;
          acc[2 + t] = __fmaf_rn(w, yy, acc[2 + t]);
        }
      }
      if (BQ <= U && (q + 1) % BQ == 0) {  // a block ends inside the step
#pragma unroll
        for (int k = 0; k < 2 + NT; ++k) {
          pair_acc(hi[k], lo[k], acc[k]);
          acc[k] = 0.f;
        }
      }
    }
    if (BQ > U && ++nb == STEPS) {
      nb = 0;
#pragma unroll
      for (int k = 0; k < 2 + NT; ++k) {
        pair_acc(hi[k], lo[k], acc[k]);
        acc[k] = 0.f;
      }
    }
  }
#pragma unroll
  for (int k = 0; k < 2 + NT; ++k) pair_acc(hi[k], lo[k], acc[k]);
}

// An FP32 re-evaluation's constants.
struct R32Setup {
  float kk, mi, mj, cshift;
  EvalErr<float> ee;
};

// Whole warp.  False when the re-evaluation does not apply: an operator
// outside the six binary ones, operands outside the FP32-safe range, or an
// a-priori test that is not valid.  Else the shift kk of a*b, a/b, b/a and
// |a-b| (the mean of the first, up to 32, values, so that the shifted sum of
// squares stays close to the centred one), the centring means of a+b and
// a-b, the shift of the sums and the evaluation-error coefficients.
__device__ __forceinline__ bool r32_setup(const ScreenArgs &A, int op, int64_t a, int64_t b, R32Setup &o) {
  const bool binop = op == DSE_OP_MUL || op == DSE_OP_DIV || op == DSE_OP_RDIV || op == DSE_OP_ADD ||
                     op == DSE_OP_SUB || op == DSE_OP_ABSDIFF;
  if (!binop || b < 0 || !DSE_OPERANDS_OK(A.F, a, b, A.err)) return false;
  if (!((A.F.flags[a] & A.F.flags[b]) & F_FP32_SAFE)) return false;
  const int lane = threadIdx.x & 31;
  const int64_t N = A.N;
  const float4 fa_a = A.F.fa[a], fa_b = A.F.fa[b];
  o.mi = fa_a.x;
  o.mj = fa_b.x;
  o.kk = 0.f;
  if (op != DSE_OP_ADD && op != DSE_OP_SUB) {
    float v0 = lane < N ? r32_plain(op, A.F.v32[a * A.F.ld + lane], A.F.v32[b * A.F.ld + lane]) : 0.f;
    for (int k = 16; k > 0; k >>= 1) v0 += __shfl_xor_sync(0xffffffffu, v0, k);
    o.kk = v0 / (float)(N < 32 ? N : 32);
    if (!isfinite(o.kk)) o.kk = 0.f;
  }
  o.cshift = op == DSE_OP_ADD ? o.mi + o.mj : op == DSE_OP_SUB ? o.mi - o.mj : o.kk;
  return binary_apriori_W<float>(A, op, a, b, fa_a, fa_b, o.kk, o.mi, o.mj, &o.ee) == DSE_VALID;
}

// The warp's sums (every lane gets them), rounded to FP32 once.
template <int OP, int NT, int U>
__device__ __forceinline__ void r32_sums_op(const ScreenArgs &A, int64_t a, int64_t b, const float *y, int nt,
                                            const R32Setup &c, float (&S)[2 + NT]) {
  float hi[2 + NT], lo[2 + NT];
#pragma unroll
  for (int k = 0; k < 2 + NT; ++k) hi[k] = lo[k] = 0.f;
  r32_pass<OP, NT, U>(A.F.v32 + a * A.F.ld, A.F.v32 + b * A.F.ld, y, A.ldy, nt, A.N, c.kk, c.mi, c.mj, hi, lo);
#pragma unroll
  for (int k = 0; k < 2 + NT; ++k) {
    double d = (double)hi[k] + (double)lo[k];
    for (int o = 16; o > 0; o >>= 1) d += __shfl_xor_sync(0xffffffffu, d, o);
    S[k] = (float)d;
  }
}

template <int NT, int U>
__device__ __forceinline__ void r32_sums(const ScreenArgs &A, int op, int64_t a, int64_t b, const float *y, int nt,
                                         const R32Setup &c, float (&S)[2 + NT]) {
  switch (op) {
    case DSE_OP_MUL: r32_sums_op<DSE_OP_MUL, NT, U>(A, a, b, y, nt, c, S); break;
    case DSE_OP_DIV: r32_sums_op<DSE_OP_DIV, NT, U>(A, a, b, y, nt, c, S); break;
    case DSE_OP_RDIV: r32_sums_op<DSE_OP_RDIV, NT, U>(A, a, b, y, nt, c, S); break;
    case DSE_OP_ADD: r32_sums_op<DSE_OP_ADD, NT, U>(A, a, b, y, nt, c, S); break;
    case DSE_OP_SUB: r32_sums_op<DSE_OP_SUB, NT, U>(A, a, b, y, nt, c, S); break;
    default: r32_sums_op<DSE_OP_ABSDIFF, NT, U>(A, a, b, y, nt, c, S); break;
  }
}

// ------------------------------------------------------ threshold filter

__device__ __forceinline__ unsigned ld_relaxed_u32(const unsigned *p) {
  unsigned v;
  asm volatile("ld.relaxed.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p));
  return v;
}

// Edges of a buffered entry's interval [s - eps, s + eps], rounded outwards
// (toward -inf / +inf) so that the FP32 edges still enclose the exact
// interval when eps is within a few ulp of s.  The histograms, the push test
// and the selection all take the edges from these two functions.
__device__ __forceinline__ float iv_lo(float s, float eps) { return __fsub_rd(s, eps); }
__device__ __forceinline__ float iv_hi(float s, float eps) { return __fadd_ru(s, eps); }

// Histogram counts of a buffered entry's lower and upper bounds.
__device__ __forceinline__ void count_bounds(const CandBufs &B, int l, float s, float eps) {
  const int bl = score_bin(iv_lo(s, eps)), bh = score_bin(iv_hi(s, eps));
  atomicAdd(&B.hist[(size_t)l * kNumBins + bl], 1u);
  atomicAdd(&B.hist_c[(size_t)l * kCoarse + bl / kFine], 1u);
  atomicAdd(&B.hist_hi[(size_t)l * kNumBins + bh], 1u);
}

// Push (id, s, eps) into list `l` if its upper edge reaches the threshold; warp-
// cooperative: every lane of the warp must call it (want = 0 to abstain).
// Returns whether this lane pushed.
__device__ __forceinline__ bool push_warp(const CandBufs &B, int l, bool want, uint64_t id, float s, float eps) {
  const unsigned lane = threadIdx.x & 31;
  float th = ld_relaxed(&B.theta[l]);
  bool p = want && (iv_hi(s, eps) >= th);
  unsigned m = __ballot_sync(0xffffffffu, p);
  if (!m) return false;
  unsigned base = 0;
  int leader = __ffs(m) - 1;
  if ((int)lane == leader) base = atomicAdd(&B.count[l], (unsigned)__popc(m));
  base = __shfl_sync(0xffffffffu, base, leader);
  if (p) {
    unsigned pos = base + __popc(m & ((1u << lane) - 1u));
    if ((int64_t)pos < B.cap) {
      size_t e = (size_t)l * (size_t)B.cap + pos;
      B.id[e] = id;
      B.score[e] = s;
      B.eps[e] = eps;
    }
    count_bounds(B, l, s, eps);
  }
  return p;
}

// Warp-staged pushes: a warp collects the candidates that reach the list's
// threshold in a shared-memory stage and writes them out with one slot
// reservation per flush, instead of one atomic round trip per batch of 32
// candidates (the same entries and bound counts as push_warp; the threshold
// is the one the caller read, refreshed by it between tiles).
template <int CAP>
struct PushStage {
  uint64_t id[CAP];
  float s[CAP], e[CAP];
};

// count_bounds for the active lanes of a warp, one atomic per distinct bin
// (entries of a flush cluster near the threshold, so bins repeat).
__device__ __forceinline__ void count_bounds_warp(const CandBufs &B, int l, bool active, float s, float eps) {
  const unsigned act = __ballot_sync(0xffffffffu, active);
  if (!active) return;
  const int lane = threadIdx.x & 31;
  const int bl = score_bin(iv_lo(s, eps)), bh = score_bin(iv_hi(s, eps)), bc = bl / kFine;
  const unsigned gl = __match_any_sync(act, bl), gc = __match_any_sync(act, bc), gh = __match_any_sync(act, bh);
  if (lane == __ffs(gl) - 1) atomicAdd(&B.hist[(size_t)l * kNumBins + bl], (unsigned)__popc(gl));
  if (lane == __ffs(gc) - 1) atomicAdd(&B.hist_c[(size_t)l * kCoarse + bc], (unsigned)__popc(gc));
  if (lane == __ffs(gh) - 1) atomicAdd(&B.hist_hi[(size_t)l * kNumBins + bh], (unsigned)__popc(gh));
}

template <int CAP>
__device__ __forceinline__ void stage_flush(const CandBufs &B, int l, PushStage<CAP> &st, int n) {
  __syncwarp();
  if (n <= 0) return;
  const unsigned lane = threadIdx.x & 31;
  unsigned base = 0;
  if (lane == 0) base = atomicAdd(&B.count[l], (unsigned)n);
  base = __shfl_sync(0xffffffffu, base, 0);
  for (int i0 = 0; i0 < n; i0 += 32) {
    const int i = i0 + (int)lane;
    const bool act = i < n;
    float s = 0.f, e = 0.f;
    if (act) {
      const unsigned pos = base + (unsigned)i;
      s = st.s[i];
      e = st.e[i];
      if ((int64_t)pos < B.cap) {
        const size_t x = (size_t)l * (size_t)B.cap + pos;
        B.id[x] = st.id[i];
        B.score[x] = s;
        B.eps[x] = e;
      }
    }
    count_bounds_warp(B, l, act, s, e);
  }
  __syncwarp();
}

// Warp-cooperative (every lane calls it); n: the stage's fill (warp-uniform),
// returned updated; *total counts the warp's pushes.
template <int CAP>
__device__ __forceinline__ int stage_push(const CandBufs &B, int l, PushStage<CAP> &st, int n, int *total, float th,
                                          bool want, uint64_t id, float s, float eps) {
  static_assert(CAP >= 32, "a stage holds at least one warp's pushes");
  const unsigned lane = threadIdx.x & 31;
  const bool p = want && (iv_hi(s, eps) >= th);
  const unsigned m = __ballot_sync(0xffffffffu, p);
  if (!m) return n;
  const int c = __popc(m);
  *total += c;
  if (n + c > CAP) {
    stage_flush(B, l, st, n);
    n = 0;
  }
  if (p) {
    const int pos = n + __popc(m & ((1u << lane) - 1u));
    st.id[pos] = id;
    st.s[pos] = s;
    st.e[pos] = eps;
  }
  return n + c;
}

// Single-lane push (no warp cooperation).
__device__ __forceinline__ bool push_one(const CandBufs &B, int l, uint64_t id, float s, float eps) {
  float th = ld_relaxed(&B.theta[l]);
  if (!(iv_hi(s, eps) >= th)) return false;
  unsigned pos = atomicAdd(&B.count[l], 1u);
  if ((int64_t)pos < B.cap) {
    size_t e = (size_t)l * (size_t)B.cap + pos;
    B.id[e] = id;
    B.score[e] = s;
    B.eps[e] = eps;
  }
  count_bounds(B, l, s, eps);
  return true;
}

// Warp-wide scan of `n` (multiple of 32) counters from the top: the highest
// index b with cum + sum(h[b..n)) >= k, or -1; *cum_out gets the sum above b.
__device__ __forceinline__ int scan_top(const unsigned *h, int n, unsigned long long cum, unsigned long long k,
                                        unsigned long long *cum_out) {
  const int lane = threadIdx.x & 31;
  for (int top = n - 1; top >= 0; top -= 32) {
    const int b = top - lane;
    const unsigned v = b >= 0 ? ld_relaxed_u32(h + b) : 0u;
    unsigned long long x = v;
    for (int o = 1; o < 32; o <<= 1) {
      unsigned long long y = __shfl_up_sync(0xffffffffu, x, o);
      if (lane >= o) x += y;
    }
    const unsigned ok = __ballot_sync(0xffffffffu, b >= 0 && cum + x >= k);
    if (ok) {
      const int first = __ffs(ok) - 1;
      const unsigned long long before = __shfl_sync(0xffffffffu, x - v, first);
      *cum_out = cum + before;
      return top - first;
    }
    cum += __shfl_sync(0xffffffffu, x, 31);
  }
  *cum_out = cum;
  return -1;
}

// Raise list l's threshold to the lower edge of the highest bin b such that at
// least k entries have lower bound >= b / kNumBins (coarse bins first, then
// the fine bins of the crossing coarse bin).  Whole warp calls.
__device__ __forceinline__ void refresh_theta(const CandBufs &B, int l, int64_t k) {
  unsigned long long above = 0, above2 = 0;
  const int c = scan_top(B.hist_c + (size_t)l * kCoarse, kCoarse, 0ull, (unsigned long long)k, &above);
  if (c < 0) return;
  const int f = scan_top(B.hist + (size_t)l * kNumBins + c * kFine, kFine, above, (unsigned long long)k, &above2);
  if (f < 0) return;
  const int bb = c * kFine + f;
  if ((threadIdx.x & 31) == 0 && bb > 0) atomic_max_nonneg(&B.theta[l], (float)bb / (float)kNumBins);
}

}  // namespace dse
