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
//     the FP64 operands) by at most u*W, W a per-candidate constant from the
//     operand magnitude bounds; the centred norm of the error vector is then
//     at most E = sqrt(N) u W, which bounds the error of sqrt(Sxx) directly
//     (triangle inequality) and of the numerator (Cauchy-Schwarz).
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

namespace dse {

template <typename R>
struct Num;
template <>
struct Num<float> {
  __device__ static float sqrt_(float x) { return sqrtf(x); }
  __device__ static float fma_(float a, float b, float c) { return fmaf(a, b, c); }
};
template <>
struct Num<double> {
  __device__ static double sqrt_(double x) { return sqrt(x); }
  __device__ static double fma_(double a, double b, double c) { return fma(a, b, c); }
};

// Centred-norm interval and realised decision of one candidate.
template <typename R>
struct CandInterval {
  R q;        // computed sqrt(Sxx)
  R q_lo, q_hi;
  R sqS2;     // sqrt(S2)
  R E;        // sqrt(N) u W
  int realised;  // 1 valid, 0 degenerate, 2 undecided
};

template <typename R>
__device__ __forceinline__ CandInterval<R> cand_interval(R S1, R S2, R N, R invN, R sqrtN, R c, R W, R gamma, R u,
                                                         R fmin) {
  CandInterval<R> o;
  const R mean = S1 * invN;
  const R Sxx = Num<R>::fma_(-S1, mean, S2);
  const R dSxx = (R(3) * gamma + R(6) * u) * S2 * R(1.01);
  o.E = sqrtN * u * W * R(1.01);
  o.q = Num<R>::sqrt_(Sxx > R(0) ? Sxx : R(0));
  const R lo2 = Sxx - dSxx;
  o.q_lo = Num<R>::sqrt_(lo2 > R(0) ? lo2 : R(0)) * (R(1) - R(4) * u) - o.E;
  o.q_hi = Num<R>::sqrt_(Sxx + dSxx) * (R(1) + R(4) * u) + o.E;
  o.sqS2 = Num<R>::sqrt_(S2);
  bool finite = isfinite(S1) && isfinite(S2) && isfinite(W);
  if (!finite) {
    o.realised = 2;
    return o;
  }
  if (fmin < R(0)) {
    o.realised = 1;
    return o;
  }
  // ||V||^2 = sum (w + c)^2 = S2 + 2 c S1 + N c^2
  const R ac = c < R(0) ? -c : c;
  const R Z = S2 + R(2) * c * S1 + N * c * c;
  const R dZ = (gamma + R(8) * u) * (S2 + R(2) * ac * sqrtN * o.sqS2 + N * c * c) * R(1.01);
  const R vlo2 = Z - dZ;
  const R V_lo = Num<R>::sqrt_(vlo2 > R(0) ? vlo2 : R(0)) * (R(1) - R(4) * u) - o.E;
  const R V_hi = Num<R>::sqrt_(Z + dZ) * (R(1) + R(4) * u) + o.E;
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

// ------------------------------------------------------ threshold filter

__device__ __forceinline__ unsigned ld_relaxed_u32(const unsigned *p) {
  unsigned v;
  asm volatile("ld.relaxed.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p));
  return v;
}

// Push (id, s, eps) into list `l` if s + eps reaches its threshold; warp-
// cooperative: every lane of the warp must call it (want = 0 to abstain).
// Returns whether this lane pushed.
__device__ __forceinline__ bool push_warp(const CandBufs &B, int l, bool want, uint64_t id, float s, float eps) {
  const unsigned lane = threadIdx.x & 31;
  float th = ld_relaxed(&B.theta[l]);
  bool p = want && (s + eps >= th);
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
    float lo = s - eps;
    int bin = lo > 0.f ? (int)(lo * (float)kNumBins) : 0;
    if (bin > kNumBins - 1) bin = kNumBins - 1;
    atomicAdd(&B.hist[(size_t)l * kNumBins + bin], 1u);
  }
  return p;
}

// Single-lane push (no warp cooperation).
__device__ __forceinline__ bool push_one(const CandBufs &B, int l, uint64_t id, float s, float eps) {
  float th = ld_relaxed(&B.theta[l]);
  if (!(s + eps >= th)) return false;
  unsigned pos = atomicAdd(&B.count[l], 1u);
  if ((int64_t)pos < B.cap) {
    size_t e = (size_t)l * (size_t)B.cap + pos;
    B.id[e] = id;
    B.score[e] = s;
    B.eps[e] = eps;
  }
  float lo = s - eps;
  int bin = lo > 0.f ? (int)(lo * (float)kNumBins) : 0;
  if (bin > kNumBins - 1) bin = kNumBins - 1;
  atomicAdd(&B.hist[(size_t)l * kNumBins + bin], 1u);
  return true;
}

// Raise list l's threshold to the lower edge of the highest bin b such that at
// least k entries have lower bound >= b / kNumBins.  Whole warp calls.
__device__ __forceinline__ void refresh_theta(const CandBufs &B, int l, int64_t k) {
  const int lane = threadIdx.x & 31;
  const unsigned *h = B.hist + (size_t)l * kNumBins;
  unsigned long long cum = 0;
  for (int top = kNumBins - 1; top >= 0; top -= 32) {
    int b = top - lane;
    unsigned v = b >= 0 ? ld_relaxed_u32(h + b) : 0u;
    unsigned long long x = v;
    for (int o = 1; o < 32; o <<= 1) {
      unsigned long long y = __shfl_up_sync(0xffffffffu, x, o);
      if (lane >= o) x += y;
    }
    unsigned ok = __ballot_sync(0xffffffffu, b >= 0 && cum + x >= (unsigned long long)k);
    if (ok) {
      int first = __ffs(ok) - 1;
      if (lane == 0) {
        int bb = top - first;
        if (bb > 0) atomic_max_nonneg(&B.theta[l], (float)bb / (float)kNumBins);
      }
      return;
    }
    cum += __shfl_sync(0xffffffffu, x, 31);
  }
}

}  // namespace dse
