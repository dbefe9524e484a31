// gram.cuh -- shared parts of the Gram-contraction screens (one target:
// screen_gram.cu; 2..16 targets and any N: screen_gmt.cu): the per-feature
// sums of the centred FP32 rows, the BF16 hi/lo row images, and the
// epilogue arithmetic that turns contraction entries into the a-priori
// decisions, score intervals and realised decisions of the candidates.
#pragma once

#include <cuda_bf16.h>
#include <math.h>

#include "dse_internal.cuh"
#include "eval64.cuh"
#include "screen_common.cuh"
#include "tcgen05.cuh"

namespace dse {
namespace gram {

// What the epilogue reads of a feature, copied once per tile into the warp's
// own shared-memory cache (5 a-features + the b-features of its patches).
struct EpiFeat {
  float4 fa;     // {mean, mean of 1/x, RU max|x|, RD max|x|}
  float2 fr;     // {RU 1/min|x|, RD 1/min|x|}
  uint32_t flags;
  int32_t cplx;
  float c[2], s1[2], s2[2], n1[2], n2[2], nu[2];  // GramFeat
  float sy[2], ny[2];                             // GramTgt
  uint64_t uk[2];                                 // packed unit key
};

}  // namespace gram

// Per-feature sums of the centred FP32 rows, family 0 = x, 1 = 1/x.
struct GramFeat {
  float c[2];   // centring constants (the FP32 means of x and of 1/x)
  float s1[2];  // sum p
  float s2[2];  // sum p^2
  float n1[2];  // RU |p|_2
  float n2[2];  // RU |p^2|_2
  float nu[2];  // RU |x|_2 and |1/x|_2 (uncentred)
  int ok[2];    // rows usable: FP32-safe values (and min |x| > 0 for 1/x)
  int pad[2];
};
// Target part: sum p y and RU |p y|_2 per family.
struct GramTgt {
  float sy[2];
  float ny[2];
};

// ------------------------------------------------------------- row images

// Centred values of feature f at samples s0 .. s0+7 (zero past N or when the
// family's rows are unusable).
__device__ __forceinline__ void gram_vals(const FeatTable &F, int64_t f, int64_t s0, int fam, float c, bool ok,
                                          float (&p)[8]) {
  if (ok && s0 + 8 <= F.N) {
    // a whole group: two 16-byte loads (rows are 16-byte aligned: ld is a
    // multiple of 4, s0 of 8)
    const float4 *src = reinterpret_cast<const float4 *>(F.v32 + f * F.ld + s0);
    const float4 a = src[0], b = src[1];
    const float x[8] = {a.x, a.y, a.z, a.w, b.x, b.y, b.z, b.w};
#pragma unroll
    for (int e = 0; e < 8; ++e) p[e] = (fam == 0 ? x[e] : __frcp_rn(x[e])) - c;
    return;
  }
#pragma unroll
  for (int e = 0; e < 8; ++e) {
    const int64_t s = s0 + e;
    float v = 0.f;
    if (ok && s < F.N) {
      const float x = F.v32[f * F.ld + s];
      v = (fam == 0 ? x : __frcp_rn(x)) - c;
    }
    p[e] = v;
  }
}

// 8 FP32 values as BF16 hi and lo parts, 16 bytes each.
__device__ __forceinline__ void split8(const float (&v)[8], uint4 &hi, uint4 &lo) {
  uint32_t h[4], l[4];
#pragma unroll
  for (int e = 0; e < 8; e += 2) {
    const __nv_bfloat162 hh = __floats2bfloat162_rn(v[e], v[e + 1]);
    const __nv_bfloat162 ll = __floats2bfloat162_rn(v[e] - __low2float(hh), v[e + 1] - __high2float(hh));
    h[e >> 1] = *reinterpret_cast<const uint32_t *>(&hh);
    l[e >> 1] = *reinterpret_cast<const uint32_t *>(&ll);
  }
  hi = make_uint4(h[0], h[1], h[2], h[3]);
  lo = make_uint4(l[0], l[1], l[2], l[3]);
}

// Compensated FP32 accumulation (TwoSum: s + c carries the exact sum of
// the terms to a few units in the last place of the result).
struct Comp32 {
  float s = 0.f, c = 0.f;
  __device__ __forceinline__ void add(float x) {
    const float t = s + x;
    const float z = t - s;
    c += (s - (t - z)) + (x - z);
    s = t;
  }
  __device__ __forceinline__ double value() const { return (double)s + (double)c; }
};

// Sum of v over the block, in thread 0 (the other threads keep their
// warp's sums).
template <int NV>
__device__ __forceinline__ void gram_block_sum(double (&v)[NV], double *sm) {
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
#pragma unroll
  for (int i = 0; i < NV; ++i) v[i] = warp_sum64(v[i]);
  __syncthreads();
  if (lane == 0)
#pragma unroll
    for (int i = 0; i < NV; ++i) sm[w * NV + i] = v[i];
  __syncthreads();
  if (threadIdx.x == 0) {  // the totals are used by thread 0 only (FP64 adds are slow on this part)
#pragma unroll
    for (int i = 0; i < NV; ++i) {
      double t = 0.0;
      for (int q = 0; q < (int)(blockDim.x >> 5); ++q) t += sm[q * NV + i];
      v[i] = t;
    }
  }
}

// A feature's GramFeat sums, accumulated per thread over its 8-sample
// groups and combined over the block: per family the compensated sums of p
// and p^2, and plain FP32 sums of p^4 and (c + p)^2 (they only bound norms,
// with a margin for their rounding).
struct GramFeatAcc {
  Comp32 cs1[2], cs2[2];
  float s4[2] = {0.f, 0.f}, su2[2] = {0.f, 0.f};

  // the 8 centred values p (and their squares p2) of family fam at samples
  // s0 .. s0+7
  __device__ __forceinline__ void add(int fam, const float (&p)[8], const float (&p2)[8], bool ok, float c, int64_t s0,
                                      int64_t N) {
#pragma unroll
    for (int e = 0; e < 8; ++e) {
      cs1[fam].add(p[e]);
      cs2[fam].add(p2[e]);
      s4[fam] = fmaf(p2[e], p2[e], s4[fam]);
      const float uv = (ok && s0 + e < N) ? p[e] + c : 0.f;
      su2[fam] = fmaf(uv, uv, su2[fam]);
    }
  }

  // Block-wide (every thread calls it; sm: 4 warps x 10 doubles); thread 0
  // writes the record.  groups: the 8-sample groups of the sample range.
  __device__ __forceinline__ void finish(double *sm, int64_t groups, const float (&c)[2], const bool (&ok)[2],
                                         GramFeat *out) {
    double acc[10] = {cs1[0].value(), cs2[0].value(), (double)s4[0], (double)su2[0], 0.0,
                      cs1[1].value(), cs2[1].value(), (double)s4[1], (double)su2[1], 0.0};
    gram_block_sum<10>(acc, sm);
    if (threadIdx.x == 0) {
      GramFeat o{};
      for (int fam = 0; fam < 2; ++fam) {
        o.c[fam] = c[fam];
        o.s1[fam] = (float)acc[5 * fam + 0];
        o.s2[fam] = (float)acc[5 * fam + 1];
        // the FP32 partial sums of squares are low by at most (terms per
        // thread + 2) u of themselves
        const double marg = 1.0 + ((double)groups * 8.0 / blockDim.x + 10.0) * 5.9604644775390625e-8;
        o.n1[fam] = __double2float_ru(sqrt(acc[5 * fam + 1] * marg) * (1.0 + 1e-15));
        o.n2[fam] = __double2float_ru(sqrt(acc[5 * fam + 2] * marg) * (1.0 + 1e-15));
        o.nu[fam] = __double2float_ru(sqrt(acc[5 * fam + 3] * marg) * (1.0 + 1e-15));
        o.ok[fam] = ok[fam] ? 1 : 0;
      }
      *out = o;
    }
  }
};

// ------------------------------------------------------------- epilogue math

struct GramCand {
  float s, eps;
  int realised;  // 1 valid, 0 degenerate, 2 undecided (escalate)
};

// Error bounds of the contraction entries of a pair.  Each entry's error
// is at most delta sum_s |a_s b_s| (the BF16x3 split, the accumulation model
// and the rounding of the rows are all relative to each term).  Two upper
// bounds of sum |a_s b_s| are taken and the smaller one used: the
// Cauchy-Schwarz product of the rows' norms, and bounds through G22 = sum
// p^2 q^2, whose terms are all nonnegative so that its computed value
// bounds its own error (G22 <= G22~ / (1 - delta)):
//   sum |p q| <= sqrt(N G22),  sum |p q^2| <= sqrt(G22) |q|,
//   sum |p^2 q| <= sqrt(G22) |p|,  sum |p q y| <= sqrt(G22) |y|  (|y| = 1).
// The second kind is much tighter for spiky rows (large values of p and q
// at different samples), where the norms' product overstates the terms.
struct GramErr {
  float dG11, dG22, dG12, dG21, h;  // h: bound of sum |p q y| for a unit y
};
__device__ __forceinline__ GramErr gram_err(float delta, float G22, float n1u, float n2u, float n1w, float n2w,
                                            float N) {
  GramErr o;
  const float g22 = fmaxf(G22, 0.f) * (1.f + 2.f * delta) * (1.f + 1.2e-7f);
  const float r = sqrtf(g22) * (1.f + 2.4e-7f);
  o.dG22 = delta * fminf(n2u * n2w, g22);
  o.dG11 = delta * fminf(n1u * n1w, sqrtf(N * g22) * (1.f + 2.4e-7f));
  o.dG12 = delta * fminf(n1u * n2w, r * n1w);
  o.dG21 = delta * fminf(n2u * n1w, r * n1u);
  o.h = r * (1.f + 4.8e-7f);
  return o;
}

__device__ __forceinline__ GramCand gram_finish(float S1, float dS1, float S2, float dS2, float Sy, float dSy,
                                                float Z, float dZ, float Vhi, float E, float N, float invN,
                                                float ysum, float fmin);

// Score interval of v = u w from the contraction entries (G11, G22, G12,
// G21, H) and the two features' sums; family fu of the a-feature, fw of the
// b-feature; kappa of the evaluation error.
// (The cached records are read in place: a run-time family index into a
// register copy would live in local memory.)
__device__ __forceinline__ GramCand gram_score(const gram::EpiFeat *Fa, int fu, const gram::EpiFeat *Fb, int fw,
                                               float G11, float G22, float G12, float G21, float H, float kappa,
                                               float delta, float N, float invN, float ysum, float fmin) {
  const float u = 5.9604644775390625e-8f;
  const float cu = Fa->c[fu], cw = Fb->c[fw];
  const float P1 = Fa->s1[fu], P2 = Fa->s2[fu], PY = Fa->sy[fu];
  const float Q1 = Fb->s1[fw], Q2 = Fb->s2[fw], QY = Fb->sy[fw];
  // statistics of v - k, k = cu cw
  const float t1a = cu * Q1, t1b = cw * P1;
  const float S1 = t1a + t1b + G11;
  const float cucw = cu * cw;
  const float t2a = cu * cu * Q2, t2b = cw * cw * P2, t2c = 2.f * cucw * G11, t2d = 2.f * cu * G12,
              t2e = 2.f * cw * G21;
  const float S2 = t2a + t2b + G22 + t2c + t2d + t2e;
  const float tya = cu * QY, tyb = cw * PY;
  const float Sy = tya + tyb + H;
  // error bounds of the three sums
  const float acu = fabsf(cu), acw = fabsf(cw);
  const GramErr ge = gram_err(delta, G22, Fa->n1[fu], Fa->n2[fu], Fb->n1[fw], Fb->n2[fw], N);
  const float dG11 = ge.dG11, dG22 = ge.dG22, dG12 = ge.dG12, dG21 = ge.dG21;
  const float dH = delta * fminf(Fa->ny[fu] * Fb->n1[fw], ge.h);
  const float dS1 = (dG11 + 10.f * u * (fabsf(t1a) + fabsf(t1b) + fabsf(G11))) * 1.01f;
  const float dS2 = (dG22 + 2.f * acu * acw * dG11 + 2.f * acu * dG12 + 2.f * acw * dG21 +
                     12.f * u * (t2a + t2b + fabsf(G22) + fabsf(t2c) + fabsf(t2d) + fabsf(t2e))) *
                    1.01f;
  // (the target sums come from the rounded products p y: u |p|_2 each)
  const float dSy =
      (dH + 10.f * u * (fabsf(tya) + fabsf(tyb) + fabsf(H)) + 1.01f * u * (acu * Fb->n1[fw] + acw * Fa->n1[fu])) *
      1.01f;
  // uncentred norm of v: Z = S2 + 2 k S1 + N k^2
  const float Z = S2 + 2.f * cucw * S1 + N * cucw * cucw;
  const float dZ = (dS2 + 2.f * fabsf(cucw) * dS1 + 10.f * u * (fabsf(S2) + 2.f * fabsf(cucw * S1) + N * cucw * cucw)) *
                   1.01f;
  const float Vhi = sqrtf(Z + dZ) * (1.f + 4.f * u);
  const float E = u * (kappa * Vhi + 1.01f * (acw * Fa->nu[fu] + acu * Fb->nu[fw])) * 1.02f;
  return gram_finish(S1, dS1, S2, dS2, Sy, dSy, Z, dZ, Vhi, E, N, invN, ysum, fmin);
}

// Target-independent part of a candidate's interval: the centred sum of
// squares Sxx = S2 - S1^2/N with its bound, q = sqrt(Sxx) with bounds
// [q_lo, q_hi] (E, the evaluation error vector's norm, included) and the
// realised decision (1 valid, 0 degenerate, 2 undecided: escalate).
struct GramVar {
  float S1, dS1, q, q_lo, q_hi, E;
  int realised;
};

// From the assembled statistics of a candidate and their error bounds: S1,
// S2 of v - k with bounds dS1, dS2, the uncentred norm Z = |v|^2 with bound
// dZ and Vhi >= |v|, and E the bound of the evaluation error vector's 2-norm.
__device__ __forceinline__ GramVar gram_var(float S1, float dS1, float S2, float dS2, float Z, float dZ, float Vhi,
                                            float E, float N, float invN, float fmin) {
  const float u = 5.9604644775390625e-8f;
  GramVar o;
  o.S1 = S1;
  o.dS1 = dS1;
  o.E = E;
  const float mean = S1 * invN;
  const float Sxx = fmaf(-S1, mean, S2);
  const float aS1 = fabsf(S1);
  const float dSxx = (dS2 + (2.f * aS1 * dS1 + dS1 * dS1) * invN + 6.f * u * (fabsf(S2) + aS1 * fabsf(mean))) * 1.01f;
  o.q = sqrtf(Sxx > 0.f ? Sxx : 0.f);
  const float lo2 = Sxx - dSxx;
  o.q_lo = sqrtf(lo2 > 0.f ? lo2 : 0.f) * (1.f - 4.f * u) - E;
  o.q_hi = sqrtf(Sxx + dSxx) * (1.f + 4.f * u) + E;
  // (a column within 2^36 of FP32 underflow, where flushed products escape
  // the relative error model, is undecided too)
  if (!(isfinite(S1) && isfinite(S2) && isfinite(Z) && isfinite(E) && isfinite(o.q_hi) &&
        S2 > N * 8.077935669463161e-28f)) {
    o.realised = 2;
    return o;
  }
  o.realised = 1;
  if (fmin >= 0.f) {
    const float vlo2 = Z - dZ;
    const float V_lo = sqrtf(vlo2 > 0.f ? vlo2 : 0.f) * (1.f - 4.f * u) - E;
    const float V_hi = Vhi + E;
    if (o.q_lo > fmin * V_hi * (1.f + 8.f * u))
      o.realised = 1;
    else if (o.q_hi < fmin * (V_lo > 0.f ? V_lo : 0.f) * (1.f - 8.f * u))
      o.realised = 0;
    else
      o.realised = 2;
  }
  return o;
}

// Score and bound for one target from the target-independent part and the
// target's sum Sy = sum (v - k) y with bound dSy: the numerator P = Sy -
// S1 ysum / N and its bound (the FP32 target is the unit-norm FP64 target to
// u per sample: 2u q_hi), s = |P| / q and the half-width of [rlo, rhi].
__device__ __forceinline__ void gram_num(const GramVar &v, float Sy, float dSy, float invN, float ysum, float *s_out,
                                         float *eps_out) {
  const float u = 5.9604644775390625e-8f;
  const float P = fmaf(-v.S1, ysum * invN, Sy);
  const float aP = fabsf(P);
  const float ays = fabsf(ysum);
  const float aS1 = fabsf(v.S1);
  const float dP = (dSy + ays * invN * v.dS1 + 6.f * u * (fabsf(Sy) + aS1 * ays * invN) + v.E * (1.f + 2.f * u) +
                    2.f * u * v.q_hi + u * aP) *
                   1.01f;
  if (!(v.q > 0.f)) {
    *s_out = 0.f;
    *eps_out = 1.f;
    return;
  }
  float s = aP / v.q;
  float rlo = (aP - dP) / v.q_hi;
  if (!(rlo > 0.f)) rlo = 0.f;
  float rhi = v.q_lo > 0.f ? (aP + dP) / v.q_lo : 1.f;
  if (!(rhi < 1.f)) rhi = 1.f;
  if (s > 1.f) s = 1.f;
  const float e1 = s - rlo, e2 = rhi - s;
  float eps = (e1 > e2 ? e1 : e2) * (1.f + 16.f * u) + 4e-12f * s;
  if (!(eps >= 0.f)) eps = 1.f;
  *s_out = s;
  *eps_out = eps;
}

// One target: the interval and realised decision of a candidate (a
// non-finite target sum leaves it undecided).
__device__ __forceinline__ GramCand gram_finish(float S1, float dS1, float S2, float dS2, float Sy, float dSy,
                                                float Z, float dZ, float Vhi, float E, float N, float invN,
                                                float ysum, float fmin) {
  GramCand o;
  const GramVar v = gram_var(S1, dS1, S2, dS2, Z, dZ, Vhi, E, N, invN, fmin);
  o.realised = isfinite(Sy) ? v.realised : 2;
  if (o.realised == 2) {
    o.s = 0.f;
    o.eps = 1.f;
    return o;
  }
  gram_num(v, Sy, dSy, invN, ysum, &o.s, &o.eps);
  return o;
}

// A-priori tests of op(ia, ib) for a*b, a/b, b/a from the cached records:
// the same tests, in the same order and arithmetic, as binary_apriori_W
// (complexity, user rules, divisor domain, FP32 directed-rounding magnitude
// interval with the exact FP64 test when it straddles the limit).
__device__ __forceinline__ int gram_apriori(const ScreenArgs &A, int opc, int64_t ia, int64_t ib,
                                            const gram::EpiFeat &a, const gram::EpiFeat &b) {
  if (A.max_complexity > 0 && a.cplx + b.cplx + 1 > A.max_complexity) return DSE_R_COMPLEXITY;
  if (rule_fails(A.F, opc, ia, ib)) return DSE_R_COMPLEXITY;
  if (opc == DSE_OP_DIV && !(b.flags & F_MINABS_POS)) return DSE_R_DOMAIN;
  if (opc == DSE_OP_RDIV && !(a.flags & F_MINABS_POS)) return DSE_R_DOMAIN;
  float lo, hi;
  if (opc == DSE_OP_MUL) {
    lo = __fmul_rd(a.fa.w, b.fa.w);
    hi = __fmul_ru(a.fa.z, b.fa.z);
  } else if (opc == DSE_OP_DIV) {
    lo = __fmul_rd(a.fa.w, b.fr.y);
    hi = __fmul_ru(a.fa.z, b.fr.x);
  } else {
    lo = __fmul_rd(b.fa.w, a.fr.y);
    hi = __fmul_ru(b.fa.z, a.fr.x);
  }
  if (hi <= A.fmax32_dn) return DSE_VALID;
  if (lo > A.fmax32_up) return DSE_R_MAGNITUDE;
  return domain_magnitude64(opc, A.F.min64[ia], A.F.max64[ia], A.F.minabs64[ia], A.F.maxabs64[ia],
                            A.F.minabs64[ib], A.F.maxabs64[ib], A.fmax64, 0.0);
}

// a + b and a - b of a pair (family x of both features, k = c_a +- c_b):
//   S1 = P1 +- Q1,  S2 = P2 + Q2 +- 2 G11,  Sy = PY +- QY
// with G11 = sum p q from the same contraction as the products (no sample is
// evaluated).  The candidate the FP32 rows represent differs from the exact
// one by at most u (2 |x| + |c|) per operand and sample.  The bounds grow
// with the operands' norms, not with the (possibly cancelling) value: a
// difference of nearly equal features gets a wide interval, or an undecided
// realised test and the FP64 escalation.
__device__ __forceinline__ GramCand gram_score_add(const gram::EpiFeat *Fa, const gram::EpiFeat *Fb, float sign,
                                                   float G11, float G22, float delta, float N, float invN, float ysum,
                                                   float fmin) {
  const float u = 5.9604644775390625e-8f;
  const float ca = Fa->c[0], cb = Fb->c[0], k = ca + sign * cb;
  const float P1 = Fa->s1[0], P2 = Fa->s2[0], PY = Fa->sy[0];
  const float Q1 = Fb->s1[0], Q2 = Fb->s2[0], QY = Fb->sy[0];
  const float S1 = P1 + sign * Q1;
  const float S2 = P2 + Q2 + sign * 2.f * G11;
  const float Sy = PY + sign * QY;
  const float dG11 = gram_err(delta, G22, Fa->n1[0], Fa->n2[0], Fb->n1[0], Fb->n2[0], N).dG11;
  const float dS1 = 8.f * u * (fabsf(P1) + fabsf(Q1)) * 1.01f;
  const float dS2 = (2.f * dG11 + 8.f * u * (P2 + Q2 + 2.f * fabsf(G11))) * 1.01f;
  const float dSy = (8.f * u * (fabsf(PY) + fabsf(QY)) + 1.01f * u * (Fa->n1[0] + Fb->n1[0])) * 1.01f;
  const float Z = S2 + 2.f * k * S1 + N * k * k;
  const float dZ = (dS2 + 2.f * fabsf(k) * dS1 + 10.f * u * (fabsf(S2) + 2.f * fabsf(k * S1) + N * k * k)) * 1.01f;
  const float Vhi = sqrtf(Z + dZ) * (1.f + 4.f * u);
  const float E = u * (2.01f * (Fa->nu[0] + Fb->nu[0]) + (fabsf(ca) + fabsf(cb)) * sqrtf(N) * (1.f + 4.f * u) +
                       Vhi) * 1.02f;
  return gram_finish(S1, dS1, S2, dS2, Sy, dSy, Z, dZ, Vhi, E, N, invN, ysum, fmin);
}

// A-priori tests of a + b and a - b from the cached records, in the order
// and arithmetic of binary_apriori_W: equal units (when checked),
// complexity, user rules, and the magnitude bound max|a| + max|b| by an FP32
// directed-rounding interval with the exact FP64 test when it straddles the
// limit.
__device__ __forceinline__ int gram_apriori_add(const ScreenArgs &A, int opc, int64_t ia, int64_t ib,
                                                const gram::EpiFeat &a, const gram::EpiFeat &b) {
  if (A.unit_check_addsub && (a.uk[0] != b.uk[0] || a.uk[1] != b.uk[1])) return DSE_R_UNIT;
  if (A.max_complexity > 0 && a.cplx + b.cplx + 1 > A.max_complexity) return DSE_R_COMPLEXITY;
  if (rule_fails(A.F, opc, ia, ib)) return DSE_R_COMPLEXITY;
  const float lo = __fadd_rd(a.fa.w, b.fa.w), hi = __fadd_ru(a.fa.z, b.fa.z);
  if (hi <= A.fmax32_dn) return DSE_VALID;
  if (lo > A.fmax32_up) return DSE_R_MAGNITUDE;
  return domain_magnitude64(opc, A.F.min64[ia], A.F.max64[ia], A.F.minabs64[ia], A.F.maxabs64[ia],
                            A.F.minabs64[ib], A.F.maxabs64[ib], A.fmax64, 0.0);
}

}  // namespace dse
