// df32.cuh -- FP32-pair ("double-float") arithmetic for the column sums of
// the re-score and the refits.
//
// GB300 runs FP64 at 2 fused multiply-adds per clock per SM and FP32 at 128,
// so the FP64 sums over samples of a candidate column (sum (v - c),
// sum (v - c)^2, sum (v - c) x_m) are bound by the FP64 pipe.  A value here
// is an unevaluated sum hi + lo of two FP32 numbers (|lo| <= ulp(hi)/2 after
// renormalisation), which carries about 48 significant bits; every step
// below is an error-free transformation or a classic correction step:
//   two_sum: Knuth's branch-free exact sum (TAOCP vol. 2, 4.2.2);
//   fast_two_sum: Dekker's exact sum for |a| >= |b| (Dekker 1971);
//   two_prod: the exact product by one fused multiply-add;
//   pair product, quotient, reciprocal and square root: Dekker's
//   double-length routines with the correction computed by FMA (Dekker 1971;
//   Karp & Markstein 1997 for the quotient / square-root correction).
// Every operation is an explicitly rounded intrinsic, so the compiler cannot
// contract a multiply and an add: the results are those of the order
// written.
//
// Range: the operands are rescaled by powers of two (exact) so that the
// largest |value| of each operand is in [1/2, 1); the caller falls back to
// FP64 when an operand is outside the FP32-safe range or when the pass
// reports values or sums out of the range where the pair format holds its
// 2^-46 relative accuracy.
#pragma once

#include "dse_internal.cuh"
#include "eval64.cuh"

namespace dse {
namespace df {

struct F2 {
  float hi, lo;
  __device__ __forceinline__ double value() const { return (double)hi + (double)lo; }
};

__device__ __forceinline__ F2 two_sum(float a, float b) {
  const float s = __fadd_rn(a, b);
  const float bb = __fsub_rn(s, a);
  const float e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
  return {s, e};
}

__device__ __forceinline__ F2 fast_two_sum(float a, float b) {
  const float s = __fadd_rn(a, b);
  return {s, __fsub_rn(b, __fsub_rn(s, a))};
}

// x + y (both pairs), renormalised; relative error about 2^-47 of |x| + |y|
__device__ __forceinline__ F2 add(F2 x, F2 y) {
  const F2 s = two_sum(x.hi, y.hi);
  const float e = __fadd_rn(s.lo, __fadd_rn(x.lo, y.lo));
  return fast_two_sum(s.hi, e);
}

__device__ __forceinline__ F2 neg(F2 x) { return {-x.hi, -x.lo}; }

// x * y, renormalised
__device__ __forceinline__ F2 mul(F2 x, F2 y) {
  const float p = __fmul_rn(x.hi, y.hi);
  float e = __fmaf_rn(x.hi, y.hi, -p);
  e = __fmaf_rn(x.hi, y.lo, e);
  e = __fmaf_rn(x.lo, y.hi, e);
  return fast_two_sum(p, e);
}

// x * x, renormalised
__device__ __forceinline__ F2 sqr(F2 x) {
  const float p = __fmul_rn(x.hi, x.hi);
  float e = __fmaf_rn(x.hi, x.hi, -p);
  e = __fmaf_rn(__fadd_rn(x.hi, x.hi), x.lo, e);
  return fast_two_sum(p, e);
}

// x / y (y != 0): q1 = x.hi / y.hi to FP32, the remainder x - q1 y in pair
// arithmetic (x.hi - q1 y.hi is exact: both are within a few ulps), then one
// correction q2 = remainder / y.hi; relative error about 2^-44
__device__ __forceinline__ F2 div(F2 x, F2 y) {
  const float r = __frcp_rn(y.hi);
  const float q1 = __fmul_rn(x.hi, r);
  const float p = __fmul_rn(q1, y.hi);
  const float pe = __fmaf_rn(q1, y.hi, -p);
  float rem = __fsub_rn(__fsub_rn(x.hi, p), pe);
  rem = __fadd_rn(rem, __fmaf_rn(-q1, y.lo, x.lo));
  return fast_two_sum(q1, __fmul_rn(rem, r));
}

__device__ __forceinline__ F2 inv(F2 y) { return div(F2{1.0f, 0.0f}, y); }

// sqrt(x) (x >= 0): s = sqrt(x.hi) to FP32, then one Newton correction with
// the exact residual x - s^2
__device__ __forceinline__ F2 sqrt_(F2 x) {
  if (!(x.hi > 0.0f)) return {0.0f, 0.0f};
  const float s = __fsqrt_rn(x.hi);
  const float p = __fmul_rn(s, s);
  const float pe = __fmaf_rn(s, s, -p);
  const float res = __fadd_rn(__fsub_rn(__fsub_rn(x.hi, p), pe), x.lo);
  const float c = __fdiv_rn(res, __fadd_rn(s, s));
  return fast_two_sum(s, c);
}

// Running sum of pair terms in Neumaier's compensated form: hi the rounded
// sum, lo the exact two-sum errors plus the terms' low parts (no
// renormalisation: the pair is read as (double)hi + (double)lo, and lo stays
// within a few ulps of hi times the number of steps a thread takes).  The
// step is symmetric in its two operands (each rounding adds a commutative
// pair), so a butterfly reduction leaves the same bits in every lane.
struct Acc {
  float hi = 0.0f, lo = 0.0f;
  __device__ __forceinline__ void add(float th, float tl) {
    const F2 s = two_sum(hi, th);
    lo = __fadd_rn(__fadd_rn(lo, tl), s.lo);
    hi = s.hi;
  }
  __device__ __forceinline__ void warp_reduce() {
    for (int o = 16; o > 0; o >>= 1) {
      const float oh = __shfl_xor_sync(0xffffffffu, hi, o), ol = __shfl_xor_sync(0xffffffffu, lo, o);
      add(oh, ol);
    }
  }
  __device__ __forceinline__ double value() const { return (double)hi + (double)lo; }
};

// 2^e as float / double (exact for the ranges used: |e| <= 126 / 1022)
__device__ __forceinline__ float pow2f(int e) { return __int_as_float((127 + e) << 23); }
__device__ __forceinline__ double pow2d(int e) { return __longlong_as_double((long long)(1023 + e) << 52); }

// Exponent e with x 2^-e in [1/2, 1) for a finite normal x > 0 (0 for x == 0
// or a non-finite x), clamped to [-1000, 1000].
__device__ __forceinline__ int scale_exp(double x) {
  if (!(x > 0.0) || !(x < INFINITY)) return 0;
  const long long bits = __double_as_longlong(x);
  const int e = (int)((bits >> 52) & 0x7ff) - 1022;
  return e < -1000 ? -1000 : e > 1000 ? 1000 : e;
}

// 1/n by an FP32 reciprocal and two Newton steps r <- r (2 - n r) (each
// doubles the correct bits: 2^-23 -> 2^-46 -> below the FP64 rounding).
__device__ __forceinline__ double recip_n(int64_t N) {
  const double n = (double)N;
  double r = (double)__frcp_rn((float)N);
  r = r * __fma_rn(-n, r, 2.0);
  r = r * __fma_rn(-n, r, 2.0);
  return r;
}

// 1/sqrt(x) for x in the FP32 normal range: FP32 estimate, two Newton steps
// y <- y (3/2 - x y^2 / 2).
__device__ __forceinline__ double rsqrt_nr(double x) {
  double y = (double)rsqrtf((float)x);
  for (int it = 0; it < 2; ++it) {
    const double h = (x * y) * y;
    y = y * __fma_rn(-0.5, h, 1.5);
  }
  return y;
}

}  // namespace df

// ----------------------------------------------------------- column sums

// One block of kColThreads threads per candidate column (threads over
// samples, warp shuffles, then the warps' partials combined in warp order in
// every thread, so that every thread holds the same bits).
constexpr int kColThreads = 128;

// The vectors a candidate column is summed against: x_m as FP64 rows (for
// the FP64 path) and as pair images (x_m 2^-e_m split into hi, lo).
struct ColVecs {
  const double *v64[kColVec];
  const float2 *vdf[kColVec];
  int e[kColVec];
  int nv;
};

// Shifted sums of one candidate column, c = v at sample 0:
//   acc[0] = sum (v - c), acc[1] = sum (v - c)^2, acc[2 + m] = sum (v - c) x_m;
// kappa = sqrt(sum m^2 / Sxx') of the scaled pass (1 on the FP64 path), m
// the magnitude the value's error is relative to (|v|, or |a| + |b| for a
// sum or difference): the factor by which the pair format's error grows
// relative to the centred column; pair = whether the pair pass produced
// them.
// s0 = |acc[2]| / sqrt(Sxx), the score against the first vector when that
// is a centred unit-norm target.
struct ColSums {
  double c;
  double acc[2 + kColVec];
  double kappa;
  double s0;
  bool pair;
};

// The block's exchange area.
struct ColShared {
  float f[kColThreads / 32][2 * (2 + kColVec) + 2];
  double d[kColThreads / 32][2 + kColVec];
  int ok;
};

namespace df {

__device__ __forceinline__ bool pair_op(int op) {
  return op != DSE_OP_EXP && op != DSE_OP_LOG;
}

// value of op(x, y) on scaled pair operands
__device__ __forceinline__ F2 eval_pair(int op, F2 x, F2 y) {
  switch (op) {
    case DSE_OP_SQUARE: return sqr(x);
    case DSE_OP_CUBE: return mul(sqr(x), x);
    case DSE_OP_INV: return inv(x);
    case DSE_OP_SQRT: return sqrt_(x);
    case DSE_OP_ADD: return add(x, y);
    case DSE_OP_SUB: return add(x, neg(y));
    case DSE_OP_MUL: return mul(x, y);
    case DSE_OP_DIV: return div(x, y);
    case DSE_OP_RDIV: return div(y, x);
    case DSE_OP_ABSDIFF: {
      const F2 d = add(x, neg(y));
      return d.hi < 0.0f ? neg(d) : d;
    }
    default: return x;  // DSE_OP_PRIMARY / identity
  }
}

// The value of op on scaled pair operands (x = a 2^-sa, y = b 2^-sb from
// their FP32 high and low rows).
__device__ __forceinline__ F2 pair_value(int op, float xh, float xl, float yh, float yl, float fa, float fb) {
  const F2 x{__fmul_rn(xh, fa), __fmul_rn(xl, fa)};
  const F2 y{__fmul_rn(yh, fb), __fmul_rn(yl, fb)};
  return eval_pair(op, x, y);
}

// One thread's samples (threadIdx.x, + kColThreads, ...) of the pair pass for
// operator OP: the shifted sums, the conditioning sum and the largest value.
// A sum or difference carries the operands' representation error (2^-48 of
// |a| + |b|), which cancellation amplifies relative to v: its conditioning
// sum takes (|a| + |b|)^2 instead of v^2.
template <int NV, int OP>
__device__ __forceinline__ void pair_pass(const float *ah, const float *al, const float *bh, const float *bl,
                                          float fa, float fb, F2 nc, int64_t N, const ColVecs &V, Acc &s1, Acc &s2,
                                          Acc (&p)[NV], float &sv, float &vmax) {
  constexpr bool additive = OP == DSE_OP_ADD || OP == DSE_OP_SUB || OP == DSE_OP_ABSDIFF;
  // two samples per thread per step, their loads issued together (the pass
  // is bound by load latency otherwise); each thread takes its samples in
  // increasing order
  constexpr int U = 2;
  for (int64_t s0 = threadIdx.x; s0 < N; s0 += U * kColThreads) {
    float lh[U], ll[U], rh[U], rl[U];
    float2 wv[U][NV];
#pragma unroll
    for (int k = 0; k < U; ++k) {
      const int64_t s = s0 + (int64_t)k * kColThreads;
      const bool in = s < N;
      lh[k] = in ? ah[s] : 0.0f;
      ll[k] = in ? al[s] : 0.0f;
      rh[k] = in ? bh[s] : 0.0f;
      rl[k] = in ? bl[s] : 0.0f;
#pragma unroll
      for (int m = 0; m < NV; ++m) wv[k][m] = in ? V.vdf[m][s] : make_float2(0.0f, 0.0f);
    }
#pragma unroll
    for (int k = 0; k < U; ++k) {
      if (s0 + (int64_t)k * kColThreads >= N) break;
      const F2 x{__fmul_rn(lh[k], fa), __fmul_rn(ll[k], fa)};
      const F2 y{__fmul_rn(rh[k], fb), __fmul_rn(rl[k], fb)};
      const F2 v = eval_pair(OP, x, y);
      const float mag = additive ? __fadd_rn(fabsf(x.hi), fabsf(y.hi)) : fabsf(v.hi);
      const F2 d = add(v, nc);
      s1.add(d.hi, d.lo);
      {
        const float q = __fmul_rn(d.hi, d.hi);
        const float qe = __fmaf_rn(__fadd_rn(d.hi, d.hi), d.lo, __fmaf_rn(d.hi, d.hi, -q));
        s2.add(q, qe);
      }
      sv = __fmaf_rn(mag, mag, sv);
      vmax = fmaxf(vmax, fabsf(v.hi));
#pragma unroll
      for (int m = 0; m < NV; ++m) {
        const float2 w = wv[k][m];
        const float q = __fmul_rn(d.hi, w.x);
        float qe = __fmaf_rn(d.hi, w.x, -q);
        qe = __fmaf_rn(d.hi, w.y, qe);
        qe = __fmaf_rn(d.lo, w.x, qe);
        p[m].add(q, qe);
      }
    }
  }
}

// The pair pass (whole block, results in warp 0); false when it does not
// apply or its result fails the range / conditioning checks (every thread
// returns the same).
template <int NV>
__device__ __forceinline__ bool col_sums_pair(const FeatTable &F, int op, int64_t a, int64_t b, int64_t N,
                                              const ColVecs &V, ColSums &out, ColShared &sh) {
  const uint32_t fl = F.flags[a] & (b >= 0 ? F.flags[b] : 0xffffffffu);
  if (!F.v32lo || !pair_op(op) || !(fl & F_FP32_SAFE)) return false;
#pragma unroll
  for (int m = 0; m < NV; ++m)
    if (!V.vdf[m]) return false;
  // power-of-two scales: operand x 2^-e with max |x 2^-e| in [1/2, 1)
  const int ea = scale_exp(F.maxabs64[a]), eb = b >= 0 ? scale_exp(F.maxabs64[b]) : 0;
  int sa = ea, sb = eb, ev;
  switch (op) {
    case DSE_OP_ADD:
    case DSE_OP_SUB:
    case DSE_OP_ABSDIFF: sa = sb = ev = ea > eb ? ea : eb; break;
    case DSE_OP_MUL: ev = ea + eb; break;
    case DSE_OP_DIV: ev = ea - eb; break;
    case DSE_OP_RDIV: ev = eb - ea; break;
    case DSE_OP_SQUARE: ev = 2 * ea; break;
    case DSE_OP_CUBE: ev = 3 * ea; break;
    case DSE_OP_INV: ev = -ea; break;
    case DSE_OP_SQRT:
      sa = ea + (ea & 1);  // even, so that the root's scale is a power of two
      ev = sa / 2;
      break;
    default: ev = ea; break;
  }
  const float fa = pow2f(-sa), fb = pow2f(-sb);
  const float *ah = F.v32 + a * F.ld, *al = F.v32lo + a * F.ld;
  const float *bh = F.v32 + (b >= 0 ? b : a) * F.ld, *bl = F.v32lo + (b >= 0 ? b : a) * F.ld;
  // a sum or difference carries the operands' representation error
  // (2^-48 of |a| + |b|), which cancellation amplifies relative to v: its
  // conditioning sum takes (|a| + |b|)^2 instead of v^2
  // (the pass over the samples is instantiated per operator, so that the
  // operator's arithmetic is not a branch inside the loop)
  const F2 c = pair_value(op, ah[0], al[0], bh[0], bl[0], fa, fb);
  Acc s1, s2, p[NV];
  float sv = 0.0f, vmax = 0.0f;
  switch (op) {
#define DSE_PAIR_CASE(OPC) \
  case OPC: pair_pass<NV, OPC>(ah, al, bh, bl, fa, fb, neg(c), N, V, s1, s2, p, sv, vmax); break;
    DSE_PAIR_CASE(DSE_OP_SQUARE)
    DSE_PAIR_CASE(DSE_OP_CUBE)
    DSE_PAIR_CASE(DSE_OP_INV)
    DSE_PAIR_CASE(DSE_OP_SQRT)
    DSE_PAIR_CASE(DSE_OP_ADD)
    DSE_PAIR_CASE(DSE_OP_SUB)
    DSE_PAIR_CASE(DSE_OP_MUL)
    DSE_PAIR_CASE(DSE_OP_DIV)
    DSE_PAIR_CASE(DSE_OP_RDIV)
    DSE_PAIR_CASE(DSE_OP_ABSDIFF)
#undef DSE_PAIR_CASE
    default: pair_pass<NV, DSE_OP_PRIMARY>(ah, al, bh, bl, fa, fb, neg(c), N, V, s1, s2, p, sv, vmax); break;
  }
  s1.warp_reduce();
  s2.warp_reduce();
#pragma unroll
  for (int m = 0; m < NV; ++m) p[m].warp_reduce();
  for (int o = 16; o > 0; o >>= 1) {
    sv = __fadd_rn(sv, __shfl_xor_sync(0xffffffffu, sv, o));
    vmax = fmaxf(vmax, __shfl_xor_sync(0xffffffffu, vmax, o));
  }
  const int w = threadIdx.x >> 5;
  if ((threadIdx.x & 31) == 0) {
    float *f = sh.f[w];
    f[0] = s1.hi;
    f[1] = s1.lo;
    f[2] = s2.hi;
    f[3] = s2.lo;
#pragma unroll
    for (int m = 0; m < NV; ++m) {
      f[4 + 2 * m] = p[m].hi;
      f[5 + 2 * m] = p[m].lo;
    }
    f[2 * (2 + kColVec)] = sv;
    f[2 * (2 + kColVec) + 1] = vmax;
  }
  __syncthreads();
  // the combination, the checks and the outputs in warp 0 only (FP64 work
  // is slow on this part); the decision reaches every thread through sh.ok
  if (threadIdx.x < 32) {
    auto combine = [&](int i) {
      Acc t;
      t.hi = sh.f[0][2 * i];
      t.lo = sh.f[0][2 * i + 1];
#pragma unroll
      for (int ww = 1; ww < kColThreads / 32; ++ww) t.add(sh.f[ww][2 * i], sh.f[ww][2 * i + 1]);
      return t.value();
    };
    const double S1 = combine(0), S2 = combine(1);
    float svt = sh.f[0][2 * (2 + kColVec)], vmx = sh.f[0][2 * (2 + kColVec) + 1];
#pragma unroll
    for (int ww = 1; ww < kColThreads / 32; ++ww) {
      svt = __fadd_rn(svt, sh.f[ww][2 * (2 + kColVec)]);
      vmx = fmaxf(vmx, sh.f[ww][2 * (2 + kColVec) + 1]);
    }
    // checks on the scaled pass, depending on the column alone (so that
    // every caller takes the same path): values within [2^-30, 2^40] at
    // their largest, finite sums, and a centred column not below 2^-24 of
    // the magnitudes its errors scale with (else the pair format's error
    // relative to the centred column could exceed 2^-34).  The vector sums
    // are then finite (|sum d x| <= sqrt(S2) |x|).
    const double Sxx = __fma_rn(-S1, S1 * recip_n(N), S2);
    const bool ok = vmx >= 9.313225746154785e-10f && vmx <= 1.099511627776e12f && isfinite(S1) &&
                    isfinite(S2) && svt > 0.0f && isfinite(svt) && Sxx >= 5.9604644775390625e-8 * (double)svt;
    if (threadIdx.x == 0) sh.ok = ok;
    if (ok) {
      double Pm[NV];
#pragma unroll
      for (int m = 0; m < NV; ++m) Pm[m] = combine(2 + m);
      // back to the unscaled sums (exact multiplications by powers of two)
      const double sc = pow2d(ev);
      out.c = c.value() * sc;
      out.acc[0] = S1 * sc;
      out.acc[1] = (S2 * sc) * sc;
#pragma unroll
      for (int m = 0; m < kColVec; ++m) {
        double v = 0.0;
        if (m < NV) {
          const int e = ev + V.e[m];
          const double pm = Pm[m < NV ? m : 0];
          v = e >= -1022 && e <= 1023 ? pm * pow2d(e) : (pm * sc) * pow2d(V.e[m]);
        }
        out.acc[2 + m] = v;
      }
      out.kappa = (double)sqrtf(svt / (float)Sxx);
      // the score against vector 0 from the scaled sums (scale-free, and
      // Sxx' is within the FP32 range here)
      out.s0 = fabs(Pm[0]) * rsqrt_nr(Sxx);
      out.pair = true;
    }
  }
  __syncthreads();
  return sh.ok != 0;
}

}  // namespace df

// The FP64 pass (whole block, results in warp 0): the same sums with c the
// FP64 value at sample 0.
// (NVB: the largest number of vectors the caller passes, known at compile
// time; the vectors past V.nv are skipped either way)
template <int NVB = kColVec>
__device__ __forceinline__ void col_sums64(const FeatTable &F, int op, int64_t a, int64_t b, int64_t N,
                                           const ColVecs &V, ColSums &out, ColShared &sh) {
  const double *xa = F.v64 + a * F.ld, *xb = F.v64 + (b >= 0 ? b : a) * F.ld;
  const double c = eval_op64(op, xa[0], xb[0]);
  double acc[2 + kColVec];
#pragma unroll
  for (int i = 0; i < 2 + kColVec; ++i) acc[i] = 0.0;
  for (int64_t s = threadIdx.x; s < N; s += kColThreads) {
    const double v = eval_op64(op, xa[s], xb[s]) - c;
    acc[0] += v;
    acc[1] = fma(v, v, acc[1]);
#pragma unroll
    for (int m = 0; m < NVB; ++m)
      if (m < V.nv) acc[2 + m] = fma(v, V.v64[m][s], acc[2 + m]);
  }
  const int w = threadIdx.x >> 5;
#pragma unroll
  for (int i = 0; i < 2 + kColVec; ++i) {
    const double t = warp_sum64(acc[i]);
    if ((threadIdx.x & 31) == 0) sh.d[w][i] = t;
  }
  __syncthreads();
  if (threadIdx.x < 32) {  // the results in warp 0
#pragma unroll
    for (int i = 0; i < 2 + kColVec; ++i) {
      double t = sh.d[0][i];
#pragma unroll
      for (int ww = 1; ww < kColThreads / 32; ++ww) t += sh.d[ww][i];
      out.acc[i] = t;
    }
    out.c = c;
    out.kappa = 1.0;
    const double sxx = out.acc[1] - out.acc[0] * (out.acc[0] / (double)N);
    out.s0 = fabs(out.acc[2]) / sqrt(sxx);
    out.pair = false;
  }
  __syncthreads();
}

// Relative error scale of a candidate's sums: for the pair pass
// (k (k/16 + 1) + 64) 2^-44 kappa with k = N/128 the steps of one thread
// (the compensation term's own rounding grows as k^2 2^-48), for FP64
// (k + 64) 2^-49 (the scale of the FP64 re-score's bound); errors of the
// shifted sums are at most this times the natural scale sqrt(Sxx) |x_m|.
__device__ __forceinline__ double col_err_scale(const ColSums &cs, int64_t N) {
  const double k = (double)(N / kColThreads + 1);
  return cs.pair ? (k * (k / 16.0 + 1.0) + 64.0) * 5.684341886080802e-14 * cs.kappa
                 : (k + 64.0) * 1.7763568394002505e-15;
}

// The column sums of one candidate (one block of kColThreads threads; the
// results are in the threads of warp 0): the pair pass where it applies,
// else FP64.  The
// choice and the arithmetic depend only on the candidate and the vectors, so
// the sums a re-score takes alongside its score and the sums a refit takes
// later agree to the bit.
__device__ __forceinline__ void col_sums(const FeatTable &F, int op, int64_t a, int64_t b, int64_t N,
                                         const ColVecs &V, ColSums &out, ColShared &sh) {
  bool done = false;
  switch (V.nv) {
    case 1: done = df::col_sums_pair<1>(F, op, a, b, N, V, out, sh); break;
    case 2: done = df::col_sums_pair<2>(F, op, a, b, N, V, out, sh); break;
    case 3: done = df::col_sums_pair<3>(F, op, a, b, N, V, out, sh); break;
    case 4: done = df::col_sums_pair<4>(F, op, a, b, N, V, out, sh); break;
    case 5: done = df::col_sums_pair<5>(F, op, a, b, N, V, out, sh); break;
    default: break;
  }
  if (!done) col_sums64(F, op, a, b, N, V, out, sh);
}

// The same for callers whose candidates are summed against one vector only
// (V.nv == 1): the same arithmetic, without the code (and registers) of the
// wider passes.
__device__ __forceinline__ void col_sums1(const FeatTable &F, int op, int64_t a, int64_t b, int64_t N,
                                          const ColVecs &V, ColSums &out, ColShared &sh) {
  if (!df::col_sums_pair<1>(F, op, a, b, N, V, out, sh)) col_sums64<1>(F, op, a, b, N, V, out, sh);
}

}  // namespace dse
