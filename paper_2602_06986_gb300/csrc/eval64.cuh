// eval64.cuh -- FP64 operator evaluation and the exact a-priori tests
// (unit, complexity, domain, magnitude) on FP64 feature summaries.
//
// Every FP64 operation is an explicitly rounded intrinsic, so the compiler
// cannot fuse a multiply and an add: the results are the IEEE results of the
// operation order written here ((x*x)*x for the cube, a single rounded
// division, a correctly rounded square root).
#pragma once

#include "dse_internal.cuh"

namespace dse {

__device__ __forceinline__ double eval_op64(int op, double a, double b) {
  switch (op) {
    case DSE_OP_SQUARE: return __dmul_rn(a, a);
    case DSE_OP_CUBE: return __dmul_rn(__dmul_rn(a, a), a);
    case DSE_OP_INV: return __drcp_rn(a);
    case DSE_OP_SQRT: return __dsqrt_rn(a);
    case DSE_OP_EXP: return exp(a);
    case DSE_OP_LOG: return log(a);
    case DSE_OP_ADD: return __dadd_rn(a, b);
    case DSE_OP_SUB: return __dsub_rn(a, b);
    case DSE_OP_MUL: return __dmul_rn(a, b);
    case DSE_OP_DIV: return __ddiv_rn(a, b);
    case DSE_OP_RDIV: return __ddiv_rn(b, a);
    case DSE_OP_ABSDIFF: return fabs(__dsub_rn(a, b));
    default: return a;  // DSE_OP_PRIMARY / identity
  }
}

// Unit rule (exact integers).  ua, ub: scaled exponent vectors.  Writes the
// result vector; returns false if the rule fails.  *bad is set if an odd
// exponent meets sqrt or the result leaves the 16-bit range.
__device__ __forceinline__ bool unit_rule(int op, const int32_t *ua, const int32_t *ub, int D, int check_addsub,
                                          int explog_dimless, int32_t *u, int *bad) {
  for (int d = 0; d < D; ++d) {
    int32_t x = ua[d], y = ub ? ub[d] : 0, r = 0;
    switch (op) {
      case DSE_OP_SQUARE: r = 2 * x; break;
      case DSE_OP_CUBE: r = 3 * x; break;
      case DSE_OP_INV: r = -x; break;
      case DSE_OP_SQRT:
        if (x & 1) *bad = 1;
        r = x / 2;
        break;
      case DSE_OP_EXP:
      case DSE_OP_LOG:
        if (explog_dimless && x != 0) return false;
        r = 0;
        break;
      case DSE_OP_ADD:
      case DSE_OP_SUB:
      case DSE_OP_ABSDIFF:
        if (check_addsub && x != y) return false;
        r = x;
        break;
      case DSE_OP_MUL: r = x + y; break;
      case DSE_OP_DIV: r = x - y; break;
      case DSE_OP_RDIV: r = y - x; break;
      default: r = x;
    }
    if (r > 32767 || r < -32767) *bad = 2;
    u[d] = r;
  }
  return true;
}

// Domain and magnitude tests on FP64 summaries of operands a (and b).
// Returns DSE_VALID, DSE_R_DOMAIN or DSE_R_MAGNITUDE.
__device__ __forceinline__ int domain_magnitude64(int op, double mina, double maxa, double minabsa, double maxabsa,
                                                  double minabsb, double maxabsb, double fmax,
                                                  double exp_arg_max) {
  switch (op) {
    case DSE_OP_LOG: if (!(mina > 0.0)) return DSE_R_DOMAIN; break;
    case DSE_OP_SQRT: if (!(mina >= 0.0)) return DSE_R_DOMAIN; break;
    case DSE_OP_INV: if (!(minabsa > 0.0)) return DSE_R_DOMAIN; break;
    case DSE_OP_EXP: if (!(maxa <= 80.0)) return DSE_R_DOMAIN; break;
    case DSE_OP_DIV: if (!(minabsb > 0.0)) return DSE_R_DOMAIN; break;
    case DSE_OP_RDIV: if (!(minabsa > 0.0)) return DSE_R_DOMAIN; break;
    default: break;
  }
  double B = 0.0;
  switch (op) {
    case DSE_OP_SQUARE: B = __dmul_rn(maxabsa, maxabsa); break;
    case DSE_OP_CUBE: B = __dmul_rn(__dmul_rn(maxabsa, maxabsa), maxabsa); break;
    case DSE_OP_INV: B = __drcp_rn(minabsa); break;
    case DSE_OP_SQRT: B = __dsqrt_rn(maxabsa); break;
    case DSE_OP_EXP: return (maxa <= exp_arg_max) ? DSE_VALID : DSE_R_MAGNITUDE;
    case DSE_OP_LOG: return DSE_VALID;
    case DSE_OP_ADD:
    case DSE_OP_SUB:
    case DSE_OP_ABSDIFF: B = __dadd_rn(maxabsa, maxabsb); break;
    case DSE_OP_MUL: B = __dmul_rn(maxabsa, maxabsb); break;
    case DSE_OP_DIV: B = __ddiv_rn(maxabsa, minabsb); break;
    case DSE_OP_RDIV: B = __ddiv_rn(maxabsb, minabsa); break;
    default: return DSE_VALID;
  }
  return (B <= fmax) ? DSE_VALID : DSE_R_MAGNITUDE;
}

// FP64 value at sample s of the candidate with global id gid (a stored
// feature for gid < n_stored, else flat slot gid - n_stored of the last rung).
__device__ __forceinline__ double candidate_value64(const FeatTable &F, const RungGeom &G, int64_t n_stored,
                                                   uint64_t gid, int64_t s) {
  int op;
  int64_t a, b;
  if (gid < (uint64_t)n_stored) {
    op = DSE_OP_PRIMARY;
    a = (int64_t)gid;
    b = -1;
  } else {
    decode_flat(G, gid - (uint64_t)n_stored, &op, &a, &b);
  }
  return eval_op64(op, F.v64[a * F.ld + s], b >= 0 ? F.v64[b * F.ld + s] : 0.0);
}

// User rules on the candidate op(a[, b]) (b < 0 for a unary op).  Both
// operands satisfy the rules already, so only the new node is checked: a
// forbidden pair with a leaf in each operand (dmask[a] is symmetric in the
// relation) and a forbidden primary below op.
__device__ __forceinline__ bool rule_fails(const FeatTable &F, int op, int64_t a, int64_t b) {
  if (!F.used) return false;
  uint64_t u = F.used[a];
  bool bad = false;
  if (b >= 0) {
    const uint64_t ub = F.used[b];
    bad = (F.dmask[a] & ub) != 0;
    u |= ub;
  }
  return bad || (u & F.op_deny[op]) != 0;
}

// Full a-priori test of op(a[, b]) against the stored table.
struct AprioriParams {
  int D, check_addsub, explog_dimless, max_complexity;
  double fmax, exp_arg_max;
};

__device__ __forceinline__ int apriori64(const FeatTable &F, const AprioriParams &P, int op, int64_t a, int64_t b,
                                         int32_t *u, int32_t *cx, int *bad) {
  const int32_t *ua = F.units + a * kMaxDims;
  const int32_t *ub = (b >= 0) ? F.units + b * kMaxDims : nullptr;
  if (!unit_rule(op, ua, ub, P.D, P.check_addsub, P.explog_dimless, u, bad)) return DSE_R_UNIT;
  int32_t c = F.cplx[a] + 1 + (b >= 0 ? F.cplx[b] : 0);
  *cx = c;
  if (P.max_complexity > 0 && c > P.max_complexity) return DSE_R_COMPLEXITY;
  if (rule_fails(F, op, a, b)) return DSE_R_COMPLEXITY;
  return domain_magnitude64(op, F.min64[a], F.max64[a], F.minabs64[a], F.maxabs64[a],
                            b >= 0 ? F.minabs64[b] : 0.0, b >= 0 ? F.maxabs64[b] : 0.0, P.fmax, P.exp_arg_max);
}

// Warp-wide reductions (all lanes get the result).
__device__ __forceinline__ double warp_sum64(double v) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}
__device__ __forceinline__ double warp_min64(double v) {
  for (int o = 16; o > 0; o >>= 1) v = fmin(v, __shfl_xor_sync(0xffffffffu, v, o));
  return v;
}
__device__ __forceinline__ double warp_max64(double v) {
  for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
  return v;
}
__device__ __forceinline__ int warp_or(int v) {
  return __any_sync(0xffffffffu, v) ? 1 : 0;
}

// Vectors a candidate column is summed against (the target and up to four
// refit vectors).
constexpr int kColVec = 5;

}  // namespace dse
