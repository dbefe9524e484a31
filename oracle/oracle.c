/*
 * oracle.c -- plain, slow, FP64 CPU oracle for Sure Independence Screening
 * (SIS) over a SISSO-style symbolic feature space, as used by DISCOVER
 * (arXiv 2602.06986).
 *
 * TEST INFRASTRUCTURE ONLY.  Only the test-suite, the smoke check and the
 * CPU-baseline leg of the benchmark may load this file's library.  The CUDA
 * product path never links, loads or calls it, and the two share no code,
 * headers, tables or helpers.
 *
 * What it computes, and the passage each part follows:
 *   - Iterative feature generation from user-provided features and an
 *     operator library ("Software Description", first paragraph; the workflow
 *     figure caption: iterative generation -> screening -> sparse selection).
 *   - Dimensional consistency and early exclusion of dimensionally invalid
 *     expressions ("Physics-Informed Constraints").  The paper tracks units
 *     with a unit library; here exponents are exact rationals held as
 *     integers over the common denominator 2^max_rung.
 *   - Restrictions on operators and expression complexity ("Design
 *     Philosophy and Constraints").
 *   - Evaluation of every candidate against the target data and SIS
 *     screening by |Pearson| ("Software Description"; SISSO, "Summary").
 *   - The greedy residual loop that approximates Eq. 1 (L0-constrained least
 *     squares, ||beta||_0 <= D) in the OMP manner named in "Software
 *     Description".
 *
 * The paper defines none of the details; this file fixes these readings:
 *   R1  Phi_0 = the primaries that pass the realised test, in input order.
 *       Rung r is generated from Phi_{r-1} = old (ids [0,o)) + new (ids
 *       [o,o+m)) as: (i) the unary block, for f in new (id order), for each
 *       enabled unary op in code order; (ii) the binary block, for i in new
 *       (id order), for j in [0,i), for each enabled binary slot in code
 *       order.  The flat index p of a rung counts every slot, valid or not.
 *       Valid rung-r candidates with r < max_rung are appended to the table in
 *       flat order; rung max_rung is never stored.  The screened set is
 *       Phi_{k-1} (global ids [0, n_{k-1})) followed by rung k (global id
 *       n_{k-1} + p).
 *   R2  Op codes (also slot order): unary ^2 ^3 ^-1 sqrt exp log = 0..5;
 *       binary + - * a/b b/a |a-b| = 6..11.  For a pair (i, j), a = f_i (the
 *       higher id), b = f_j.
 *   R3  Units: ^2 doubles, ^3 triples, ^-1 negates, sqrt halves; exp and log
 *       require a dimensionless operand when explog_dimensionless is set and
 *       always give a dimensionless result; + - |a-b| require equal operand
 *       units when unit_check_addsub is set and keep them; * adds; a/b
 *       subtracts b from a; b/a subtracts a from b.
 *   R4  Complexity = number of operator nodes; a candidate above a positive
 *       max_complexity is excluded.
 *   R5  Domain: log needs min > 0; sqrt needs min >= 0; ^-1, and the divisor
 *       of a/b and b/a, need min|.| > 0; exp needs max <= 80.
 *   R6  Magnitude: an a-priori bound on max|v| from the operand summaries
 *       (M = max|.|, m = min|.|) must be <= fmax_max: ^2 M*M; ^3 (M*M)*M;
 *       ^-1 1/m; sqrt sqrt(M); exp: max <= log(fmax_max); log: exempt;
 *       + - |a-b| Ma+Mb; * Ma*Mb; a/b Ma/mb; b/a Mb/ma.
 *   R7  Realised: every value finite and, unless fmin_std_rel < 0, the
 *       candidate is not degenerate: std(v) > fmin_std_rel * rms(v), with
 *       std = sqrt(sum (v - mean)^2 / N) and rms = sqrt(sum v^2 / N).
 *   R8  Reasons are attributed in the order unit, complexity, domain,
 *       magnitude, realised (first failing test).
 *   R9  Score (SIS): |sum (v - vbar)(y - ybar)| / sqrt(sum (v - vbar)^2 *
 *       sum (y - ybar)^2), two-pass, Neumaier-compensated sums, per target.
 *       Aggregated mode: sqrt(mean over targets of score^2).
 *   R10 Top-k order: score descending, then global id ascending.
 *   R11 Residual loop: r_0 = y; for D = 1..Dmax: S_D = SIS top-k against
 *       r_{D-1}; for each s in S_D not already chosen, least squares with
 *       intercept of y on [d_1..d_{D-1}, s] (Householder QR); d_D = the s with
 *       the smallest RMSE (ties: lower id); r_D = y - fit.
 *   R15 User rules on variable combinations and functional forms ("Design
 *       Philosophy and Constraints"), optional, for at most 64 primaries:
 *       pair_deny[p] bit q (made symmetric) forbids primaries p and q in one
 *       expression (p = q: p may occur as a leaf at most once); op_deny[o]
 *       bit p forbids primary p anywhere below an application of op o.  A
 *       failing candidate takes reason 2 (the "form" reason: complexity cap
 *       or rule), tested after the complexity cap.  Primaries are named by
 *       their input index.
 *   R16 Redundancy: two valid candidates are equivalent when the FP64
 *       Pearson correlation of their values has |rho| >= 1 - tau; a candidate
 *       is redundant when an equivalent valid candidate with a smaller global
 *       id exists.  The deduplicated SIS list is the top-k (R10) of the
 *       non-redundant candidates.  Equivalent candidates' scores differ by at
 *       most sqrt(2 tau) (unit vectors at distance sqrt(2(1-|rho|))), so the
 *       search for an equivalent partner is confined to that score window.
 *
 * All arithmetic is IEEE FP64; compile with -ffp-contract=off so that no
 * multiply-add is fused.
 */
#include <math.h>
#include <stdint.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define ORC_MAX_DIMS 8
#define ORC_MAX_RUNG 4

enum {
  ORC_SQUARE = 0, ORC_CUBE = 1, ORC_INV = 2, ORC_SQRT = 3, ORC_EXP = 4, ORC_LOG = 5,
  ORC_ADD = 6, ORC_SUB = 7, ORC_MUL = 8, ORC_DIV = 9, ORC_RDIV = 10, ORC_ABSDIFF = 11,
  ORC_PRIMARY = 15
};
enum {
  ORC_VALID = 0, ORC_R_UNIT = 1, ORC_R_COMPLEXITY = 2, ORC_R_DOMAIN = 3,
  ORC_R_MAGNITUDE = 4, ORC_R_REALISED = 5
};

typedef struct {
  int64_t n_samples, n_primary;
  int32_t n_dims, max_rung;
  const double *X;      /* [n_primary][n_samples] */
  const int32_t *units; /* [n_primary][n_dims] integer exponents */
  uint32_t op_mask;     /* bit (1 << code) per enabled op */
  int32_t max_complexity;
  int32_t unit_check_addsub;
  int32_t explog_dimensionless;
  double fmax_max;
  double fmin_std_rel; /* < 0 disables the degeneracy test */
  const uint64_t *pair_deny; /* R15, NULL or [n_primary] rows; n_primary <= 64 */
  const uint64_t *op_deny;   /* R15, NULL or [12] rows */
} orc_params;

typedef struct {
  orc_params P;
  int64_t N;
  int D;
  int64_t nfeat;
  int32_t *op, *rung, *cplx;
  int64_t *ca, *cb;
  int64_t *unit; /* [nfeat][D], exponents scaled by 2^max_rung */
  double *val;   /* [nfeat][N] */
  double *vmin, *vmax, *vminabs, *vmaxabs;
  int64_t rung_begin[ORC_MAX_RUNG + 2];
  int64_t slots[ORC_MAX_RUNG + 1];
  int64_t reasons[ORC_MAX_RUNG + 1][6];
  int have_counts[ORC_MAX_RUNG + 1];
  int uops[6], nu;
  int bops[6], nb;
  double exp_arg_max;
  int rules;          /* R15 active */
  uint64_t deny[64];  /* symmetric pair rule, by primary input index */
  uint64_t opdeny[12];
  uint64_t *leaves;   /* [nfeat] set of primary input indices among the leaves */
} orc_space;

/* ---------------------------------------------------------------- sums */

typedef struct { double s, c; } nsum;

static void nadd(nsum *a, double x) {
  double t = a->s + x;
  if (fabs(a->s) >= fabs(x)) a->c += (a->s - t) + x;
  else a->c += (x - t) + a->s;
  a->s = t;
}
static double nval(const nsum *a) { return a->s + a->c; }

/* --------------------------------------------------------- small helpers */

static uint64_t tri(uint64_t n) { return n * (n - 1) / 2; } /* T(n) = n(n-1)/2 */

static void summarise(const double *v, int64_t N, double *mn, double *mx, double *mna,
                      double *mxa) {
  double a = v[0], b = v[0], c = fabs(v[0]), d = fabs(v[0]);
  for (int64_t s = 1; s < N; ++s) {
    if (v[s] < a) a = v[s];
    if (v[s] > b) b = v[s];
    if (fabs(v[s]) < c) c = fabs(v[s]);
    if (fabs(v[s]) > d) d = fabs(v[s]);
  }
  *mn = a; *mx = b; *mna = c; *mxa = d;
}

/* R7: realised test on a fully evaluated candidate. */
static int realised_ok(const orc_space *S, const double *v) {
  const int64_t N = S->N;
  for (int64_t s = 0; s < N; ++s)
    if (!isfinite(v[s])) return 0;
  if (S->P.fmin_std_rel < 0) return 1;
  nsum a = {0, 0};
  for (int64_t s = 0; s < N; ++s) nadd(&a, v[s]);
  double mean = nval(&a) / (double)N;
  nsum q = {0, 0}, r = {0, 0};
  for (int64_t s = 0; s < N; ++s) {
    double d = v[s] - mean;
    nadd(&q, d * d);
    nadd(&r, v[s] * v[s]);
  }
  double sd = sqrt(nval(&q) / (double)N);
  double rms = sqrt(nval(&r) / (double)N);
  return sd > S->P.fmin_std_rel * rms;
}

static int is_unary(int op) { return op >= ORC_SQUARE && op <= ORC_LOG; }

/* R15.  The operands satisfy the rules themselves (every stored feature
   passed this test when it was generated), so only what the new node adds is
   checked: a forbidden pair with one leaf in each operand (a leaf shared by
   both operands occurs twice), and a forbidden leaf below op. */
static int rule_fails(const orc_space *S, int op, int64_t a, int64_t b) {
  const uint64_t la = S->leaves[a], lb = is_unary(op) ? 0 : S->leaves[b];
  for (int p = 0; p < 64; ++p) {
    if (!((la >> p) & 1)) continue;
    for (int q = 0; q < 64; ++q)
      if (((lb >> q) & 1) && ((S->deny[p] >> q) & 1)) return 1;
  }
  const uint64_t all = la | lb;
  for (int p = 0; p < 64; ++p)
    if (((all >> p) & 1) && ((S->opdeny[op] >> p) & 1)) return 1;
  return 0;
}

/* R3-R6: a-priori tests of op(a[, b]).  Returns the reason code (0 = pass)
   and writes the result's unit vector and complexity. */
static int apriori(const orc_space *S, int op, int64_t a, int64_t b, int64_t *u, int32_t *cx) {
  const int D = S->D;
  const int64_t *ua = S->unit + a * D;
  const int64_t *ub = is_unary(op) ? NULL : S->unit + b * D;
  int k;
  switch (op) {
  case ORC_SQUARE: for (k = 0; k < D; ++k) u[k] = 2 * ua[k]; break;
  case ORC_CUBE: for (k = 0; k < D; ++k) u[k] = 3 * ua[k]; break;
  case ORC_INV: for (k = 0; k < D; ++k) u[k] = -ua[k]; break;
  case ORC_SQRT:
    for (k = 0; k < D; ++k) {
      if (ua[k] % 2 != 0) { fprintf(stderr, "oracle: odd exponent under sqrt\n"); abort(); }
      u[k] = ua[k] / 2;
    }
    break;
  case ORC_EXP:
  case ORC_LOG:
    if (S->P.explog_dimensionless)
      for (k = 0; k < D; ++k)
        if (ua[k] != 0) return ORC_R_UNIT;
    for (k = 0; k < D; ++k) u[k] = 0;
    break;
  case ORC_ADD:
  case ORC_SUB:
  case ORC_ABSDIFF:
    if (S->P.unit_check_addsub)
      for (k = 0; k < D; ++k)
        if (ua[k] != ub[k]) return ORC_R_UNIT;
    for (k = 0; k < D; ++k) u[k] = ua[k];
    break;
  case ORC_MUL: for (k = 0; k < D; ++k) u[k] = ua[k] + ub[k]; break;
  case ORC_DIV: for (k = 0; k < D; ++k) u[k] = ua[k] - ub[k]; break;
  case ORC_RDIV: for (k = 0; k < D; ++k) u[k] = ub[k] - ua[k]; break;
  default: abort();
  }
  int32_t c = S->cplx[a] + 1 + (is_unary(op) ? 0 : S->cplx[b]);
  *cx = c;
  if (S->P.max_complexity > 0 && c > S->P.max_complexity) return ORC_R_COMPLEXITY;
  if (S->rules && rule_fails(S, op, a, b)) return ORC_R_COMPLEXITY;

  const double mna = S->vminabs[a], mxa = S->vmaxabs[a];
  switch (op) {
  case ORC_LOG: if (!(S->vmin[a] > 0)) return ORC_R_DOMAIN; break;
  case ORC_SQRT: if (!(S->vmin[a] >= 0)) return ORC_R_DOMAIN; break;
  case ORC_INV: if (!(mna > 0)) return ORC_R_DOMAIN; break;
  case ORC_EXP: if (!(S->vmax[a] <= 80.0)) return ORC_R_DOMAIN; break;
  case ORC_DIV: if (!(S->vminabs[b] > 0)) return ORC_R_DOMAIN; break;
  case ORC_RDIV: if (!(mna > 0)) return ORC_R_DOMAIN; break;
  default: break;
  }

  double B = 0;
  switch (op) {
  case ORC_SQUARE: B = mxa * mxa; break;
  case ORC_CUBE: B = (mxa * mxa) * mxa; break;
  case ORC_INV: B = 1.0 / mna; break;
  case ORC_SQRT: B = sqrt(mxa); break;
  case ORC_EXP:
    if (!(S->vmax[a] <= S->exp_arg_max)) return ORC_R_MAGNITUDE;
    return ORC_VALID;
  case ORC_LOG: return ORC_VALID;
  case ORC_ADD:
  case ORC_SUB:
  case ORC_ABSDIFF: B = mxa + S->vmaxabs[b]; break;
  case ORC_MUL: B = mxa * S->vmaxabs[b]; break;
  case ORC_DIV: B = mxa / S->vminabs[b]; break;
  case ORC_RDIV: B = S->vmaxabs[b] / mna; break;
  default: abort();
  }
  if (!(B <= S->P.fmax_max)) return ORC_R_MAGNITUDE;
  return ORC_VALID;
}

static void evaluate(const orc_space *S, int op, int64_t a, int64_t b, double *v) {
  const int64_t N = S->N;
  const double *x = S->val + a * N;
  const double *y = is_unary(op) ? NULL : S->val + b * N;
  int64_t s;
  switch (op) {
  case ORC_SQUARE: for (s = 0; s < N; ++s) v[s] = x[s] * x[s]; break;
  case ORC_CUBE: for (s = 0; s < N; ++s) v[s] = (x[s] * x[s]) * x[s]; break;
  case ORC_INV: for (s = 0; s < N; ++s) v[s] = 1.0 / x[s]; break;
  case ORC_SQRT: for (s = 0; s < N; ++s) v[s] = sqrt(x[s]); break;
  case ORC_EXP: for (s = 0; s < N; ++s) v[s] = exp(x[s]); break;
  case ORC_LOG: for (s = 0; s < N; ++s) v[s] = log(x[s]); break;
  case ORC_ADD: for (s = 0; s < N; ++s) v[s] = x[s] + y[s]; break;
  case ORC_SUB: for (s = 0; s < N; ++s) v[s] = x[s] - y[s]; break;
  case ORC_MUL: for (s = 0; s < N; ++s) v[s] = x[s] * y[s]; break;
  case ORC_DIV: for (s = 0; s < N; ++s) v[s] = x[s] / y[s]; break;
  case ORC_RDIV: for (s = 0; s < N; ++s) v[s] = y[s] / x[s]; break;
  case ORC_ABSDIFF: for (s = 0; s < N; ++s) v[s] = fabs(x[s] - y[s]); break;
  default: abort();
  }
}

/* R1: flat index p of rung r -> (op, a, b).  The pair index is recovered by
   bisection on the integers, T(i) <= q* < T(i+1). */
static int decode_flat(const orc_space *S, int r, uint64_t p, int *op, int64_t *a, int64_t *b) {
  const int64_t o = S->rung_begin[r - 1];
  const int64_t m = S->rung_begin[r] - o;
  const uint64_t nun = (uint64_t)S->nu * (uint64_t)m;
  if (p < nun) {
    *a = o + (int64_t)(p / (uint64_t)S->nu);
    *op = S->uops[p % (uint64_t)S->nu];
    *b = -1;
    return 0;
  }
  if (S->nb == 0) return -1;
  const uint64_t pp = p - nun;
  const uint64_t q = pp / (uint64_t)S->nb;
  const int slot = (int)(pp % (uint64_t)S->nb);
  const uint64_t qs = q + tri((uint64_t)o);
  int64_t lo = o, hi = o + m - 1;
  if (m <= 0) return -1;
  while (lo < hi) {
    int64_t mid = lo + (hi - lo + 1) / 2;
    if (tri((uint64_t)mid) <= qs) lo = mid;
    else hi = mid - 1;
  }
  const uint64_t j = qs - tri((uint64_t)lo);
  if (j >= (uint64_t)lo) return -1;
  *op = S->bops[slot];
  *a = lo;
  *b = (int64_t)j;
  return 0;
}

static uint64_t rung_slots(const orc_space *S, int r) {
  const uint64_t o = (uint64_t)S->rung_begin[r - 1];
  const uint64_t m = (uint64_t)(S->rung_begin[r] - S->rung_begin[r - 1]);
  const uint64_t pairs = (m == 0) ? 0 : tri(m) + m * o;
  return (uint64_t)S->nu * m + (uint64_t)S->nb * pairs;
}

/* Reason code of slot p of rung r; v is scratch of length N. */
static int slot_reason(const orc_space *S, int r, uint64_t p, double *v) {
  int op; int64_t a, b;
  int64_t u[ORC_MAX_DIMS]; int32_t cx;
  if (decode_flat(S, r, p, &op, &a, &b) != 0) return -1;
  int why = apriori(S, op, a, b, u, &cx);
  if (why) return why;
  evaluate(S, op, a, b, v);
  return realised_ok(S, v) ? ORC_VALID : ORC_R_REALISED;
}

static int grow(orc_space *S, int64_t n) {
  const int64_t N = S->N, D = S->D > 0 ? S->D : 1;
#define GROW(ptr, type, per)                                                            \
  do {                                                                                  \
    void *q = realloc(S->ptr, (size_t)(n) * (size_t)(per) * sizeof(type));              \
    if (!q) return -1;                                                                  \
    S->ptr = (type *)q;                                                                 \
  } while (0)
  GROW(op, int32_t, 1); GROW(rung, int32_t, 1); GROW(cplx, int32_t, 1);
  GROW(ca, int64_t, 1); GROW(cb, int64_t, 1); GROW(leaves, uint64_t, 1);
  GROW(unit, int64_t, D);
  GROW(val, double, N);
  GROW(vmin, double, 1); GROW(vmax, double, 1); GROW(vminabs, double, 1); GROW(vmaxabs, double, 1);
#undef GROW
  return 0;
}

static void set_summary(orc_space *S, int64_t f) {
  summarise(S->val + f * S->N, S->N, &S->vmin[f], &S->vmax[f], &S->vminabs[f], &S->vmaxabs[f]);
}

/* ------------------------------------------------------------ public API */

void orc_space_free(orc_space *S) {
  if (!S) return;
  free(S->op); free(S->rung); free(S->cplx); free(S->ca); free(S->cb); free(S->unit); free(S->leaves);
  free(S->val); free(S->vmin); free(S->vmax); free(S->vminabs); free(S->vmaxabs);
  free(S);
}

int orc_space_build(const orc_params *P, orc_space **out) {
  *out = NULL;
  if (P->n_samples < 2 || P->n_primary < 1 || P->n_dims < 0 || P->n_dims > ORC_MAX_DIMS ||
      P->max_rung < 1 || P->max_rung > ORC_MAX_RUNG)
    return -1;
  orc_space *S = (orc_space *)calloc(1, sizeof(orc_space));
  if (!S) return -2;
  S->P = *P;
  S->P.X = NULL; S->P.units = NULL; S->P.pair_deny = NULL; S->P.op_deny = NULL;
  if (P->pair_deny || P->op_deny) {
    if (P->n_primary > 64) { free(S); return -1; }
    S->rules = 1;
    for (int64_t p = 0; p < P->n_primary; ++p)
      for (int64_t q = 0; q < P->n_primary; ++q)
        if (P->pair_deny && (((P->pair_deny[p] >> q) & 1) || ((P->pair_deny[q] >> p) & 1)))
          S->deny[p] |= (uint64_t)1 << q;
    for (int o = 0; o < 12; ++o) S->opdeny[o] = P->op_deny ? P->op_deny[o] : 0;
  }
  S->N = P->n_samples;
  S->D = P->n_dims;
  S->exp_arg_max = log(P->fmax_max);
  for (int c = 0; c <= 5; ++c)
    if (P->op_mask & (1u << c)) S->uops[S->nu++] = c;
  for (int c = 6; c <= 11; ++c)
    if (P->op_mask & (1u << c)) S->bops[S->nb++] = c;

  const int64_t N = S->N;
  const int64_t scale = (int64_t)1 << P->max_rung;
  if (grow(S, P->n_primary)) { orc_space_free(S); return -2; }
  /* Rung 0: primaries that pass the realised test (R1, R7). */
  int64_t nf = 0;
  S->slots[0] = P->n_primary;
  for (int64_t p = 0; p < P->n_primary; ++p) {
    const double *x = P->X + p * N;
    if (!realised_ok(S, x)) { S->reasons[0][ORC_R_REALISED]++; continue; }
    memcpy(S->val + nf * N, x, (size_t)N * sizeof(double));
    S->op[nf] = ORC_PRIMARY; S->rung[nf] = 0; S->cplx[nf] = 0;
    S->ca[nf] = p; S->cb[nf] = -1;
    S->leaves[nf] = S->rules ? (uint64_t)1 << p : 0;
    for (int k = 0; k < S->D; ++k) S->unit[nf * S->D + k] = (int64_t)P->units[p * S->D + k] * scale;
    set_summary(S, nf);
    S->reasons[0][ORC_VALID]++;
    ++nf;
  }
  S->nfeat = nf;
  S->have_counts[0] = 1;
  S->rung_begin[0] = 0;
  S->rung_begin[1] = nf;

  /* Rungs 1..max_rung-1 are materialised (R1). */
  for (int r = 1; r < P->max_rung; ++r) {
    const uint64_t ns = rung_slots(S, r);
    S->slots[r] = (int64_t)ns;
    signed char *why = (signed char *)malloc(ns ? ns : 1);
    if (!why) { orc_space_free(S); return -2; }
#pragma omp parallel
    {
      double *v = (double *)malloc((size_t)N * sizeof(double));
#pragma omp for schedule(dynamic, 4096)
      for (int64_t p = 0; p < (int64_t)ns; ++p) why[p] = (signed char)slot_reason(S, r, (uint64_t)p, v);
      free(v);
    }
    int64_t nvalid = 0;
    for (uint64_t p = 0; p < ns; ++p) {
      if (why[p] < 0) { free(why); orc_space_free(S); return -3; }
      S->reasons[r][(int)why[p]]++;
      if (why[p] == ORC_VALID) ++nvalid;
    }
    if (grow(S, S->nfeat + nvalid)) { free(why); orc_space_free(S); return -2; }
    for (uint64_t p = 0; p < ns; ++p) {
      if (why[p] != ORC_VALID) continue;
      int op; int64_t a, b; int32_t cx;
      int64_t u[ORC_MAX_DIMS];
      decode_flat(S, r, p, &op, &a, &b);
      apriori(S, op, a, b, u, &cx);
      const int64_t f = S->nfeat++;
      evaluate(S, op, a, b, S->val + f * N);
      S->op[f] = op; S->rung[f] = r; S->cplx[f] = cx; S->ca[f] = a; S->cb[f] = b;
      S->leaves[f] = S->leaves[a] | (is_unary(op) ? 0 : S->leaves[b]);
      for (int k = 0; k < S->D; ++k) S->unit[f * S->D + k] = u[k];
      set_summary(S, f);
    }
    free(why);
    S->have_counts[r] = 1;
    S->rung_begin[r + 1] = S->nfeat;
  }
  *out = S;
  return 0;
}

int64_t orc_n_features(const orc_space *S) { return S->nfeat; }
int64_t orc_rung_begin(const orc_space *S, int r) { return S->rung_begin[r]; }
uint64_t orc_rung_slots(const orc_space *S, int r) {
  if (r == 0) return (uint64_t)S->slots[0];
  return rung_slots(S, r);
}
uint64_t orc_total_candidates(const orc_space *S) {
  return (uint64_t)S->nfeat + rung_slots(S, S->P.max_rung);
}

/* Counts of rung r by reason (index 0 = valid).  Rung max_rung is evaluated
   in full on the first call. */
int orc_rung_counts(orc_space *S, int r, int64_t *slots, int64_t *reasons6) {
  if (r < 0 || r > S->P.max_rung) return -1;
  if (!S->have_counts[r]) {
    const uint64_t ns = rung_slots(S, r);
    int64_t cnt[6] = {0, 0, 0, 0, 0, 0};
    int bad = 0;
#pragma omp parallel
    {
      int64_t lc[6] = {0, 0, 0, 0, 0, 0};
      double *v = (double *)malloc((size_t)S->N * sizeof(double));
#pragma omp for schedule(dynamic, 4096)
      for (int64_t p = 0; p < (int64_t)ns; ++p) {
        int w = slot_reason(S, r, (uint64_t)p, v);
        if (w < 0) bad = 1;
        else lc[w]++;
      }
      free(v);
#pragma omp critical
      for (int c = 0; c < 6; ++c) cnt[c] += lc[c];
    }
    if (bad) return -3;
    S->slots[r] = (int64_t)ns;
    for (int c = 0; c < 6; ++c) S->reasons[r][c] = cnt[c];
    S->have_counts[r] = 1;
  }
  *slots = S->slots[r];
  for (int c = 0; c < 6; ++c) reasons6[c] = S->reasons[r][c];
  return 0;
}

/* Global id -> (rung, op, a, b).  Returns 0 on success. */
int orc_decode(const orc_space *S, uint64_t id, int32_t *rung, int32_t *op, int64_t *a, int64_t *b) {
  if (id < (uint64_t)S->nfeat) {
    *rung = S->rung[id]; *op = S->op[id]; *a = S->ca[id]; *b = S->cb[id];
    return 0;
  }
  const int r = S->P.max_rung;
  const uint64_t p = id - (uint64_t)S->nfeat;
  if (p >= rung_slots(S, r)) return -1;
  int o; int64_t x, y;
  if (decode_flat(S, r, p, &o, &x, &y)) return -1;
  *rung = r; *op = o; *a = x; *b = y;
  return 0;
}

static int write_expr(const orc_space *S, int64_t f, int op, int64_t a, int64_t b, char *buf, int64_t len);

static int write_feature(const orc_space *S, int64_t f, char *buf, int64_t len) {
  return write_expr(S, f, S->op[f], S->ca[f], S->cb[f], buf, len);
}

/* Canonical strings: x<p>, sq(A), cb(A), inv(A), sqrt(A), exp(A), log(A),
   (A+B), (A-B), (A*B), (A/B), (B/A), |A-B| with A = f_a, B = f_b. */
static int write_expr(const orc_space *S, int64_t f, int op, int64_t a, int64_t b, char *buf, int64_t len) {
  (void)f;
  if (op == ORC_PRIMARY) return snprintf(buf, (size_t)len, "x%lld", (long long)a) >= len ? -1 : 0;
  char *A = (char *)malloc((size_t)len), *B = (char *)malloc((size_t)len);
  int rc = 0;
  if (!A || !B) { free(A); free(B); return -1; }
  if (write_feature(S, a, A, len)) rc = -1;
  if (!rc && !is_unary(op) && write_feature(S, b, B, len)) rc = -1;
  if (!rc) {
    int n = 0;
    switch (op) {
    case ORC_SQUARE: n = snprintf(buf, (size_t)len, "sq(%s)", A); break;
    case ORC_CUBE: n = snprintf(buf, (size_t)len, "cb(%s)", A); break;
    case ORC_INV: n = snprintf(buf, (size_t)len, "inv(%s)", A); break;
    case ORC_SQRT: n = snprintf(buf, (size_t)len, "sqrt(%s)", A); break;
    case ORC_EXP: n = snprintf(buf, (size_t)len, "exp(%s)", A); break;
    case ORC_LOG: n = snprintf(buf, (size_t)len, "log(%s)", A); break;
    case ORC_ADD: n = snprintf(buf, (size_t)len, "(%s+%s)", A, B); break;
    case ORC_SUB: n = snprintf(buf, (size_t)len, "(%s-%s)", A, B); break;
    case ORC_MUL: n = snprintf(buf, (size_t)len, "(%s*%s)", A, B); break;
    case ORC_DIV: n = snprintf(buf, (size_t)len, "(%s/%s)", A, B); break;
    case ORC_RDIV: n = snprintf(buf, (size_t)len, "(%s/%s)", B, A); break;
    case ORC_ABSDIFF: n = snprintf(buf, (size_t)len, "|%s-%s|", A, B); break;
    default: rc = -1;
    }
    if (n >= len) rc = -1;
  }
  free(A); free(B);
  return rc;
}

int orc_expr_string(const orc_space *S, uint64_t id, char *buf, int64_t len) {
  int32_t r, op; int64_t a, b;
  if (orc_decode(S, id, &r, &op, &a, &b)) return -1;
  if (id < (uint64_t)S->nfeat) return write_feature(S, (int64_t)id, buf, len);
  return write_expr(S, -1, op, a, b, buf, len);
}

/* Values of candidate id (length N) and its reason code (0 = valid).  For an
   a-priori invalid candidate the values are left untouched. */
int orc_candidate(const orc_space *S, uint64_t id, double *v, int32_t *reason) {
  if (id < (uint64_t)S->nfeat) {
    memcpy(v, S->val + id * S->N, (size_t)S->N * sizeof(double));
    *reason = ORC_VALID;
    return 0;
  }
  const int r = S->P.max_rung;
  const uint64_t p = id - (uint64_t)S->nfeat;
  if (p >= rung_slots(S, r)) return -1;
  int op; int64_t a, b; int64_t u[ORC_MAX_DIMS]; int32_t cx;
  decode_flat(S, r, p, &op, &a, &b);
  int why = apriori(S, op, a, b, u, &cx);
  if (why) { *reason = why; return 0; }
  evaluate(S, op, a, b, v);
  *reason = realised_ok(S, v) ? ORC_VALID : ORC_R_REALISED;
  return 0;
}

/* Reason code of every candidate with global id in [id_begin, id_end), one
   byte each (R8: the first failing test; stored features are valid by
   construction).  The mask "Physics-Informed Constraints" describes, candidate
   by candidate.  Returns 0, or -1 for a range outside the space. */
int orc_reasons(const orc_space *S, uint64_t id_begin, uint64_t id_end, int8_t *why) {
  const uint64_t total = orc_total_candidates(S);
  if (id_end < id_begin || id_end > total) return -1;
  const int r = S->P.max_rung;
#pragma omp parallel
  {
    double *v = (double *)malloc((size_t)S->N * sizeof(double));
#pragma omp for schedule(dynamic, 1024)
    for (int64_t i = (int64_t)id_begin; i < (int64_t)id_end; ++i) {
      if (i < S->nfeat) why[i - (int64_t)id_begin] = ORC_VALID;
      else why[i - (int64_t)id_begin] = (int8_t)slot_reason(S, r, (uint64_t)(i - S->nfeat), v);
    }
    free(v);
  }
  return 0;
}

/* Unit vector of candidate id (R3: exponents as integers over the common
   denominator 2^max_rung) into unit[n_dims].  Returns 1 when the op's unit
   rule holds, 0 when it fails (unit left unspecified), -1 for an id outside
   the space. */
int orc_candidate_unit(const orc_space *S, uint64_t id, int64_t *unit) {
  if (id < (uint64_t)S->nfeat) {
    for (int k = 0; k < S->D; ++k) unit[k] = S->unit[id * S->D + k];
    return 1;
  }
  const uint64_t p = id - (uint64_t)S->nfeat;
  if (p >= rung_slots(S, S->P.max_rung)) return -1;
  int op; int64_t a, b; int32_t cx;
  if (decode_flat(S, S->P.max_rung, p, &op, &a, &b)) return -1;
  return apriori(S, op, a, b, unit, &cx) == ORC_R_UNIT ? 0 : 1;
}

int orc_feature_info(const orc_space *S, int64_t f, int32_t *cplx, int64_t *unit, double *summ4) {
  if (f < 0 || f >= S->nfeat) return -1;
  *cplx = S->cplx[f];
  for (int k = 0; k < S->D; ++k) unit[k] = S->unit[f * S->D + k];
  summ4[0] = S->vmin[f]; summ4[1] = S->vmax[f]; summ4[2] = S->vminabs[f]; summ4[3] = S->vmaxabs[f];
  return 0;
}

/* --------------------------------------------------------------- scoring */

typedef struct {
  int T;
  int64_t N;
  double *yc;  /* [T][N] centred targets */
  double *syy; /* [T] */
} targets;

static int targets_init(targets *G, const double *Y, int T, int64_t N) {
  G->T = T; G->N = N;
  G->yc = (double *)malloc((size_t)T * (size_t)N * sizeof(double));
  G->syy = (double *)malloc((size_t)T * sizeof(double));
  if (!G->yc || !G->syy) return -2;
  for (int t = 0; t < T; ++t) {
    nsum a = {0, 0};
    for (int64_t s = 0; s < N; ++s) nadd(&a, Y[t * N + s]);
    double mean = nval(&a) / (double)N;
    nsum q = {0, 0};
    for (int64_t s = 0; s < N; ++s) {
      double d = Y[t * N + s] - mean;
      G->yc[t * N + s] = d;
      nadd(&q, d * d);
    }
    G->syy[t] = nval(&q);
    if (!(G->syy[t] > 0)) return -1;
  }
  return 0;
}
static void targets_free(targets *G) { free(G->yc); free(G->syy); }

/* R9 for every target. */
static void score_values(const targets *G, const double *v, double *out) {
  const int64_t N = G->N;
  nsum a = {0, 0};
  for (int64_t s = 0; s < N; ++s) nadd(&a, v[s]);
  const double mean = nval(&a) / (double)N;
  nsum q = {0, 0};
  for (int64_t s = 0; s < N; ++s) {
    double d = v[s] - mean;
    nadd(&q, d * d);
  }
  const double sxx = nval(&q);
  for (int t = 0; t < G->T; ++t) {
    nsum c = {0, 0};
    const double *y = G->yc + (int64_t)t * N;
    for (int64_t s = 0; s < N; ++s) nadd(&c, (v[s] - mean) * y[s]);
    out[t] = fabs(nval(&c)) / sqrt(sxx * G->syy[t]);
  }
}

typedef struct { double score; uint64_t id; } hit;

static int hit_cmp(const void *x, const void *y) {
  const hit *a = (const hit *)x, *b = (const hit *)y;
  if (a->score > b->score) return -1;
  if (a->score < b->score) return 1;
  return (a->id < b->id) ? -1 : (a->id > b->id);
}

typedef struct { hit *h; int64_t n, cap; } hitlist;

static int hl_push(hitlist *L, double s, uint64_t id, int64_t k) {
  if (L->n == L->cap) {
    if (L->n >= 2 * k && L->n >= 4096) {
      qsort(L->h, (size_t)L->n, sizeof(hit), hit_cmp);
      L->n = k;
    } else {
      int64_t nc = L->cap ? 2 * L->cap : 1024;
      hit *q = (hit *)realloc(L->h, (size_t)nc * sizeof(hit));
      if (!q) return -2;
      L->h = q; L->cap = nc;
    }
  }
  L->h[L->n].score = s; L->h[L->n].id = id; L->n++;
  return 0;
}

/* SIS screen of global ids [id_begin, id_end) (R1, R9, R10).  mode 0: one
   top-k list per target; mode 1: one aggregated list.  out_ids/out_scores
   are [L][k] with L = T (mode 0) or 1; n_out[L] gets each list's length.
   counts6 (optional) receives the reason counts of the screened range. */
int orc_screen(const orc_space *S, const double *Y, int T, int64_t k, int mode, uint64_t id_begin,
               uint64_t id_end, uint64_t *out_ids, double *out_scores, int64_t *n_out, int64_t *counts6) {
  const uint64_t total = orc_total_candidates(S);
  if (T < 1 || k < 1 || id_begin > id_end || id_end > total || (mode != 0 && mode != 1)) return -1;
  targets G;
  int rc = targets_init(&G, Y, T, S->N);
  if (rc) { targets_free(&G); return rc; }
  const int L = mode == 0 ? T : 1;
  int nth = 1;
#ifdef _OPENMP
  nth = omp_get_max_threads();
#endif
  hitlist *lists = (hitlist *)calloc((size_t)nth * (size_t)L, sizeof(hitlist));
  int64_t cnt[6] = {0, 0, 0, 0, 0, 0};
  int err = 0;
#pragma omp parallel
  {
    int tid = 0;
#ifdef _OPENMP
    tid = omp_get_thread_num();
#endif
    double *v = (double *)malloc((size_t)S->N * sizeof(double));
    double *sc = (double *)malloc((size_t)T * sizeof(double));
    int64_t lc[6] = {0, 0, 0, 0, 0, 0};
#pragma omp for schedule(dynamic, 1024)
    for (int64_t g = (int64_t)id_begin; g < (int64_t)id_end; ++g) {
      int32_t why;
      if (orc_candidate(S, (uint64_t)g, v, &why)) { err = 1; continue; }
      lc[why]++;
      if (why) continue;
      score_values(&G, v, sc);
      if (mode == 0) {
        for (int t = 0; t < T; ++t)
          if (hl_push(&lists[tid * L + t], sc[t], (uint64_t)g, k)) err = 1;
      } else {
        double a = 0;
        for (int t = 0; t < T; ++t) a += sc[t] * sc[t];
        if (hl_push(&lists[tid * L], sqrt(a / T), (uint64_t)g, k)) err = 1;
      }
    }
    free(v); free(sc);
#pragma omp critical
    for (int c = 0; c < 6; ++c) cnt[c] += lc[c];
  }
  if (!err) {
    for (int l = 0; l < L; ++l) {
      int64_t tot = 0;
      for (int th = 0; th < nth; ++th) tot += lists[th * L + l].n;
      hit *all = (hit *)malloc((size_t)(tot ? tot : 1) * sizeof(hit));
      int64_t w = 0;
      for (int th = 0; th < nth; ++th) {
        memcpy(all + w, lists[th * L + l].h, (size_t)lists[th * L + l].n * sizeof(hit));
        w += lists[th * L + l].n;
      }
      qsort(all, (size_t)tot, sizeof(hit), hit_cmp);
      int64_t n = tot < k ? tot : k;
      for (int64_t i = 0; i < n; ++i) {
        out_ids[l * k + i] = all[i].id;
        out_scores[l * k + i] = all[i].score;
      }
      n_out[l] = n;
      free(all);
    }
  }
  for (int i = 0; i < nth * L; ++i) free(lists[i].h);
  free(lists);
  targets_free(&G);
  if (counts6)
    for (int c = 0; c < 6; ++c) counts6[c] = cnt[c];
  return err ? -3 : 0;
}

/* Reason and per-target score of each listed id (scores of invalid ids are
   set to NaN).  scores is [n][T]. */
int orc_score_ids(const orc_space *S, const double *Y, int T, const uint64_t *ids, int64_t n,
                  double *scores, int32_t *reasons) {
  targets G;
  int rc = targets_init(&G, Y, T, S->N);
  if (rc) { targets_free(&G); return rc; }
  const uint64_t total = orc_total_candidates(S);
  int err = 0;
#pragma omp parallel
  {
    double *v = (double *)malloc((size_t)S->N * sizeof(double));
#pragma omp for schedule(dynamic, 16)
    for (int64_t i = 0; i < n; ++i) {
      int32_t why = -1;
      if (ids[i] >= total || orc_candidate(S, ids[i], v, &why)) { err = 1; continue; }
      reasons[i] = why;
      if (why) {
        for (int t = 0; t < T; ++t) scores[i * T + t] = NAN;
        continue;
      }
      score_values(&G, v, scores + i * T);
    }
    free(v);
  }
  targets_free(&G);
  return err ? -1 : 0;
}

/* ------------------------------------------------- redundancy (R16) */

/* FP64 Pearson correlation of two value vectors, two-pass with
   Neumaier-compensated sums. */
static double pearson(const double *a, const double *b, int64_t N) {
  nsum sa = {0, 0}, sb = {0, 0};
  for (int64_t s = 0; s < N; ++s) { nadd(&sa, a[s]); nadd(&sb, b[s]); }
  const double ma = nval(&sa) / (double)N, mb = nval(&sb) / (double)N;
  nsum qa = {0, 0}, qb = {0, 0}, c = {0, 0};
  for (int64_t s = 0; s < N; ++s) {
    const double da = a[s] - ma, db = b[s] - mb;
    nadd(&qa, da * da);
    nadd(&qb, db * db);
    nadd(&c, da * db);
  }
  return nval(&c) / sqrt(nval(&qa) * nval(&qb));
}

/* R16.  orc_screen (mode 0 or 1) followed by redundancy removal: each list
   holds the top-k of the non-redundant candidates of the screened range
   (partners are sought in the same range).  The lists are screened with a
   larger length kk and walked in rank order; an entry is decided only when
   every candidate within sqrt(2 tau) of its score is in the list, else kk
   doubles.  n_redundant (optional, per list) counts the redundant entries
   passed over; margin (optional) gets min | (1 - |rho|) - tau | over the
   correlations computed. */
int orc_screen_dedup(const orc_space *S, const double *Y, int T, int64_t k, int mode, double tau,
                     uint64_t id_begin, uint64_t id_end, uint64_t *out_ids, double *out_scores, int64_t *n_out,
                     int64_t *n_redundant, double *margin) {
  if (!(tau > 0) || !(tau < 1) || k < 1 || T < 1 || (mode != 0 && mode != 1) || id_begin > id_end) return -1;
  const int L = mode == 0 ? T : 1;
  const int64_t N = S->N;
  const double w = sqrt(2.0 * tau) * (1.0 + 1e-9) + 1e-13;
  const int64_t range = (int64_t)(id_end - id_begin);
  int64_t kk = 4 * k;
  double mg = INFINITY;
  double *va = (double *)malloc((size_t)N * sizeof(double));
  double *vb = (double *)malloc((size_t)N * sizeof(double));
  int rc = 0;
  for (;;) {
    if (kk > range) kk = range > 0 ? range : 1;
    uint64_t *ids = (uint64_t *)malloc((size_t)L * (size_t)kk * sizeof(uint64_t));
    double *sc = (double *)malloc((size_t)L * (size_t)kk * sizeof(double));
    int64_t *nl = (int64_t *)malloc((size_t)L * sizeof(int64_t));
    rc = orc_screen(S, Y, T, kk, mode, id_begin, id_end, ids, sc, nl, NULL);
    int undecided = 0;
    for (int l = 0; l < L && rc == 0 && !undecided; ++l) {
      const uint64_t *li = ids + (int64_t)l * kk;
      const double *ls = sc + (int64_t)l * kk;
      const int64_t n = nl[l];
      const int full = (n == kk) && (kk < range);
      int64_t kept = 0, red = 0;
      for (int64_t i = 0; i < n && kept < k; ++i) {
        if (full && !(ls[i] - w > ls[n - 1])) { undecided = 1; break; }
        int redundant = 0;
        for (int dir = -1; dir <= 1 && !redundant; dir += 2)
          for (int64_t j = i + dir; j >= 0 && j < n && fabs(ls[j] - ls[i]) <= w; j += dir) {
            if (li[j] >= li[i]) continue;
            int32_t r1, r2;
            if (orc_candidate(S, li[i], va, &r1) || orc_candidate(S, li[j], vb, &r2)) { rc = -3; break; }
            const double rho = fabs(pearson(va, vb, N));
            const double d = fabs((1.0 - rho) - tau);
            if (d < mg) mg = d;
            if (rho >= 1.0 - tau) { redundant = 1; break; }
          }
        if (redundant) { ++red; continue; }
        out_ids[(int64_t)l * k + kept] = li[i];
        out_scores[(int64_t)l * k + kept] = ls[i];
        ++kept;
      }
      n_out[l] = kept;
      if (n_redundant) n_redundant[l] = red;
    }
    free(ids); free(sc); free(nl);
    if (rc || !undecided || kk >= range) break;
    kk *= 2;
  }
  free(va); free(vb);
  if (margin) *margin = mg;
  return rc;
}

/* ------------------------------------------------------- residual loop */

/* Least squares with intercept of y on the columns C[0..p-1] (each length N)
   by Householder QR of the N x (p+1) design matrix [1, C].  Writes the
   coefficients beta[0..p] (intercept first) and returns the RMSE of the
   explicit residual y - A beta; returns INFINITY if A is rank deficient. */
static double ls_qr(const double *const *C, int p, const double *y, int64_t N, double *beta) {
  const int q = p + 1;
  double *A = (double *)malloc((size_t)N * (size_t)q * sizeof(double));
  double *b = (double *)malloc((size_t)N * sizeof(double));
  double *w = (double *)malloc((size_t)N * sizeof(double));
  for (int64_t s = 0; s < N; ++s) {
    A[s * q] = 1.0;
    for (int c = 0; c < p; ++c) A[s * q + c + 1] = C[c][s];
    b[s] = y[s];
  }
  double R[5][5], cn[5];
  int ok = 1;
  for (int c = 0; c < q; ++c) {
    double t = 0;
    for (int64_t s = 0; s < N; ++s) t += A[s * q + c] * A[s * q + c];
    cn[c] = sqrt(t);
  }
  for (int c = 0; c < q; ++c) {
    double nrm = 0, scale = 0;
    for (int64_t s = c; s < N; ++s) if (fabs(A[s * q + c]) > scale) scale = fabs(A[s * q + c]);
    if (scale == 0) { ok = 0; break; }
    for (int64_t s = c; s < N; ++s) { double t = A[s * q + c] / scale; nrm += t * t; }
    nrm = scale * sqrt(nrm);
    double alpha = A[c * q + c] > 0 ? -nrm : nrm;
    /* Householder vector w = x - alpha e1, reflect columns c..q-1 and b. */
    for (int64_t s = c; s < N; ++s) w[s] = A[s * q + c];
    w[c] -= alpha;
    double ww = 0;
    for (int64_t s = c; s < N; ++s) ww += w[s] * w[s];
    if (ww == 0) { ok = 0; break; }
    for (int cc = c; cc < q; ++cc) {
      double d = 0;
      for (int64_t s = c; s < N; ++s) d += w[s] * A[s * q + cc];
      double f = 2.0 * d / ww;
      for (int64_t s = c; s < N; ++s) A[s * q + cc] -= f * w[s];
    }
    double d = 0;
    for (int64_t s = c; s < N; ++s) d += w[s] * b[s];
    double f = 2.0 * d / ww;
    for (int64_t s = c; s < N; ++s) b[s] -= f * w[s];
    for (int cc = 0; cc < q; ++cc) R[c][cc] = cc >= c ? A[c * q + cc] : 0.0;
  }
  double rmse = INFINITY;
  if (ok) /* a column (numerically) in the span of the earlier ones */
    for (int c = 0; c < q; ++c) if (!(fabs(R[c][c]) > 1e-12 * cn[c])) ok = 0;
  if (ok) {
    for (int c = q - 1; c >= 0; --c) {
      double t = b[c];
      for (int cc = c + 1; cc < q; ++cc) t -= R[c][cc] * beta[cc];
      beta[c] = t / R[c][c];
    }
    nsum e = {0, 0};
    for (int64_t s = 0; s < N; ++s) {
      double f = beta[0];
      for (int c = 0; c < p; ++c) f += beta[c + 1] * C[c][s];
      double r = y[s] - f;
      nadd(&e, r * r);
    }
    rmse = sqrt(nval(&e) / (double)N);
  }
  free(A); free(b); free(w);
  return rmse;
}

/* R11.  desc_ids[Dmax], rmse[Dmax], coefs[Dmax][Dmax+1] (intercept first,
   zero-padded), sis_ids[Dmax][k], n_sis[Dmax], residual[N] (final r_D). */
int orc_residual_loop(const orc_space *S, const double *y, int Dmax, int64_t k, uint64_t *desc_ids,
                      double *rmse, double *coefs, uint64_t *sis_ids, int64_t *n_sis, double *residual) {
  const int64_t N = S->N;
  if (Dmax < 1 || Dmax > 4 || k < 1) return -1;
  double *r = (double *)malloc((size_t)N * sizeof(double));
  double *cols = (double *)malloc((size_t)(Dmax + 1) * (size_t)N * sizeof(double));
  double *sc = (double *)malloc((size_t)k * sizeof(double));
  memcpy(r, y, (size_t)N * sizeof(double));
  int rc = 0;
  for (int D = 1; D <= Dmax && !rc; ++D) {
    int64_t nk = 0;
    uint64_t *S_D = sis_ids + (int64_t)(D - 1) * k;
    rc = orc_screen(S, r, 1, k, 0, 0, orc_total_candidates(S), S_D, sc, &nk, NULL);
    if (rc) break;
    n_sis[D - 1] = nk;
    double best = INFINITY;
    uint64_t best_id = UINT64_MAX;
    double best_beta[5] = {0, 0, 0, 0, 0};
    int err = 0;
#pragma omp parallel
    {
      double *v = (double *)malloc((size_t)N * sizeof(double));
      const double *C[5];
      double beta[5];
      for (int d = 0; d < D - 1; ++d) C[d] = cols + (int64_t)d * N;
      C[D - 1] = v;
#pragma omp for schedule(dynamic, 4)
      for (int64_t i = 0; i < nk; ++i) {
        int dup = 0;
        for (int d = 0; d < D - 1; ++d) if (desc_ids[d] == S_D[i]) dup = 1;
        if (dup) continue;
        int32_t why;
        if (orc_candidate(S, S_D[i], v, &why) || why) { err = 1; continue; }
        double e = ls_qr(C, D, y, N, beta);
#pragma omp critical
        if (e < best || (e == best && S_D[i] < best_id)) {
          best = e; best_id = S_D[i];
          for (int c = 0; c <= D; ++c) best_beta[c] = beta[c];
        }
      }
      free(v);
    }
    if (err || best_id == UINT64_MAX) { rc = -3; break; }
    desc_ids[D - 1] = best_id;
    rmse[D - 1] = best;
    for (int c = 0; c <= Dmax; ++c) coefs[(D - 1) * (Dmax + 1) + c] = c <= D ? best_beta[c] : 0.0;
    int32_t why;
    orc_candidate(S, best_id, cols + (int64_t)(D - 1) * N, &why);
    for (int64_t s = 0; s < N; ++s) {
      double f = best_beta[0];
      for (int d = 0; d < D; ++d) f += best_beta[d + 1] * cols[(int64_t)d * N + s];
      r[s] = y[s] - f;
    }
  }
  if (!rc) memcpy(residual, r, (size_t)N * sizeof(double));
  free(r); free(cols); free(sc);
  return rc;
}

/* ------------------------------------------------------ exhaustive L0 */

typedef struct { double rmse; int64_t pos[4]; } l0_hit;

/* (rmse ascending, positions lexicographically ascending) */
static int l0_before(const l0_hit *a, const l0_hit *b, int D) {
  if (a->rmse != b->rmse) return a->rmse < b->rmse;
  for (int c = 0; c < D; ++c)
    if (a->pos[c] != b->pos[c]) return a->pos[c] < b->pos[c];
  return 0;
}

static void l0_insert(l0_hit *top, int64_t *n, int64_t m, const l0_hit *h, int D) {
  if (*n == m && !l0_before(h, &top[m - 1], D)) return;
  int64_t i = *n < m ? (*n)++ : m - 1;
  while (i > 0 && l0_before(h, &top[i - 1], D)) { top[i] = top[i - 1]; --i; }
  top[i] = *h;
}

/* Eq. 1 solved exhaustively over a listed subspace (the sparsifying step of
   SISSO that follows SIS): among all D-subsets {p_0 < .. < p_{D-1}} of the
   positions of ids[0..n), the least-squares fit with intercept of y on the
   candidates' columns (ls_qr: Householder QR, rank rule of R11) with the
   smallest RMSE.  Keeps the m_top best full-rank subsets in the order
   (RMSE ascending, positions lexicographically ascending); best_pos[m_top][D],
   best_rmse[m_top]; *n_found = how many were kept. */
int orc_l0_search(const orc_space *S, const double *y, const uint64_t *ids, int64_t n, int D, int64_t m_top,
                  int64_t *best_pos, double *best_rmse, int64_t *n_found) {
  const int64_t N = S->N;
  if (D < 1 || D > 4 || n < D || m_top < 1) return -1;
  double *cols = (double *)malloc(sizeof(double) * (size_t)n * (size_t)N);
  if (!cols) return -1;
  int err = 0;
  for (int64_t i = 0; i < n; ++i) {
    int32_t why = 0;
    if (ids[i] >= orc_total_candidates(S) || orc_candidate(S, ids[i], cols + i * N, &why) || why) err = 1;
  }
  if (err) { free(cols); return -1; }
  l0_hit *all = NULL;
  int64_t n_all = 0;
#pragma omp parallel
  {
    l0_hit *top = (l0_hit *)malloc(sizeof(l0_hit) * (size_t)m_top);
    int64_t nt = 0;
#pragma omp for schedule(dynamic, 1)
    for (int64_t p0 = 0; p0 < n; ++p0) {
      int64_t p[4] = {p0, 0, 0, 0};
      /* the remaining positions in lexicographic order */
      int c = 1;
      if (D > 1) p[1] = p0;
      for (;;) {
        if (c == D) {
          const double *C[4];
          double beta[5];
          for (int q = 0; q < D; ++q) C[q] = cols + p[q] * N;
          l0_hit h;
          h.rmse = ls_qr(C, D, y, N, beta);
          for (int q = 0; q < 4; ++q) h.pos[q] = q < D ? p[q] : 0;
          if (h.rmse < INFINITY) l0_insert(top, &nt, m_top, &h, D);
          --c;
          if (c < 1) break;
          continue;
        }
        /* advance position c (c >= 1) */
        ++p[c];
        if (p[c] > n - (D - c)) {  /* no room for the later positions */
          --c;
          if (c < 1) break;
          continue;
        }
        ++c;
        if (c < D) p[c] = p[c - 1];
      }
    }
#pragma omp critical
    if (nt > 0) {  /* (realloc to zero bytes may return NULL) */
      l0_hit *grown = (l0_hit *)realloc(all, sizeof(l0_hit) * (size_t)(n_all + nt));
      if (grown) {
        all = grown;
        memcpy(all + n_all, top, sizeof(l0_hit) * (size_t)nt);
        n_all += nt;
      } else {
        err = 1;
      }
    }
    free(top);
  }
  int64_t nf = 0;
  if (!err) {
    l0_hit *top = (l0_hit *)malloc(sizeof(l0_hit) * (size_t)m_top);
    for (int64_t i = 0; i < n_all; ++i) l0_insert(top, &nf, m_top, &all[i], D);
    for (int64_t i = 0; i < nf; ++i) {
      best_rmse[i] = top[i].rmse;
      for (int q = 0; q < D; ++q) best_pos[i * D + q] = top[i].pos[q];
    }
    free(top);
  }
  *n_found = nf;
  free(all);
  free(cols);
  return err ? -1 : 0;
}

/* Margins of the threshold tests (R5-R7) over flat slots [p0, p1) of rung r:
   how close any decision came to flipping, as relative distances, so that a
   1-ulp difference in an FP64 library function (exp, log) between two
   implementations cannot change a mask when every margin is well above the
   rounding level.  out[0] magnitude: |B - fmax_max| / fmax_max over slots
   reaching the magnitude test (exp: |max - log(fmax_max)| / log(fmax_max));
   out[1] exp domain: |max - 80| / 80; out[2] realised: |sd - f*rms| / (f*rms)
   over slots reaching the realised test with finite values; out[3] the
   number of slots whose tests were examined.  Minima start at +inf. */
int orc_margins(const orc_space *S, int r, uint64_t p0, uint64_t p1, double *out) {
  if (r < 1 || r > S->P.max_rung) return -1;
  const uint64_t slots = rung_slots(S, r);
  if (p1 > slots) p1 = slots;
  double m_mag = INFINITY, m_exp = INFINITY, m_real = INFINITY, n_seen = 0;
  const int64_t N = S->N;
#pragma omp parallel reduction(min : m_mag, m_exp, m_real) reduction(+ : n_seen)
  {
    double *v = (double *)malloc(sizeof(double) * (size_t)N);
#pragma omp for schedule(dynamic, 256)
    for (int64_t pi = (int64_t)p0; pi < (int64_t)p1; ++pi) {
      int op; int64_t a, b;
      int64_t u[ORC_MAX_DIMS]; int32_t cx;
      if (decode_flat(S, r, (uint64_t)pi, &op, &a, &b) != 0) continue;
      n_seen += 1;
      const int why = apriori(S, op, a, b, u, &cx);
      if (why == ORC_R_UNIT || why == ORC_R_COMPLEXITY) continue;
      if (op == ORC_EXP) {
        const double d = fabs(S->vmax[a] - 80.0) / 80.0;
        if (d < m_exp) m_exp = d;
        if (why == ORC_R_DOMAIN) continue;
        const double e = fabs(S->vmax[a] - S->exp_arg_max) / fabs(S->exp_arg_max);
        if (e < m_mag) m_mag = e;
      } else if (why != ORC_R_DOMAIN && op != ORC_LOG) {
        const double mna = S->vminabs[a], mxa = S->vmaxabs[a];
        double B = 0;
        switch (op) {
        case ORC_SQUARE: B = mxa * mxa; break;
        case ORC_CUBE: B = (mxa * mxa) * mxa; break;
        case ORC_INV: B = 1.0 / mna; break;
        case ORC_SQRT: B = sqrt(mxa); break;
        case ORC_ADD: case ORC_SUB: case ORC_ABSDIFF: B = mxa + S->vmaxabs[b]; break;
        case ORC_MUL: B = mxa * S->vmaxabs[b]; break;
        case ORC_DIV: B = mxa / S->vminabs[b]; break;
        case ORC_RDIV: B = S->vmaxabs[b] / mna; break;
        default: break;
        }
        const double d = fabs(B - S->P.fmax_max) / S->P.fmax_max;
        if (d < m_mag) m_mag = d;
      }
      if (why != ORC_VALID || S->P.fmin_std_rel < 0) continue;
      evaluate(S, op, a, b, v);
      int fin = 1;
      for (int64_t t = 0; t < N; ++t) fin &= isfinite(v[t]) != 0;
      if (!fin) continue;
      nsum q0 = {0, 0};
      for (int64_t t = 0; t < N; ++t) nadd(&q0, v[t]);
      const double mean = nval(&q0) / (double)N;
      nsum q = {0, 0}, rr = {0, 0};
      for (int64_t t = 0; t < N; ++t) {
        const double d = v[t] - mean;
        nadd(&q, d * d);
        nadd(&rr, v[t] * v[t]);
      }
      const double sd = sqrt(nval(&q) / (double)N), lim = S->P.fmin_std_rel * sqrt(nval(&rr) / (double)N);
      if (lim > 0) {
        const double d = fabs(sd - lim) / lim;
        if (d < m_real) m_real = d;
      }
    }
    free(v);
  }
  out[0] = m_mag;
  out[1] = m_exp;
  out[2] = m_real;
  out[3] = n_seen;
  return 0;
}

int orc_num_threads(void) {
#ifdef _OPENMP
  return omp_get_max_threads();
#else
  return 1;
#endif
}
