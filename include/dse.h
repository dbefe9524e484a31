/*
 * dse.h -- C ABI of the GB300 (sm_103a) descriptor-screening engine.
 *
 * The engine implements the data-parallel hot path of SISSO-style symbolic
 * regression as used by DISCOVER (arXiv 2602.06986): generate rung-k
 * candidate features from user-provided primary features and an operator
 * library, drop dimensionally invalid ones, evaluate every candidate on every
 * sample and keep the top k by Sure Independence Screening (|Pearson|
 * correlation) against one or many targets or residuals.
 *
 * Passages of the paper each call follows:
 *   dse_build_space     "Software Description": candidates are generated from
 *                       user features and operator libraries, iteratively;
 *                       "Physics-Informed Constraints": dimensionally invalid
 *                       expressions are excluded early; "Design Philosophy
 *                       and Constraints": restrictions on operators and
 *                       complexity.
 *   dse_sis_screen      "Software Description": candidates are evaluated
 *                       against target data; SIS is the screening of SISSO
 *                       ("Summary"); the workflow figure places screening
 *                       between generation and sparse model selection.
 *   dse_ls_refit        Eq. 1 (L0-constrained least squares, ||beta||_0 <= D)
 *                       approximated greedily, OMP being one of the strategies
 *                       named in "Software Description".
 *   dse_residual_loop   the two above chained on the device for D = 1..n_iter
 *                       (screen the residual, refit, new residual).
 *   dse_sis_screen_batched  dse_sis_screen over many independent data sets at
 *                       once (no counterpart in the paper: an engineering form).
 *
 * Conventions (all calls):
 *   - Every entry point returns a dse_status; 0 is success.  No C++ exception
 *     crosses the ABI.  dse_last_error() gives a message for the last failure
 *     of the calling thread.
 *   - Buffers passed in are owned by the caller and are copied (or read in
 *     place on the device) before the call returns or, for device buffers,
 *     before the enqueued work completes; they must stay valid until then.
 *   - Handles (dse_space, dse_result) are owned by the library and released
 *     with the matching *_free call.
 *   - Work is enqueued on the stream given in the descriptor (a cudaStream_t,
 *     NULL for the legacy default stream).  dse_build_space,
 *     dse_topk_fetch, dse_result_stats, dse_space_counts, dse_ls_refit,
 *     dse_residual_loop, dse_batch_fetch and dse_batch_stats wait for it.
 *   - There is no CPU fallback: without a usable CUDA device every call that
 *     computes returns DSE_ECUDA.
 *
 * Operator codes are also the slot order of a pair and the bit positions of
 * op_mask: unary  0 x^2, 1 x^3, 2 x^-1, 3 sqrt, 4 exp, 5 log;
 *          binary 6 a+b, 7 a-b, 8 a*b, 9 a/b, 10 b/a, 11 |a-b|.
 * The "/" of the paper's operator lists is the two slots 9 and 10.
 *
 * Global candidate ids: ids [0, n_stored) are the stored features of rungs
 * 0..max_rung-1 (rung by rung, each rung in generation order); id
 * n_stored + p is flat index p of rung max_rung, whose unary block
 * (feature-major, op-minor) precedes its binary block (pair (i, j), i from the
 * newest stored rung, j < i, slot-minor).  Flat indices count every slot,
 * valid or not.
 */
#ifndef DSE_H
#define DSE_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef int32_t dse_status;
#define DSE_OK 0
#define DSE_EINVAL (-1)    /* bad argument or descriptor */
#define DSE_ENOMEM (-2)    /* device or host allocation failed */
#define DSE_ECUDA (-3)     /* CUDA runtime error or no usable device */
#define DSE_ERANGE (-4)    /* id or id range outside the candidate space */
#define DSE_ETIMEOUT (-5)  /* a bounded device-side wait ran out */
#define DSE_EOVERFLOW (-6) /* space, unit exponent or buffer beyond limits */
#define DSE_EBOUNDS (-7)   /* bounds-checked build only: an index check
                              failed (the access was skipped)              */

enum {
  DSE_OP_SQUARE = 0, DSE_OP_CUBE = 1, DSE_OP_INV = 2, DSE_OP_SQRT = 3, DSE_OP_EXP = 4,
  DSE_OP_LOG = 5, DSE_OP_ADD = 6, DSE_OP_SUB = 7, DSE_OP_MUL = 8, DSE_OP_DIV = 9,
  DSE_OP_RDIV = 10, DSE_OP_ABSDIFF = 11, DSE_OP_PRIMARY = 15
};

/* Why a candidate is excluded; tests are applied in this order. */
enum {
  DSE_VALID = 0,
  DSE_R_UNIT = 1,       /* unit rule of the op fails                        */
  DSE_R_COMPLEXITY = 2, /* form: more operator nodes than max_complexity, or
                           a user rule (pair_deny / op_deny) fails          */
  DSE_R_DOMAIN = 3,     /* log/sqrt/inverse/divisor/exp domain from summaries */
  DSE_R_MAGNITUDE = 4,  /* a-priori bound on max|value| above fmax_max       */
  DSE_R_REALISED = 5    /* non-finite value or degenerate (std <= f * rms)   */
};

enum { DSE_MODE_PER_TARGET = 0, DSE_MODE_AGGREGATED = 1 };

enum {
  DSE_PREC_FP32 = 0,   /* FP32 evaluation and sums with error bounds, FP64
                          re-score of the top-k boundary                    */
  DSE_PREC_FP64 = 1,   /* plain FP64 evaluation and sums (the comparator)   */
  DSE_PREC_BF16X3 = 2, /* FP32 evaluation, BF16x3 tensor-core contraction   */
  DSE_PREC_AUTO = 3    /* FP32 for few targets, BF16x3 for many             */
};

typedef struct dse_space dse_space;
typedef struct dse_result dse_result;

/* Feature space.  X holds n_primary rows of FP64 samples (row stride ld_x
   elements).  With sample_idx (host array of n_samples column indices,
   duplicates allowed, e.g. a bootstrap resample) the space is built on those
   columns; without it on columns [0, n_samples).  units holds n_primary rows
   of n_dims integer exponents (host).  Rungs 0..max_rung-1 are materialised in
   FP64 (and FP32) on the device; rung max_rung is never stored. */
typedef struct {
  int64_t n_samples;            /* N >= 2                                     */
  int64_t n_primary;            /* >= 1                                       */
  int32_t n_dims;               /* unit dimensions, 0..8                      */
  int32_t max_rung;             /* 1..3                                       */
  const double *X;              /* [n_primary][ld_x], host or device          */
  int64_t ld_x;                 /* >= n_samples, or >= max(sample_idx)+1      */
  int32_t x_on_device;          /* 1: X is a device pointer                   */
  int32_t reserved0;
  const int64_t *sample_idx;    /* optional host gather list, NULL = identity */
  const int32_t *units;         /* host [n_primary][n_dims]; NULL iff n_dims 0 */
  uint32_t op_mask;             /* bit per op code                            */
  int32_t max_complexity;       /* <= 0: no cap                               */
  int32_t unit_check_addsub;    /* + - |a-b| need equal units                 */
  int32_t explog_dimensionless; /* exp and log need dimensionless operands    */
  double fmax_max;              /* magnitude limit, finite and > 0 (1e15)     */
  double fmin_std_rel;          /* degeneracy limit (1e-8); < 0 disables       */
  void *stream;                 /* cudaStream_t                               */
  /* Optional user rules on variable combinations and functional forms
     ("Design Philosophy and Constraints"); either may be NULL; non-NULL
     needs n_primary <= 64.  Primaries are named by their input index.
     pair_deny: host [n_primary] rows; bit q of row p (or of row q, bit p)
       forbids primaries p and q in one expression; bit p of row p lets p
       occur as a leaf at most once.
     op_deny: host [12] rows by op code; bit p of row o forbids primary p
       anywhere below an application of op o.
     A candidate failing a rule gets reason DSE_R_COMPLEXITY, tested after
     the complexity cap; rung-0 primaries are never excluded by a rule. */
  const uint64_t *pair_deny;
  const uint64_t *op_deny;
} dse_space_desc;

dse_status dse_build_space(const dse_space_desc *desc, dse_space **out);
void dse_space_free(dse_space *space);

/* Number of stored features (rungs 0..max_rung-1) and of all candidate ids. */
dse_status dse_space_size(const dse_space *space, int64_t *n_stored, uint64_t *n_total);

/* Per-rung counts.  slots = flat slots of the rung; reasons[6] = counts by
   reason code (index 0 = valid).  For rungs below max_rung the counts are
   exact after every test.  For rung max_rung the a-priori tests (unit,
   complexity, domain, magnitude) are counted by a device pass over all slots;
   reasons[0] is then the a-priori valid count and reasons[5] is -1 (the
   realised test needs evaluation: see dse_result_stats). Synchronises. */
dse_status dse_space_counts(dse_space *space, int32_t rung, uint64_t *slots, int64_t reasons[6]);

/* Expression of a candidate: its rung, op code and operand ids (stored
   feature ids; for a primary a = primary index, b = -1; for unary ops b = -1). */
typedef struct {
  int32_t rung, op;
  int64_t a, b;
} dse_expr;

dse_status dse_decode(const dse_space *space, uint64_t id, dse_expr *out);
/* Unit vectors of n candidates ("Physics-Informed Constraints": the units
   an expression carries follow from its op's exponent rule): for ids[i]
   (host array), n_dims exponents as integers over the common denominator
   2^max_rung into units[i * n_dims ...] (host; may be NULL when n_dims is
   0) and unit_ok[i] = 1 when the op's unit rule holds, 0 when the candidate
   is dimensionally invalid (its row is then 0).  Stored features are read
   from the table, last-rung candidates computed by the screen's own device
   rule.  DSE_ERANGE for an id outside the space.  Synchronises. */
dse_status dse_candidate_units(dse_space *space, const uint64_t *ids, int64_t n, int64_t *units,
                               int8_t *unit_ok);
/* Canonical text: x<p>, sq(A), cb(A), inv(A), sqrt(A), exp(A), log(A),
   (A+B), (A-B), (A*B), (A/B), (B/A), |A-B| with A the higher-id operand. */
dse_status dse_expr_string(const dse_space *space, uint64_t id, char *buf, int64_t len);

/* SIS screen.  Y holds n_targets rows of N FP64 target (or residual) values,
   row stride ld_y elements.  Candidates with global ids in [id_begin, id_end)
   are screened (id_end = 0 means all).  PER_TARGET keeps k per target,
   AGGREGATED keeps k by sqrt(mean_t score_t^2).  The top-k is exact: set and
   order (score descending, id ascending) equal those of FP64 scores, apart
   from candidates whose scores differ by less than the reported bounds. */
typedef struct {
  const double *Y;       /* [n_targets][ld_y], host or device               */
  int64_t ld_y;          /* >= N                                            */
  int32_t y_on_device;
  int32_t n_targets;     /* >= 1                                            */
  int64_t k;             /* >= 1                                            */
  int32_t mode;          /* DSE_MODE_*                                      */
  int32_t precision;     /* DSE_PREC_*                                      */
  uint64_t id_begin, id_end;
  void *stream;          /* cudaStream_t                                    */
  int32_t flags;         /* DSE_FLAG_* bits                                 */
  int32_t reserved0;
  double dedup_tau;      /* with DSE_FLAG_DEDUP: 0 < tau < 0.5 (0: 1e-10)   */
  /* Optional DEVICE buffer of (id_end - id_begin) bytes, id_end as resolved
     (0: the whole space), or NULL.  The screen writes, in id order, the
     reason code (DSE_VALID or DSE_R_*) it assigned to each candidate of the
     range: the per-candidate mask of "Physics-Informed Constraints" (units)
     and of the domain, magnitude and realised tests, the same decisions the
     reasons counts of dse_stats sum up.  Not a device pointer: DSE_EINVAL. */
  int8_t *reasons;
  /* Optional DEVICE buffer of 2 x n_lists x (id_end - id_begin) floats, or
     NULL: for each candidate of the range (id order) and each list, the
     score s and error bound eps that the screening kernels computed for it
     before any re-score (the FP32 or tensor-core interval, or the FP64
     value of an escalated candidate), as (s, eps) pairs; NaN where a
     candidate has none (excluded by a test).  For checking the error bounds
     candidate by candidate.  Not a device pointer: DSE_EINVAL. */
  float *intervals;
} dse_screen_desc;

/* dse_screen_desc.flags: record CUDA events around each kernel group so that
   dse_result_stats reports their device time (kernel_ms). */
#define DSE_FLAG_TIMING 1
/* Score-based redundancy removal ("Design Philosophy and Constraints": the
   search space is reduced by rules; SISSO's convention of keeping one of
   several interchangeable features).  Two valid candidates are equivalent
   when the FP64 Pearson correlation of their values has |rho| >= 1 - tau
   (then they are interchangeable in any linear model with intercept); a
   candidate is redundant when an equivalent candidate of the screened range
   has a smaller id.  Each list then holds the top-k of the non-redundant
   candidates.  Equivalent candidates' scores differ by at most sqrt(2 tau),
   so partners are sought only within that score window of a longer list
   (4k entries, doubled until every decision is covered); an entry is
   decided only when the list holds every candidate of its window.  The
   call synchronises the stream (it reads the list state between rounds).
   Not available in dse_residual_loop or the batched screens. */
#define DSE_FLAG_DEDUP 2
/* Evaluate the binary slots sample by sample.  Without it a single-target
   FP32 screen with 16 <= N <= 2048 takes the statistics of a*b, a/b, b/a,
   a+b and a-b from Gram contractions on the tensor cores, and a per-target
   screen of 2..16 targets (DSE_PREC_AUTO or DSE_PREC_BF16X3) does the same
   for any N >= 16 (same results: the same bounds contract, the same
   re-score of the list); |a-b| is always evaluated sample by sample.  With
   the flag, those screens run the CUDA-core kernels (one target) or the
   sample-by-sample tensor-core kernel (2..16 targets). */
#define DSE_FLAG_DIRECT 4
/* Time only the product/quotient kernel group (kernel_ms[1]; the other
   entries 0): two events per screen instead of five, for timing that kernel
   inside a longer measured region.  DSE_FLAG_TIMING takes precedence. */
#define DSE_FLAG_TIMING_MAIN 8

dse_status dse_sis_screen(dse_space *space, const dse_screen_desc *desc, dse_result **out);
void dse_result_free(dse_result *result);

/* Copies list `list` (a target index, or 0 in AGGREGATED mode) of a result:
   up to cap entries of (id, score, err_bound) in rank order, host or device
   pointers (checked with cudaPointerGetAttributes); n_out gets the list
   length.  Any of idx/score/err_bound may be NULL.  Synchronises. */
dse_status dse_topk_fetch(dse_result *result, int32_t list, uint64_t *idx, double *score,
                          double *err_bound, int64_t cap, int64_t *n_out);

typedef struct {
  int64_t screened;        /* candidate ids in the screened range            */
  int64_t reasons[6];      /* over the screened range, by reason code        */
  int64_t evaluated;       /* candidates whose statistics were accumulated   */
  int64_t buffered;        /* candidate-target entries that passed threshold */
  int64_t escalated;       /* FP64 decisions of the realised test            */
  int64_t rescored;        /* candidate-target pairs re-scored (FP32-pair
                              sums with a bound, FP64 where they do not
                              apply)                                         */
  int32_t reruns;          /* screens repeated after a buffer overflow       */
  int32_t precision_used;  /* DSE_PREC_* actually run                        */
  double max_err_bound;    /* largest bound among returned scores            */
  int64_t valid_by_group[3];  /* valid candidates scored by the stored/unary,
                                 product/quotient and sum/difference kernels */
  double kernel_ms[4];     /* with DSE_FLAG_TIMING (DSE_FLAG_TIMING_MAIN:
                              the second entry only): device time of the
                              stored/unary kernel (with the Gram operand
                              images when the products take that path), the
                              product/quotient kernel, the sum/difference
                              kernel and the selection kernels; else 0     */
  int64_t kernel_launches; /* kernels this screen launched                   */
  int64_t redundant;       /* DSE_FLAG_DEDUP: redundant entries passed over
                              while filling the lists (all lists)           */
  int32_t dedup_rounds;    /* DSE_FLAG_DEDUP: list lengths tried (0: off)    */
  int32_t binary_path;     /* DSE_PATH_* that scored the product/quotient
                              slots (0: none in the range)                   */
} dse_stats;

/* dse_stats.binary_path */
#define DSE_PATH_CUDA_CORE 1   /* sample by sample on the CUDA cores        */
#define DSE_PATH_TENSOR 2      /* sample by sample, tensor-core numerators  */
#define DSE_PATH_GRAM 3        /* Gram contraction, one target              */
#define DSE_PATH_GRAM_MT 4     /* Gram contraction, 2..16 targets           */

dse_status dse_result_stats(dse_result *result, dse_stats *out);

/* Batched SIS screen: many independent problems, each with its own space
   (its own primaries, or a sample gather list of a shared data set: a
   cross-validation fold, a bootstrap resample) and its own target, screened
   together with the same semantics as dse_sis_screen in PER_TARGET mode over
   the whole space (stored features and rung max_rung), k per problem.  Each
   kernel group runs once over all problems: work is cut into per-problem
   jobs (candidate runs, pair tiles, pair-list runs) that warps and CTAs take
   from device counters, so small and large problems share the GPU.  The
   paper screens one data set at a time ("Software Description": candidates
   evaluated against the target); batching independent problems is an
   engineering form of the same step with no counterpart there.

   dse_sis_screen_batched plans (job and tile lists, per-problem arguments,
   every buffer, allocated once) and enqueues the first screen on
   desc->stream.  dse_batch_rescreen screens again with new targets (same
   problems) without host-side planning or allocation; with DSE_BATCH_GRAPH
   the whole screen (resets and kernels) is captured once into a CUDA graph
   and replayed.  Results are read with dse_batch_fetch / dse_batch_stats,
   which synchronise; if a problem's candidate buffer overflowed, the batch
   is screened again (eagerly, thresholds kept) before they return.  The
   spaces must outlive the batch and must not be used concurrently by other
   calls while it runs.  The target of problem i has the n_samples of its
   space. */
typedef struct {
  dse_space *space;
  const double *y;        /* n_samples values, host or device              */
  int32_t y_on_device;
  int32_t reserved0;
} dse_batch_item;

typedef struct {
  int64_t k;              /* per problem, >= 1                              */
  int32_t precision;      /* DSE_PREC_FP32 / AUTO (FP32) or DSE_PREC_FP64   */
  int32_t flags;          /* DSE_BATCH_* bits                               */
  void *stream;           /* cudaStream_t                                   */
} dse_batch_desc;

/* dse_batch_desc.flags: replay the screen as a CUDA graph in
   dse_batch_rescreen (captured at its first call). */
#define DSE_BATCH_GRAPH 1

typedef struct dse_batch dse_batch;

dse_status dse_sis_screen_batched(const dse_batch_item *items, int32_t n_items, const dse_batch_desc *desc,
                                  dse_batch **out);
/* Y: the new targets of every problem, concatenated in item order (problem i
   has its space's n_samples values), host or device.  Enqueued. */
dse_status dse_batch_rescreen(dse_batch *batch, const double *Y, int32_t y_on_device);
/* As dse_topk_fetch, for problem `item`. */
dse_status dse_batch_fetch(dse_batch *batch, int32_t item, uint64_t *idx, double *score, double *err_bound,
                           int64_t cap, int64_t *n_out);
/* As dse_result_stats, for problem `item` (kernel_ms: 0; kernel_launches:
   launches of the whole batch screen). */
dse_status dse_batch_stats(dse_batch *batch, int32_t item, dse_stats *out);
void dse_batch_free(dse_batch *batch);

/* One step of the residual loop: least squares with intercept of y (N FP64
   values) on the columns of the `n_fixed` candidates `fixed` plus one
   candidate from `cand` (n_cand ids), for every candidate; picks the one with
   the smallest RMSE (ties: lower id) and writes its id, RMSE, coefficients
   (intercept first, n_fixed + 2 values, host) and the residual y - fit
   (N FP64 values; host or device).  Ids already in `fixed` are skipped.
   Every fit is solved from its column sums (FP32-pair arithmetic, FP64
   where that does not apply) with a bound on its RSS error; every fit that
   could be the best within its bound is redone in FP64, so the pick, its
   RMSE, coefficients and residual are an FP64 fit's.  Synchronises. */
typedef struct {
  const double *y;        /* N values, host or device                       */
  int32_t y_on_device;
  int32_t n_fixed;        /* 0..3                                           */
  const uint64_t *fixed;  /* host                                           */
  const uint64_t *cand;   /* host or device (cand_on_device)                */
  int64_t n_cand;
  int32_t cand_on_device;
  int32_t reserved0;
  void *stream;
} dse_refit_desc;

dse_status dse_ls_refit(dse_space *space, const dse_refit_desc *desc, uint64_t *best_id,
                        double *best_rmse, double *coefs, double *residual);

/* The whole residual loop on the device ("Software Description": SIS to
   retain candidates, then a sparsifying step, OMP being one of the named
   strategies; Eq. 1 approximated greedily): r_0 = y; for D = 1..n_iter the
   SIS screen of r_{D-1} over the whole space (top k, same semantics as
   dse_sis_screen in PER_TARGET mode), then the least-squares refits of
   every retained candidate with the D-1 descriptors chosen so far (as
   dse_ls_refit), the pick of the smallest RMSE and the new residual
   r_D = y - fit.  The screen is planned once and every iteration is
   enqueued back to back with no host round trip; the call waits once at
   the end (and re-runs an iteration on the host-driven path if its
   candidate buffer overflowed).  Synchronises.  Errors: DSE_EINVAL when an
   iteration finds no full-rank fit, DSE_EOVERFLOW on a persistent overflow,
   the codes of dse_sis_screen otherwise.

   Resume: with n_fixed > 0 the descriptors d_1..d_n_fixed are taken as
   chosen (a checkpoint of an earlier call), the fit with all of them and
   its residual r_n_fixed are recomputed on the device (the same refit
   kernels, so the same bits as the iteration that chose d_n_fixed), and the
   loop continues with D = n_fixed + 1..n_iter.  out gets the fixed ids in
   chosen[0..n_fixed), the recomputed fit's RMSE and coefficients in entry
   n_fixed - 1, NaN RMSEs and zero statistics for the earlier entries (the
   checkpoint holds them), and sis_ids rows only for the iterations run. */
typedef struct {
  const double *y;        /* N values, host or device                       */
  int32_t y_on_device;
  int32_t n_iter;         /* 1..4                                           */
  int64_t k;              /* retained candidates per iteration, >= 1        */
  int32_t precision;      /* DSE_PREC_FP32 / AUTO (FP32) or DSE_PREC_FP64   */
  int32_t flags;          /* DSE_FLAG_TIMING / _TIMING_MAIN: kernel_ms of
                             each screen                                     */
  void *stream;           /* cudaStream_t                                   */
  int32_t n_fixed;        /* 0..n_iter-1 descriptors already chosen         */
  int32_t reserved0;
  const uint64_t *fixed;  /* host, n_fixed distinct candidate ids           */
} dse_loop_desc;

typedef struct {
  uint64_t chosen[4];     /* descriptor ids d_1..d_n_iter                   */
  double rmse[4];         /* RMSE of the fit after each iteration           */
  double coefs[4][5];     /* per iteration: intercept, then D coefficients  */
  dse_stats stats[4];     /* statistics of each iteration's screen          */
} dse_loop_result;

/* sis_ids: optional [n_iter][k] (host or device) -- each iteration's SIS
   subspace in rank order, 2^64-1 past its length; residual: optional final
   residual r_n_iter (N values, host or device). */
dse_status dse_residual_loop(dse_space *space, const dse_loop_desc *desc, dse_loop_result *out,
                             uint64_t *sis_ids, double *residual);

/* Exhaustive L0 search over a listed subspace: Eq. 1 (least squares with
   intercept, ||beta||_0 <= D) solved exactly over the n_ids listed candidates
   (typically the union of the SIS subspaces of dse_residual_loop) -- every
   D-subset, the sparsifying step SISSO applies after SIS ("Summary";
   exhaustive search over the subspace rather than the greedy loop).  On the
   device: centred columns, their FP64 Gram matrix, a scan of every subset by
   an incremental Cholesky step (rank rule of dse_ls_refit, pivots in position
   order), the 32 best by explained variance, each refit explicitly in FP64.
   Returns the n_top best subsets by (RMSE ascending, positions ascending):
   top_pos[n_top][dim] positions into ids (ascending within a subset),
   top_rmse[n_top], top_coefs[n_top][dim+1] (intercept first; may be NULL),
   host arrays; n_found = how many (fewer if fewer subsets have full rank).
   Limits: dim 1..3, n_ids <= 65536 (the Gram matrix takes 8 n_ids^2 bytes),
   n_top <= 32.  Synchronises. */
typedef struct {
  const double *y;        /* N values, host or device                       */
  int32_t y_on_device;
  int32_t dim;            /* D: 1..3                                        */
  const uint64_t *ids;    /* n_ids candidate ids, host or device            */
  int64_t n_ids;
  int32_t ids_on_device;
  int32_t n_top;          /* 1..32                                          */
  void *stream;           /* cudaStream_t                                   */
} dse_l0_desc;

dse_status dse_l0_search(dse_space *space, const dse_l0_desc *desc, int64_t *top_pos, double *top_rmse,
                         double *top_coefs, int32_t *n_found);

/* dse_ls_refit without any device allocation.  The paper has no counterpart:
   this is an engineering variant of the same refit step for callers that
   cannot allocate device memory while they run -- applications that hand all
   device memory to their own pool allocator, run under a hard memory budget,
   or have reserved the whole device for other work.  Same arguments and
   results as dse_ls_refit; like it, the call waits for its stream and copies
   the winner to host memory, so it must not be issued on a stream that is
   being captured into a CUDA graph.  Its scratch is one fixed 8 MiB area per
   device, held by every device that loads the library until the process
   exits; the limits are N <= 32768 samples and n_cand <= 16384 candidates,
   and larger requests return DSE_EOVERFLOW with a message (the area is left
   as it was and later calls are unaffected).  The first call on a device
   looks the area's address up (cudaGetSymbolAddress) and keeps it; the
   library must not be used across a cudaDeviceReset.  All calls on a device
   share the one area, which keeps the last call's contents: calls that
   overlap on the GPU (other streams or threads) race, so the caller must
   serialise them. */
dse_status dse_ls_refit_noalloc(dse_space *space, const dse_refit_desc *desc, uint64_t *best_id,
                                double *best_rmse, double *coefs, double *residual);

/* Launch and tile parameters of the planner, process-wide.  An autotuner
   (the package's autotune module) times candidate values on the device and
   installs the fastest.  A zero field keeps the built-in default.  They
   decide which work goes to which kernel and in what order, not what is
   computed: the returned lists are the same apart from ties, the reported
   bounds may differ (e.g. Gram contraction against sample by sample). */
typedef struct {
  int32_t tile_group;        /* consecutive 16/32-row i-blocks per group of
                                pair tiles, 1..64 (defaults: 8 on the tensor
                                cores, 4 on the CUDA cores)                   */
  int32_t seed_stride;       /* every seed_stride-th product tile is launched
                                first to raise the thresholds, 2..4096 (64)   */
  int32_t gram_max_n;        /* largest N for the product Gram contraction,
                                16..2048 (2048)                               */
  int32_t tc_min_targets;    /* DSE_PREC_AUTO takes the tensor cores from this
                                many targets, 1..4096 (8)                     */
  int32_t batch_job_samples; /* batched screens: candidate-samples per job,
                                1024..2^20 (16384)                           */
  int32_t gmt_group;         /* multi-target Gram tiles: a-blocks (128
                                features each) per group of the tile order
                                (the b-blocks are swept once per group),
                                1..4096 (2)                                  */
  int32_t gmt_cluster;       /* multi-target Gram kernel: CTAs per thread-
                                block cluster sharing each b-image chunk by
                                multicast, 1 or 2 (2; one CTA per tile also
                                where the device cannot co-schedule pairs)   */
  int32_t reserved[1];
} dse_tuning;

/* Installs t (NULL: every default).  DSE_EINVAL for a value outside its
   range.  Affects screens planned afterwards. */
dse_status dse_set_tuning(const dse_tuning *t);
/* The values in effect (defaults filled in; tile_group 0 when the two
   defaults differ). */
dse_status dse_get_tuning(dse_tuning *t);

/* Failure detection without a fault.  dse_check_wait runs the bounded
   device wait the pipelined kernels use (an mbarrier polled at most `polls`
   times) on a barrier that completes only when `arrive` is nonzero: it
   returns DSE_ETIMEOUT when the wait runs out, DSE_OK otherwise, and the
   context stays usable either way.  Synchronises. */
dse_status dse_check_wait(uint32_t polls, int32_t arrive, void *stream);

/* Issue rates of the pipes the CUDA-core kernels are bound by, measured on
   the current device: FP32 fused multiply-adds, special-function (MUFU
   ex2) operations and FP64 fused multiply-adds per second over the whole
   device (lane operations; register-resident independent chains in 64
   warps per SM, best of three timed rounds after a warm-up round).  The
   denominators of the ALU rooflines.  Synchronises. */
dse_status dse_measure_peaks(double *fp32_fma_per_s, double *sfu_per_s, double *fp64_fma_per_s, void *stream);

/* Bounds-checked builds (compiled with DSE_CHECK_BOUNDS, libdse_checked.so;
   the substitute for a memory checker where none can run): the screening
   kernels check their gathered and computed indices (feature rows and
   samples, tile coordinates against the operand images, candidate ids
   against the screened range, list positions) and, on a violation, skip
   the access and store DSE_EBOUNDS in the screen's error word, which the
   screen then returns.  dse_bounds_probe runs one such check on the device
   (index against limit) and returns DSE_EBOUNDS when it fails, DSE_OK when
   it holds; in a normal build it returns DSE_EINVAL (no checks compiled). */
dse_status dse_bounds_probe(int64_t index, int64_t limit, void *stream);

/* Test hook: the device allocation after `after` more successful ones
   fails with DSE_ENOMEM (once); a negative value switches the hook off.
   Process-wide. */
void dse_debug_fail_alloc(int64_t after);

/* Number of kernels the library has launched in this process so far. */
int64_t dse_kernel_launches(void);

/* Message of the last failed call on this thread ("" if none). */
const char *dse_last_error(void);

/* Library version string. */
const char *dse_version(void);

#ifdef __cplusplus
}
#endif

#endif /* DSE_H */
