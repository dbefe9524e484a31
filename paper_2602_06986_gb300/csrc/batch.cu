// batch.cu -- batched SIS screens: many independent problems (each its own
// space and target, k per problem, one list per problem) screened with one
// launch per kernel group.
//
// Layout: the problems' targets share one [n][ldy] FP64/FP32 array (row p =
// problem p, ldy = the largest row stride), the candidate buffers are one
// CandBufs with n lists, the escalation list records each entry's problem,
// and every kernel reads its problem's arguments from a device array of
// ScreenArgs (one per problem; a second copy for the additive tiles, whose
// rows are the unit-class order).  Work is cut on the host into jobs of one
// problem each -- runs of stored/unary candidates, pair tiles, runs of the
// concatenated equal-unit pair lists -- whose sizes follow the problem's
// sample count, and warps/CTAs take them from device counters.  A re-screen
// with new targets is a fixed sequence of resets and kernels with no host
// work, which the library can capture once into a CUDA graph and replay.
#include <math.h>
#include <string.h>

#include <algorithm>
#include <new>
#include <vector>

#include "dse_internal.cuh"
#include "plan.cuh"
#include "screen_kernels.cuh"
#include "util.cuh"

namespace dse {
FeatTable table_of(const dse_space *S);
}

using namespace dse;

struct dse_batch {
  int32_t n = 0;
  int32_t prec64 = 0;
  int64_t k = 0;
  int32_t flags = 0;
  cudaStream_t stream = nullptr;
  std::vector<dse_space *> spaces;
  std::vector<int64_t> yoff_h;     // offset of each problem's target in the concatenated input
  int64_t ytotal = 0;
  int32_t ldy = 0;
  std::vector<uint64_t> total, add_total;
  // device state (one allocation)
  void *scratch = nullptr;
  size_t scratch_bytes = 0;
  ScreenArgs *args = nullptr, *args_add = nullptr;
  ScreenArgs A0_mul{}, A0_add{}, A0_esc{};
  SelectArgs S{};
  CandBufs B{};
  Job *feat_jobs = nullptr, *pl_jobs = nullptr;
  int32_t n_feat_jobs = 0, n_pl_jobs = 0;
  int2 *pairs = nullptr;
  Tile *tmul = nullptr, *tadd = nullptr;
  int32_t n_mul = 0, n_add = 0;
  unsigned int *counters = nullptr;  // feature jobs, product tiles, sum tiles, pair-list jobs
  double *Ycat = nullptr;
  int64_t *yoff = nullptr;
  double *y64 = nullptr;
  float *y32 = nullptr, *ysum32 = nullptr;
  unsigned long long *stats = nullptr;  // [n][ST_COUNT]
  int *err = nullptr;
  unsigned int *overflow = nullptr;
  uint64_t *out_id = nullptr;
  double *out_score = nullptr, *out_eps = nullptr;
  int64_t *out_n = nullptr;
  // CUDA graph of the screen (DSE_BATCH_GRAPH)
  cudaStream_t cap_stream = nullptr;
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  int64_t graph_launches = 0;
  // host results of the last screen
  bool fetched = false;
  int32_t reruns = 0;
  int64_t launches = 0;
  std::vector<dse_stats> host_stats;
  std::vector<int64_t> h_out_n;
};

namespace {


int32_t job_len(int64_t N) {
  return (int32_t)std::max<int64_t>(4, std::min<int64_t>(64, (int64_t)tuning().batch_job_samples / N));
}

// Resets, target preparation (with_targets) and every kernel of one screen of
// the batch, enqueued on st.  reset_theta: start the thresholds from zero
// (new targets); a re-run after an overflow keeps them.
dse_status enqueue(dse_batch *b, cudaStream_t st, bool with_targets, bool reset_theta) {
  const int n = b->n;
  const int sms = sm_count();
  const int64_t l0 = launches_so_far();
  DSE_CUDA(cudaMemsetAsync(b->B.count, 0, sizeof(unsigned) * n, st));
  DSE_CUDA(cudaMemsetAsync(b->B.hist, 0, sizeof(unsigned) * n * kNumBins, st));
  DSE_CUDA(cudaMemsetAsync(b->B.hist_hi, 0, sizeof(unsigned) * n * kNumBins, st));
  DSE_CUDA(cudaMemsetAsync(b->B.hist_c, 0, sizeof(unsigned) * n * kCoarse, st));
  DSE_CUDA(cudaMemsetAsync(b->A0_esc.esc_count, 0, sizeof(unsigned), st));
  DSE_CUDA(cudaMemsetAsync(b->stats, 0, sizeof(unsigned long long) * ST_COUNT * n, st));
  DSE_CUDA(cudaMemsetAsync(b->S.n_jobs, 0, sizeof(unsigned), st));
  DSE_CUDA(cudaMemsetAsync(b->counters, 0, sizeof(unsigned) * 4, st));
  DSE_CUDA(cudaMemsetAsync(b->err, 0, sizeof(int), st));
  if (reset_theta) DSE_CUDA(cudaMemsetAsync(b->B.theta, 0, sizeof(float) * n, st));
  if (with_targets)
    launch_targets_batched(b->Ycat, b->yoff, b->args, n, b->ldy, b->y64, b->y32, b->ysum32, b->err, st);
  launch_feature_batched(b->prec64, b->args, b->feat_jobs, b->n_feat_jobs, b->counters, sms, st);
  DSE_TRY(launch_pair_batched(b->prec64, KIND_MUL, b->A0_mul, b->args, sms, st));
  DSE_TRY(launch_pair_batched(b->prec64, KIND_ADD, b->A0_add, b->args_add, sms, st));
  launch_pairlist_batched(b->prec64, b->args, b->pairs, b->pl_jobs, b->n_pl_jobs, b->counters + 3, sms, st);
  launch_escalate(b->A0_esc, sms, st, b->args);
  DSE_TRY(launch_select(b->S, b->A0_esc, sms, st, b->args));
  DSE_CUDA(cudaGetLastError());
  b->launches = launches_so_far() - l0;
  return DSE_OK;
}

dse_status upload_targets(dse_batch *b, const double *Y, bool on_device) {
  if (on_device) {
    DSE_CUDA(cudaMemcpyAsync(b->Ycat, Y, sizeof(double) * b->ytotal, cudaMemcpyDeviceToDevice, b->stream));
  } else {
    DSE_CUDA(cudaMemcpyAsync(b->Ycat, Y, sizeof(double) * b->ytotal, cudaMemcpyHostToDevice, b->stream));
  }
  return DSE_OK;
}

// Screen with the targets now in Ycat: replay the graph (captured at the
// first use) or enqueue eagerly.
dse_status run(dse_batch *b, bool use_graph) {
  b->fetched = false;
  b->reruns = 0;
  if (!use_graph) return enqueue(b, b->stream, true, true);
  if (!b->exec) {
    if (!b->cap_stream) DSE_CUDA(cudaStreamCreateWithFlags(&b->cap_stream, cudaStreamNonBlocking));
    DSE_CUDA(cudaStreamBeginCapture(b->cap_stream, cudaStreamCaptureModeThreadLocal));
    const dse_status s = enqueue(b, b->cap_stream, true, true);
    cudaGraph_t g = nullptr;
    const cudaError_t e = cudaStreamEndCapture(b->cap_stream, &g);
    if (s != DSE_OK) {
      if (g) cudaGraphDestroy(g);
      return s;
    }
    if (e != cudaSuccess) return cuda_status(e, "batch graph capture");
    b->graph = g;
    DSE_CUDA(cudaGraphInstantiate(&b->exec, g, 0));
    b->graph_launches = b->launches;
    note_launches(-b->graph_launches);  // captured, not run: counted at each replay
  }
  DSE_CUDA(cudaGraphLaunch(b->exec, b->stream));
  note_launches(b->graph_launches);
  b->launches = b->graph_launches;
  return DSE_OK;
}

// Wait for the screen; re-run it (eagerly, thresholds kept) while a list
// overflowed its buffer; gather every problem's statistics.
dse_status finish(dse_batch *b) {
  if (b->fetched) return DSE_OK;
  const int n = b->n;
  cudaStream_t st = b->stream;
  for (int attempt = 0;; ++attempt) {
    std::vector<unsigned> ov(n), bc(n);
    std::vector<unsigned long long> hs((size_t)n * ST_COUNT);
    int herr = 0;
    DSE_CUDA(cudaMemcpyAsync(ov.data(), b->overflow, sizeof(unsigned) * n, cudaMemcpyDeviceToHost, st));
    DSE_CUDA(cudaMemcpyAsync(hs.data(), b->stats, sizeof(unsigned long long) * hs.size(), cudaMemcpyDeviceToHost,
                             st));
    DSE_CUDA(cudaMemcpyAsync(&herr, b->err, sizeof(int), cudaMemcpyDeviceToHost, st));
    DSE_CUDA(cudaMemcpyAsync(bc.data(), b->B.count, sizeof(unsigned) * n, cudaMemcpyDeviceToHost, st));
    DSE_CUDA(cudaStreamSynchronize(st));
    if (herr) {
      set_error(herr == DSE_ETIMEOUT   ? "a bounded device wait timed out"
                : herr == DSE_EBOUNDS ? "an index check of the bounds-checked build failed"
                                      : "invalid target (zero variance or not finite)");
      return herr;
    }
    for (int p = 0; p < n; ++p)
      if (hs[(size_t)p * ST_COUNT + ST_ESC_OVERFLOW]) {
        set_error("escalation list overflow");
        return DSE_EOVERFLOW;
      }
    bool any = false;
    for (unsigned v : ov) any |= v != 0;
    if (any && attempt < 8) {
      ++b->reruns;
      DSE_TRY(enqueue(b, st, false, false));
      continue;
    }
    if (any) {
      set_error("candidate buffer overflow persisted");
      return DSE_EOVERFLOW;
    }
    std::vector<int64_t> nout(n);
    std::vector<double> mxe(n);
    DSE_CUDA(cudaMemcpy(nout.data(), b->out_n, sizeof(int64_t) * n, cudaMemcpyDeviceToHost));
    DSE_CUDA(cudaMemcpy(mxe.data(), b->S.max_eps, sizeof(double) * n, cudaMemcpyDeviceToHost));
    b->h_out_n = nout;
    b->host_stats.assign(n, dse_stats{});
    for (int p = 0; p < n; ++p) {
      const unsigned long long *h = hs.data() + (size_t)p * ST_COUNT;
      dse_stats &o = b->host_stats[p];
      o.screened = (int64_t)b->total[p];
      for (int c = 0; c < 6; ++c) o.reasons[c] = (int64_t)h[ST_REASON0 + c];
      o.reasons[DSE_R_UNIT] += (int64_t)b->add_total[p] - (int64_t)h[ST_ADD_SEEN];
      o.evaluated = (int64_t)h[ST_EVALUATED];
      o.buffered = bc[p];
      o.escalated = (int64_t)h[ST_ESCALATED];
      o.rescored = (int64_t)h[ST_RESCORED];
      o.reruns = b->reruns;
      o.precision_used = b->prec64 ? DSE_PREC_FP64 : DSE_PREC_FP32;
      for (int g = 0; g < 3; ++g) o.valid_by_group[g] = (int64_t)h[ST_VALID_G0 + g];
      o.kernel_launches = b->launches;
      o.max_err_bound = nout[p] > 0 ? mxe[p] : 0.0;
    }
    b->fetched = true;
    return DSE_OK;
  }
}

void release(dse_batch *b) {
  if (!b) return;
  if (b->exec) cudaGraphExecDestroy(b->exec);
  if (b->graph) cudaGraphDestroy(b->graph);
  if (b->cap_stream) cudaStreamDestroy(b->cap_stream);
  if (b->scratch) {
    AllocStream as(b->stream);
    dfree(b->scratch);
  }
  delete b;
}

// Plan the batch: per-problem arguments, job and tile lists, buffers.
dse_status plan(const dse_batch_item *items, int32_t n, const dse_batch_desc *d, dse_batch *b) {
  cudaStream_t st = b->stream;
  const int64_t k = d->k;
  b->n = n;
  b->k = k;
  b->prec64 = d->precision == DSE_PREC_FP64;
  b->flags = d->flags;
  b->spaces.resize(n);
  b->yoff_h.resize(n);
  b->total.resize(n);
  b->add_total.resize(n);
  int64_t ldy = 4;
  for (int p = 0; p < n; ++p) {
    dse_space *sp = items[p].space;
    b->spaces[p] = sp;
    b->yoff_h[p] = b->ytotal;
    b->ytotal += sp->N;
    ldy = std::max(ldy, sp->ld);
  }
  b->ldy = (int32_t)ldy;

  // jobs, tiles, pair lists
  std::vector<Job> fjobs, pjobs;
  std::vector<Tile> mul, add;
  std::vector<int64_t> pair_off(n, 0), pair_cnt(n, 0);
  int64_t n_pairs = 0;
  for (int p = 0; p < n; ++p) {
    dse_space *sp = b->spaces[p];
    const RungGeom &g = sp->geom;
    b->total[p] = (uint64_t)sp->n + g.slots;
    const int32_t len = job_len(sp->N);
    const int64_t nf = sp->n + (int64_t)g.um;
    for (int64_t f = 0; f < nf; f += len) fjobs.push_back(Job{p, (int32_t)std::min<int64_t>(len, nf - f), f});
    if (g.nb == 0 || g.n <= g.o) continue;
    bool any_mul = false, any_add = false;
    std::vector<int> addpos;
    for (int s = 0; s < g.nb; ++s) {
      const int op = g.bops[s];
      if (op == DSE_OP_MUL || op == DSE_OP_DIV || op == DSE_OP_RDIV) any_mul = true;
      else {
        any_add = true;
        addpos.push_back(s);
      }
    }
    if (any_mul) {
      const size_t t0 = mul.size();
      triangle_tiles(g.o, g.n - 1, 32, 32, mul);
      for (size_t t = t0; t < mul.size(); ++t) mul[t].prob = p;
    }
    if (any_add) {
      b->add_total[p] = count_slots_mod(g.slots - g.um, g.nb, addpos);
      bool listed = false;
      const bool one_class = !(sp->unit_check_addsub && sp->D > 0) || sp->h_class_begin.size() <= 2;
      if (!one_class) {
        DSE_TRY(equal_unit_pairs(sp, st));
        const uint64_t mm = (uint64_t)(g.n - g.o), oo = (uint64_t)g.o;
        const uint64_t all_pairs = mm ? tri(mm) + mm * oo : 0;
        listed = (uint64_t)sp->n_eq_pairs * 4 <= all_pairs;
      }
      if (listed) {
        pair_off[p] = n_pairs;
        pair_cnt[p] = sp->n_eq_pairs;
        for (int64_t q = 0; q < sp->n_eq_pairs; q += len)
          pjobs.push_back(Job{p, (int32_t)std::min<int64_t>(len, sp->n_eq_pairs - q), n_pairs + q});
        n_pairs += sp->n_eq_pairs;
      } else {
        // one class: class order is id order, so the id triangle of the
        // products serves; else tiles over the unit classes
        const size_t t0 = add.size();
        if (one_class)
          triangle_tiles(g.o, g.n - 1, 32, 32, add);
        else
          class_tiles(sp->h_class_begin, sp->n, 32, 32, 0, add);
        for (size_t t = t0; t < add.size(); ++t) add[t].prob = p;
      }
    }
  }
  if (fjobs.size() > (size_t)INT32_MAX || pjobs.size() > (size_t)INT32_MAX || mul.size() > (size_t)INT32_MAX ||
      add.size() > (size_t)INT32_MAX) {
    set_error("batch too large");
    return DSE_EINVAL;
  }
  b->n_feat_jobs = (int32_t)fjobs.size();
  b->n_pl_jobs = (int32_t)pjobs.size();
  b->n_mul = (int32_t)mul.size();
  b->n_add = (int32_t)add.size();

  // buffers
  const int64_t cap = std::max<int64_t>(8 * k, k + 32768);
  const int64_t esc_cap = 1 << 20;
  SelectArgs &S = b->S;
  CandBufs &B = b->B;
  uint64_t *esc_id = nullptr;
  unsigned *esc_count = nullptr;
  uint32_t *esc_prob = nullptr;
  Scratch sc;
  sc.add(&b->args, (size_t)n);
  sc.add(&b->args_add, (size_t)n);
  sc.add(&b->feat_jobs, fjobs.size());
  sc.add(&b->pl_jobs, pjobs.size());
  sc.add(&b->pairs, (size_t)n_pairs);
  sc.add(&b->tmul, mul.size());
  sc.add(&b->tadd, add.size());
  sc.add(&b->counters, 4);
  sc.add(&b->Ycat, (size_t)b->ytotal);
  sc.add(&b->yoff, (size_t)n);
  sc.add(&b->y64, (size_t)n * ldy);
  sc.add(&b->y32, (size_t)n * ldy);
  sc.add(&b->ysum32, (size_t)n);
  sc.add(&b->stats, (size_t)n * ST_COUNT);
  sc.add(&b->err, 1);
  sc.add(&b->overflow, (size_t)n);
  sc.add(&B.id, (size_t)n * cap);
  sc.add(&B.score, (size_t)n * cap);
  sc.add(&B.eps, (size_t)n * cap);
  sc.add(&B.count, (size_t)n);
  sc.add(&B.hist, (size_t)n * kNumBins);
  sc.add(&B.hist_hi, (size_t)n * kNumBins);
  sc.add(&B.hist_c, (size_t)n * kCoarse);
  sc.add(&B.theta, (size_t)n);
  sc.add(&esc_id, (size_t)esc_cap);
  sc.add(&esc_prob, (size_t)esc_cap);
  sc.add(&esc_count, 1);
  sc.add(&S.state, (size_t)n);
  sc.add(&S.colL, (size_t)n * cap);
  sc.add(&S.colH, (size_t)n * cap);
  sc.add(&S.r_id, (size_t)n * cap);
  sc.add(&S.r_s32, (size_t)n * cap);
  sc.add(&S.r_e32, (size_t)n * cap);
  sc.add(&S.r_s64, (size_t)n * cap);
  sc.add(&S.r_e64, (size_t)n * cap);
  sc.add(&S.r_need, (size_t)n * cap);
  sc.add(&S.r_count, (size_t)n);
  sc.add(&S.job, (size_t)n * cap);
  sc.add(&S.job_list, (size_t)n * cap);
  sc.add(&S.n_jobs, 1);
  sc.add(&b->out_id, (size_t)n * k);
  sc.add(&b->out_score, (size_t)n * k);
  sc.add(&b->out_eps, (size_t)n * k);
  sc.add(&b->out_n, (size_t)n);
  sc.add(&S.max_eps, (size_t)n);
  sc.add(&S.r_rank, (size_t)n * cap);
  sc.add(&S.r_key, (size_t)n * cap);
  DSE_TRY(sc.alloc(&b->scratch, &b->scratch_bytes));
  B.cap = cap;

  // per-problem arguments
  std::vector<ScreenArgs> args(n), args_add(n);
  const double u = b->prec64 ? 1.1102230246251565e-16 : 5.9604644775390625e-8;
  for (int p = 0; p < n; ++p) {
    dse_space *sp = b->spaces[p];
    ScreenArgs A{};
    A.F = table_of(sp);
    A.G = sp->geom;
    A.n_stored = sp->n;
    A.id_begin = 0;
    A.id_end = b->total[p];
    A.N = (int32_t)sp->N;
    A.invN = 1.0 / (double)sp->N;
    A.ldy = (int32_t)ldy;
    A.T = 1;
    A.t0 = p;
    A.mode = DSE_MODE_PER_TARGET;
    A.n_lists = n;
    A.y32 = b->y32;
    A.y64 = b->y64;
    A.ysum32 = b->ysum32;
    A.max_complexity = sp->max_complexity;
    A.fmax64 = sp->fmax_max;
    {
      const double f = sp->fmax_max;
      float fd = (float)f, fu = (float)f;
      if ((double)fd > f) fd = nextafterf(fd, 0.f);
      if ((double)fu < f) fu = nextafterf(fu, INFINITY);
      A.fmax32_dn = fd;
      A.fmax32_up = fu;
    }
    A.fmin_std_rel = (float)sp->fmin_std_rel;
    A.fmin_std_rel64 = sp->fmin_std_rel;
    accum_factors(sp->N, b->prec64, &A.gamma_lane, &A.gamma, &A.block_len);
    A.u = (float)u;
    A.k = k;
    A.unit_check_addsub = sp->unit_check_addsub && sp->D > 0;
    A.explog_dimensionless = sp->explog_dimensionless;
    A.B = B;
    A.esc_id = esc_id;
    A.esc_count = esc_count;
    A.esc_cap = esc_cap;
    A.esc_prob = esc_prob;
    A.prob = p;
    A.stats = b->stats + (size_t)p * ST_COUNT;
    A.err = b->err;
    A.rowid = sp->rowid_ident;
    for (int c = 0; c < 6; ++c) A.slot_pos[c] = -1;
    for (int s2 = 0; s2 < sp->geom.nb; ++s2) A.slot_pos[sp->geom.bops[s2] - 6] = s2;
    A.first_pass = 1;
    A.group = 0;
    args[p] = A;
    A.rowid = sp->class_rows;
    args_add[p] = A;
  }
  // launch-level arguments: tile lists, counters, escalation list, error flag
  ScreenArgs L{};
  L.err = b->err;
  L.B = B;
  L.esc_id = esc_id;
  L.esc_count = esc_count;
  L.esc_cap = esc_cap;
  L.esc_prob = esc_prob;
  L.mode = DSE_MODE_PER_TARGET;
  L.first_pass = 1;
  b->A0_esc = L;
  b->A0_mul = L;
  b->A0_mul.tiles = b->tmul;
  b->A0_mul.n_tiles = b->n_mul;
  b->A0_mul.tile_counter = b->counters + 1;
  b->A0_add = L;
  b->A0_add.tiles = b->tadd;
  b->A0_add.n_tiles = b->n_add;
  b->A0_add.tile_counter = b->counters + 2;

  S.B = B;
  S.n_lists = n;
  S.k = k;
  S.all64 = b->prec64;
  S.overflow = b->overflow;
  S.out_id = b->out_id;
  S.out_score = b->out_score;
  S.out_eps = b->out_eps;
  S.out_n = b->out_n;
  S.stats = b->stats;

  // uploads (pageable host memory: the copies complete before the call returns)
  auto up = [&](void *dst, const void *src, size_t bytes) -> dse_status {
    if (bytes) DSE_CUDA(cudaMemcpyAsync(dst, src, bytes, cudaMemcpyHostToDevice, st));
    return DSE_OK;
  };
  DSE_TRY(up(b->args, args.data(), sizeof(ScreenArgs) * n));
  DSE_TRY(up(b->args_add, args_add.data(), sizeof(ScreenArgs) * n));
  DSE_TRY(up(b->feat_jobs, fjobs.data(), sizeof(Job) * fjobs.size()));
  DSE_TRY(up(b->pl_jobs, pjobs.data(), sizeof(Job) * pjobs.size()));
  DSE_TRY(up(b->tmul, mul.data(), sizeof(Tile) * mul.size()));
  DSE_TRY(up(b->tadd, add.data(), sizeof(Tile) * add.size()));
  DSE_TRY(up(b->yoff, b->yoff_h.data(), sizeof(int64_t) * n));
  for (int p = 0; p < n; ++p)
    if (pair_cnt[p])
      DSE_CUDA(cudaMemcpyAsync(b->pairs + pair_off[p], b->spaces[p]->eq_pairs, sizeof(int2) * pair_cnt[p],
                               cudaMemcpyDeviceToDevice, st));
  DSE_CUDA(cudaStreamSynchronize(st));
  return DSE_OK;
}

}  // namespace

// ================================================================ C ABI

extern "C" {

dse_status dse_sis_screen_batched(const dse_batch_item *items, int32_t n_items, const dse_batch_desc *d,
                                  dse_batch **out) {
  dse::NvtxRange nvtx_range_("dse_sis_screen_batched");
  clear_error();
  if (!items || !d || !out || n_items < 1 || d->k < 1 || d->k > (1 << 20) ||
      !(d->precision == DSE_PREC_FP32 || d->precision == DSE_PREC_FP64 || d->precision == DSE_PREC_AUTO) ||
      (d->flags & ~DSE_BATCH_GRAPH)) {
    set_error("invalid batch descriptor");
    return DSE_EINVAL;
  }
  *out = nullptr;
  for (int32_t p = 0; p < n_items; ++p)
    if (!items[p].space || !items[p].y) {
      set_error("batch item %d: null space or target", (int)p);
      return DSE_EINVAL;
    }
  DSE_TRY(check_device());
  AllocStream as((cudaStream_t)d->stream);
  dse_batch *b = new (std::nothrow) dse_batch();
  if (!b) {
    set_error("out of host memory");
    return DSE_ENOMEM;
  }
  b->stream = (cudaStream_t)d->stream;
  dse_status s = plan(items, n_items, d, b);
  // targets: each item's values into its slice of the concatenated array
  for (int32_t p = 0; s == DSE_OK && p < n_items; ++p) {
    const cudaError_t e =
        cudaMemcpyAsync(b->Ycat + b->yoff_h[p], items[p].y, sizeof(double) * b->spaces[p]->N,
                        items[p].y_on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, b->stream);
    if (e != cudaSuccess) s = cuda_status(e, "batch targets");
  }
  if (s == DSE_OK) s = run(b, false);
  if (s != DSE_OK) {
    release(b);
    return s;
  }
  *out = b;
  return DSE_OK;
}

dse_status dse_batch_rescreen(dse_batch *b, const double *Y, int32_t y_on_device) {
  dse::NvtxRange nvtx_range_("dse_batch_rescreen");
  clear_error();
  if (!b || !Y) {
    set_error("null argument");
    return DSE_EINVAL;
  }
  AllocStream as(b->stream);
  DSE_TRY(upload_targets(b, Y, y_on_device != 0));
  return run(b, (b->flags & DSE_BATCH_GRAPH) != 0);
}

dse_status dse_batch_fetch(dse_batch *b, int32_t item, uint64_t *idx, double *score, double *err_bound, int64_t cap,
                           int64_t *n_out) {
  dse::NvtxRange nvtx_range_("dse_batch_fetch");
  clear_error();
  if (!b || item < 0 || item >= b->n || cap < 0) {
    set_error("bad batch or item");
    return DSE_EINVAL;
  }
  AllocStream as(b->stream);
  DSE_TRY(finish(b));
  const int64_t n = b->h_out_n[item];
  if (n_out) *n_out = n;
  const int64_t m = std::min(n, cap);
  if (m == 0) return DSE_OK;
  const size_t off = (size_t)item * b->k;
  if (idx) DSE_CUDA(cudaMemcpy(idx, b->out_id + off, 8 * m, cudaMemcpyDefault));
  if (score) DSE_CUDA(cudaMemcpy(score, b->out_score + off, 8 * m, cudaMemcpyDefault));
  if (err_bound) DSE_CUDA(cudaMemcpy(err_bound, b->out_eps + off, 8 * m, cudaMemcpyDefault));
  return DSE_OK;
}

dse_status dse_batch_stats(dse_batch *b, int32_t item, dse_stats *out) {
  clear_error();
  if (!b || !out || item < 0 || item >= b->n) {
    set_error("bad batch or item");
    return DSE_EINVAL;
  }
  AllocStream as(b->stream);
  DSE_TRY(finish(b));
  *out = b->host_stats[item];
  return DSE_OK;
}

void dse_batch_free(dse_batch *b) { release(b); }

}  // extern "C"
