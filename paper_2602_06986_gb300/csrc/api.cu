// api.cu -- the C ABI: argument checks, handles, and the orchestration of the
// build, screen and selection kernels.
#include <math.h>
#include <stdio.h>
#include <string.h>

#include <algorithm>
#include <new>
#include <string>
#include <functional>
#include <vector>

#include "dse_internal.cuh"
#include "plan.cuh"
#include "screen_kernels.cuh"
#include "util.cuh"

namespace dse {
const char *last_error();
dse_status build_space(const dse_space_desc *d, dse_space **out);
dse_status space_release(dse_space *S);
dse_status count_last_rung(dse_space *S, cudaStream_t st);
FeatTable table_of(const dse_space *S);
RungGeom make_geom(const dse_space *S, int r);
dse_status refit_impl(dse_space *S, const dse_refit_desc *d, uint64_t *best_id, double *best_rmse, double *coefs,
                      double *residual);

// Blocked-summation error factors of the CUDA-core kernels for N samples:
// warp-per-candidate kernels (each lane sums its samples in blocks of 16,
// then a 5-level shuffle tree) and the pair kernel (blocks of block_len
// samples, about sqrt(N)); FP64 sums are plain.
void accum_factors(int64_t N, int prec64, float *gamma_lane, float *gamma_pair, int *block_len) {
  const double u = prec64 ? 1.1102230246251565e-16 : 5.9604644775390625e-8;
  int bl = (int)ceil(sqrt((double)N));
  bl = std::max(16, (bl + 1) / 2 * 2);
  *block_len = bl;
  const double nlane = ceil((double)N / 32.0);
  *gamma_lane = prec64 ? (float)((nlane + 8.0) * u * 1.05) : (float)((16.0 + ceil(nlane / 16.0) + 8.0) * u * 1.05);
  *gamma_pair = prec64 ? (float)((double)(N + 4) * u * 1.05)
                       : (float)(((double)bl + ceil((double)N / bl) + 4.0) * u * 1.05);
}

int sm_count() {
  int dev = 0, n = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev);
  return n > 0 ? n : 1;
}

dse_status check_device() {
  int n = 0;
  cudaError_t e = cudaGetDeviceCount(&n);
  if (e != cudaSuccess || n == 0) {
    cudaGetLastError();
    set_error("no usable CUDA device (%s)", e != cudaSuccess ? cudaGetErrorString(e) : "0 devices");
    return DSE_ECUDA;
  }
  return DSE_OK;
}

// ----------------------------------------------------------- tile lists

// Pair tiles over the positions of `rows` grouped in consecutive classes
// (class c = positions [cb[c], cb[c+1])): for every block of BI positions, the
// blocks of BJ positions from the start of the first class touching it up to
// the block itself.  Pairs are taken for position_i > position_j only.
void class_tiles(const std::vector<int64_t> &cb, int64_t npos, int BI, int BJ, int64_t i_from,
                        std::vector<Tile> &out) {
  // class start of every position
  std::vector<int64_t> start(npos);
  for (size_t c = 0; c + 1 < cb.size(); ++c)
    for (int64_t p = cb[c]; p < cb[c + 1]; ++p) start[p] = cb[c];
  for (int64_t i0 = i_from; i0 < npos; i0 += BI) {
    int64_t i1 = std::min(i0 + BI, npos);
    int64_t jlo = start[i0];
    int64_t bj0 = jlo / BJ * BJ;
    for (int64_t j0 = bj0; j0 < i1 - 1; j0 += BJ) {
      Tile t;
      t.ibase = (int32_t)i0;
      t.ni = (int16_t)(i1 - i0);
      t.jbase = (int32_t)j0;
      t.nj = (int16_t)std::min<int64_t>(BJ, npos - j0);
      t.prob = 0;
      out.push_back(t);
    }
  }
}

// The pairs (i > j) of equal unit vectors with i in the newest stored rung,
// built once per space from its unit classes and kept on the device.
dse_status equal_unit_pairs(dse_space *sp, cudaStream_t st) {
  if (sp->n_eq_pairs >= 0) return DSE_OK;
  const int64_t o = sp->geom.o;
  std::vector<int2> pairs;
  for (size_t c = 0; c + 1 < sp->h_class_begin.size(); ++c) {
    const int64_t b = sp->h_class_begin[c], e = sp->h_class_begin[c + 1];
    for (int64_t x = b + 1; x < e; ++x) {
      const int32_t i = sp->h_class_rows[x];  // ids ascend within a class
      if (i < o) continue;
      for (int64_t y = b; y < x; ++y) pairs.push_back(make_int2(i, sp->h_class_rows[y]));
    }
  }
  DSE_TRY(dalloc(&sp->eq_pairs, pairs.size(), "equal-unit pairs"));
  if (!pairs.empty())
    DSE_CUDA(cudaMemcpyAsync(sp->eq_pairs, pairs.data(), sizeof(int2) * pairs.size(), cudaMemcpyHostToDevice, st));
  DSE_CUDA(cudaStreamSynchronize(st));
  sp->n_eq_pairs = (int64_t)pairs.size();
  return DSE_OK;
}

// Triangle tiles over ids: i in [ia, ib] (the rows touched by the pair range),
// j < i.
void triangle_tiles(int64_t ia, int64_t ib, int BI, int BJ, std::vector<Tile> &out) {
  for (int64_t i0 = ia; i0 <= ib; i0 += BI) {
    int64_t i1 = std::min(i0 + BI, ib + 1);
    for (int64_t j0 = 0; j0 < i1 - 1; j0 += BJ) {
      Tile t;
      t.ibase = (int32_t)i0;
      t.ni = (int16_t)(i1 - i0);
      t.jbase = (int32_t)j0;
      t.nj = (int16_t)std::min<int64_t>(BJ, i1 - 1 - j0);
      t.prob = 0;
      out.push_back(t);
    }
  }
}

// Order pair tiles so that the tiles resident at the same time share their
// operand rows: groups of G consecutive i-blocks, j-block major inside a
// group.  A wave of one CTA per SM then covers a compact block of the
// triangle (e.g. 8 i-blocks x 19 j-blocks) whose rows stay in L2, instead of
// one i-block against hundreds of j-blocks.
void group_tiles(std::vector<Tile> &t, int64_t ia, int BI, int G) {
  const int64_t span = (int64_t)BI * G;
  std::stable_sort(t.begin(), t.end(), [&](const Tile &a, const Tile &b) {
    const int64_t ga = (a.ibase - ia) / span, gb = (b.ibase - ia) / span;
    if (ga != gb) return ga < gb;
    if (a.jbase != b.jbase) return a.jbase < b.jbase;
    return a.ibase < b.ibase;
  });
}

// ------------------------------------------------------------- screening

struct ScreenPlan {
  int prec64, nt, passes;
  int64_t cap;
  std::vector<Tile> mul_tiles, add_tiles;
  bool use_pairlist = false;     // additive slots from the equal-unit pair list
  bool add_by_id = false;        // additive tiles over ids (one unit class): rows = identity
  uint64_t id0, id1, p0, p1;     // stored ids and unary flat range
  uint64_t add_total;            // additive slots of the binary block in range
  float gamma_lane, gamma_pair;
  int block_len;
  // tensor-core path (BF16x3 contraction of the binary block)
  bool use_tc = false;
  int ntp = 0, tc_passes = 0, gen_blk = 1;
  int32_t n_seed_tiles = 0;      // leading product/quotient tiles launched first
  float gamma_gen = 0.f, gamma_num = 0.f;
  unsigned char *bsplit = nullptr;
  // Gram path of the product/quotient slots (single-target FP32 screens)
  bool use_gram = false;
  bool gram_addsub = false;      // a+b and a-b in the Gram kernel too
  std::vector<int2> gram_tiles;
  int2 *gram_tiles_dev = nullptr;
  void *gram_scr = nullptr;
  // multi-target Gram path (2..16 targets, per-target lists)
  bool use_gmt = false;
  std::vector<int2> gmt_tiles;
  int2 *gmt_tiles_dev = nullptr;
  void *gmt_scr = nullptr;
};

bool gram_eligible(int64_t N);
size_t gram_space_bytes(int64_t n, int64_t N);
size_t gram_screen_bytes(int64_t n, int64_t N);
void gram_build_space(const FeatTable &F, void *buf, cudaStream_t st);
void gram_tiles(const dse_space *sp, uint64_t id_begin, uint64_t id_end, std::vector<int2> &out);
void launch_gram_arows(const ScreenArgs &A, const void *space_buf, void *scr, cudaStream_t st);
dse_status launch_pair_gram(const ScreenArgs &A, const void *space_buf, void *scr, const int2 *tiles, int n_tiles,
                            int sms, cudaStream_t st);

bool gmt_eligible(int T, int64_t N);
size_t gmt_space_bytes(int64_t n, int64_t N);
size_t gmt_screen_bytes(int64_t n, int64_t N);
void gmt_build_space(const FeatTable &F, void *buf, cudaStream_t st);
void gmt_tiles(const dse_space *sp, uint64_t id_begin, uint64_t id_end, std::vector<int2> &out);
void launch_gmt_brows(const ScreenArgs &A, const void *space_buf, void *scr, cudaStream_t st);
dse_status launch_pair_gmt(const ScreenArgs &A, const void *space_buf, void *scr, const int2 *tiles, int n_tiles,
                           int sms, cudaStream_t st);

int tc_ntp_for(int T, int N);
int tc_gen_samples();
int tc_gen_parts();
size_t tc_bsplit_bytes(int ntp, int N);
void launch_tc_targets(const float *y32, int32_t ldy, int t0, int T, int N, int ntp, unsigned char *out,
                       cudaStream_t st);
dse_status launch_pair_tc(int kind, int ntp, const ScreenArgs &A, const unsigned char *bsplit, const float *rows,
                          const float *rcp_rows, int64_t nrows, float gamma_gen, float gamma_num, int gen_blk, int sms,
                          cudaStream_t st);
void launch_rcp_rows(const float *v32, int64_t count, float *out, int sms, cudaStream_t st);
void launch_gather_rows(const float *v32, int64_t ld, const int32_t *rows, int64_t n, float *out, int sms,
                        cudaStream_t st);

// The tensor-core pass structure: each pass contracts `ntp` targets; the
// CUDA-core kernels (stored/unary candidates, sparse additive pairs) cover the
// same targets in sub-passes of 16.
static dse_status run_tc_passes(dse_result *R, const ScreenPlan &plan, void *scr_tiles_mul, void *scr_tiles_add,
                                ScreenArgs &A, int sms, cudaStream_t st,
                                const std::function<dse_status(int)> &mark) {
  dse_space *sp = R->space;
  for (int tp = 0; tp < plan.tc_passes; ++tp) {
    const int t0 = tp * plan.ntp, tn = std::min(plan.ntp, R->T - t0);
    launch_tc_targets(R->y32, R->ldy, t0, tn, (int)sp->N, plan.ntp, plan.bsplit, st);
    DSE_TRY(mark(0));
    for (int s0 = 0; s0 < tn; s0 += 16) {
      A.t0 = t0 + s0;
      A.T = std::min(16, tn - s0);
      A.first_pass = tp == 0 && s0 == 0;
      launch_feature(0, 16, A, plan.id0, plan.id1, plan.p0, plan.p1, plan.gamma_lane, sms, st);
      if (plan.use_pairlist)
        launch_pairlist(0, 16, A, sp->eq_pairs, sp->n_eq_pairs, plan.gamma_lane, sms, st);
    }
    A.t0 = t0;
    A.T = tn;
    A.first_pass = tp == 0;
    DSE_TRY(mark(1));
    if (!plan.mul_tiles.empty()) {
      if (!sp->rcp32) {
        // reciprocal rows of the stored features, built at the first use
        const int64_t cnt = sp->n * sp->ld;
        DSE_TRY(dmalloc(reinterpret_cast<void **>(&sp->rcp32), sizeof(float) * (size_t)cnt, "reciprocal rows"));
        launch_rcp_rows(sp->v32, cnt, sp->rcp32, sms, st);
      }
      A.rowid = sp->rowid_ident;
      const Tile *t0p = reinterpret_cast<const Tile *>(scr_tiles_mul);
      const int32_t nall = (int32_t)plan.mul_tiles.size(), ns = plan.n_seed_tiles;
      if (ns > 0) {
        A.tiles = t0p;
        A.n_tiles = ns;
        DSE_TRY(launch_pair_tc(KIND_MUL, plan.ntp, A, plan.bsplit, sp->v32, sp->rcp32, sp->n, plan.gamma_gen, plan.gamma_num, plan.gen_blk,
                               sms, st));
      }
      A.tiles = t0p + ns;
      A.n_tiles = nall - ns;
      DSE_TRY(launch_pair_tc(KIND_MUL, plan.ntp, A, plan.bsplit, sp->v32, sp->rcp32, sp->n, plan.gamma_gen, plan.gamma_num, plan.gen_blk, sms,
                             st));
    }
    DSE_TRY(mark(2));
    if (!plan.use_pairlist && !plan.add_tiles.empty()) {
      A.tiles = reinterpret_cast<const Tile *>(scr_tiles_add);
      A.n_tiles = (int32_t)plan.add_tiles.size();
      A.rowid = plan.add_by_id ? sp->rowid_ident : sp->class_rows;
      if (!plan.add_by_id && !sp->v32_class) {
        // the rows in unit-class order, built at the first use
        DSE_TRY(dmalloc(reinterpret_cast<void **>(&sp->v32_class), sizeof(float) * (size_t)(sp->n * sp->ld),
                        "class-ordered rows"));
        launch_gather_rows(sp->v32, sp->ld, sp->class_rows, sp->n, sp->v32_class, sms, st);
      }
      DSE_TRY(launch_pair_tc(KIND_ADD, plan.ntp, A, plan.bsplit, plan.add_by_id ? sp->v32 : sp->v32_class, nullptr, sp->n,
                             plan.gamma_gen, plan.gamma_num, plan.gen_blk, sms,
                             st));
    }
  }
  return DSE_OK;
}

uint64_t count_slots_mod(uint64_t x, int nb, const std::vector<int> &posset) {
  // number of p' in [0, x) with p' mod nb in posset
  uint64_t full = x / (uint64_t)nb, rem = x % (uint64_t)nb;
  uint64_t c = full * posset.size();
  for (int p : posset)
    if ((uint64_t)p < rem) ++c;
  return c;
}

// Zero a screen's buffer counts, bound histograms, escalation count,
// statistics and re-score job counts (n_jobs[0..2)).
__global__ void k_screen_reset(unsigned *count, unsigned *hist, unsigned *hist_hi, unsigned *hist_c, int nl,
                               unsigned *esc_count, unsigned long long *stats, unsigned *n_jobs) {
  const int64_t nh = (int64_t)nl * kNumBins, nc = (int64_t)nl * kCoarse;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < nh; e += (int64_t)gridDim.x * blockDim.x) {
    hist[e] = 0u;
    hist_hi[e] = 0u;
    if (e < nc) hist_c[e] = 0u;
    if (e < nl) count[e] = 0u;
    if (e < ST_COUNT) stats[e] = 0ull;
    if (e == 0) {
      *esc_count = 0u;
      n_jobs[0] = 0u;
      n_jobs[1] = 0u;
    }
  }
}

static dse_status run_screen(dse_result *R, const ScreenPlan &plan, void *scr_tiles_mul, void *scr_tiles_add,
                             ScreenArgs &A, SelectArgs &S, unsigned int *tile_ctr) {
  dse_space *sp = R->space;
  cudaStream_t st = R->stream;
  const int sms = sm_count();
  const int nl = R->n_lists;
  const int64_t launches0 = launches_so_far();
  // the screen's counters and histograms, zeroed by one kernel
  note_launches(1);
  k_screen_reset<<<std::max(1, std::min(sms, (int)((nl * kNumBins + 255) / 256))), 256, 0, st>>>(
      A.B.count, A.B.hist, A.B.hist_hi, A.B.hist_c, nl, A.esc_count, A.stats, S.n_jobs);
  // per-candidate reasons: -1 until a kernel decides the candidate
  if (A.why) DSE_CUDA(cudaMemsetAsync(A.why, 0xff, (size_t)(A.id_end - A.id_begin), st));
  // intervals: NaN (all bits set) until a kernel writes one
  if (A.ivl) DSE_CUDA(cudaMemsetAsync(A.ivl, 0xff, sizeof(float2) * (size_t)(A.id_end - A.id_begin) * nl, st));
  // optional device timing of each kernel group
  const bool timing = (R->flags & (DSE_FLAG_TIMING | DSE_FLAG_TIMING_MAIN)) != 0;
  const bool main_only = !(R->flags & DSE_FLAG_TIMING);
  cudaEvent_t ev_open = nullptr;
  int open_group = -1;
  // one event per group boundary: it closes the open group and opens the
  // next (main_only: events around group 1 only)
  auto mark = [&](int group) -> dse_status {
    if (!timing) return DSE_OK;
    const bool need = !main_only || group == 1 || open_group == 1;
    if (!need) {
      open_group = group;
      return DSE_OK;
    }
    cudaEvent_t e;
    DSE_CUDA(cudaEventCreate(&e));
    R->events.push_back(e);
    DSE_CUDA(cudaEventRecord(e, st));
    if (ev_open) R->timing.push_back({open_group, {ev_open, e}});
    ev_open = group >= 0 && (!main_only || group == 1) ? e : nullptr;
    open_group = group;
    return DSE_OK;
  };

  if (plan.use_tc) DSE_TRY(run_tc_passes(R, plan, scr_tiles_mul, scr_tiles_add, A, sms, st, mark));
  for (int pass = 0; pass < (plan.use_tc ? 0 : plan.passes); ++pass) {
    A.t0 = pass * plan.nt;
    A.T = std::min(plan.nt, R->T - A.t0);
    A.first_pass = pass == 0;
    DSE_TRY(mark(0));
    launch_feature(plan.prec64, plan.nt, A, plan.id0, plan.id1, plan.p0, plan.p1, plan.gamma_lane, sms, st);
    if (plan.use_gram) {
      // the operand images (timed with the stored/unary group)
      if (!sp->gram_buf) {
        DSE_TRY(dmalloc(&sp->gram_buf, gram_space_bytes(sp->n, sp->N), "product Gram images"));
        gram_build_space(table_of(sp), sp->gram_buf, st);
      }
      launch_gram_arows(A, sp->gram_buf, plan.gram_scr, st);
    } else if (plan.use_gmt) {
      // the operand images (timed with the stored/unary group)
      if (!sp->gmt_buf) {
        DSE_TRY(dmalloc(&sp->gmt_buf, gmt_space_bytes(sp->n, sp->N), "multi-target Gram images"));
        gmt_build_space(table_of(sp), sp->gmt_buf, st);
      }
      launch_gmt_brows(A, sp->gmt_buf, plan.gmt_scr, st);
    }
    DSE_TRY(mark(1));
    if (plan.use_gram) {
      DSE_TRY(launch_pair_gram(A, sp->gram_buf, plan.gram_scr, plan.gram_tiles_dev, (int)plan.gram_tiles.size(), sms,
                               st));
    } else if (plan.use_gmt) {
      DSE_TRY(launch_pair_gmt(A, sp->gmt_buf, plan.gmt_scr, plan.gmt_tiles_dev, (int)plan.gmt_tiles.size(), sms,
                              st));
    } else if (!plan.mul_tiles.empty()) {
      A.rowid = sp->rowid_ident;
      A.tile_counter = tile_ctr;
      const Tile *t0p = reinterpret_cast<const Tile *>(scr_tiles_mul);
      const int32_t nall = (int32_t)plan.mul_tiles.size(), ns = plan.n_seed_tiles;
      if (ns > 0) {
        A.tiles = t0p;
        A.n_tiles = ns;
        DSE_CUDA(cudaMemsetAsync(tile_ctr, 0, sizeof(unsigned), st));
        DSE_TRY(launch_pair(plan.prec64, KIND_MUL, plan.nt, A, plan.block_len, sms, st));
      }
      A.tiles = t0p + ns;
      A.n_tiles = nall - ns;
      DSE_CUDA(cudaMemsetAsync(tile_ctr, 0, sizeof(unsigned), st));
      DSE_TRY(launch_pair(plan.prec64, KIND_MUL, plan.nt, A, plan.block_len, sms, st));
    }
    DSE_TRY(mark(2));
    if (plan.use_pairlist) {
      launch_pairlist(plan.prec64, plan.nt, A, sp->eq_pairs, sp->n_eq_pairs, plan.gamma_lane, sms, st);
    } else if (!plan.add_tiles.empty()) {
      A.tiles = reinterpret_cast<const Tile *>(scr_tiles_add);
      A.n_tiles = (int32_t)plan.add_tiles.size();
      A.rowid = plan.add_by_id ? sp->rowid_ident : sp->class_rows;
      A.tile_counter = tile_ctr + 1;
      DSE_CUDA(cudaMemsetAsync(tile_ctr + 1, 0, sizeof(unsigned), st));
      DSE_TRY(launch_pair(plan.prec64, KIND_ADD, plan.nt, A, plan.block_len, sms, st));
    }
  }
  DSE_TRY(mark(3));
  ScreenArgs E = A;
  E.t0 = 0;
  E.T = R->T;
  launch_escalate(E, sms, st);
  launch_why_fixup(A, sms, st);
  DSE_TRY(launch_select(S, E, sms, st));
  DSE_TRY(mark(-1));
  DSE_CUDA(cudaGetLastError());
  R->launches += launches_so_far() - launches0;
  return DSE_OK;
}

// What a re-run of a screen needs (launch arguments, plan, tile lists).
struct Keep {
  ScreenPlan plan;
  ScreenArgs A;
  SelectArgs S;
  Tile *tmul, *tadd;
  unsigned *tile_ctr;
};

// Plan a screen and allocate everything; with launch, also upload the
// targets and enqueue it (otherwise d->Y is ignored and the screen is run
// later by screen_enqueue_target).
static dse_status screen_impl(dse_space *sp, const dse_screen_desc *d, dse_result **out, bool launch = true) {
  cudaStream_t st = (cudaStream_t)d->stream;
  const int64_t N = sp->N;
  const uint64_t total = (uint64_t)sp->n + sp->geom.slots;
  uint64_t id_begin = d->id_begin, id_end = d->id_end ? d->id_end : total;
  if (id_begin > id_end || id_end > total) {
    set_error("id range [%llu, %llu) outside [0, %llu)", (unsigned long long)id_begin,
              (unsigned long long)id_end, (unsigned long long)total);
    return DSE_ERANGE;
  }
  if ((d->reasons && !is_device_pointer(d->reasons)) || (d->intervals && !is_device_pointer(d->intervals))) {
    set_error("the reasons and intervals buffers must be device memory");
    return DSE_EINVAL;
  }
  int prec = d->precision;
  ScreenPlan plan{};
  // the tensor-core contraction for many targets (per-target lists only)
  if (d->mode == DSE_MODE_PER_TARGET &&
      (prec == DSE_PREC_BF16X3 || (prec == DSE_PREC_AUTO && d->n_targets >= tuning().tc_min_targets))) {
    plan.use_tc = true;
    prec = DSE_PREC_BF16X3;
  } else if (prec == DSE_PREC_AUTO || prec == DSE_PREC_BF16X3) {
    prec = DSE_PREC_FP32;
  }
  plan.prec64 = prec == DSE_PREC_FP64;
  plan.nt = d->n_targets == 1 ? 1 : 16;
  plan.passes = (d->n_targets + plan.nt - 1) / plan.nt;
  if (d->mode == DSE_MODE_AGGREGATED && plan.passes > 1) {
    set_error("aggregated mode supports at most %d targets", plan.nt);
    return DSE_EINVAL;
  }
  const int n_lists = d->mode == DSE_MODE_AGGREGATED ? 1 : d->n_targets;
  plan.cap = std::max<int64_t>(8 * d->k, d->k + 131072);

  // ranges of each candidate group
  const uint64_t ns = (uint64_t)sp->n;
  const RungGeom &g = sp->geom;
  plan.id0 = std::min(id_begin, ns);
  plan.id1 = std::min(id_end, ns);
  auto clampp = [&](uint64_t id) { return id <= ns ? 0ull : std::min<uint64_t>(id - ns, g.slots); };
  const uint64_t pb = clampp(id_begin), pe = clampp(id_end);
  plan.p0 = std::min(pb, g.um);
  plan.p1 = std::min(pe, g.um);
  // binary block range in pair space
  const uint64_t bb = std::max(pb, g.um), be = std::max(pe, g.um);
  int BI = plan.nt == 1 ? 32 : 16, BJ = BI;
  if (plan.use_tc) {
    BI = 16;  // 128-pair tensor-core tiles
    BJ = 8;
  }
  std::vector<int> addpos;
  if (g.nb > 0 && be > bb) {
    const uint64_t q0 = (bb - g.um) / g.nb, q1 = (be - g.um - 1) / g.nb;
    uint64_t ia, ja, ib2, jb;
    pair_from_index(q0 + g.tri_o, &ia, &ja);
    pair_from_index(q1 + g.tri_o, &ib2, &jb);
    bool any_mul = false, any_add = false, any_addsub = false, any_absdiff = false;
    for (int s = 0; s < g.nb; ++s) {
      int op = g.bops[s];
      if (op == DSE_OP_MUL || op == DSE_OP_DIV || op == DSE_OP_RDIV) any_mul = true;
      else {
        any_add = true;
        addpos.push_back(s);
        (op == DSE_OP_ABSDIFF ? any_absdiff : any_addsub) = true;
      }
    }
    plan.use_gram = (any_mul || any_addsub) && !plan.prec64 && !plan.use_tc && d->n_targets == 1 &&
                    gram_eligible(N) && !(d->flags & DSE_FLAG_DIRECT);
    // 2..16 targets: the multi-target Gram contraction instead of the
    // sample-by-sample tensor-core kernel (DSE_FLAG_DIRECT keeps the latter);
    // the stored/unary and |a-b| candidates go to the CUDA-core kernels
    plan.use_gmt = plan.use_tc && (any_mul || any_addsub) && gmt_eligible(d->n_targets, N) &&
                   !(d->flags & DSE_FLAG_DIRECT);
    if (plan.use_gmt) {
      plan.use_tc = false;
      BI = BJ = 16;
    }
    // a+b and a-b come from the same contraction (the centred cross term);
    // the additive kernels then run for |a-b| alone, or not at all
    plan.gram_addsub = (plan.use_gram || plan.use_gmt) && any_addsub;
    const bool add_kernels = any_add && !(plan.gram_addsub && !any_absdiff);
    if (plan.use_gram) {
      gram_tiles(sp, id_begin, id_end, plan.gram_tiles);
    } else if (plan.use_gmt) {
      gmt_tiles(sp, id_begin, id_end, plan.gmt_tiles);
    } else if (any_mul) {
      triangle_tiles((int64_t)ia, (int64_t)ib2, BI, BJ, plan.mul_tiles);
      const Tuning tn = tuning();
      group_tiles(plan.mul_tiles, (int64_t)ia, BI, plan.use_tc ? tn.tile_group_tc : tn.tile_group_cc);
      // A large tile list is launched in two parts: every seed_stride-th
      // tile first (64 by default), so that the thresholds have risen from a
      // spread sample of the space before the bulk of the candidates is
      // filtered.
      const size_t nt = plan.mul_tiles.size(), stride = (size_t)tn.seed_stride;
      if (nt >= 64 * stride) {
        std::vector<Tile> seed, rest;
        seed.reserve(nt / stride + 1);
        rest.reserve(nt);
        for (size_t t = 0; t < nt; ++t) (t % stride == 0 ? seed : rest).push_back(plan.mul_tiles[t]);
        plan.n_seed_tiles = (int32_t)seed.size();
        seed.insert(seed.end(), rest.begin(), rest.end());
        plan.mul_tiles.swap(seed);
      }
    }
    if (add_kernels) {
      const bool one_class = !(sp->unit_check_addsub && sp->D > 0) || sp->h_class_begin.size() <= 2;
      if (one_class) {
        // every pair may be added: the same id triangle as the products,
        // restricted to the rows of the range
        triangle_tiles((int64_t)ia, (int64_t)ib2, BI, BJ, plan.add_tiles);
        plan.add_by_id = true;
      } else {
        // sparse equal-unit pairs: an explicit list (built once per space);
        // dense: tiles over the unit classes (positions within class_rows;
        // classes interleave old and new ids, so every block is visited)
        DSE_TRY(equal_unit_pairs(sp, st));
        const uint64_t mm = (uint64_t)(g.n - g.o), oo = (uint64_t)g.o;
        const uint64_t all_pairs = mm ? tri(mm) + mm * oo : 0;
        if ((uint64_t)sp->n_eq_pairs * 4 <= all_pairs)
          plan.use_pairlist = true;
        else
          class_tiles(sp->h_class_begin, sp->n, BI, BJ, 0, plan.add_tiles);
      }
    }
    if (any_add)
      plan.add_total = count_slots_mod(be - g.um, g.nb, addpos) - count_slots_mod(bb - g.um, g.nb, addpos);
  }
  // accumulation error factors
  const double u32 = 5.9604644775390625e-8, u64 = 1.1102230246251565e-16;
  const double u = plan.prec64 ? u64 : u32;
  accum_factors(N, plan.prec64, &plan.gamma_lane, &plan.gamma_pair, &plan.block_len);
  if (plan.use_tc) {
    plan.ntp = tc_ntp_for(d->n_targets, (int)N);
    plan.tc_passes = (d->n_targets + plan.ntp - 1) / plan.ntp;
    const int nchunks = (int)((N + 31) / 32);
    // generation sums: spp samples of each chunk per thread, blocks of
    // gen_blk chunks, the parts' partial sums added at the end
    const double spp = tc_gen_samples(), parts = tc_gen_parts();
    plan.gen_blk = std::max(1, (int)lround(sqrt(nchunks / spp)));
    plan.gamma_gen =
        (float)((spp * plan.gen_blk + ceil((double)nchunks / plan.gen_blk) + parts + 4.0) * u32 * 1.05);
    // contraction: BF16x3 split (w = wh + wl + ew with |ew| <= 2^-16 |w|, the
    // same for y; dropping wl*yl, ew*y and w*ey leaves at most 3.01 * 2^-16
    // of sum |w y|) plus 2u per tensor-core
    // accumulation step (3 products x 2 k-steps per chunk, up to 16 chunks per
    // TMEM block; with 16 targets the products go to two accumulators of at
    // most 2 x 2 steps per chunk, whose halves are added once: fewer steps)
    // and the register drain of the blocks, times a safety factor 4
    const int nblocks = (nchunks + 15) / 16;
    const double steps = 3.0 * 2.0 * std::min(nchunks, 16);
    plan.gamma_num = (float)(4.0 * (2.0 * steps + nblocks + 2.0) * u32 + 3.02 * 1.52587890625e-5 +
                             (double)plan.gamma_gen);
  }

  dse_result *R = new (std::nothrow) dse_result();
  if (!R) {
    set_error("out of host memory");
    return DSE_ENOMEM;
  }
  R->space = sp;
  R->n_lists = n_lists;
  R->T = d->n_targets;
  R->mode = d->mode;
  R->precision = prec;
  R->k = d->k;
  R->id_begin = id_begin;
  R->id_end = id_end;
  R->stream = st;
  R->ldy = (int32_t)sp->ld;

  // one scratch allocation
  Scratch sc;
  ScreenArgs A{};
  SelectArgs S{};
  double *Yd = nullptr;
  Tile *tmul = nullptr, *tadd = nullptr;
  unsigned *tile_ctr = nullptr;
  const int64_t cap = plan.cap;
  const int64_t T = d->n_targets;
  if (launch && !d->y_on_device) sc.add(&Yd, (size_t)T * d->ld_y);
  sc.add(&R->y64, (size_t)T * R->ldy);
  sc.add(&R->y32, (size_t)T * R->ldy);
  sc.add(&R->ydf, (size_t)T * R->ldy);
  sc.add(&R->ysum32, (size_t)T);
  sc.add(&A.B.id, (size_t)n_lists * cap);
  sc.add(&A.B.score, (size_t)n_lists * cap);
  sc.add(&A.B.eps, (size_t)n_lists * cap);
  sc.add(&A.B.count, (size_t)n_lists);
  sc.add(&A.B.hist, (size_t)n_lists * kNumBins);
  sc.add(&A.B.hist_hi, (size_t)n_lists * kNumBins);
  sc.add(&A.B.hist_c, (size_t)n_lists * kCoarse);
  sc.add(&S.state, (size_t)n_lists);
  sc.add(&S.colL, (size_t)n_lists * cap);
  sc.add(&S.colH, (size_t)n_lists * cap);
  sc.add(&A.B.theta, (size_t)n_lists);
  const int64_t esc_cap = 1 << 20;
  sc.add(&A.esc_id, (size_t)esc_cap);
  sc.add(&A.esc_count, 1);
  sc.add(&A.esc2_id, (size_t)esc_cap);
  sc.add(&A.esc2_count, 1);
  sc.add(&R->stats, ST_COUNT);
  sc.add(&R->err, 1);
  sc.add(&S.r_id, (size_t)n_lists * cap);
  sc.add(&S.r_s32, (size_t)n_lists * cap);
  sc.add(&S.r_e32, (size_t)n_lists * cap);
  sc.add(&S.r_s64, (size_t)n_lists * cap);
  sc.add(&S.r_e64, (size_t)n_lists * cap);
  sc.add(&S.r_need, (size_t)n_lists * cap);
  sc.add(&S.r_count, (size_t)n_lists);
  sc.add(&R->overflow, (size_t)n_lists);
  sc.add(&S.job, (size_t)n_lists * cap);
  sc.add(&S.job_list, (size_t)n_lists * cap);
  sc.add(&S.job32, (size_t)n_lists * cap);
  sc.add(&S.job32_list, (size_t)n_lists * cap);
  sc.add(&S.n_jobs, 2);
  sc.add(&R->out_id, (size_t)n_lists * d->k);
  sc.add(&R->out_score, (size_t)n_lists * d->k);
  sc.add(&R->out_eps, (size_t)n_lists * d->k);
  sc.add(&R->out_n, (size_t)n_lists);
  sc.add(&S.max_eps, (size_t)n_lists);
  sc.add(&S.r_rank, (size_t)n_lists * cap);
  sc.add(&S.r_key, (size_t)n_lists * cap);
  sc.add(&tmul, plan.mul_tiles.size());
  sc.add(&tadd, plan.add_tiles.size());
  sc.add(&tile_ctr, 2);
  sc.add(&plan.bsplit, plan.use_tc ? tc_bsplit_bytes(plan.ntp, (int)N) : 1);
  unsigned char *gram_scr = nullptr;
  sc.add(&plan.gram_tiles_dev, plan.gram_tiles.size());
  sc.add(&gram_scr, plan.use_gram ? gram_screen_bytes(sp->n, N) : 1);
  unsigned char *gmt_scr = nullptr;
  sc.add(&plan.gmt_tiles_dev, plan.gmt_tiles.size());
  sc.add(&gmt_scr, plan.use_gmt ? gmt_screen_bytes(sp->n, N) : 1);
  dse_status s = sc.alloc(&R->scratch, &R->scratch_bytes);
  plan.gram_scr = gram_scr;
  plan.gmt_scr = gmt_scr;
  if (s != DSE_OK) {
    delete R;
    return s;
  }
  auto fail = [&](dse_status e) {
    dfree(R->scratch);
    delete R;
    return e;
  };
  cudaError_t e = cudaSuccess;
  const double *Ysrc = d->Y;
  if (launch && !d->y_on_device) {
    e = cudaMemcpyAsync(Yd, d->Y, sizeof(double) * T * d->ld_y, cudaMemcpyHostToDevice, st);
    Ysrc = Yd;
  }
  if (!e && !plan.mul_tiles.empty())
    e = cudaMemcpyAsync(tmul, plan.mul_tiles.data(), sizeof(Tile) * plan.mul_tiles.size(), cudaMemcpyHostToDevice,
                        st);
  if (!e && !plan.add_tiles.empty())
    e = cudaMemcpyAsync(tadd, plan.add_tiles.data(), sizeof(Tile) * plan.add_tiles.size(), cudaMemcpyHostToDevice,
                        st);
  if (!e && !plan.gram_tiles.empty())
    e = cudaMemcpyAsync(plan.gram_tiles_dev, plan.gram_tiles.data(), sizeof(int2) * plan.gram_tiles.size(),
                        cudaMemcpyHostToDevice, st);
  if (!e && !plan.gmt_tiles.empty())
    e = cudaMemcpyAsync(plan.gmt_tiles_dev, plan.gmt_tiles.data(), sizeof(int2) * plan.gmt_tiles.size(),
                        cudaMemcpyHostToDevice, st);
  if (!e) e = cudaMemsetAsync(R->err, 0, sizeof(int), st);
  if (!e) e = cudaMemsetAsync(A.B.theta, 0, sizeof(float) * n_lists, st);
  if (e) return fail(cuda_status(e, "screen setup"));
  A.why = d->reasons;
  A.ivl = reinterpret_cast<float2 *>(d->intervals);
  if (launch) launch_targets(Ysrc, d->ld_y, (int)T, N, R->ldy, R->y64, R->y32, R->ydf, R->ysum32, R->err, st);
  R->launches = launch ? 1 : 0;
  R->flags = d->flags;

  A.F = table_of(sp);
  A.G = g;
  A.n_stored = sp->n;
  A.id_begin = id_begin;
  A.id_end = id_end;
  A.N = (int32_t)N;
  A.invN = 1.0 / (double)N;
  A.ldy = R->ldy;
  A.mode = d->mode;
  A.n_lists = n_lists;
  A.y32 = R->y32;
  A.ydf = R->ydf;
  A.y64 = R->y64;
  A.ysum32 = R->ysum32;
  A.max_complexity = sp->max_complexity;
  A.fmax64 = sp->fmax_max;
  {
    double f = sp->fmax_max;
    float fd = (float)f, fu = (float)f;
    if ((double)fd > f) fd = nextafterf(fd, 0.f);
    if ((double)fu < f) fu = nextafterf(fu, INFINITY);
    A.fmax32_dn = fd;
    A.fmax32_up = fu;
  }
  A.fmin_std_rel = (float)sp->fmin_std_rel;
  A.fmin_std_rel64 = sp->fmin_std_rel;
  A.gamma = plan.gamma_pair;
  A.u = (float)u;
  A.k = d->k;
  A.unit_check_addsub = sp->unit_check_addsub && sp->D > 0;
  A.explog_dimensionless = sp->explog_dimensionless;
  A.B.cap = cap;
  A.esc_cap = esc_cap;
  A.stats = R->stats;
  A.err = R->err;
  for (int c = 0; c < 6; ++c) A.slot_pos[c] = -1;
  for (int s2 = 0; s2 < g.nb; ++s2) A.slot_pos[g.bops[s2] - 6] = s2;
  A.gram_addsub = plan.gram_addsub ? 1 : 0;

  S.B = A.B;
  S.n_lists = n_lists;
  S.k = d->k;
  S.all64 = plan.prec64;
  S.overflow = R->overflow;
  S.out_id = R->out_id;
  S.out_score = R->out_score;
  S.out_eps = R->out_eps;
  S.out_n = R->out_n;
  R->max_eps = S.max_eps;
  S.stats = R->stats;

  if (launch) {
    s = run_screen(R, plan, tmul, tadd, A, S, tile_ctr);
    if (s != DSE_OK) return fail(s);
  }

  // keep what a re-run after a buffer overflow needs
  R->host_stats = dse_stats{};
  R->host_stats.screened = (int64_t)(id_end - id_begin);
  R->host_stats.precision_used = prec;
  R->host_stats.binary_path = plan.use_gmt                               ? DSE_PATH_GRAM_MT
                              : plan.use_gram                            ? DSE_PATH_GRAM
                              : plan.use_tc && !plan.mul_tiles.empty()   ? DSE_PATH_TENSOR
                              : !plan.mul_tiles.empty()                  ? DSE_PATH_CUDA_CORE
                                                                         : 0;
  Keep *keep = new (std::nothrow) Keep{plan, A, S, tmul, tadd, tile_ctr};
  if (!keep) return fail(DSE_ENOMEM);
  R->keep = keep;
  R->keep_free = [](void *p) { delete reinterpret_cast<Keep *>(p); };
  R->rerun = [](dse_result *r) -> dse_status {
    Keep *k = reinterpret_cast<Keep *>(r->keep);
    return run_screen(r, k->plan, k->tmul, k->tadd, k->A, k->S, k->tile_ctr);
  };
  R->add_total = plan.add_total;
  R->buf_count = A.B.count;
  *out = R;
  return DSE_OK;
}

// Screen a prepared result (screen_impl without launch) against new targets
// already on the device (T rows of stride ld_y): thresholds start from zero.
// clear: zero the error flag and the thresholds first (the loop's snapshot
// kernel leaves them zeroed for the iterations after the first).
static dse_status screen_enqueue_target(dse_result *R, const double *Y, int64_t ld_y, bool clear = true) {
  cudaStream_t st = R->stream;
  Keep *k = reinterpret_cast<Keep *>(R->keep);
  if (clear) {
    DSE_CUDA(cudaMemsetAsync(R->err, 0, sizeof(int), st));
    DSE_CUDA(cudaMemsetAsync(k->A.B.theta, 0, sizeof(float) * R->n_lists, st));
  }
  launch_targets(Y, ld_y, R->T, R->space->N, R->ldy, R->y64, R->y32, R->ydf, R->ysum32, R->err, st);
  R->launches = 1;
  R->fetched = false;
  R->reruns = 0;
  return run_screen(R, k->plan, k->tmul, k->tadd, k->A, k->S, k->tile_ctr);
}

// The statistics of a finished screen from its device counters (stats,
// per-list buffered counts, list lengths and largest bounds).
static void stats_from_counters(const dse_result *R, const unsigned long long *hs, const unsigned *bc,
                                const int64_t *nout, const double *mx, dse_stats &o) {
  for (int c = 0; c < 6; ++c) o.reasons[c] = (int64_t)hs[ST_REASON0 + c];
  o.reasons[DSE_R_UNIT] += (int64_t)R->add_total - (int64_t)hs[ST_ADD_SEEN];
  o.evaluated = (int64_t)hs[ST_EVALUATED];
  for (int g = 0; g < 3; ++g) o.valid_by_group[g] = (int64_t)hs[ST_VALID_G0 + g];
  o.kernel_launches = R->launches;
  o.buffered = 0;
  for (int l = 0; l < R->n_lists; ++l) o.buffered += bc[l];
  o.escalated = (int64_t)hs[ST_ESCALATED];
  o.rescored = (int64_t)hs[ST_RESCORED];
  o.reruns = R->reruns;
  double m = 0.0;
  for (int l = 0; l < R->n_lists; ++l)
    if (nout[l] > 0) m = std::max(m, mx[l]);
  o.max_err_bound = m;
}

// Wait for a result, re-running the screen while any list overflowed its
// buffer (the thresholds reached so far stay valid lower bounds).  Every
// small device result is copied asynchronously into the thread's pinned
// staging area, so each attempt costs one stream synchronisation.
static dse_status finish(dse_result *R) {
  if (R->fetched) return DSE_OK;
  cudaStream_t st = R->stream;
  const int nl = R->n_lists;
  // staging layout: stats | out_n | max_eps | overflow | buf_count | err
  const size_t o_stats = 0, o_n = o_stats + 8 * ST_COUNT, o_eps = o_n + 8 * (size_t)nl,
               o_ov = o_eps + 8 * (size_t)nl, o_bc = o_ov + 4 * (size_t)nl, o_err = o_bc + 4 * (size_t)nl,
               bytes = o_err + 8;
  for (int attempt = 0;; ++attempt) {
    char *h = static_cast<char *>(pinned_staging(bytes));
    if (!h) return DSE_ENOMEM;
    DSE_CUDA(cudaMemcpyAsync(h + o_stats, R->stats, 8 * ST_COUNT, cudaMemcpyDeviceToHost, st));
    DSE_CUDA(cudaMemcpyAsync(h + o_n, R->out_n, 8 * (size_t)nl, cudaMemcpyDeviceToHost, st));
    DSE_CUDA(cudaMemcpyAsync(h + o_eps, R->max_eps, 8 * (size_t)nl, cudaMemcpyDeviceToHost, st));
    DSE_CUDA(cudaMemcpyAsync(h + o_ov, R->overflow, 4 * (size_t)nl, cudaMemcpyDeviceToHost, st));
    DSE_CUDA(cudaMemcpyAsync(h + o_bc, R->buf_count, 4 * (size_t)nl, cudaMemcpyDeviceToHost, st));
    DSE_CUDA(cudaMemcpyAsync(h + o_err, R->err, sizeof(int), cudaMemcpyDeviceToHost, st));
    DSE_CUDA(cudaStreamSynchronize(st));
    const unsigned long long *hs = reinterpret_cast<const unsigned long long *>(h + o_stats);
    const int herr = *reinterpret_cast<const int *>(h + o_err);
    if (herr) {
      set_error(herr == DSE_ETIMEOUT   ? "a bounded device wait timed out"
                : herr == DSE_EBOUNDS ? "an index check of the bounds-checked build failed"
                                      : "invalid target (zero variance or not finite)");
      return herr;
    }
    if (hs[ST_ESC_OVERFLOW]) {
      set_error("escalation list overflow");
      return DSE_EOVERFLOW;
    }
    const unsigned *ov = reinterpret_cast<const unsigned *>(h + o_ov);
    bool any = false;
    for (int l = 0; l < nl; ++l) any |= ov[l] != 0;
    if (any && attempt < 8) {
      ++R->reruns;
      DSE_TRY(R->rerun(R));
      continue;
    }
    if (any) {
      set_error("candidate buffer overflow persisted");
      return DSE_EOVERFLOW;
    }
    dse_stats &o = R->host_stats;
    stats_from_counters(R, hs, reinterpret_cast<const unsigned *>(h + o_bc),
                        reinterpret_cast<const int64_t *>(h + o_n), reinterpret_cast<const double *>(h + o_eps), o);
    for (int g = 0; g < 4; ++g) o.kernel_ms[g] = 0.0;
    for (auto &t : R->timing) {
      float ms = 0.f;
      if (cudaEventElapsedTime(&ms, t.second.first, t.second.second) == cudaSuccess && t.first >= 0 && t.first < 4)
        o.kernel_ms[t.first] += ms;
    }
    const int64_t *nout = reinterpret_cast<const int64_t *>(h + o_n);
    R->h_out_n.assign(nout, nout + nl);
    R->fetched = true;
    return DSE_OK;
  }
}


// ------------------------------------------------- redundancy removal

dse_status dedup_result(dse_result *R, int64_t k, double tau, bool full, bool *undecided, int64_t *n_redundant);

// DSE_FLAG_DEDUP: screen for lists of kk = 4k entries, remove redundant
// entries within the score window, and double kk while an entry's window
// may reach past the end of its list.
static dse_status dedup_screen(dse_space *sp, const dse_screen_desc *d, dse_result **out) {
  const double tau = d->dedup_tau > 0.0 ? d->dedup_tau : 1e-10;
  const uint64_t total = (uint64_t)sp->n + sp->geom.slots;
  const uint64_t id_end = d->id_end ? d->id_end : total;
  const uint64_t range = id_end > d->id_begin ? id_end - d->id_begin : 0;
  const int64_t kmax = (int64_t)1 << 24;
  int64_t kk = std::min<int64_t>(4 * d->k, kmax);
  dse_screen_desc d2 = *d;
  d2.flags &= ~DSE_FLAG_DEDUP;
  for (int round = 1;; ++round) {
    if ((uint64_t)kk > range) kk = (int64_t)std::max<uint64_t>(range, 1);
    d2.k = kk;
    dse_result *R = nullptr;
    DSE_TRY(screen_impl(sp, &d2, &R));
    dse_status s = finish(R);
    bool undecided = false;
    int64_t nred = 0;
    const bool full = (uint64_t)kk < range;
    if (s == DSE_OK) s = dedup_result(R, d->k, tau, full, &undecided, &nred);
    if (s != DSE_OK) {
      dse_result_free(R);
      return s;
    }
    if (!undecided) {
      R->host_stats.redundant = nred;
      R->host_stats.dedup_rounds = round;
      *out = R;
      return DSE_OK;
    }
    dse_result_free(R);
    if (kk >= kmax) {
      set_error("redundancy removal needs lists longer than %lld", (long long)kmax);
      return DSE_EOVERFLOW;
    }
    kk = std::min<int64_t>(2 * kk, kmax);
  }
}

// ------------------------------------------------------ residual loop

size_t refit_chain_bytes(int64_t N, int64_t cap);
void refit_chain_prep(dse_space *S, const double *y, const uint64_t *fid, int nf, void *scratch, int64_t cap,
                      cudaStream_t st);
void refit_chain_vectors(void *scratch, int64_t N, int64_t cap, const double **vec, const float2 **vdf,
                         const int **vexp, double **outx);
void refit_chain_fit(dse_space *S, const double *y, const uint64_t *fid, int nf, const uint64_t *cand, int64_t cap,
                     const int64_t *n_dev, void *scratch, bool have_sums, double *res, double *report,
                     uint64_t *chosen, cudaStream_t st);

constexpr int kLoopMax = 4;  // descriptors (the refit fits up to 4 columns)
constexpr int kReport = 8;   // winner's index, id, rmse, intercept + 4 coefficients
constexpr int kSmall = ST_COUNT + 5;  // per iteration: counters, overflow, buffered, list length, max bound, error

// The residual loop with every iteration enqueued back to back: screen of
// the current residual (one plan, reused), then the refits of its top k
// against the descriptors chosen so far, all on the device; the host reads
// the reports once at the end.  An iteration whose candidate buffer
// overflowed is repeated, with the rest of the loop, on the host-driven
// path (wait, re-run from the thresholds reached, refit).
// One iteration's small results into the loop's report rows (counters,
// overflow flag, buffered count, list length, largest bound, error flag as
// 64-bit words) and its list of ids, in one launch.
__global__ void k_loop_snapshot(const unsigned long long *stats, const unsigned *overflow, const unsigned *buf_count,
                                const int64_t *out_n, const double *max_eps, int *err, const uint64_t *out_id,
                                int64_t k, unsigned long long *small, uint64_t *ids, float *theta, int n_lists) {
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t < ST_COUNT) small[t] = stats[t];
  if (t == 0) {
    small[ST_COUNT] = *overflow;
    small[ST_COUNT + 1] = *buf_count;
    small[ST_COUNT + 2] = (unsigned long long)*out_n;
    small[ST_COUNT + 3] = (unsigned long long)__double_as_longlong(*max_eps);
    small[ST_COUNT + 4] = (unsigned long long)(unsigned)*err;
    // the next iteration's screen starts from a clear error flag and zero
    // thresholds (what its target step would otherwise reset)
    *err = 0;
    for (int l = 0; l < n_lists; ++l) theta[l] = 0.0f;
  }
  for (int64_t i = t; i < k; i += (int64_t)gridDim.x * blockDim.x) ids[i] = out_id[i];
}

static dse_status residual_loop_impl(dse_space *sp, const dse_loop_desc *d, dse_loop_result *out, uint64_t *sis_ids,
                                     double *residual) {
  cudaStream_t st = (cudaStream_t)d->stream;
  const int D = d->n_iter;
  const int it0 = d->n_fixed;  // first iteration run (resume after it0 chosen descriptors)
  const int64_t N = sp->N, k = d->k;
  dse_screen_desc sd{};
  sd.ld_y = N;
  sd.n_targets = 1;
  sd.k = k;
  sd.mode = DSE_MODE_PER_TARGET;
  sd.precision = d->precision == DSE_PREC_FP64 ? DSE_PREC_FP64 : DSE_PREC_FP32;
  sd.stream = d->stream;
  sd.flags = d->flags & (DSE_FLAG_TIMING | DSE_FLAG_TIMING_MAIN);
  dse_result *R = nullptr;
  DSE_TRY(screen_impl(sp, &sd, &R, false));
  struct Owner {
    dse_result *R;
    void *scratch = nullptr;
    ~Owner() {
      dfree(scratch);
      dse_result_free(R);
    }
  } own{R};

  double *ydev = nullptr, *r = nullptr, *rep = nullptr;
  uint64_t *fid = nullptr, *ids = nullptr;
  unsigned long long *small = nullptr;
  unsigned char *rscr = nullptr;
  double *rx = nullptr;
  Keep *kp = reinterpret_cast<Keep *>(R->keep);
  // the re-score takes the refit sums alongside (one warp per candidate:
  // N <= 4096); rx holds them per retained entry
  const bool fused = N <= 4096;
  Scratch sc;
  if (!d->y_on_device) sc.add(&ydev, (size_t)N);
  sc.add(&r, (size_t)D * N);
  sc.add(&fid, kLoopMax);
  sc.add(&rep, (size_t)D * kReport);
  sc.add(&small, (size_t)D * kSmall);
  sc.add(&ids, (size_t)D * k);
  sc.add(&rscr, refit_chain_bytes(N, k));
  sc.add(&rx, fused ? (size_t)R->n_lists * kp->plan.cap * 8 : 1);
  uint64_t *cand1 = nullptr;
  int64_t *n1 = nullptr;
  sc.add(&cand1, 1);
  sc.add(&n1, 1);
  size_t bytes = 0;
  DSE_TRY(sc.alloc(&own.scratch, &bytes));
  const double *y = d->y;
  if (!d->y_on_device) {
    DSE_CUDA(cudaMemcpyAsync(ydev, d->y, sizeof(double) * N, cudaMemcpyHostToDevice, st));
    y = ydev;
  }
  DSE_CUDA(cudaMemsetAsync(fid, 0xFF, sizeof(uint64_t) * kLoopMax, st));
  DSE_CUDA(cudaMemsetAsync(r, 0, sizeof(double) * D * N, st));
  DSE_CUDA(cudaMemsetAsync(small, 0, sizeof(unsigned long long) * D * kSmall, st));
  DSE_CUDA(cudaMemsetAsync(ids, 0xFF, sizeof(uint64_t) * D * k, st));
  if (it0 > 0) {
    // resume: the chosen descriptors, and the fit with all of them (the
    // last one as the only candidate of iteration it0 - 1's refit) for the
    // residual r_it0 the next screen takes
    uint64_t *h = static_cast<uint64_t *>(pinned_staging(sizeof(uint64_t) * (kLoopMax + 1) + sizeof(int64_t)));
    if (!h) return DSE_ENOMEM;
    for (int i = 0; i < it0; ++i) h[i] = d->fixed[i];
    int64_t one = 1;
    memcpy(h + kLoopMax, &one, sizeof(int64_t));
    DSE_CUDA(cudaMemcpyAsync(fid, h, sizeof(uint64_t) * it0, cudaMemcpyHostToDevice, st));
    DSE_CUDA(cudaMemcpyAsync(cand1, h + it0 - 1, sizeof(uint64_t), cudaMemcpyHostToDevice, st));
    DSE_CUDA(cudaMemcpyAsync(n1, h + kLoopMax, sizeof(int64_t), cudaMemcpyHostToDevice, st));
    DSE_CUDA(cudaStreamSynchronize(st));  // (the staging area is reused)
    refit_chain_prep(sp, y, fid, it0 - 1, rscr, 1, st);
    refit_chain_fit(sp, y, fid, it0 - 1, cand1, 1, n1, rscr, false, r + (size_t)(it0 - 1) * N,
                    rep + (size_t)(it0 - 1) * kReport, fid + it0 - 1, st);
    DSE_CUDA(cudaGetLastError());
  }

  auto snapshot = [&](int it) -> dse_status {
    note_launches(1);
    k_loop_snapshot<<<(unsigned)std::max<int64_t>(1, std::min<int64_t>(64, (k + 255) / 256)), 256, 0, st>>>(
        R->stats, R->overflow, R->buf_count, R->out_n, R->max_eps, R->err, R->out_id, k,
        small + (size_t)it * kSmall, ids + (size_t)it * k, kp->A.B.theta, R->n_lists);
    return DSE_OK;
  };
  // before iteration it's screen: the fixed columns' fit, and the vectors
  // the re-score takes the candidates' sums against
  auto prepare = [&](int it) {
    refit_chain_prep(sp, y, fid, it, rscr, k, st);
    if (fused) {
      const double *vec[4];
      const float2 *vdf[4];
      const int *vexp = nullptr;
      double *outx = nullptr;
      refit_chain_vectors(rscr, N, k, vec, vdf, &vexp, &outx);
      for (int m = 0; m < 4; ++m) {
        kp->S.xv[m] = vec[m];
        kp->S.xdf[m] = vdf[m];
      }
      kp->S.xexp = vexp;
      kp->S.nx = 1 + it;
      kp->S.r_x = rx;
      kp->S.out_x = outx;
    }
  };
  auto fit = [&](int it) {
    refit_chain_fit(sp, y, fid, it, R->out_id, k, R->out_n, rscr, fused, r + (size_t)it * N,
                    rep + (size_t)it * kReport, fid + it, st);
  };
  auto step = [&](int it) -> dse_status {
    const double *src = it == 0 ? y : r + (size_t)(it - 1) * N;
    prepare(it);
    DSE_TRY(screen_enqueue_target(R, src, N, it == it0));
    DSE_TRY(snapshot(it));
    fit(it);
    DSE_CUDA(cudaGetLastError());
    return DSE_OK;
  };
  const size_t hbytes = sizeof(unsigned long long) * D * kSmall + sizeof(double) * D * kReport;
  auto read_back = [&](unsigned long long **hs, double **hr) -> dse_status {
    char *h = static_cast<char *>(pinned_staging(hbytes));
    if (!h) return DSE_ENOMEM;
    DSE_CUDA(cudaMemcpyAsync(h, small, sizeof(unsigned long long) * D * kSmall, cudaMemcpyDeviceToHost, st));
    DSE_CUDA(cudaMemcpyAsync(h + sizeof(unsigned long long) * D * kSmall, rep, sizeof(double) * D * kReport,
                             cudaMemcpyDeviceToHost, st));
    DSE_CUDA(cudaStreamSynchronize(st));
    *hs = reinterpret_cast<unsigned long long *>(h);
    *hr = reinterpret_cast<double *>(h + sizeof(unsigned long long) * D * kSmall);
    return DSE_OK;
  };

  // all iterations back to back, one wait
  size_t tmark[kLoopMax + 1];  // each iteration's range of timing events
  for (int it = 0; it < D; ++it) {
    tmark[it] = R->timing.size();
    if (it >= it0) DSE_TRY(step(it));
  }
  tmark[D] = R->timing.size();
  unsigned long long *hs = nullptr;
  double *hr = nullptr;
  DSE_TRY(read_back(&hs, &hr));
  int first_bad = D;
  for (int it = it0; it < D && first_bad == D; ++it) {
    const unsigned long long *sm = hs + (size_t)it * kSmall;
    if ((unsigned)sm[ST_COUNT] != 0u) first_bad = it;  // buffer overflow
  }
  if (first_bad < D) {
    // repeat from the overflowed iteration with the host-driven path
    for (int it = first_bad; it < D; ++it) {
      const double *src = it == 0 ? y : r + (size_t)(it - 1) * N;
      tmark[it] = R->timing.size();
      prepare(it);
      DSE_TRY(screen_enqueue_target(R, src, N));
      DSE_TRY(finish(R));
      DSE_TRY(snapshot(it));
      fit(it);
      DSE_CUDA(cudaGetLastError());
      out->stats[it] = R->host_stats;
      tmark[it + 1] = R->timing.size();
    }
    DSE_TRY(read_back(&hs, &hr));
  }
  for (int it = 0; it < D; ++it) {
    if (it < it0 - 1) {  // chosen in the call being resumed
      out->chosen[it] = d->fixed[it];
      out->rmse[it] = NAN;
      continue;
    }
    const unsigned long long *sm = hs + (size_t)it * kSmall;
    const int herr = (int)(unsigned)sm[ST_COUNT + 4];
    if (herr) {
      set_error(herr == DSE_ETIMEOUT   ? "a bounded device wait timed out"
                : herr == DSE_EBOUNDS ? "an index check of the bounds-checked build failed"
                                      : "invalid target or residual (zero variance or not finite)");
      return herr;
    }
    if (sm[ST_ESC_OVERFLOW]) {
      set_error("escalation list overflow");
      return DSE_EOVERFLOW;
    }
    const double *rr = hr + (size_t)it * kReport;
    long long bi, bid;
    memcpy(&bi, &rr[0], 8);
    memcpy(&bid, &rr[1], 8);
    if (bi < 0) {
      set_error("iteration %d: no candidate gives a full-rank fit", it + 1);
      return DSE_EINVAL;
    }
    out->chosen[it] = (uint64_t)bid;
    out->rmse[it] = rr[2];
    for (int c = 0; c < 5; ++c) out->coefs[it][c] = c < it + 2 ? rr[3 + c] : 0.0;
    if (it < it0) continue;  // the resumed fit: no screen of its own
    if (it < first_bad) {
      const unsigned bc = (unsigned)sm[ST_COUNT + 1];
      const int64_t nout = (int64_t)sm[ST_COUNT + 2];
      double mx;
      memcpy(&mx, &sm[ST_COUNT + 3], 8);
      dse_stats &o = out->stats[it];
      o = dse_stats{};
      o.screened = R->host_stats.screened;
      o.precision_used = R->host_stats.precision_used;
      o.binary_path = R->host_stats.binary_path;
      R->reruns = 0;
      stats_from_counters(R, sm, &bc, &nout, &mx, o);
    }
    // device time of the kernel groups of this iteration's screen
    dse_stats &o = out->stats[it];
    for (int g = 0; g < 4; ++g) o.kernel_ms[g] = 0.0;
    for (size_t e = tmark[it]; e < tmark[it + 1] && e < R->timing.size(); ++e) {
      float ms = 0.f;
      const auto &t = R->timing[e];
      if (cudaEventElapsedTime(&ms, t.second.first, t.second.second) == cudaSuccess && t.first >= 0 && t.first < 4)
        o.kernel_ms[t.first] += ms;
    }
  }
  // outputs
  if (sis_ids) {
    DSE_CUDA(cudaMemcpyAsync(sis_ids, ids, sizeof(uint64_t) * D * k, cudaMemcpyDefault, st));
  }
  if (residual) DSE_CUDA(cudaMemcpyAsync(residual, r + (size_t)(D - 1) * N, sizeof(double) * N, cudaMemcpyDefault, st));
  DSE_CUDA(cudaStreamSynchronize(st));
  return DSE_OK;
}

}  // namespace dse

using namespace dse;

// ================================================================ C ABI

extern "C" {

const char *dse_last_error(void) { return dse::last_error(); }
const char *dse_version(void) { return "dse 0.1 (sm_103a)"; }
int64_t dse_kernel_launches(void) { return launches_so_far(); }

dse_status dse_build_space(const dse_space_desc *d, dse_space **out) {
  dse::NvtxRange nvtx_range_("dse_build_space");
  clear_error();
  if (!d || !out) {
    set_error("null argument");
    return DSE_EINVAL;
  }
  *out = nullptr;
  if (d->n_samples < 2 || d->n_samples > (1 << 30) || d->n_primary < 1 || d->n_primary > (1 << 24) ||
      d->n_dims < 0 || d->n_dims > kMaxDims || d->max_rung < 1 || d->max_rung > kMaxRung || !d->X ||
      (d->n_dims > 0 && !d->units) || (d->op_mask & ~0xFFFu) || d->op_mask == 0 || !(d->fmax_max > 0) ||
      !isfinite(d->fmax_max) || isnan(d->fmin_std_rel)) {
    set_error("invalid space descriptor");
    return DSE_EINVAL;
  }
  if ((d->pair_deny || d->op_deny) && d->n_primary > 64) {
    set_error("user rules need n_primary <= 64");
    return DSE_EINVAL;
  }
  if (d->sample_idx) {
    for (int64_t s = 0; s < d->n_samples; ++s)
      if (d->sample_idx[s] < 0 || d->sample_idx[s] >= d->ld_x) {
        set_error("sample_idx[%lld] out of range", (long long)s);
        return DSE_EINVAL;
      }
  } else if (d->ld_x < d->n_samples) {
    set_error("ld_x < n_samples");
    return DSE_EINVAL;
  }
  DSE_TRY(check_device());
  AllocStream as((cudaStream_t)d->stream);
  dse_status st = build_space(d, out);
  if (st == DSE_OK) (*out)->stream = (cudaStream_t)d->stream;
  return st;
}

void dse_space_free(dse_space *s) {
  if (!s) return;
  AllocStream as(s->stream);
  space_release(s);
}

dse_status dse_space_size(const dse_space *s, int64_t *n_stored, uint64_t *n_total) {
  clear_error();
  if (!s) {
    set_error("null space");
    return DSE_EINVAL;
  }
  if (n_stored) *n_stored = s->n;
  if (n_total) *n_total = (uint64_t)s->n + s->geom.slots;
  return DSE_OK;
}

dse_status dse_space_counts(dse_space *s, int32_t rung, uint64_t *slots, int64_t reasons[6]) {
  dse::NvtxRange nvtx_range_("dse_space_counts");
  clear_error();
  if (!s || rung < 0 || rung > s->max_rung) {
    set_error("bad space or rung");
    return DSE_EINVAL;
  }
  if (rung == s->max_rung) DSE_TRY(count_last_rung(s, 0));
  if (slots) *slots = s->slots[rung];
  if (reasons)
    for (int c = 0; c < 6; ++c) reasons[c] = s->reasons[rung][c];
  return DSE_OK;
}

dse_status dse_decode(const dse_space *s, uint64_t id, dse_expr *out) {
  clear_error();
  if (!s || !out) {
    set_error("null argument");
    return DSE_EINVAL;
  }
  if (id < (uint64_t)s->n) {
    out->rung = s->h_rung[id];
    out->op = s->h_op[id];
    out->a = s->h_ca[id];
    out->b = s->h_cb[id];
    return DSE_OK;
  }
  int op;
  int64_t a, b;
  if (!decode_flat(s->geom, id - (uint64_t)s->n, &op, &a, &b)) {
    set_error("id %llu outside the space", (unsigned long long)id);
    return DSE_ERANGE;
  }
  out->rung = s->max_rung;
  out->op = op;
  out->a = a;
  out->b = b;
  return DSE_OK;
}

static std::string expr_text(const dse_space *s, int op, int64_t a, int64_t b);
static std::string feat_text(const dse_space *s, int64_t f) {
  return expr_text(s, s->h_op[f], s->h_ca[f], s->h_cb[f]);
}
static std::string expr_text(const dse_space *s, int op, int64_t a, int64_t b) {
  if (op == DSE_OP_PRIMARY) return "x" + std::to_string(a);
  std::string A = feat_text(s, a);
  std::string B = b >= 0 ? feat_text(s, b) : std::string();
  switch (op) {
    case DSE_OP_SQUARE: return "sq(" + A + ")";
    case DSE_OP_CUBE: return "cb(" + A + ")";
    case DSE_OP_INV: return "inv(" + A + ")";
    case DSE_OP_SQRT: return "sqrt(" + A + ")";
    case DSE_OP_EXP: return "exp(" + A + ")";
    case DSE_OP_LOG: return "log(" + A + ")";
    case DSE_OP_ADD: return "(" + A + "+" + B + ")";
    case DSE_OP_SUB: return "(" + A + "-" + B + ")";
    case DSE_OP_MUL: return "(" + A + "*" + B + ")";
    case DSE_OP_DIV: return "(" + A + "/" + B + ")";
    case DSE_OP_RDIV: return "(" + B + "/" + A + ")";
    case DSE_OP_ABSDIFF: return "|" + A + "-" + B + "|";
    default: return "?";
  }
}

dse_status dse_expr_string(const dse_space *s, uint64_t id, char *buf, int64_t len) {
  dse_expr e;
  DSE_TRY(dse_decode(s, id, &e));
  if (!buf || len < 1) {
    set_error("null buffer");
    return DSE_EINVAL;
  }
  std::string t = id < (uint64_t)s->n ? feat_text(s, (int64_t)id) : expr_text(s, e.op, e.a, e.b);
  if ((int64_t)t.size() + 1 > len) {
    set_error("buffer too small (%zu needed)", t.size() + 1);
    return DSE_EOVERFLOW;
  }
  memcpy(buf, t.c_str(), t.size() + 1);
  return DSE_OK;
}

dse_status dse_sis_screen(dse_space *s, const dse_screen_desc *d, dse_result **out) {
  dse::NvtxRange nvtx_range_("dse_sis_screen");
  clear_error();
  if (!s || !d || !out) {
    set_error("null argument");
    return DSE_EINVAL;
  }
  *out = nullptr;
  if (!d->Y || d->n_targets < 1 || d->n_targets > 4096 || d->k < 1 || d->k > (1 << 24) || d->ld_y < s->N ||
      (d->mode != DSE_MODE_PER_TARGET && d->mode != DSE_MODE_AGGREGATED) || d->precision < 0 ||
      d->precision > DSE_PREC_AUTO) {
    set_error("invalid screen descriptor");
    return DSE_EINVAL;
  }
  if ((d->flags & DSE_FLAG_DEDUP) && !(d->dedup_tau == 0.0 || (d->dedup_tau > 0.0 && d->dedup_tau < 0.5))) {
    set_error("dedup_tau outside (0, 0.5)");
    return DSE_EINVAL;
  }
  DSE_TRY(check_device());
  AllocStream as((cudaStream_t)d->stream);
  if (d->flags & DSE_FLAG_DEDUP) return dedup_screen(s, d, out);
  return screen_impl(s, d, out);
}

void dse_result_free(dse_result *r) {
  if (!r) return;
  AllocStream as(r->stream);  // the free is ordered after the result's work
  dfree(r->scratch);
  dfree(r->extra);
  if (r->keep && r->keep_free) r->keep_free(r->keep);
  for (cudaEvent_t e : r->events) cudaEventDestroy(e);
  delete r;
}

dse_status dse_topk_fetch(dse_result *r, int32_t list, uint64_t *idx, double *score, double *err_bound, int64_t cap,
                          int64_t *n_out) {
  dse::NvtxRange nvtx_range_("dse_topk_fetch");
  clear_error();
  if (!r || list < 0 || list >= r->n_lists || cap < 0) {
    set_error("bad result or list");
    return DSE_EINVAL;
  }
  DSE_TRY(finish(r));
  const int64_t n = r->h_out_n[list];
  if (n_out) *n_out = n;
  int64_t m = std::min(n, cap);
  if (m == 0) return DSE_OK;
  const size_t off = (size_t)list * r->k;
  // copies on the result's stream; wait only when one lands in host memory
  bool host = false;
  auto cp = [&](void *dst, const void *src, size_t bytes) {
    host |= !is_device_pointer(dst);
    return cudaMemcpyAsync(dst, src, bytes, cudaMemcpyDefault, r->stream);
  };
  if (idx) DSE_CUDA(cp(idx, r->out_id + off, 8 * m));
  if (score) DSE_CUDA(cp(score, r->out_score + off, 8 * m));
  if (err_bound) DSE_CUDA(cp(err_bound, r->out_eps + off, 8 * m));
  if (host) DSE_CUDA(cudaStreamSynchronize(r->stream));
  return DSE_OK;
}

dse_status dse_result_stats(dse_result *r, dse_stats *out) {
  clear_error();
  if (!r || !out) {
    set_error("null argument");
    return DSE_EINVAL;
  }
  DSE_TRY(finish(r));
  *out = r->host_stats;
  return DSE_OK;
}

dse_status dse_residual_loop(dse_space *s, const dse_loop_desc *d, dse_loop_result *out, uint64_t *sis_ids,
                             double *residual) {
  dse::NvtxRange nvtx_range_("dse_residual_loop");
  clear_error();
  if (!s || !d || !out || !d->y || d->n_iter < 1 || d->n_iter > kLoopMax || d->k < 1 || d->k > (1 << 20) ||
      d->precision < 0 || d->precision > DSE_PREC_AUTO || d->n_fixed < 0 || d->n_fixed >= d->n_iter ||
      (d->n_fixed > 0 && !d->fixed)) {
    set_error("invalid loop descriptor");
    return DSE_EINVAL;
  }
  for (int i = 0; i < d->n_fixed; ++i) {
    bool dup = false;
    for (int j = 0; j < i; ++j) dup = dup || d->fixed[j] == d->fixed[i];
    if (dup || d->fixed[i] >= (uint64_t)s->n + s->geom.slots) {
      set_error("fixed descriptor %d is out of range or repeated", i);
      return DSE_EINVAL;
    }
  }
  *out = dse_loop_result{};
  DSE_TRY(check_device());
  AllocStream as((cudaStream_t)d->stream);
  return residual_loop_impl(s, d, out, sis_ids, residual);
}

dse_status dse_ls_refit(dse_space *s, const dse_refit_desc *d, uint64_t *best_id, double *best_rmse, double *coefs,
                        double *residual) {
  dse::NvtxRange nvtx_range_("dse_ls_refit");
  clear_error();
  if (!s || !d || !d->y || d->n_fixed < 0 || d->n_fixed > 3 || (d->n_fixed > 0 && !d->fixed) || !d->cand ||
      d->n_cand < 1 || !best_id || !best_rmse) {
    set_error("invalid refit descriptor");
    return DSE_EINVAL;
  }
  DSE_TRY(check_device());
  AllocStream as((cudaStream_t)d->stream);
  return refit_impl(s, d, best_id, best_rmse, coefs, residual);
}

}  // extern "C"
