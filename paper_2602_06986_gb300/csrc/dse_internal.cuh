// dse_internal.cuh -- shared definitions of the GB300 descriptor-screening
// library: device tables, launch arguments, the flat-index codec and the
// inline-PTX helpers (mbarrier, bulk async copies) used by the kernels.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <string>
#include <vector>

#include "dse.h"

namespace dse {

constexpr int kMaxDims = 8;
constexpr int kMaxRung = 3;
constexpr int kNumBins = 4096;      // threshold histogram bins over [0, 1]
constexpr float kTol = 1e-5f;       // relative tolerance of a reported score

// Per-feature flag bits (exact FP64 tests on the feature's summaries).
enum : uint32_t {
  F_MINABS_POS = 1u << 0,   // min|x| > 0
  F_MIN_POS = 1u << 1,      // min x > 0
  F_MIN_NONNEG = 1u << 2,   // min x >= 0
  F_EXP_DOMAIN = 1u << 3,   // max x <= 80
  F_EXP_MAG = 1u << 4,      // max x <= log(fmax_max)
  F_FP32_SAFE = 1u << 5,    // every nonzero |x| in [2^-60, 2^60]
  F_DIMLESS = 1u << 6,      // unit vector is zero
};

// Device view of the stored features Phi_{k-1} (structure of arrays).
struct FeatTable {
  int64_t n;        // number of stored features
  int64_t N;        // samples
  int64_t ld;       // row stride (elements) of v64 / v32, multiple of 4
  const double *v64;
  const float *v32;                          // RN(v64)
  const float *v32lo;                        // RN(v64 - v32): v64 = v32 + v32lo to 2^-48 relative
                                             // for F_FP32_SAFE features (nullptr while building)
  const double *mean64, *rmean64;            // mean of x, mean of 1/x (0 if min|x| == 0)
  const double *min64, *max64, *minabs64, *maxabs64;
  const float4 *fa;                          // {mean32, rmean32, RU(max|x|), RD(max|x|)}
  const float2 *fr;                          // {RU(1/min|x|), RD(1/min|x|)} (0 if min|x| == 0)
  const uint32_t *flags;
  const int32_t *cplx;
  const int32_t *op;
  const int64_t *ca, *cb;
  const int32_t *units;                      // [n][kMaxDims] scaled exponents
  const uint64_t *ukey;                      // [n][2] packed exponents (16 bits each)
  const float *fnorm;                        // RU(sqrt(sum_s x_s^2))
  // user rules (all three nullptr when the space has none): used[f] = the
  // primaries among f's leaves; dmask[f] = the primaries that may not meet
  // any of them; op_deny[o] = the primaries forbidden below op o
  const uint64_t *used, *dmask, *op_deny;
};

// Rung-k geometry: global id = n_stored + p.
struct RungGeom {
  int64_t o;          // first id of the newest stored rung
  int64_t n;          // stored features
  int32_t nu, nb;     // enabled unary ops / binary slots
  int32_t uops[6];    // op codes of the unary ops in order
  int32_t bops[6];    // op codes of the binary slots in order
  uint64_t um;        // nu * (n - o): size of the unary block
  uint64_t slots;     // total flat slots of rung k
  uint64_t tri_o;     // o(o-1)/2
};

__host__ __device__ inline uint64_t tri(uint64_t n) { return n * (n - 1) / 2; }

// Pair index qs (>= 0) -> (i, j) with i(i-1)/2 <= qs < i(i+1)/2, j = qs - i(i-1)/2.
// A square root estimate, then an exact integer fix-up.
__host__ __device__ inline void pair_from_index(uint64_t qs, uint64_t *i, uint64_t *j) {
#ifdef __CUDA_ARCH__
  // on the device an FP32 root (the FP64 pipe is slow on this part): within
  // one unit of the row for qs < 2^44 (2^22 stored features); the loops
  // below correct whatever is left
  const float d = sqrtf(8.0f * (float)qs + 1.0f);
  uint64_t r = (uint64_t)((1.0f + d) * 0.5f);
#else
  double d = sqrt(8.0 * (double)qs + 1.0);
  uint64_t r = (uint64_t)((1.0 + d) * 0.5);
#endif
  if (r < 1) r = 1;
  while (tri(r) > qs) --r;
  while (tri(r + 1) <= qs) ++r;
  *i = r;
  *j = qs - tri(r);
}

// Flat index p of rung k -> (op, a, b); b = -1 for unary.  Returns false if p
// is outside the rung.
__host__ __device__ inline bool decode_flat(const RungGeom &g, uint64_t p, int *op, int64_t *a,
                                            int64_t *b) {
  if (p >= g.slots) return false;
  if (p < g.um) {
    *a = g.o + (int64_t)(p / (uint64_t)g.nu);
    *op = g.uops[p % (uint64_t)g.nu];
    *b = -1;
    return true;
  }
  uint64_t pp = p - g.um;
  uint64_t q = pp / (uint64_t)g.nb;
  int slot = (int)(pp % (uint64_t)g.nb);
  uint64_t i, j;
  pair_from_index(q + g.tri_o, &i, &j);
  *op = g.bops[slot];
  *a = (int64_t)i;
  *b = (int64_t)j;
  return true;
}

__host__ __device__ inline bool is_unary(int op) { return op >= DSE_OP_SQUARE && op <= DSE_OP_LOG; }

// ------------------------------------------------------------------ buffers

// Per-list candidate buffer: entries (global id, FP32 score, error bound).
struct CandBufs {
  uint64_t *id;        // [lists][cap]
  float *score;        // [lists][cap]
  float *eps;          // [lists][cap]
  unsigned int *count; // [lists]
  int64_t cap;
  unsigned int *hist;  // [lists][kNumBins]   buffered lower bounds by bin
  unsigned int *hist_c;// [lists][kCoarse]    the same, kFine bins per coarse bin
  unsigned int *hist_hi;// [lists][kNumBins]  buffered upper bounds by bin
  float *theta;        // [lists] (as float; raised monotonically with atomicMax on bits)
};

constexpr int kFine = 64;
constexpr int kCoarse = kNumBins / kFine;

__host__ __device__ inline int score_bin(float x) {
  int b = x > 0.f ? (int)(x * (float)kNumBins) : 0;
  return b > kNumBins - 1 ? kNumBins - 1 : b;
}

// Statistics counters on the device (unsigned long long for atomics).
enum {
  ST_REASON0 = 0,      // 6 reason counters
  ST_EVALUATED = 6,
  ST_BUFFERED = 7,
  ST_ESCALATED = 8,
  ST_RESCORED = 9,
  ST_ESC_OVERFLOW = 10,
  ST_TIMEOUT = 11,
  ST_ADD_SEEN = 12,    // additive slots examined by the additive pair kernel
  ST_VALID_G0 = 13,    // valid candidates scored per kernel group (3)
  ST_COUNT = 16
};

// Tile of the pair triangle: rows rowid[ibase .. ibase+ni) x rowid[jbase .. jbase+nj);
// a pair (x, y) is taken iff position(x) > position(y).
struct Tile {
  int32_t ibase, jbase;
  int16_t ni, nj;
  int32_t prob;  // problem of a batched screen (0 otherwise)
};

// A run of consecutive work units of one problem of a batched screen
// (candidates of the stored/unary group, or pairs of the pair list).
struct Job {
  int32_t prob;
  int32_t count;
  int64_t first;
};

// Arguments common to the screen kernels.
struct ScreenArgs {
  FeatTable F;
  RungGeom G;
  int64_t n_stored;
  uint64_t id_begin, id_end;   // global id range
  int32_t N;
  double invN;                 // 1/N (rounded to the evaluation type by each kernel)
  int32_t ldy;                 // row stride of y32 / y64
  int32_t T;                   // targets in this pass
  int32_t t0;                  // first target of this pass (list offset)
  int32_t mode;                // DSE_MODE_*
  int32_t n_lists;
  const float *y32;            // [T][ldy] centred, unit-norm targets (FP32)
  const float2 *ydf;           // [T][ldy] the same as pairs (hi, lo) = (y32, RN(y64 - y32)), or nullptr
  const double *y64;           // [T][ldy] centred, unit-norm targets (FP64)
  const float *ysum32;         // [T] sum of the FP32 targets
  int32_t max_complexity;
  float fmax32_dn, fmax32_up;  // RD / RU of fmax_max
  double fmax64;
  float fmin_std_rel;          // < 0: degeneracy test off
  double fmin_std_rel64;
  float gamma;                 // accumulation error factor (FP32 path)
  float u;                     // unit roundoff of the evaluation type
  int64_t k;
  int32_t unit_check_addsub, explog_dimensionless;
  CandBufs B;
  uint64_t *esc_id;            // escalation list (global ids)
  unsigned int *esc_count;
  int64_t esc_cap;
  unsigned long long *stats;
  int *err;                    // device error flag (timeouts)
  // pair kernels
  const Tile *tiles;
  int32_t n_tiles;
  unsigned int *tile_counter;
  const int32_t *rowid;
  int32_t slot_pos[6];         // flat slot position of each binary op code 6..11 (-1 = off)
  int32_t first_pass;          // count statistics and escalate only in the first target pass
  int32_t group;               // kernel group for the per-group valid counters
  // batched screens: per-problem accumulation factors and the problem index
  // recorded with each escalated candidate
  float gamma_lane;            // warp-per-candidate kernels
  int32_t block_len;           // pair kernel blocking of the FP32 sums
  int32_t prob;
  uint32_t *esc_prob;          // escalation list: problem of each entry (batched only)
  int8_t *why;                 // optional: reason code of each id of [id_begin, id_end) (device)
  float2 *ivl;                 // optional: (s, eps) of each id of the range and list, before re-scores
  int32_t gram_addsub;         // a+b and a-b are scored by the Gram kernel: the additive kernels take |a-b| only
  // the entries of the escalation list that its FP32 stage left undecided
  // (single screens; nullptr: no FP32 stage)
  uint64_t *esc2_id = nullptr;
  unsigned int *esc2_count = nullptr;
};

// Planner parameters in effect (dse_set_tuning, defaults filled in).
struct Tuning {
  int tile_group_tc, tile_group_cc, seed_stride, gram_max_n, tc_min_targets, batch_job_samples, gmt_group,
      gmt_cluster;
};
Tuning tuning();

// Launch bookkeeping (process-wide count of the library's kernel launches).
void note_launches(int64_t n);

// ---------------------------------------------------- bounds-checked build
// DSE_IN_BOUNDS(i, n, err): with DSE_CHECK_BOUNDS, whether 0 <= i < n; on a
// violation DSE_EBOUNDS goes to the error word *err (when not null) and the
// caller skips the access.  Always true otherwise (no code).
#ifdef DSE_CHECK_BOUNDS
__device__ __forceinline__ bool dse_in_bounds(int64_t i, int64_t n, int *err) {
  if (i >= 0 && i < n) return true;
  if (err) atomicExch(err, DSE_EBOUNDS);
  return false;
}
#define DSE_IN_BOUNDS(i, n, err) ::dse::dse_in_bounds((int64_t)(i), (int64_t)(n), (err))
#else
#define DSE_IN_BOUNDS(i, n, err) true
#endif
// the operands a (and b >= 0) of a decoded candidate are rows of F
#define DSE_OPERANDS_OK(F, a, b, err) (DSE_IN_BOUNDS((a), (F).n, (err)) && ((b) < 0 || DSE_IN_BOUNDS((b), (F).n, (err))))

// ----------------------------------------------------------- PTX helpers

__device__ __forceinline__ uint32_t smem_u32(const void *p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ void mbar_init(uint64_t *bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_fence_init() {
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t *bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
               : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t *bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}

// Bounded wait on an mbarrier phase; returns false (and the caller records a
// timeout) if the phase did not complete within `limit` polls.
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t *bar, uint32_t parity, uint32_t limit) {
  for (uint32_t it = 0; it < limit; ++it)
    if (mbar_try_wait(bar, parity)) return true;
  return false;
}

// 2-D tensor copy (TMA) of one box at element coordinates (x, y) of the
// tensor map into shared memory, completing on an mbarrier.  x times the
// element size must be a multiple of 16 bytes.
__device__ __forceinline__ void tma_load_2d(void *dst, const void *map, int x, int y, uint64_t *bar) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];" ::"r"(
          smem_u32(dst)),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(smem_u32(bar))
      : "memory");
}

// 1-D bulk async copy global -> shared, completing on an mbarrier.
// dst, src 16-byte aligned, bytes a multiple of 16.
__device__ __forceinline__ void bulk_g2s(void *dst, const void *src, uint32_t bytes, uint64_t *bar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
          smem_u32(dst)),
      "l"(src), "r"(bytes), "r"(smem_u32(bar))
      : "memory");
}

// The same copy delivered to this offset of every CTA of the cluster named
// by ctaMask, each completing on its own mbarrier at the offset of bar.
__device__ __forceinline__ void bulk_g2s_mc(void *dst, const void *src, uint32_t bytes, uint64_t *bar,
                                            uint16_t mask) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes.multicast::cluster [%0], [%1], %2, [%3], "
      "%4;" ::"r"(smem_u32(dst)),
      "l"(src), "r"(bytes), "r"(smem_u32(bar)), "h"(mask)
      : "memory");
}

__device__ __forceinline__ uint32_t cluster_ctarank() {
  uint32_t r;
  asm volatile("mov.u32 %0, %%cluster_ctarank;" : "=r"(r));
  return r;
}

// All threads of every CTA of the cluster (release / acquire).
__device__ __forceinline__ void cluster_sync_all() {
  asm volatile("barrier.cluster.arrive.release.aligned;\n\tbarrier.cluster.wait.acquire.aligned;" ::: "memory");
}

__device__ __forceinline__ float rcp_approx(float x) {
  float r;
  asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
  return r;
}

// Raise a non-negative float threshold monotonically.
__device__ __forceinline__ void atomic_max_nonneg(float *addr, float v) {
  atomicMax(reinterpret_cast<int *>(addr), __float_as_int(v));
}

__device__ __forceinline__ float ld_relaxed(const float *p) {
  float v;
  asm volatile("ld.relaxed.gpu.global.f32 %0, [%1];" : "=f"(v) : "l"(p));
  return v;
}

}  // namespace dse

// ----------------------------------------------------- host-side handles

struct dse_space {
  // description
  int64_t N, ld, n_primary;
  int32_t D, max_rung;
  uint32_t op_mask;
  int32_t max_complexity, unit_check_addsub, explog_dimensionless;
  double fmax_max, fmin_std_rel, exp_arg_max;
  int device;
  // stored features (device)
  int64_t n;                     // stored
  int64_t rung_begin[dse::kMaxRung + 2];
  uint64_t slots[dse::kMaxRung + 1];
  int64_t reasons[dse::kMaxRung + 1][6];
  bool have_counts[dse::kMaxRung + 1];
  double *v64 = nullptr;
  float *v32 = nullptr, *v32lo = nullptr;
  double *mean64 = nullptr, *rmean64 = nullptr, *min64 = nullptr, *max64 = nullptr,
         *minabs64 = nullptr, *maxabs64 = nullptr;
  float4 *fa = nullptr;
  float2 *fr = nullptr;
  float *fnorm = nullptr;
  uint32_t *flags = nullptr;
  int32_t *cplx = nullptr, *op = nullptr, *units = nullptr;
  int64_t *ca = nullptr, *cb = nullptr;
  uint64_t *ukey = nullptr;
  uint64_t *used = nullptr, *dmask = nullptr, *op_deny = nullptr;  // user rules (nullptr: none)
  int32_t *rowid_ident = nullptr;   // identity row list [0, n)
  void *gram_buf = nullptr;         // product Gram images and sums (built at the first use)
  void *gmt_buf = nullptr;          // multi-target Gram a-images and sums (built at the first use)
  float *rcp32 = nullptr;           // [n][ld] rcp.approx of v32 (tensor-core products, built at the first use)
  float *v32_class = nullptr;       // v32 rows in unit-class order (tensor-core additive tiles, first use)
  // host copies for decoding
  std::vector<int32_t> h_op, h_rung, h_cplx;
  std::vector<int64_t> h_ca, h_cb;
  std::vector<uint64_t> h_ukey;     // [n][2]
  // unit classes for the additive pair kernels
  std::vector<int32_t> h_class_rows;            // feature ids sorted by (unit key, id)
  std::vector<int64_t> h_class_begin;           // class boundaries into h_class_rows
  int32_t *class_rows = nullptr;
  int2 *eq_pairs = nullptr;                     // equal-unit pairs (i > j, i in the newest rung)
  int64_t n_eq_pairs = -1;                      // -1: not built yet
  dse::RungGeom geom;
  cudaStream_t stream = nullptr;   // build stream: the space's memory is freed in its order
  dse::FeatTable table() const;
};

struct dse_result {
  dse_space *space;
  int32_t n_lists, T, mode, precision;
  int64_t k;
  uint64_t id_begin, id_end;
  cudaStream_t stream;
  // outputs (device)
  uint64_t *out_id = nullptr;       // [lists][k]
  double *out_score = nullptr;      // [lists][k]
  double *out_eps = nullptr;        // [lists][k]
  int64_t *out_n = nullptr;         // [lists]
  double *max_eps = nullptr;        // [lists] largest returned bound
  std::vector<int64_t> h_out_n;     // list lengths (host, after the wait)
  unsigned long long *stats = nullptr;
  int *err = nullptr;
  unsigned int *overflow = nullptr; // [lists]
  // working state kept for a re-run
  double *y64 = nullptr;
  float *y32 = nullptr;
  float2 *ydf = nullptr;
  float *ysum32 = nullptr;
  int32_t ldy = 0;
  int32_t reruns = 0;
  bool fetched = false;
  dse_stats host_stats{};
  void *scratch = nullptr;          // one allocation for buffers
  void *extra = nullptr;            // deduplicated lists (out_* point into it)
  size_t scratch_bytes = 0;
  unsigned int *buf_count = nullptr;
  uint64_t add_total = 0;           // additive slots of the screened binary range
  void *keep = nullptr;             // launch state for a re-run
  void (*keep_free)(void *) = nullptr;
  dse_status (*rerun)(dse_result *) = nullptr;
  int32_t flags = 0;
  std::vector<std::pair<int, std::pair<cudaEvent_t, cudaEvent_t>>> timing;  // (group, start, stop)
  std::vector<cudaEvent_t> events;  // every event of timing (one may close a group and open the next)
  int64_t launches = 0;
};
