// screen_tc.cu -- the multi-target screen on the 5th-generation tensor cores.
//
// With T targets (residuals or tasks) screened at once, the numerators
// sum_s w_s y_{t,s} of every candidate are a dense contraction
// D[m][t] = sum_s A[m][s] B[t][s] between the candidate values A (generated on
// the fly, never written to HBM) and the targets B.  This kernel evaluates the
// binary block of rung k tile by tile (128 pairs per tile, the three slots of
// one kind) and contracts on tcgen05 in BF16x3: A = Ah + Al, B = Bh + Bl (BF16
// splits of the FP32 values), D += Ah Bh + Ah Bl + Al Bh with FP32
// accumulation in TMEM.  S1 = sum w and S2 = sum w^2 stay on the CUDA cores in
// FP32.
//
// Warp roles (one CTA per SM, persistent over a static tile stride):
//   warp 0        producer: per 32-sample chunk, 2-D tensor copies (TMA,
//                 boxes of 8 rows, 128-byte swizzle) of the tile's 24
//                 operand rows and of their reciprocal rows, and a bulk copy
//                 of the pre-split target block into a 3-stage ring
//                 (mbarrier expect-tx);
//   warp 1        TMEM allocation and the MMA issuer (one elected thread):
//                 3 slots x 2 k-steps x 3 products per chunk; tcgen05.commit to
//                 the stage's "empty" barrier and, after the last chunk of an
//                 accumulation block, to the accumulator's "full" barrier;
//   warps 2-9     generation: row m (a pair) x one half of each chunk's samples:
//                 candidate values (quotients from reciprocal rows copied
//                 next to the value rows), FP32 S1/S2, BF16 hi/lo split,
//                 16-byte stores into the canonical K-major layout (8x8 core
//                 matrices, no swizzle), proxy fence, arrive;
//   warps 10-13   epilogue: tcgen05.ld of TMEM lane quadrant (warp % 4),
//                 block accumulation, scores, error bounds, threshold pushes.
// Accumulators are double-buffered in TMEM by accumulation block (up to 16
// chunks = 512 samples), so the epilogue of one block overlaps the MMAs of
// the next; longer sample ranges drain each block into a running FP32 sum
// that the epilogue keeps in further TMEM columns.
//
// Error model of the contraction (used for the reported bound, and the
// reason reported TC scores above the 1e-5 tolerance are re-scored):
// the BF16x3 split drops Al Bl and the splits' residuals (BF16 rounds to
// 8 significant bits, so each two-term split leaves at most 2^-16 of the
// value), at most 3.01 * 2^-16 of sum |w y|; each tensor-core accumulation
// step is modelled with a relative error of 2u on the running sum of
// |terms|, with a safety factor of 4 (the accumulation order and rounding
// inside an MMA are not documented, so this part is a model, not a proof).
#include <cuda.h>
#include <cuda_bf16.h>
#include <math.h>

#include "dse_internal.cuh"
#include "eval64.cuh"
#include "screen_common.cuh"
#include "screen_kernels.cuh"
#include "tcgen05.cuh"
#include "util.cuh"

namespace dse {

namespace tc {

constexpr int M = 128;  // pairs per tile
constexpr int BI = 16, BJ = 8, ROWS = BI + BJ;
constexpr int NS = 3;     // stages of the A operands (and, with A in shared memory, of everything)
constexpr int NR_MAX = 6;  // stages of the operand rows and target blocks with A in TMEM
constexpr int KB = 16;    // chunks per accumulation block (512 samples)
constexpr int NGEN = 8;   // generation warps: two per row quadrant, one per half of a chunk
constexpr int NPART = NGEN / 4;  // parts of a chunk's samples
constexpr int SPP = 32 / NPART;  // samples per part (a multiple of 8)
constexpr int WARPS = 2 + NGEN + 4;
constexpr int THREADS = WARPS * 32;
constexpr uint32_t kWait = 1u << 22;
// polls of the epilogue's waits, each followed by a short sleep (the
// epilogue has a whole accumulation block of slack, so it polls gently)
constexpr uint32_t kWaitLazy = 1u << 22;

// Operand rows in shared memory: the 16 i-rows, then the 8 j-rows, 128 bytes
// (32 samples) each, written by 2-D tensor copies (boxes of 8 rows) with the
// 128-byte swizzle: 16-byte group q of row r sits at group q ^ (r & 7), so
// the rows a warp reads at one sample offset lie in different banks.
constexpr uint32_t ROWS_BYTES = 2 * ROWS * 128;  // 6144: the rows, then their reciprocals (products)
constexpr int RCP_ROW = ROWS;                      // row index of the first reciprocal row
constexpr uint32_t A_TILE = M * KC * 2;         // 8192 per slot per hi/lo
constexpr uint32_t A_OFF = ROWS_BYTES;
// With 16 targets a pass the A operands (candidate values, BF16 hi/lo) live
// in tensor memory: the MMA then reads only B from shared memory, whose
// bandwidth an N = 16 MMA with a shared-memory A would exhaust.  Wider target
// blocks keep A in shared memory (their accumulators leave no room).
__host__ __device__ constexpr bool tmem_a(int ntp) { return ntp == 16; }
__host__ __device__ constexpr uint32_t b_off(int ntp) { return tmem_a(ntp) ? ROWS_BYTES : A_OFF + 6 * A_TILE; }
__host__ __device__ constexpr uint32_t b_bytes(int ntp) { return 2u * (uint32_t)ntp * KC * 2; }
__host__ __device__ constexpr uint32_t stage_bytes(int ntp) { return b_off(ntp) + b_bytes(ntp); }
static_assert(A_OFF % 1024 == 0 && b_off(16) % 1024 == 0 && b_off(32) % 1024 == 0 && stage_bytes(16) % 1024 == 0 &&
                  stage_bytes(32) % 1024 == 0 && stage_bytes(48) % 1024 == 0 && stage_bytes(64) % 1024 == 0,
              "the swizzled row boxes need 1024-byte aligned stages");
// TMEM columns: two accumulator buffers of 3 slots x acc_w columns, the
// running sums of longer sample ranges (3 x NTP, NTP = 32; with A in TMEM
// they are kept in shared memory), then (A in TMEM) per stage 3 slots x
// hi/lo x KC/2 columns (two BF16 per 32-bit column).  With A in TMEM each
// slot's accumulator is 2 NTP wide: one N = 2 NTP MMA takes wh against the
// stacked [yh; yl] block and an N = NTP MMA adds wl yh onto the first half,
// so the numerator is the sum of the two halves (two MMAs per K-step and
// slot instead of three).
__host__ __device__ constexpr int acc_w(int ntp) { return tmem_a(ntp) ? 2 * ntp : ntp; }
__host__ __device__ constexpr int acc_cols(int ntp) {
  return tmem_a(ntp) ? 6 * acc_w(ntp) : ntp <= 32 ? 9 * ntp : 6 * ntp;
}
constexpr int A_STAGE_COLS = 3 * 2 * (KC / 2);  // 96
__host__ __device__ constexpr int tmem_cols_needed(int ntp) {
  return acc_cols(ntp) + (tmem_a(ntp) ? NS * A_STAGE_COLS : 0);
}

// Byte offset of samples s .. s+3 (s a multiple of 4) of swizzled row r.
__host__ __device__ constexpr uint32_t row_off(int r, int s) {
  return (uint32_t)(r * 128 + ((((s >> 2) ^ (r & 7))) << 4));
}

// Offsets of the eight samples s .. s+7 a generation thread reads from each
// of its four rows (value rows ri, rj and their reciprocals); the same in
// every stage, so computed once.
struct GenAddr {
  uint32_t a[2], b[2], ia[2], ib[2];
};
__device__ __forceinline__ GenAddr gen_addr(int ri, int rj, int s) {
  GenAddr g;
  for (int h = 0; h < 2; ++h) {
    g.a[h] = row_off(ri, s + 4 * h);
    g.b[h] = row_off(rj, s + 4 * h);
    g.ia[h] = row_off(RCP_ROW + ri, s + 4 * h);
    g.ib[h] = row_off(RCP_ROW + rj, s + 4 * h);
  }
  return g;
}

struct Shared {
  uint64_t full_rows[NR_MAX], empty[NR_MAX];  // row stages: copies landed / MMAs done with them
  uint64_t full_a[NS], empty_a[NS];           // A stages: generated / MMAs done (A in TMEM)
  uint64_t acc_full[2], acc_empty[2], gen_done[2], epi_free[2];
  uint64_t drain;  // last tcgen05.commit of the MMA issuer, before TMEM is freed
  uint32_t tmem_base;
  int abort;
  float hand[2][NPART][M][6];  // [tile parity][sample part][row][S1, S2 per slot]
  float theta[4][64];        // each epilogue warp's copy of the pass's list thresholds
  float ysum[4][64];         // and of the targets' sums
  float sy[4][16][32];       // each epilogue warp's spill of 16 numerators for its rare full scores
};

constexpr size_t shared_bytes() { return (sizeof(Shared) + 1023) / 1024 * 1024; }
// With A in TMEM, each row's running numerator sums (3 slots x NTP, rows 49
// floats apart) follow the stages in shared memory.
constexpr int RUN_W = 49;
__host__ __device__ constexpr size_t run_bytes(int ntp) { return tmem_a(ntp) ? (size_t)M * RUN_W * 4 : 0; }

}  // namespace tc

// Pre-split targets: for chunk c, {hi, lo} x ntp x KC BF16 in the core-matrix
// layout (targets beyond T and samples beyond N are zero).
__global__ void k_tc_targets(const float *y32, int32_t ldy, int t0, int T, int N, int ntp, int nchunks,
                             unsigned char *out) {
  const int64_t total = (int64_t)nchunks * ntp * tc::KC;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
    const int c = (int)(e / ((int64_t)ntp * tc::KC));
    const int rem = (int)(e % ((int64_t)ntp * tc::KC));
    const int t = rem / tc::KC, k = rem % tc::KC;
    const int s = c * tc::KC + k;
    const float v = (t < T && s < N) ? y32[(int64_t)(t0 + t) * ldy + s] : 0.f;
    const __nv_bfloat16 h = __float2bfloat16_rn(v);
    const __nv_bfloat16 l = __float2bfloat16_rn(v - __bfloat162float(h));
    unsigned char *base = out + (size_t)c * tc::b_bytes(ntp);
    *reinterpret_cast<__nv_bfloat16 *>(base + tc::core_off(t, k)) = h;
    *reinterpret_cast<__nv_bfloat16 *>(base + (size_t)ntp * tc::KC * 2 + tc::core_off(t, k)) = l;
  }
}

// Epilogue of one candidate (row m, slot k), in two parts: the tests that
// do not depend on the target (a-priori, realised; escalation) and the
// target-independent terms of the score bound, then the targets 16 at a
// time straight from the tensor memory (no per-thread array of NTP values).
struct TcCand {
  bool ok;
  uint64_t gid;
  CandInterval<float> ci;
  float S1, a0, a1, a2, qlo;
};

__device__ __forceinline__ TcCand tc_prepare(const ScreenArgs &A, LaneStats &ls, bool pv, int64_t ia, int64_t ib,
                                             int opc, uint64_t pbase, const float4 &fa_a, const float4 &fa_b,
                                             float kk, float mi, float mj, float S1, float S2, float gamma_gen,
                                             float gamma_num) {
  TcCand o;
  o.ok = false;
  const bool additive = opc == DSE_OP_ADD || opc == DSE_OP_SUB || opc == DSE_OP_ABSDIFF;
  const int pos = A.slot_pos[opc - 6];
  o.gid = (uint64_t)A.n_stored + pbase + (uint64_t)(pos < 0 ? 0 : pos);
  const bool cand = pv && pos >= 0 && o.gid >= A.id_begin && o.gid < A.id_end;
  if (!cand) return o;
  if (additive) ls.seen++;
  EvalErr<float> ee{0.f, 0.f};
  const int reason = binary_apriori_W<float>(A, opc, ia, ib, fa_a, fa_b, kk, mi, mj, &ee);
  if (reason != DSE_VALID) {
    ls.r[reason]++;
    note_why(A, o.gid, reason);
    return o;
  }
  if (!((A.F.flags[ia] & A.F.flags[ib]) & F_FP32_SAFE)) {
    escalate(A, o.gid);
    ls.escalated++;
    return o;
  }
  const float u = 5.9604644775390625e-8f;
  const float N = (float)A.N, invN = (float)A.invN, sqrtN = sqrtf(N);
  const float cshift = opc == DSE_OP_ADD ? mi + mj : opc == DSE_OP_SUB ? mi - mj : kk;
  o.ci = cand_interval<float>(S1, S2, N, invN, sqrtN, cshift, ee, gamma_gen, u, (float)A.fmin_std_rel64);
  if (o.ci.realised == 0) {
    ls.r[DSE_R_REALISED]++;
    note_why(A, o.gid, DSE_R_REALISED);
    return o;
  }
  if (o.ci.realised == 2) {
    escalate(A, o.gid);
    ls.escalated++;
    return o;
  }
  ls.r[DSE_VALID]++;
  ls.evaluated++;
  note_why(A, o.gid, DSE_VALID);
  // The largest score the interval of target t can reach is
  // rhi = (|P_t| a2 + a0 + a1 |ysum_t|) / q_lo (the terms of cand_score_num's
  // numerator bound, split into what depends on the target and what does
  // not); a candidate whose rhi is below the list's threshold (a lower bound
  // of the final k-th lower bound) cannot be in the top k.
  o.S1 = S1;
  o.a0 = (gamma_num * o.ci.sqS2 * (1.0f + 2.0f * u) + o.ci.E * (1.0f + 2.0f * u) + 2.0f * u * o.ci.q_hi) * 1.01f;
  o.a1 = fabsf(S1) * invN * (gamma_gen + 4.0f * u) * 1.01f;
  o.a2 = 1.0f + u * 1.01f;
  o.qlo = o.ci.q_lo * (1.0f - 8.0f * u);
  o.ok = true;
  return o;
}

// Targets t0 .. t0+15 of a prepared candidate; returns the lists pushed to.
// The cheap bound is evaluated for all 16 without branches (independent
// chains); the few survivors are scored in full from a per-lane copy of
// their numerators in shared memory (sy: [16][32] of this warp).
__device__ __forceinline__ uint64_t tc_targets16(const ScreenArgs &A, const TcCand &c, const float (&Sy)[16], int t0,
                                                 float gamma_gen, float gamma_num, const float *ysum,
                                                 const float *theta, float (*sy)[32]) {
  const float u = 5.9604644775390625e-8f;
  const float invN = (float)A.invN;
  const int lane = threadIdx.x & 31;
  if (A.ivl) {
    // every target's interval, for checking the error model
#pragma unroll
    for (int i = 0; i < 16; ++i) {
      const int t = t0 + i;
      if (t >= A.T) continue;
      float s, e;
      cand_score_num<float>(c.ci, c.S1, Sy[i], invN, ysum[t], gamma_gen, gamma_num, u, &s, &e);
      note_ivl(A, c.gid, A.t0 + t, s, e * (1.0f + 2.4e-7f));
    }
  }
  unsigned mask = 0;
#pragma unroll
  for (int i = 0; i < 16; ++i) {
    const int t = t0 + i;
    const float ys = ysum[t];
    const float aP = fabsf(fmaf(-c.S1, ys * invN, Sy[i]));
    const float num = fmaf(aP, c.a2, fmaf(c.a1, fabsf(ys), c.a0)) * (1.0f + 8.0f * u);
    const bool pass = t < A.T && !(c.qlo > 0.0f && num < theta[t] * c.qlo);
    mask |= pass ? 1u << i : 0u;
  }
  if (!mask) return 0;
#pragma unroll
  for (int i = 0; i < 16; ++i) sy[i][lane] = Sy[i];
  uint64_t pushed = 0;
  while (mask) {
    const int i = __ffs(mask) - 1;
    mask &= mask - 1;
    const int t = t0 + i;
    const float v = sy[i][lane];
    float s, e;
    cand_score_num<float>(c.ci, c.S1, v, invN, ysum[t], gamma_gen, gamma_num, u, &s, &e);
    if (iv_hi(s, e) < theta[t]) continue;
    if (push_one(A.B, A.t0 + t, c.gid, s, e * (1.0f + 2.4e-7f))) pushed |= 1ull << t;
  }
  return pushed;
}

// Generation state of one row (pair) of a tile: the shift constants of the
// three slots (products: the FMA constants of a*b, a/b, b/a; sums: the two
// centring means and the |a-b| constant) and the running blocked sums.
struct TcGen {
  float c0, c1, c2;
  float t1[3], t2[3];
};

// Eight samples of the three slots of one row: samples kbase + k .. +7 of
// the stage's operand rows ri, rj and of their reciprocal rows (swizzled,
// see row_ld4).  Candidate values, FP32 sum w
// and sum w^2, BF16 hi/lo splits (two values per conversion) and 16-byte
// stores into the canonical K-major layout of the A tiles.  CHECK: entries at
// or beyond `lim` are zero (the last, partial chunk).
template <int KIND, bool CHECK, bool TA>
__device__ __forceinline__ void tc_gen8(TcGen &g, const unsigned char *S, const tc::GenAddr &ad, int k, int kbase, int lim,
                                        unsigned char *Aop, uint32_t acol, int m) {
  using namespace tc;
  float av[8], bv[8], iav[8], ibv[8];
#pragma unroll
  for (int h = 0; h < 2; ++h) {
    *reinterpret_cast<float4 *>(av + 4 * h) = *reinterpret_cast<const float4 *>(S + ad.a[h]);
    *reinterpret_cast<float4 *>(bv + 4 * h) = *reinterpret_cast<const float4 *>(S + ad.b[h]);
    if (KIND == KIND_MUL) {
      *reinterpret_cast<float4 *>(iav + 4 * h) = *reinterpret_cast<const float4 *>(S + ad.ia[h]);
      *reinterpret_cast<float4 *>(ibv + 4 * h) = *reinterpret_cast<const float4 *>(S + ad.ib[h]);
    }
  }
  float wv[3][8];
#pragma unroll
  for (int e = 0; e < 8; ++e) {
    if (!CHECK || k + e < lim) {
      const float a = av[e], b = bv[e];
      if (KIND == KIND_MUL) {
        wv[0][e] = fmaf(a, b, -g.c0);
        wv[1][e] = fmaf(a, ibv[e], -g.c1);
        wv[2][e] = fmaf(b, iav[e], -g.c2);
      } else {
        const float ac = a - g.c0, bc = b - g.c1, d = a - b;
        wv[0][e] = ac + bc;
        wv[1][e] = ac - bc;
        wv[2][e] = fabsf(d) - g.c2;
      }
#pragma unroll
      for (int sl = 0; sl < 3; ++sl) {
        g.t1[sl] += wv[sl][e];
        g.t2[sl] = fmaf(wv[sl][e], wv[sl][e], g.t2[sl]);
      }
    } else {
      wv[0][e] = wv[1][e] = wv[2][e] = 0.f;
    }
  }
#pragma unroll
  for (int sl = 0; sl < 3; ++sl) {
    uint32_t hi[4], lo[4];
#pragma unroll
    for (int e = 0; e < 8; e += 2) {
      const __nv_bfloat162 h = __floats2bfloat162_rn(wv[sl][e], wv[sl][e + 1]);
      const __nv_bfloat162 l = __floats2bfloat162_rn(wv[sl][e] - __low2float(h), wv[sl][e + 1] - __high2float(h));
      hi[e >> 1] = *reinterpret_cast<const uint32_t *>(&h);
      lo[e >> 1] = *reinterpret_cast<const uint32_t *>(&l);
    }
    if (TA) {
      // this lane's row: four columns (eight samples) per component
      const uint32_t col = acol + (uint32_t)sl * KC + (uint32_t)(kbase + k) / 2;
      tmem_st4(col, hi);
      tmem_st4(col + KC / 2, lo);
    } else {
      *reinterpret_cast<uint4 *>(Aop + (2 * sl) * A_TILE + core_off(m, kbase + k)) =
          make_uint4(hi[0], hi[1], hi[2], hi[3]);
      *reinterpret_cast<uint4 *>(Aop + (2 * sl + 1) * A_TILE + core_off(m, kbase + k)) =
          make_uint4(lo[0], lo[1], lo[2], lo[3]);
    }
  }
}

template <int KIND, int NTP>
__global__ void __launch_bounds__(tc::THREADS, 1) k_pair_tc(const ScreenArgs A, const unsigned char *bsplit,
                                                             const __grid_constant__ CUtensorMap rows_map,
                                                             const __grid_constant__ CUtensorMap rcp_map,
                                                             float gamma_gen, float gamma_num, int gen_blk) {
  using namespace tc;
  extern __shared__ __align__(1024) unsigned char smem[];
  Shared &sh = *reinterpret_cast<Shared *>(smem);
  unsigned char *stages = smem + shared_bytes();
  constexpr uint32_t SB = stage_bytes(NTP);
  constexpr bool TA = tmem_a(NTP);
  // row stages: with A in TMEM they are small and outnumber the A stages, so
  // the copies run further ahead; otherwise rows and A share the NS stages
  constexpr int NR = TA ? NR_MAX : NS;
  constexpr uint32_t B_OFF = b_off(NTP);
  constexpr int ACOL = acc_cols(NTP);  // first A column (A in TMEM)
  constexpr int ACW = acc_w(NTP);      // accumulator columns per slot
  float *run_sm = reinterpret_cast<float *>(stages + (size_t)NR * SB);
  // the swizzled row boxes need 1024-byte aligned stages (no static shared
  // memory here, so the dynamic window starts aligned); refuse otherwise
  if (smem_u32(stages) & 1023u) {
    if (threadIdx.x == 0) atomicExch(A.err, DSE_EINVAL);
    return;
  }
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int nchunks = (A.N + KC - 1) / KC;
  const int nblocks = (nchunks + KB - 1) / KB;
  constexpr int COLS = tmem_cols_needed(NTP);
  constexpr int TMEM_COLS = (COLS <= 32)    ? 32
                            : (COLS <= 64)  ? 64
                            : (COLS <= 128) ? 128
                            : (COLS <= 256) ? 256
                                            : 512;
  static_assert(COLS <= 512, "too many targets for the TMEM accumulators");

  if (threadIdx.x == 0) {
    for (int s = 0; s < NR; ++s) {
      mbar_init(&sh.full_rows[s], 1);
      mbar_init(&sh.empty[s], 1);
    }
    for (int s = 0; s < NS; ++s) {
      mbar_init(&sh.full_a[s], NGEN);
      mbar_init(&sh.empty_a[s], 1);
    }
    for (int b = 0; b < 2; ++b) {
      mbar_init(&sh.acc_full[b], 1);
      mbar_init(&sh.acc_empty[b], 4);
      mbar_init(&sh.gen_done[b], NGEN);
      mbar_init(&sh.epi_free[b], 4);
    }
    mbar_init(&sh.drain, 1);
    sh.abort = 0;
    mbar_fence_init();
  }
  if (warp == 1) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&sh.tmem_base)),
                 "r"((uint32_t)TMEM_COLS)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  fence_before();
  __syncthreads();
  fence_after();
  const uint32_t tmem = sh.tmem_base;

  // Every wait is bounded: on expiry the kernel records DSE_ETIMEOUT, raises
  // the CTA's abort flag and every role leaves its loop.  wait() is for the
  // single-thread roles, wait_warp() for whole warps (warp-uniform result).
  volatile int *abort_flag = &sh.abort;
  auto wait = [&](uint64_t *bar, uint32_t parity) -> bool {
    if (mbar_wait_bounded(bar, parity, kWait)) return true;
    atomicExch(A.err, DSE_ETIMEOUT);
    *abort_flag = 1;
    return false;
  };
  auto wait_warp = [&](uint64_t *bar, uint32_t parity) -> bool {
    const bool ok = __all_sync(0xffffffffu, mbar_wait_bounded(bar, parity, kWait));
    if (!ok && lane == 0) {
      atomicExch(A.err, DSE_ETIMEOUT);
      *abort_flag = 1;
    }
    return ok;
  };
  auto wait_warp_lazy = [&](uint64_t *bar, uint32_t parity) -> bool {
    bool done = false;
    for (uint32_t it = 0; it < kWaitLazy && !done; ++it) {
      done = mbar_try_wait(bar, parity);
      if (!done) __nanosleep(200);
    }
    const bool ok = __all_sync(0xffffffffu, done);
    if (!ok && lane == 0) {
      atomicExch(A.err, DSE_ETIMEOUT);
      *abort_flag = 1;
    }
    return ok;
  };
  auto aborted_warp = [&]() -> bool { return __any_sync(0xffffffffu, *abort_flag != 0); };

  if (warp == 0) {
    // ------------------------------------------------------------ producer
    // lane 0: three 2-D tensor copies of the chunk's operand rows (i-rows
    // 0-7, 8-15, j-rows 0-7 at the tile's row positions; rows past the end
    // and samples past N arrive as zeros), three more of their reciprocal
    // rows for the products and quotients, and one bulk copy of the target
    // block
    int lt = 0;
    uint32_t issued = 0;  // chunks whose copies were issued
    for (int tile = blockIdx.x; tile < A.n_tiles && !aborted_warp(); tile += gridDim.x, ++lt) {
      const Tile tl = A.tiles[tile];
      bool ok = true;
      for (int c = 0; c < nchunks; ++c) {
        const uint32_t gc = (uint32_t)lt * nchunks + c, st = gc % NR, u = gc / NR;
        if (u >= 1 && !wait_warp(&sh.empty[st], (u - 1) & 1)) {
          ok = false;
          break;
        }
        unsigned char *S = stages + (size_t)st * SB;
        if (lane == 0) {
          mbar_arrive_expect_tx(&sh.full_rows[st], (KIND == KIND_MUL ? 6u : 3u) * 1024u + b_bytes(NTP));
          const int x = c * KC;
          tma_load_2d(S, &rows_map, x, tl.ibase, &sh.full_rows[st]);
          tma_load_2d(S + 1024, &rows_map, x, tl.ibase + 8, &sh.full_rows[st]);
          tma_load_2d(S + 2048, &rows_map, x, tl.jbase, &sh.full_rows[st]);
          if (KIND == KIND_MUL) {
            tma_load_2d(S + 3072, &rcp_map, x, tl.ibase, &sh.full_rows[st]);
            tma_load_2d(S + 4096, &rcp_map, x, tl.ibase + 8, &sh.full_rows[st]);
            tma_load_2d(S + 5120, &rcp_map, x, tl.jbase, &sh.full_rows[st]);
          }
          bulk_g2s(S + B_OFF, bsplit + (size_t)c * b_bytes(NTP), b_bytes(NTP), &sh.full_rows[st]);
        }
        __syncwarp();
        issued = gc + 1;
      }
      if (!ok) break;
    }
    // no copy may still be landing when the CTA exits (normally these
    // phases completed long ago and the waits return at once)
    if (lane == 0)
      for (uint32_t st = 0; st < (uint32_t)NR && st < issued; ++st) {
        const uint32_t last = (issued - 1 - st) / NR * NR + st;  // last use of stage st
        mbar_wait_bounded(&sh.full_rows[st], (last / NR) & 1, kWait);
      }
  } else if (warp == 1) {
    // ----------------------------------------------------------------- MMA
    if (lane == 0) {
      constexpr uint32_t IDESC = idesc_bf16(M, NTP);
      int lt = 0;
      for (int tile = blockIdx.x; tile < A.n_tiles && !*abort_flag; tile += gridDim.x, ++lt) {
        for (int b = 0; b < nblocks && !*abort_flag; ++b) {
          const uint32_t gb = (uint32_t)lt * nblocks + b, buf = gb & 1, ub = gb >> 1;
          if (ub >= 1 && !wait(&sh.acc_empty[buf], (ub - 1) & 1)) break;
          fence_after();
          const int c_end = min(nchunks, (b + 1) * KB);
          for (int c = b * KB; c < c_end; ++c) {
            const uint32_t gc = (uint32_t)lt * nchunks + c, st = gc % NR, u = gc / NR;
            const uint32_t sa = gc % NS, ua = gc / NS;
            if (!wait(&sh.full_rows[st], u & 1) || !wait(&sh.full_a[sa], ua & 1)) break;
            fence_after();
            const uint32_t sbase = smem_u32(stages + (size_t)st * SB);
            const uint32_t bh = sbase + B_OFF, bl = bh + (uint32_t)NTP * KC * 2;
            constexpr uint32_t IDESC2 = idesc_bf16(M, 2 * NTP);  // wh against [yh; yl]
#pragma unroll
            for (int k = 0; k < 3; ++k) {
              const uint32_t d = tmem + (buf * 3 + k) * ACW;
              const uint32_t ah = sbase + A_OFF + (2 * k) * A_TILE, al = ah + A_TILE;
              const uint32_t tah = tmem + ACOL + sa * A_STAGE_COLS + k * KC, tal = tah + KC / 2;
#pragma unroll
              for (int kk = 0; kk < KC / 16; ++kk) {
                const uint32_t koff = kk * 2 * LBO;
                const uint32_t acc = (c == b * KB && kk == 0) ? 0u : 1u;
                if (TA) {
                  mma_bf16_ta(d, tah + kk * 8, smem_desc(bh + koff), IDESC2, acc);
                  mma_bf16_ta(d, tal + kk * 8, smem_desc(bh + koff), IDESC, 1u);
                } else {
                  mma_bf16(d, smem_desc(ah + koff), smem_desc(bh + koff), IDESC, acc);
                  mma_bf16(d, smem_desc(ah + koff), smem_desc(bl + koff), IDESC, 1u);
                  mma_bf16(d, smem_desc(al + koff), smem_desc(bh + koff), IDESC, 1u);
                }
              }
            }
            mma_commit(&sh.empty[st]);
            if (TA) mma_commit(&sh.empty_a[sa]);
            if (c == c_end - 1) mma_commit(&sh.acc_full[buf]);
          }
        }
      }
      // every MMA this thread issued has completed before TMEM is freed
      mma_commit(&sh.drain);
      mbar_wait_bounded(&sh.drain, 0, kWait);
    }
  } else if (warp < 2 + NGEN) {
    // ---------------------------------------------------------- generation
    // warp g = warp - 2 writes rows m = 32 (g & 3) + lane (one pair each)
    // for samples [SPP h, SPP h + SPP) of every chunk, h = g >> 2 (all
    // generation warps work on the same chunk, so each waits only for fills
    // whose predecessors it consumed itself)
    const int gw = warp - 2;
    // row = pair; the warp's rows are its TMEM lane quadrant (warp % 4), the
    // lanes its tcgen05 stores may address
    const int m = (warp & 3) * 32 + lane;
    const int part = gw >> 2;            // which SPP samples of a chunk
    static_assert(SPP == 8 || SPP == 16, "one or two eight-sample steps per chunk and thread");
    const GenAddr gad = gen_addr(m >> 3, BI + (m & 7), part * SPP);
    const GenAddr gad2 = gen_addr(m >> 3, BI + (m & 7), part * SPP + (SPP - 8));
    const int ti = m >> 3, tj = m & 7;
    int lt = 0;
    for (int tile = blockIdx.x; tile < A.n_tiles && !aborted_warp(); tile += gridDim.x, ++lt) {
      const Tile tl = A.tiles[tile];
      const int fi = ti < tl.ni ? A.rowid[tl.ibase + ti] : -1;
      const int fj = tj < tl.nj ? A.rowid[tl.jbase + tj] : -1;
      const float4 fa_i = fi >= 0 ? A.F.fa[fi] : make_float4(0.f, 0.f, 0.f, 0.f);
      const float4 fa_j = fj >= 0 ? A.F.fa[fj] : make_float4(0.f, 0.f, 0.f, 0.f);
      const float mi = fa_i.x, mj = fa_j.x;
      TcGen g;
      if (KIND == KIND_MUL) {
        g.c0 = mi * mj;
        g.c1 = mi * fa_j.y;
        g.c2 = mj * fa_i.y;
      } else {
        g.c0 = mi;
        g.c1 = mj;
        g.c2 = fabsf(mi - mj);
      }
      float s1[3] = {0.f, 0.f, 0.f}, s2[3] = {0.f, 0.f, 0.f};
#pragma unroll
      for (int k = 0; k < 3; ++k) g.t1[k] = g.t2[k] = 0.f;
      int blk = 0;
      bool ok = true;
      for (int c = 0; c < nchunks; ++c) {
        const uint32_t gc = (uint32_t)lt * nchunks + c, st = gc % NR, u = gc / NR;
        const uint32_t sa = gc % NS, ua = gc / NS;
        // with A in TMEM: the MMAs that read this A stage before (chunk
        // gc - NS, which these warps generated) have completed
        if (!wait_warp(&sh.full_rows[st], u & 1) || (TA && ua >= 1 && !wait_warp(&sh.empty_a[sa], (ua - 1) & 1))) {
          ok = false;
          break;
        }
        if (TA) fence_after();
        unsigned char *S = stages + (size_t)st * SB;
        unsigned char *Aop = S + A_OFF;
        const uint32_t acol = tmem + ((uint32_t)((warp & 3) * 32) << 16) + ACOL + sa * A_STAGE_COLS;
        if ((c + 1) * KC <= A.N) {
          tc_gen8<KIND, false, TA>(g, S, gad, 0, part * SPP, 0, Aop, acol, m);
          if (SPP == 16) tc_gen8<KIND, false, TA>(g, S, gad2, 8, part * SPP, 0, Aop, acol, m);
        } else {
          const int lim = A.N - c * KC - part * SPP;
          tc_gen8<KIND, true, TA>(g, S, gad, 0, part * SPP, lim, Aop, acol, m);
          if (SPP == 16) tc_gen8<KIND, true, TA>(g, S, gad2, 8, part * SPP, lim, Aop, acol, m);
        }
        if (++blk == gen_blk) {
          blk = 0;
#pragma unroll
          for (int k = 0; k < 3; ++k) {
            s1[k] += g.t1[k];
            s2[k] += g.t2[k];
            g.t1[k] = g.t2[k] = 0.f;
          }
        }
        if (TA) {
          tmem_wait_st();
          fence_before();
        } else {
          fence_proxy_async();
        }
        __syncwarp();
        if (lane == 0) mbar_arrive(&sh.full_a[sa]);
      }
      if (!ok) break;
      // hand this part's S1/S2 of the row to the epilogue warps
      const int p = lt & 1;
      if (lt >= 2 && !wait_warp(&sh.epi_free[p], ((lt >> 1) - 1) & 1)) break;
#pragma unroll
      for (int k = 0; k < 3; ++k) {
        sh.hand[p][part][m][2 * k] = s1[k] + g.t1[k];
        sh.hand[p][part][m][2 * k + 1] = s2[k] + g.t2[k];
      }
      __syncwarp();
      if (lane == 0) mbar_arrive(&sh.gen_done[p]);
    }
  } else {
    // ------------------------------------------------------------ epilogue
    const int q = warp & 3;
    const int m = q * 32 + lane;
    const int ti = m >> 3, tj = m & 7;
    const uint32_t lane_base = (uint32_t)(q * 32) << 16;
    LaneStats ls;
    ls.zero();
    int lt = 0;
    for (int tile = blockIdx.x; tile < A.n_tiles && !aborted_warp(); tile += gridDim.x, ++lt) {
      const Tile tl = A.tiles[tile];
      const int64_t x = ti < tl.ni ? A.rowid[tl.ibase + ti] : -1;
      const int64_t y = tj < tl.nj ? A.rowid[tl.jbase + tj] : -1;
      bool pv = x >= 0 && y >= 0 && (tl.ibase + ti) > (tl.jbase + tj);
      const int64_t ia = x > y ? x : y, ib = x > y ? y : x;
      pv = pv && ia >= A.G.o;
      uint64_t pbase = 0;
      if (pv) pbase = A.G.um + (tri((uint64_t)ia) + (uint64_t)ib - A.G.tri_o) * (uint64_t)A.G.nb;
      const float4 fa_x = x >= 0 ? A.F.fa[x] : make_float4(0.f, 0.f, 0.f, 0.f);
      const float4 fa_y = y >= 0 ? A.F.fa[y] : make_float4(0.f, 0.f, 0.f, 0.f);
      const float4 fa_a = x > y ? fa_x : fa_y, fa_b = x > y ? fa_y : fa_x;
      const float mi = fa_x.x, mj = fa_y.x;  // evaluation order: row i, row j
      float kks[3];
      if (KIND == KIND_MUL) {
        kks[0] = mi * mj;
        kks[1] = mi * fa_y.y;
        kks[2] = mj * fa_x.y;
      } else {
        kks[0] = kks[1] = 0.f;
        kks[2] = fabsf(mi - mj);
      }
      // numerators: one block stays in TMEM until the end; longer sample
      // ranges drain each block into a running FP32 sum kept in TMEM
      // columns [6 NTP, 9 NTP) (added in registers, block by block)
      if (nblocks > 1 && NTP <= 32) {
        for (int b = 0; b < nblocks; ++b) {
          const uint32_t gb = (uint32_t)lt * nblocks + b, buf = gb & 1, ub = gb >> 1;
          if (!wait_warp_lazy(&sh.acc_full[buf], ub & 1)) break;
          fence_after();
#pragma unroll
          for (int k = 0; k < 3; ++k)
#pragma unroll
            for (int c16 = 0; c16 < NTP; c16 += 16) {
              float v[16], r[16];
              tmem_ld16(tmem + lane_base + (buf * 3 + k) * ACW + c16, v);
              if (TA) {
                tmem_ld16(tmem + lane_base + (buf * 3 + k) * ACW + NTP + c16, r);
#pragma unroll
                for (int i = 0; i < 16; ++i) v[i] = v[i] + r[i];
                float *rs = run_sm + m * RUN_W + k * NTP + c16;
#pragma unroll
                for (int i = 0; i < 16; ++i) rs[i] = b > 0 ? rs[i] + v[i] : v[i];
              } else {
                const uint32_t run = tmem + lane_base + (6 + k) * NTP + c16;
                if (b > 0) {
                  tmem_ld16(run, r);
#pragma unroll
                  for (int i = 0; i < 16; ++i) v[i] = r[i] + v[i];
                }
                tmem_st16(run, v);
              }
            }
          fence_before();
          __syncwarp();
          if (lane == 0) mbar_arrive(&sh.acc_empty[buf]);
        }
      }
      const uint32_t gb_last = (uint32_t)lt * nblocks + (nblocks - 1), buf_last = gb_last & 1;
      if (nblocks == 1 && !wait_warp_lazy(&sh.acc_full[buf_last], (gb_last >> 1) & 1)) break;
      if (aborted_warp()) break;
      fence_after();
      const int p = lt & 1;
      if (!wait_warp_lazy(&sh.gen_done[p], (lt >> 1) & 1)) break;
      // this warp's copy of the list thresholds (they only rise, so an older
      // copy is still a valid lower bound)
      for (int t = lane; t < NTP; t += 32) {
        sh.theta[q][t] = t < A.T ? ld_relaxed(&A.B.theta[A.t0 + t]) : 0.f;
        sh.ysum[q][t] = t < A.T ? A.ysum32[A.t0 + t] : 0.f;
      }
      __syncwarp();
      float st12[6];
#pragma unroll
      for (int i = 0; i < 6; ++i) {
        float v = sh.hand[p][0][m][i];
#pragma unroll
        for (int h = 1; h < NPART; ++h) v += sh.hand[p][h][m][i];
        st12[i] = v;
      }
      __syncwarp();
      if (lane == 0) mbar_arrive(&sh.epi_free[p]);
      uint64_t pushed = 0;
#pragma unroll
      for (int k = 0; k < 3; ++k) {
        const int opc = KIND == KIND_MUL ? (k == 0 ? DSE_OP_MUL : k == 1 ? DSE_OP_DIV : DSE_OP_RDIV)
                                         : (k == 0 ? DSE_OP_ADD : k == 1 ? DSE_OP_SUB : DSE_OP_ABSDIFF);
        const TcCand tcc = tc_prepare(A, ls, pv, ia, ib, opc, pbase, fa_a, fa_b, kks[k], mi, mj, st12[2 * k],
                                      st12[2 * k + 1], gamma_gen, gamma_num);
#pragma unroll(NTP <= 32 ? 2 : 1)
        for (int c16 = 0; c16 < NTP; c16 += 16) {
          float v[16];
          if (nblocks == 1) {
            tmem_ld16(tmem + lane_base + (buf_last * 3 + k) * ACW + c16, v);  // whole warp
            if (TA) {
              float r[16];
              tmem_ld16(tmem + lane_base + (buf_last * 3 + k) * ACW + NTP + c16, r);
#pragma unroll
              for (int i = 0; i < 16; ++i) v[i] = v[i] + r[i];
            }
          } else if (TA) {
#pragma unroll
            for (int i = 0; i < 16; ++i) v[i] = run_sm[m * RUN_W + k * NTP + c16 + i];
          } else {
            tmem_ld16(tmem + lane_base + (6 + k) * NTP + c16, v);
          }
          if (tcc.ok) pushed |= tc_targets16(A, tcc, v, c16, gamma_gen, gamma_num, sh.ysum[q], sh.theta[q], sh.sy[q]);
        }
      }
      if (nblocks == 1) {
        fence_before();
        __syncwarp();
        if (lane == 0) mbar_arrive(&sh.acc_empty[buf_last]);
      }
      // raise the thresholds of the lists this warp pushed to
      unsigned lo = (unsigned)pushed, hi = (unsigned)(pushed >> 32);
      lo = __reduce_or_sync(0xffffffffu, lo);
      hi = __reduce_or_sync(0xffffffffu, hi);
      const uint64_t all = (uint64_t)lo | ((uint64_t)hi << 32);
      for (int t = 0; t < NTP && t < 64; ++t)
        if (all & (1ull << t)) refresh_theta(A.B, A.t0 + t, A.k);
    }
    flush_stats(A, ls);
  }
  fence_before();
  __syncthreads();
  fence_after();
  __syncwarp();
  if (warp == 1)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"((uint32_t)TMEM_COLS)
                 : "memory");
}

// --------------------------------------------------------------- launcher

// Tensor map of the FP32 operand rows [nrows][ld] (N valid samples per row)
// for the kernel's 2-D copies: boxes of 32 samples x 8 rows, 128-byte
// swizzle, zero fill outside.  cuTensorMapEncodeTiled comes from the driver
// through the runtime's entry-point query (the library links the runtime
// only).
typedef CUresult (*EncodeTiledFn)(CUtensorMap *, CUtensorMapDataType, cuuint32_t, void *, const cuuint64_t *,
                                  const cuuint64_t *, const cuuint32_t *, const cuuint32_t *, CUtensorMapInterleave,
                                  CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

static dse_status rows_tensor_map(const float *base, int64_t nrows, int64_t N, int64_t ld, CUtensorMap *out) {
  static EncodeTiledFn encode = nullptr;
  if (!encode) {
    void *fn = nullptr;
    cudaDriverEntryPointQueryResult q = cudaDriverEntryPointSymbolNotFound;
    cudaError_t e = cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault, &q);
    if (e != cudaSuccess || q != cudaDriverEntryPointSuccess || !fn) {
      cudaGetLastError();
      set_error("cuTensorMapEncodeTiled is not available from the driver");
      return DSE_ECUDA;
    }
    encode = reinterpret_cast<EncodeTiledFn>(fn);
  }
  const cuuint64_t dims[2] = {(cuuint64_t)N, (cuuint64_t)(nrows > 0 ? nrows : 1)};
  const cuuint64_t strides[1] = {(cuuint64_t)ld * sizeof(float)};
  const cuuint32_t box[2] = {(cuuint32_t)tc::KC, 8u};
  const cuuint32_t elem[2] = {1u, 1u};
  const CUresult r = encode(out, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, const_cast<float *>(base), dims, strides, box,
                            elem, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
                            CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  if (r != CUDA_SUCCESS) {
    set_error("cuTensorMapEncodeTiled failed (%d)", (int)r);
    return DSE_ECUDA;
  }
  return DSE_OK;
}

template <int KIND, int NTP>
static dse_status launch_tc_t(const ScreenArgs &A, const unsigned char *bsplit, const CUtensorMap &map,
                              const CUtensorMap &rmap, float gamma_gen, float gamma_num, int gen_blk, int sms,
                              cudaStream_t st) {
  const size_t smem = tc::shared_bytes() + (size_t)(tc::tmem_a(NTP) ? tc::NR_MAX : tc::NS) * tc::stage_bytes(NTP) +
                      tc::run_bytes(NTP);
  static bool attr[64] = {false};
  int dev = 0;
  cudaGetDevice(&dev);
  if (!attr[dev & 63]) {
    DSE_CUDA(cudaFuncSetAttribute(k_pair_tc<KIND, NTP>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    attr[dev & 63] = true;
  }
  int grid = sms < A.n_tiles ? sms : A.n_tiles;
  if (grid < 1) return DSE_OK;
  note_launches(1);
  ScreenArgs B = A;
  B.group = KIND == KIND_MUL ? 1 : 2;
  k_pair_tc<KIND, NTP><<<grid, tc::THREADS, smem, st>>>(B, bsplit, map, rmap, gamma_gen, gamma_num, gen_blk);
  return DSE_OK;
}

// Reciprocal rows of the stored FP32 rows (the rcp.approx the error model
// assumes), read by the product/quotient kernel next to the rows.
__global__ void k_rcp_rows(const float *v32, int64_t count, float *out) {
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < count; e += (int64_t)gridDim.x * blockDim.x)
    out[e] = rcp_approx(v32[e]);
}

void launch_rcp_rows(const float *v32, int64_t count, float *out, int sms, cudaStream_t st) {
  int64_t blocks = (count + 255) / 256;
  if (blocks > (int64_t)sms * 16) blocks = (int64_t)sms * 16;
  if (blocks < 1) return;
  note_launches(1);
  k_rcp_rows<<<(unsigned)blocks, 256, 0, st>>>(v32, count, out);
}

// Rows in the order of a row list (the unit-class order of the additive
// tiles): out[p] = v32[rows[p]], so that a tile's rows are consecutive for
// the 2-D copies.
__global__ void k_gather_rows(const float *v32, int64_t ld, const int32_t *rows, int64_t n, float *out) {
  const int64_t total = n * ld;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x)
    out[e] = v32[(int64_t)rows[e / ld] * ld + e % ld];
}

void launch_gather_rows(const float *v32, int64_t ld, const int32_t *rows, int64_t n, float *out, int sms,
                        cudaStream_t st) {
  int64_t blocks = (n * ld + 255) / 256;
  if (blocks > (int64_t)sms * 16) blocks = (int64_t)sms * 16;
  if (blocks < 1) return;
  note_launches(1);
  k_gather_rows<<<(unsigned)blocks, 256, 0, st>>>(v32, ld, rows, n, out);
}

// Samples of each chunk one generation thread sums (the blocked FP32 sums
// inner length per chunk) and the number of partial sums per row.
int tc_gen_samples() { return tc::SPP; }
int tc_gen_parts() { return tc::NPART; }

int tc_ntp_for(int T, int N) {
  // one accumulation block keeps every target in TMEM; longer sample ranges
  // drain blocks into registers, which bounds the targets per pass at 32
  const int nchunks = (N + tc::KC - 1) / tc::KC;
  const int cap = nchunks > tc::KB ? 32 : 64;
  int t = T < cap ? T : cap;
  return t <= 16 ? 16 : t <= 32 ? 32 : t <= 48 ? 48 : 64;
}

size_t tc_bsplit_bytes(int ntp, int N) {
  const int nchunks = (N + tc::KC - 1) / tc::KC;
  return (size_t)nchunks * tc::b_bytes(ntp);
}

void launch_tc_targets(const float *y32, int32_t ldy, int t0, int T, int N, int ntp, unsigned char *out,
                       cudaStream_t st) {
  const int nchunks = (N + tc::KC - 1) / tc::KC;
  const int64_t total = (int64_t)nchunks * ntp * tc::KC;
  int64_t blocks = (total + 255) / 256;
  if (blocks > 4096) blocks = 4096;
  note_launches(1);
  k_tc_targets<<<(unsigned)blocks, 256, 0, st>>>(y32, ldy, t0, T, N, ntp, nchunks, out);
}

dse_status launch_pair_tc(int kind, int ntp, const ScreenArgs &A, const unsigned char *bsplit, const float *rows,
                          const float *rcp_rows, int64_t nrows, float gamma_gen, float gamma_num, int gen_blk, int sms,
                          cudaStream_t st) {
  if (A.n_tiles <= 0) return DSE_OK;
  if (kind == KIND_MUL && !rcp_rows) {
    set_error("reciprocal rows missing");
    return DSE_EINVAL;
  }
  CUtensorMap map, rmap;
  DSE_TRY(rows_tensor_map(rows, nrows, A.N, A.F.ld, &map));
  DSE_TRY(rows_tensor_map(kind == KIND_MUL ? rcp_rows : rows, nrows, A.N, A.F.ld, &rmap));
  if (ntp > 32 && (A.N + tc::KC - 1) / tc::KC > tc::KB) {
    set_error("target block %d needs N <= %d samples", ntp, tc::KB * tc::KC);
    return DSE_EINVAL;
  }
#define DSE_TC_CASE(NTPV)                                                                                   \
  case NTPV:                                                                                                \
    return kind == KIND_MUL                                                                                  \
               ? launch_tc_t<KIND_MUL, NTPV>(A, bsplit, map, rmap, gamma_gen, gamma_num, gen_blk, sms, st)         \
               : launch_tc_t<KIND_ADD, NTPV>(A, bsplit, map, rmap, gamma_gen, gamma_num, gen_blk, sms, st);
  switch (ntp) {
    DSE_TC_CASE(16)
    DSE_TC_CASE(32)
    DSE_TC_CASE(48)
    DSE_TC_CASE(64)
    default:
      set_error("unsupported target block %d", ntp);
      return DSE_EINVAL;
  }
#undef DSE_TC_CASE
}

}  // namespace dse
