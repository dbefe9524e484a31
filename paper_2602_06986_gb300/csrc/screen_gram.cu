// screen_gram.cu -- the product and quotient slots of rung k from Gram
// matrices on the 5th-generation tensor cores (single-target FP32 screens).
//
// The SIS statistics of a product are bilinear in the operands' rows, so
// they need no per-sample evaluation of the candidate: for a pair (i, j),
// i > j, each slot a*b, a/b, b/a is v = u w with u one of x_i, 1/x_i and w
// one of x_j, 1/x_j.  With u = c_u + p and w = c_w + q (c = the feature's
// FP32 mean, of x or of 1/x; p, q the centred FP32 rows), the statistics of
// v shifted by k = c_u c_w are exactly
//   S1 = sum (v - k)     = c_u Q1 + c_w P1 + G11
//   S2 = sum (v - k)^2   = c_u^2 Q2 + c_w^2 P2 + G22 + 2 c_u c_w G11 + 2 c_u G12 + 2 c_w G21
//   Sy = sum (v - k) y   = c_u QY + c_w PY + H
// with per-feature sums P1 = sum p, P2 = sum p^2, PY = sum p y (Q* of w)
// and five contractions G11 = sum p q, G22 = sum p^2 q^2, G12 = sum p q^2,
// G21 = sum p^2 q, H = sum (p y) q.  One contraction of six rows per "a"
// feature ([p, p^2, p y] of x and of 1/x) against four rows per "b" feature
// ([q, q^2] of x and of 1/x) gives all three slots of every pair of a tile:
// 20 a-features (128 rows, two per 32-row group unused) x 64 b-features
// (256 columns).  The contraction runs on tcgen05 in BF16x3 with FP32
// accumulation in tensor memory; the rest (a-priori tests, intervals,
// realised test, threshold pushes) is the FP32 path's epilogue on the
// statistics above.  This is a reformulation of the evaluation by the
// algebra of the statistics; the paper evaluates candidates directly.
//
// Error bounds (the reported eps contains the FP64 score of the exact
// candidate, as on the direct path):
//   * each contraction entry: |G~ - G| <= delta |a|_2 |b|_2 with delta the
//     BF16x3 split (3.01 * 2^-16), the tensor-core accumulation model of the
//     multi-target kernel (2u per accumulation step, safety factor 4) and
//     one rounding of each squared or target-weighted row;
//   * the FP32 assembly of S1, S2, Sy: a few roundings of the sum of the
//     absolute terms;
//   * the evaluation error of the candidate represented by the FP32 rows
//     ((c + p) reproduces x32 to u (|x| + |c|), x32 is x to u, 1/x32 is
//     1/x to 2u): per sample u (kappa |u w| + |u| |c_w| + |w| |c_u|) with
//     kappa 4.01 for a*b and 5.01 for the quotients, as the vector bound
//     E = u (kappa |V| + |c_w| |U| + |c_u| |W|).
// Candidates whose realised test the bounds cannot decide, or whose
// operands leave the FP32-safe range, go to the FP64 escalation.
//
// Warp roles (one CTA per SM, persistent over a static tile stride):
//   warp 0      producer: two 1-D bulk copies per stage (the a- and
//               b-images of a 32-sample chunk, each already in the canonical
//               K-major core-matrix layout), 5-stage ring;
//   warp 1      TMEM allocation (256 columns: two 128-column accumulators)
//               and the MMA issuer: 2 k-steps x 3 products per chunk;
//   warps 2-9   epilogue: warp w reads the TMEM lanes of quadrant w % 4,
//               which hold its five a-features' rows, 32 columns at a time
//               (every other patch: two warps per quadrant) through a private
//               shared-memory patch, and scores the 120 candidates (5 a x 8 b
//               x 3 slots) of each patch from a private copy of the 21
//               features' records (loaded while the tile's MMAs run); the
//               passing candidates are staged per warp and written out with
//               one slot reservation per flush, and the warps' statistics
//               meet in shared memory before one set of global atomics.
#include <cuda_bf16.h>
#include <math.h>

#include <algorithm>
#include <vector>

#include "dse_internal.cuh"
#include "eval64.cuh"
#include "screen_common.cuh"
#include "gram.cuh"
#include "screen_kernels.cuh"
#include "tcgen05.cuh"
#include "util.cuh"

namespace dse {

namespace gram {

constexpr int FA = 20;  // a-features per tile
constexpr int FB = 32;  // b-features per tile (about 2.6 tiles per CTA on medium, so
                        // that a tile's MMAs run under the previous tile's epilogue)
constexpr int FW = 5;   // a-features per epilogue warp (6 rows each)
constexpr int M = 128, NCOL = 4 * FB;
constexpr int TMEM_COLS = 2 * NCOL;  // two accumulator buffers (a power of two >= 32)
constexpr int NS = 5;  // stages: the ring is bound by the copies' latency (about 2k cycles)
constexpr uint32_t A_HALF = M * tc::KC * 2;     // hi or lo part of an a-image chunk
constexpr uint32_t B_HALF = NCOL * tc::KC * 2;  // hi or lo part of a b-image chunk
constexpr uint32_t A_IMG = 2 * A_HALF, B_IMG = 2 * B_HALF;
constexpr uint32_t STAGE = A_IMG + B_IMG;
constexpr int EPI = 8;  // epilogue warps: two per TMEM lane quadrant
constexpr int THREADS = (2 + EPI) * 32;
constexpr uint32_t kWait = 1u << 22;
constexpr int EC = 32;  // TMEM columns per epilogue patch (8 b-features)
constexpr int PATCHES = NCOL / EC;
constexpr int PW = PATCHES / 2;  // patches per epilogue warp (two warps per quadrant)

// Row of a-feature f (0..19), type t (0..5: p, p^2, p y of x, then of 1/x):
// epilogue warp f / 5 owns TMEM lanes 32 (f / 5) .. + 31.
__host__ __device__ inline int arow(int f, int t) { return 32 * (f / FW) + 6 * (f % FW) + t; }
// Column of b-feature g (0..63), type t (0..3: q, q^2 of x, then of 1/x).
__host__ __device__ inline int bcol(int g, int t) { return 4 * g + t; }

constexpr int NCACHE = FW + 8 * PW;

struct Shared {
  uint64_t full[NS], empty[NS];
  uint64_t acc_full[2], acc_empty[2];
  uint64_t drain;
  uint32_t tmem_base;
  int abort;
  float E[EPI][32][EC + 1];        // each epilogue warp's patch: its 32 lanes x 32 columns
  EpiFeat cache[EPI][NCACHE];      // each epilogue warp's feature records
  PushStage<64> stage[EPI];        // each epilogue warp's pending pushes
  unsigned st[10];                 // the epilogue warps' statistics, summed per CTA
};

constexpr size_t shared_bytes() { return (sizeof(Shared) + 1023) / 1024 * 1024; }
constexpr size_t smem_total() { return shared_bytes() + (size_t)NS * STAGE; }
static_assert(smem_total() <= 227 * 1024, "shared memory of one CTA");

}  // namespace gram


// Space part, one block per stored feature f: the b-image rows (q, q^2 of x
// and of 1/x) and the sums of GramFeat.  Images are zero-initialised by the
// caller (unused rows, samples past N).
__global__ void __launch_bounds__(128) k_gram_space(FeatTable F, int nchunks, unsigned char *bimg, GramFeat *gf) {
  __shared__ double sm[4 * 10];
  const int64_t f = blockIdx.x;
  if (f >= F.n) return;
  const uint32_t fl = F.flags[f];
  const float4 fa = F.fa[f];
  const bool okx = (fl & F_FP32_SAFE) != 0;
  const bool okr = okx && (fl & F_MINABS_POS) != 0;
  const float c[2] = {fa.x, fa.y};
  const bool ok[2] = {okx, okr};
  const int64_t gb = f / gram::FB;
  const int g = (int)(f % gram::FB);
  GramFeatAcc acc;
  const int64_t groups = (int64_t)nchunks * (tc::KC / 8);
  for (int64_t gi = threadIdx.x; gi < groups; gi += blockDim.x) {
    const int64_t s0 = gi * 8;
    const int ch = (int)(s0 / tc::KC), k0 = (int)(s0 % tc::KC);
    unsigned char *base = bimg + ((size_t)gb * nchunks + ch) * gram::B_IMG;
#pragma unroll
    for (int fam = 0; fam < 2; ++fam) {
      float p[8], p2[8];
      gram_vals(F, f, s0, fam, c[fam], ok[fam], p);
#pragma unroll
      for (int e = 0; e < 8; ++e) p2[e] = p[e] * p[e];
      acc.add(fam, p, p2, ok[fam], c[fam], s0, F.N);
      uint4 h, l;
      split8(p, h, l);
      const uint32_t o1 = tc::core_off(gram::bcol(g, 2 * fam), k0);
      *reinterpret_cast<uint4 *>(base + o1) = h;
      *reinterpret_cast<uint4 *>(base + gram::B_HALF + o1) = l;
      split8(p2, h, l);
      const uint32_t o2 = tc::core_off(gram::bcol(g, 2 * fam + 1), k0);
      *reinterpret_cast<uint4 *>(base + o2) = h;
      *reinterpret_cast<uint4 *>(base + gram::B_HALF + o2) = l;
    }
  }
  acc.finish(sm, groups, c, ok, gf + f);
}

// Per screen, one block per stored feature f: the a-image rows (p, p^2,
// p y of x and of 1/x, y the FP32 target) and the target sums.
__global__ void __launch_bounds__(128) k_gram_arows(FeatTable F, int nchunks, const float *y32, const GramFeat *gf,
                                                    unsigned char *aimg, GramTgt *gt) {
  __shared__ double sm[4 * 4];
  const int64_t f = blockIdx.x;
  if (f >= F.n) return;
  const GramFeat G = gf[f];
  const int64_t ab = f / gram::FA;
  const int fa = (int)(f % gram::FA);
  // per family: sum p y (compensated) and sum (p y)^2 (plain FP32, a norm)
  Comp32 csy[2];
  float sq[2] = {0.f, 0.f};
  const int64_t groups = (int64_t)nchunks * (tc::KC / 8);
  for (int64_t gi = threadIdx.x; gi < groups; gi += blockDim.x) {
    const int64_t s0 = gi * 8;
    const int ch = (int)(s0 / tc::KC), k0 = (int)(s0 % tc::KC);
    unsigned char *base = aimg + ((size_t)ab * nchunks + ch) * gram::A_IMG;
    float y[8];
#pragma unroll
    for (int e = 0; e < 8; ++e) y[e] = s0 + e < F.N ? y32[s0 + e] : 0.f;
#pragma unroll
    for (int fam = 0; fam < 2; ++fam) {
      float p[8], p2[8], py[8];
      gram_vals(F, f, s0, fam, G.c[fam], G.ok[fam] != 0, p);
#pragma unroll
      for (int e = 0; e < 8; ++e) {
        p2[e] = p[e] * p[e];
        py[e] = p[e] * y[e];
        csy[fam].add(py[e]);
        sq[fam] = fmaf(py[e], py[e], sq[fam]);
      }
      uint4 h, l;
      const float *rows[3] = {p, p2, py};
#pragma unroll
      for (int t = 0; t < 3; ++t) {
        float r8[8];
#pragma unroll
        for (int e = 0; e < 8; ++e) r8[e] = rows[t][e];
        split8(r8, h, l);
        const uint32_t o = tc::core_off(gram::arow(fa, 3 * fam + t), k0);
        *reinterpret_cast<uint4 *>(base + o) = h;
        *reinterpret_cast<uint4 *>(base + gram::A_HALF + o) = l;
      }
    }
  }
  double acc[4] = {csy[0].value(), (double)sq[0], csy[1].value(), (double)sq[1]};
  gram_block_sum<4>(acc, sm);
  if (threadIdx.x == 0) {
    GramTgt o;
    for (int fam = 0; fam < 2; ++fam) {
      const double marg = 1.0 + ((double)groups * 8.0 / blockDim.x + 10.0) * 5.9604644775390625e-8;
      o.sy[fam] = (float)acc[2 * fam];
      o.ny[fam] = __double2float_ru(sqrt(acc[2 * fam + 1] * marg) * (1.0 + 1e-15));
    }
    gt[f] = o;
  }
}


// ------------------------------------------------------------------ kernel

struct GramArgs {
  const unsigned char *aimg, *bimg;
  const GramFeat *gf;
  const GramTgt *gt;
  const int2 *tiles;  // (a-block, b-block)
  int n_tiles;
  int nchunks;
  float delta;
  int na, nb;  // a-blocks and b-blocks of the images
};

__global__ void __launch_bounds__(gram::THREADS, 1) k_pair_gram(const ScreenArgs A, const GramArgs GA) {
  using namespace gram;
  using namespace tc;
  extern __shared__ __align__(1024) unsigned char smem[];
  Shared &sh = *reinterpret_cast<Shared *>(smem);
  unsigned char *stages = smem + shared_bytes();
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int nchunks = GA.nchunks;

  if (threadIdx.x == 0) {
    for (int s = 0; s < NS; ++s) {
      mbar_init(&sh.full[s], 1);
      mbar_init(&sh.empty[s], 1);
    }
    for (int b = 0; b < 2; ++b) {
      mbar_init(&sh.acc_full[b], 1);
      mbar_init(&sh.acc_empty[b], EPI);
    }
    mbar_init(&sh.drain, 1);
    sh.abort = 0;
    for (int k = 0; k < 10; ++k) sh.st[k] = 0;
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
  auto aborted_warp = [&]() -> bool { return __any_sync(0xffffffffu, *abort_flag != 0); };

  if (warp == 0) {
    // ------------------------------------------------------------ producer
    if (lane == 0) {
      int lt = 0;
      uint32_t issued = 0;
      for (int tile = blockIdx.x; tile < GA.n_tiles && !*abort_flag; tile += gridDim.x, ++lt) {
        int2 tl = GA.tiles[tile];
        if (!(DSE_IN_BOUNDS(tl.x, GA.na, A.err) && DSE_IN_BOUNDS(tl.y, GA.nb, A.err))) tl = make_int2(0, 0);
        bool ok = true;
        for (int c = 0; c < nchunks; ++c) {
          const uint32_t gc = (uint32_t)lt * nchunks + c, st = gc % NS, u = gc / NS;
          if (u >= 1 && !wait(&sh.empty[st], (u - 1) & 1)) {
            ok = false;
            break;
          }
          unsigned char *S = stages + (size_t)st * STAGE;
          mbar_arrive_expect_tx(&sh.full[st], STAGE);
          bulk_g2s(S, GA.aimg + ((size_t)tl.x * nchunks + c) * A_IMG, A_IMG, &sh.full[st]);
          bulk_g2s(S + A_IMG, GA.bimg + ((size_t)tl.y * nchunks + c) * B_IMG, B_IMG, &sh.full[st]);
          issued = gc + 1;
        }
        if (!ok) break;
      }
      // no copy may still be landing when the CTA exits
      for (uint32_t st = 0; st < (uint32_t)NS && st < issued; ++st) {
        const uint32_t last = (issued - 1 - st) / NS * NS + st;
        mbar_wait_bounded(&sh.full[st], (last / NS) & 1, kWait);
      }
    }
  } else if (warp == 1) {
    // ----------------------------------------------------------------- MMA
    if (lane == 0) {
      constexpr uint32_t IDESC = idesc_bf16(M, NCOL);
      int lt = 0;
      for (int tile = blockIdx.x; tile < GA.n_tiles && !*abort_flag; tile += gridDim.x, ++lt) {
        const uint32_t buf = lt & 1, ub = lt >> 1;
        if (ub >= 1 && !wait(&sh.acc_empty[buf], (ub - 1) & 1)) break;
        fence_after();
        const uint32_t d = tmem + buf * NCOL;
        bool ok = true;
        for (int c = 0; c < nchunks; ++c) {
          const uint32_t gc = (uint32_t)lt * nchunks + c, st = gc % NS, u = gc / NS;
          if (!wait(&sh.full[st], u & 1)) {
            ok = false;
            break;
          }
          fence_after();
          const uint32_t ah = smem_u32(stages + (size_t)st * STAGE), al = ah + A_HALF;
          const uint32_t bh = ah + A_IMG, bl = bh + B_HALF;
#pragma unroll
          for (int kk = 0; kk < KC / 16; ++kk) {
            const uint32_t koff = kk * 2 * LBO;
            const uint32_t acc = (c == 0 && kk == 0) ? 0u : 1u;
            mma_bf16(d, smem_desc(ah + koff), smem_desc(bh + koff), IDESC, acc);
            mma_bf16(d, smem_desc(ah + koff), smem_desc(bl + koff), IDESC, 1u);
            mma_bf16(d, smem_desc(al + koff), smem_desc(bh + koff), IDESC, 1u);
          }
          mma_commit(&sh.empty[st]);
          if (c == nchunks - 1) mma_commit(&sh.acc_full[buf]);
        }
        if (!ok) break;
      }
      // every MMA issued has completed before TMEM is freed
      mma_commit(&sh.drain);
      mbar_wait_bounded(&sh.drain, 0, kWait);
    }
  } else {
    // ------------------------------------------------------------ epilogue
    const int ew = warp - 2;         // 0 .. EPI-1
    const int q = warp & 3;          // TMEM lane quadrant = a-features 5q .. 5q+4
    const int h = ew >> 2;           // patches h, h + 2, ...
    const uint32_t lane_base = (uint32_t)(q * 32) << 16;
    float(*E)[EC + 1] = sh.E[ew];
    EpiFeat *cache = sh.cache[ew];
    PushStage<64> &stg = sh.stage[ew];
    LaneStats ls;
    ls.zero();
    const float N = (float)A.N, invN = (float)A.invN;
    const float fmin = (float)A.fmin_std_rel64;
    const float ysum = A.ysum32[A.t0];
    const int64_t n = A.F.n, o = A.G.o;
    int lt = 0;
    for (int tile = blockIdx.x; tile < GA.n_tiles && !aborted_warp(); tile += gridDim.x, ++lt) {
      const int2 tl = GA.tiles[tile];
      // this warp's feature records: a-features 0..4, then the b-features of
      // its patches (8 each), while the tile's MMAs run
      for (int e = lane; e < NCACHE; e += 32) {
        int64_t f;
        if (e < FW) {
          f = (int64_t)tl.x * FA + q * FW + e;
        } else {
          const int k = e - FW;
          f = (int64_t)tl.y * FB + (2 * (k >> 3) + h) * (EC / 4) + (k & 7);
        }
        if (f < n) {
          EpiFeat c;
          c.fa = A.F.fa[f];
          c.fr = A.F.fr[f];
          c.flags = A.F.flags[f];
          c.cplx = A.F.cplx[f];
          c.uk[0] = A.F.ukey[2 * f];
          c.uk[1] = A.F.ukey[2 * f + 1];
          const GramFeat g = GA.gf[f];
          const GramTgt t = GA.gt[f];
#pragma unroll
          for (int m = 0; m < 2; ++m) {
            c.c[m] = g.c[m];
            c.s1[m] = g.s1[m];
            c.s2[m] = g.s2[m];
            c.n1[m] = g.n1[m];
            c.n2[m] = g.n2[m];
            c.nu[m] = g.nu[m];
            c.sy[m] = t.sy[m];
            c.ny[m] = t.ny[m];
          }
          cache[e] = c;
        }
      }
      __syncwarp();
      const uint32_t buf = lt & 1, ub = lt >> 1;
      if (!wait_warp(&sh.acc_full[buf], ub & 1)) break;
      fence_after();
      // pushes are staged per warp and written out once per tile (or when
      // the stage fills); the threshold is read afresh for every batch (it
      // rises while other warps finish their tiles)
      int staged = 0, pushed = 0;
      for (int pcl = 0; pcl < PW; ++pcl) {
        const int pc = 2 * pcl + h;
        float v[EC];
        tmem_ld32(tmem + lane_base + buf * NCOL + pc * EC, v);
#pragma unroll
        for (int e = 0; e < EC; ++e) E[lane][e] = v[e];
        __syncwarp();
        // 5 a-features x 8 b-features x 3 slots = 120 products and
        // quotients (iterations 0-3), then 5 x 8 x 2 = 80 sums and
        // differences (iterations 4-6, when this kernel takes them)
        const int iters = A.gram_addsub ? 7 : 4;
        for (int it = 0; it < iters; ++it) {
          const float th = ld_relaxed(&A.B.theta[A.t0]);  // issued first: its latency hides behind the scoring
          const bool add = it >= 4;
          int idx, fi, gj, opc;
          if (!add) {
            idx = it * 32 + lane;
            const int rem = idx % 24, slot = rem % 3;
            fi = idx / 24;
            gj = rem / 3;
            opc = slot == 0 ? DSE_OP_MUL : slot == 1 ? DSE_OP_DIV : DSE_OP_RDIV;
          } else {
            idx = (it - 4) * 32 + lane;
            fi = idx >> 4;
            gj = (idx >> 1) & 7;
            opc = (idx & 1) ? DSE_OP_SUB : DSE_OP_ADD;
          }
          const int64_t i = (int64_t)tl.x * FA + q * FW + fi;
          const int64_t j = (int64_t)tl.y * FB + pc * (EC / 4) + gj;
          bool want = false;
          uint64_t gid = 0;
          float s = 0.f, eps = 0.f;
          const bool pair = idx < (add ? 80 : 120) && i < n && i >= o && j < i;
          const int pos = A.slot_pos[opc - 6];
          if (pair && pos >= 0) {
            const uint64_t pbase = A.G.um + (tri((uint64_t)i) + (uint64_t)j - A.G.tri_o) * (uint64_t)A.G.nb;
            gid = (uint64_t)A.n_stored + pbase + (uint64_t)pos;
            if (gid >= A.id_begin && gid < A.id_end) {
              const EpiFeat &ca = cache[fi], &cb = cache[FW + pcl * 8 + gj];
              const int reason = add ? gram_apriori_add(A, opc, i, j, ca, cb) : gram_apriori(A, opc, i, j, ca, cb);
              if (add) ls.seen++;
              if (reason != DSE_VALID) {
                ls.r[reason]++;
                note_why(A, gid, reason);
              } else if (!((ca.flags & cb.flags) & F_FP32_SAFE)) {
                escalate(A, gid);
                ls.escalated++;
              } else {
                GramCand gc;
                if (add) {
                  gc = gram_score_add(&ca, &cb, opc == DSE_OP_ADD ? 1.f : -1.f, E[6 * fi][4 * gj],
                                      E[6 * fi + 1][4 * gj + 1], GA.delta, N, invN, ysum, fmin);
                } else {
                  const int fu = opc == DSE_OP_RDIV ? 1 : 0, fw = opc == DSE_OP_DIV ? 1 : 0;
                  const int ra = 6 * fi + 3 * fu, cl = 4 * gj + 2 * fw;
                  gc = gram_score(&ca, fu, &cb, fw, E[ra][cl], E[ra + 1][cl + 1], E[ra][cl + 1], E[ra + 1][cl],
                                  E[ra + 2][cl], opc == DSE_OP_MUL ? 4.01f : 5.01f, GA.delta, N, invN, ysum, fmin);
                }
                if (gc.realised == 0) {
                  ls.r[DSE_R_REALISED]++;
                  note_why(A, gid, DSE_R_REALISED);
                } else if (gc.realised == 2) {
                  escalate(A, gid);
                  ls.escalated++;
                } else {
                  ls.r[DSE_VALID]++;
                  ls.evaluated++;
                  note_why(A, gid, DSE_VALID);
                  want = true;
                  s = gc.s;
                  eps = gc.eps * (1.0f + 2.4e-7f);
                  note_ivl(A, gid, A.t0, s, eps);
                }
              }
            }
          }
          staged = stage_push(A.B, A.t0, stg, staged, &pushed, th, want, gid, s, eps);
        }
        __syncwarp();
      }
      fence_before();
      __syncwarp();
      if (lane == 0) mbar_arrive(&sh.acc_empty[buf]);
      stage_flush(A.B, A.t0, stg, staged);
      if (pushed > 0) refresh_theta(A.B, A.t0, A.k);
    }
    // statistics: the warps' counters meet in shared memory, then one set of
    // global atomics per CTA (thousands of warps adding to the same few
    // counters at once would queue at the L2)
    {
      const unsigned v[10] = {ls.seen, ls.r[0], ls.r[1], ls.r[2], ls.r[3], ls.r[4], ls.r[5], ls.r[DSE_VALID],
                              ls.evaluated, ls.escalated};
#pragma unroll
      for (int k = 0; k < 10; ++k) {
        unsigned t = v[k];
        for (int off = 16; off > 0; off >>= 1) t += __shfl_xor_sync(0xffffffffu, t, off);
        if (lane == 0 && t) atomicAdd(&sh.st[k], t);
      }
      asm volatile("bar.sync 1, %0;" ::"r"(EPI * 32) : "memory");
      if (ew == 0 && lane < 10 && A.first_pass) {
        const unsigned t = sh.st[lane];
        const int dst = lane == 0   ? ST_ADD_SEEN
                        : lane < 7  ? ST_REASON0 + (lane - 1)
                        : lane == 7 ? ST_VALID_G0 + 1
                        : lane == 8 ? ST_EVALUATED
                                    : ST_ESCALATED;
        if (t) atomicAdd(&A.stats[dst], (unsigned long long)t);
      }
    }
  }
  fence_before();
  __syncthreads();
  fence_after();
  if (warp == 1)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"((uint32_t)TMEM_COLS) : "memory");
}

// ------------------------------------------------------------------- host

// Whether a screen may take the Gram path: FP32, one target, N up to 2048
// samples (the accumulation bound grows with the chunks per accumulator).
bool gram_eligible(int64_t N) { return N >= 16 && N <= tuning().gram_max_n; }

size_t gram_space_bytes(int64_t n, int64_t N) {
  const int64_t nchunks = (N + tc::KC - 1) / tc::KC;
  const int64_t nb = (n + gram::FB - 1) / gram::FB;
  return (size_t)nb * nchunks * gram::B_IMG + (size_t)n * sizeof(GramFeat) + 256;
}

size_t gram_screen_bytes(int64_t n, int64_t N) {
  const int64_t nchunks = (N + tc::KC - 1) / tc::KC;
  const int64_t na = (n + gram::FA - 1) / gram::FA;
  return (size_t)na * nchunks * gram::A_IMG + (size_t)n * sizeof(GramTgt) + 256;
}

// Space part: b-images and feature sums, built once per space into `buf`
// (gram_space_bytes).
void gram_build_space(const FeatTable &F, void *buf, cudaStream_t st) {
  const int64_t n = F.n, N = F.N;
  const int nchunks = (int)((N + tc::KC - 1) / tc::KC);
  const int64_t nb = (n + gram::FB - 1) / gram::FB;
  unsigned char *bimg = static_cast<unsigned char *>(buf);
  GramFeat *gf = reinterpret_cast<GramFeat *>(bimg + (size_t)nb * nchunks * gram::B_IMG);
  cudaMemsetAsync(bimg, 0, (size_t)nb * nchunks * gram::B_IMG, st);
  note_launches(1);
  k_gram_space<<<(unsigned)n, 128, 0, st>>>(F, nchunks, bimg, gf);
}

// The tiles (a-block, b-block) holding a pair of the binary block of rung k
// with a candidate id in [id_begin, id_end).
void gram_tiles(const dse_space *sp, uint64_t id_begin, uint64_t id_end, std::vector<int2> &out) {
  const RungGeom &g = sp->geom;
  const int64_t n = sp->n, o = g.o;
  out.clear();
  if (g.nb == 0 || n < 2) return;
  const uint64_t p_lo = id_begin > (uint64_t)sp->n ? id_begin - (uint64_t)sp->n : 0;
  const uint64_t p_hi = id_end > (uint64_t)sp->n ? id_end - (uint64_t)sp->n : 0;
  if (p_hi <= p_lo) return;
  auto pidx = [&](int64_t i, int64_t j) { return g.um + (tri((uint64_t)i) + (uint64_t)j - g.tri_o) * (uint64_t)g.nb; };
  const int64_t na = (n + gram::FA - 1) / gram::FA;
  for (int64_t b = 0; b < na; ++b) {
    const int64_t i0 = std::max<int64_t>(b * gram::FA, o), i1 = std::min<int64_t>(b * gram::FA + gram::FA, n) - 1;
    if (i0 > i1) continue;
    for (int64_t c = 0; c * gram::FB < i1; ++c) {
      const int64_t j0 = c * gram::FB, j1 = std::min<int64_t>(j0 + gram::FB - 1, i1 - 1);
      // smallest and largest flat index of the tile's pairs (i > j)
      const int64_t ia = std::max<int64_t>(i0, j0 + 1);
      const uint64_t lo = pidx(ia, j0), hi = pidx(i1, std::min<int64_t>(j1, i1 - 1)) + (uint64_t)g.nb;
      if (hi <= p_lo || lo >= p_hi) continue;
      out.push_back(make_int2((int)b, (int)c));
    }
  }
}

// delta of the contraction entries for N samples (see the header).
float gram_delta(int64_t N) {
  const double u32 = 5.9604644775390625e-8;
  const int64_t nchunks = (N + tc::KC - 1) / tc::KC;
  const double steps = 3.0 * (tc::KC / 16) * (double)nchunks;
  return (float)(4.0 * (2.0 * steps + 2.0) * u32 + 3.02 * 1.52587890625e-5 + 4.0 * u32);
}

// One screen's a-images and target sums into `scr` (gram_screen_bytes).
void launch_gram_arows(const ScreenArgs &A, const void *space_buf, void *scr, cudaStream_t st) {
  const int64_t n = A.F.n, N = A.N;
  const int nchunks = (int)((N + tc::KC - 1) / tc::KC);
  const int64_t na = (n + gram::FA - 1) / gram::FA, nb = (n + gram::FB - 1) / gram::FB;
  const unsigned char *bimg = static_cast<const unsigned char *>(space_buf);
  const GramFeat *gf = reinterpret_cast<const GramFeat *>(bimg + (size_t)nb * nchunks * gram::B_IMG);
  unsigned char *aimg = static_cast<unsigned char *>(scr);
  GramTgt *gt = reinterpret_cast<GramTgt *>(aimg + (size_t)na * nchunks * gram::A_IMG);
  // (every row the epilogue reads is written for every chunk; the unused
  // rows only feed TMEM lanes that are never read)
  note_launches(1);
  k_gram_arows<<<(unsigned)n, 128, 0, st>>>(A.F, nchunks, A.y32 + (int64_t)A.t0 * A.ldy, gf, aimg, gt);
}

// One screen's product/quotient slots: the kernel over `tiles` (device,
// n_tiles) after launch_gram_arows.
dse_status launch_pair_gram(const ScreenArgs &A, const void *space_buf, void *scr, const int2 *tiles, int n_tiles,
                            int sms, cudaStream_t st) {
  if (n_tiles <= 0) return DSE_OK;
  const int64_t n = A.F.n, N = A.N;
  const int nchunks = (int)((N + tc::KC - 1) / tc::KC);
  const int64_t na = (n + gram::FA - 1) / gram::FA, nb = (n + gram::FB - 1) / gram::FB;
  const unsigned char *bimg = static_cast<const unsigned char *>(space_buf);
  const GramFeat *gf = reinterpret_cast<const GramFeat *>(bimg + (size_t)nb * nchunks * gram::B_IMG);
  unsigned char *aimg = static_cast<unsigned char *>(scr);
  GramTgt *gt = reinterpret_cast<GramTgt *>(aimg + (size_t)na * nchunks * gram::A_IMG);
  note_launches(1);
  static bool attr[64] = {false};
  int dev = 0;
  cudaGetDevice(&dev);
  if (!attr[dev & 63]) {
    DSE_CUDA(cudaFuncSetAttribute(k_pair_gram, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)gram::smem_total()));
    attr[dev & 63] = true;
  }
  GramArgs GA{aimg, bimg, gf, gt, tiles, n_tiles, nchunks, gram_delta(N), (int)na, (int)nb};
  ScreenArgs B = A;
  B.group = 1;
  const int grid = sms < n_tiles ? sms : n_tiles;
  k_pair_gram<<<grid, gram::THREADS, gram::smem_total(), st>>>(B, GA);
  return DSE_OK;
}

}  // namespace dse
