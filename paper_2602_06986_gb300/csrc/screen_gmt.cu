// screen_gmt.cu -- products, quotients, sums and differences of the binary
// block for 2..16 targets and any number of samples, from Gram contractions
// on the 5th-generation tensor cores (per-target lists).
//
// The statistics of a product slot v = u w (u = x_i, w = x_j or 1/x_j) are
// bilinear in the centred FP32 rows p (of x_i) and q (of x_j or 1/x_j):
// with the per-feature sums P1 = sum p, P2 = sum p^2, PY_t = sum p y_t (Q*
// of w), they need G11 = sum p q, G12 = sum p q^2, G21 = sum p^2 q, G22 =
// sum p^2 q^2 and H_t = sum p (q y_t) for every target t (the algebra of the
// single-target Gram kernel, screen_gram.cu).  Here the targets sit on the
// B side of one contraction over ORDERED pairs (i, j) of a tile:
//   A rows (TMEM lanes): p of 128 features, then p^2 of the same features;
//   B rows: per b-feature [q y_t (x), q' y_t (1/x)] for 16 targets (the H
//           block, 192 rows for 6 b-features), then [q, q^2, q', q'^2]
//           (the G block, 24 rows + 8 zero rows);
//   MMA 1: p x (H|G) -> 224 columns: H_t and G11/G12 of both families;
//   MMA 2: p^2 x G   ->  32 columns: G21/G22 of both families.
// Entry (i, j) with w = 1/x_j is a/b of the pair (i, j) when i > j and b/a
// of the pair (j, i) when i < j, so the full square of ordered pairs gives
// every quotient once; a*b, a+b and a-b are taken from the entries with
// i > j (a+b and a-b need only G11 of the x family and the target sums).
// A tile is 128 a-features x 6 b-features = 768 ordered pairs, contracted
// in 32-sample chunks (BF16x3: hi*hi + hi*lo + lo*hi, FP32 accumulation in
// tensor memory).  Long sample ranges are accumulated in blocks of 16
// chunks (512 samples) into one of two TMEM column sets and drained by the
// epilogue into FP32 running sums in registers, so that the accumulation
// bound stays that of one block (the same model as the multi-target
// tensor-core kernel) and the drain overlaps the next block's MMAs.
//
// Warp roles (one CTA per SM, persistent over a static tile stride):
//   warp 0      producer: two 1-D bulk copies per stage (the a-image chunk,
//               32 KB: p and p^2 hi/lo; the b-image chunk, 28 KB: H|G
//               hi/lo), 3-stage ring;
//   warp 1      TMEM allocation (512 columns: two sets of 256) and the MMA
//               issuer: 2 k-steps x 3 products x 2 MMAs per chunk;
//   warps 2-13  epilogue: warp w reads TMEM lane quadrant w % 4 (its 32
//               a-features) and third (w - 2) / 4 of the b-features (2
//               each); after the tile's last block it scores its a-feature
//               against its 2 b-features, every slot and target, with the
//               a-priori tests, intervals, realised test, escalation and
//               threshold pushes of the single-target Gram epilogue.
// The a-images and the per-feature sums are built once per space, the
// b-images and the target sums per screen (their rows depend on the
// targets).
#include <cuda_bf16.h>
#include <math.h>

#include <algorithm>
#include <vector>

#include "dse_internal.cuh"
#include "eval64.cuh"
#include "gram.cuh"
#include "screen_common.cuh"
#include "screen_kernels.cuh"
#include "tcgen05.cuh"
#include "util.cuh"

namespace dse {

namespace gmt {

constexpr int FA = 128;            // a-features per tile (one TMEM lane each)
constexpr int FB = 6;              // b-features per tile
constexpr int NTP = 16;            // targets per screen (rows beyond T are zero)
constexpr int HC = 2 * NTP;        // H rows per b-feature: q y_t of x, then of 1/x
constexpr int NH = FB * HC;        // 192
constexpr int NG = 32;             // G rows: [q, q^2, q', q'^2] per b-feature + zero rows
constexpr int N1 = NH + NG;        // 224: B of the first MMA (H rows, then G rows)
constexpr int SET = N1 + NG;       // 256 columns per accumulator set: H | G0 (p) | G1 (p^2)
constexpr int TMEM_COLS = 2 * SET; // 512
constexpr uint32_t A_PART = FA * tc::KC * 2;  // 8 KB: 128 rows x 32 samples, BF16
constexpr uint32_t A_IMG = 4 * A_PART;        // p hi, p^2 hi, p lo, p^2 lo
constexpr uint32_t B_PART = N1 * tc::KC * 2;  // 14 KB
constexpr uint32_t B_IMG = 2 * B_PART;        // hi, lo
constexpr uint32_t STAGE = A_IMG + B_IMG;     // 60 KB
constexpr uint32_t G_OFF = (NH / 8) * tc::SBO;  // byte offset of the G rows in a B part
constexpr int NS = 3;
constexpr int DB = 16;             // chunks per accumulation block
constexpr int EPI = 12;            // epilogue warps: three per TMEM lane quadrant
constexpr int THREADS = (2 + EPI) * 32;
constexpr int BPW = FB / 3;        // b-features per epilogue warp
constexpr int RUN = BPW * (HC + 8);  // running sums per epilogue thread (80)
constexpr int RG0 = BPW * HC, RG1 = RG0 + 4 * BPW;  // offsets of the G0 and G1 sums in them
constexpr uint32_t kWait = 1u << 22;
constexpr int kStage = 64;         // pending pushes per epilogue warp

static_assert(N1 % 16 == 0 && N1 <= 256 && NG % 16 == 0, "MMA shapes (M = 128)");
static_assert(FB * 4 <= NG, "G rows");

struct Shared {
  uint64_t full[NS], empty[NS];
  uint64_t acc_full[2], acc_empty[2];
  uint64_t drain;
  uint32_t tmem_base;
  int abort;
  float theta[EPI][NTP];  // each epilogue warp's copy of the list thresholds
  float ysum[NTP];
  float py[EPI][NTP][32];  // each epilogue warp's a-features' target sums (target-major)
  // each epilogue warp's pending pushes (list, id, score, bound), written
  // out a b-feature at a time
  uint64_t pid[EPI][kStage];
  float ps[EPI][kStage], pe[EPI][kStage];
  uint8_t pl[EPI][kStage];
  int pn[EPI];
};

constexpr size_t shared_bytes() { return (sizeof(Shared) + 1023) / 1024 * 1024; }
constexpr size_t smem_total() { return shared_bytes() + (size_t)NS * STAGE; }
static_assert(smem_total() <= 227 * 1024, "shared memory of one CTA");

// B-image row of b-feature g: H row of target t and family fam, G row of
// type k (0..3: q, q^2 of x, then of 1/x).
__host__ __device__ inline int hrow(int g, int fam, int t) { return g * HC + fam * NTP + t; }
__host__ __device__ inline int grow(int g, int k) { return NH + 4 * g + k; }

}  // namespace gmt

// Target sums of a feature, per family and target: sum fl(p y_t)
// (compensated) and RU |fl(p y_t)|_2.
struct GmtTgt {
  float sy[2][gmt::NTP];
  float ny[2][gmt::NTP];
};

// ------------------------------------------------------------- row images

// Space part, one block per feature slot f of the a-blocks (slots past n
// write zero rows): the a-image rows p, p^2 of x and the feature's sums.
__global__ void __launch_bounds__(128) k_gmt_space(FeatTable F, int nchunks, unsigned char *aimg, GramFeat *gf) {
  __shared__ double sm[4 * 10];
  const int64_t f = blockIdx.x;
  const bool real = f < F.n;
  uint32_t fl = 0;
  float4 fa = make_float4(0.f, 0.f, 0.f, 0.f);
  if (real) {
    fl = F.flags[f];
    fa = F.fa[f];
  }
  const bool okx = real && (fl & F_FP32_SAFE) != 0;
  const bool okr = okx && (fl & F_MINABS_POS) != 0;
  const float c[2] = {fa.x, fa.y};
  const bool ok[2] = {okx, okr};
  const int64_t ab = f / gmt::FA;
  const int r = (int)(f % gmt::FA);
  GramFeatAcc acc;
  const int64_t groups = (int64_t)nchunks * (tc::KC / 8);
  for (int64_t gi = threadIdx.x; gi < groups; gi += blockDim.x) {
    const int64_t s0 = gi * 8;
    const int ch = (int)(s0 / tc::KC), k0 = (int)(s0 % tc::KC);
    unsigned char *base = aimg + ((size_t)ab * nchunks + ch) * gmt::A_IMG;
#pragma unroll
    for (int fam = 0; fam < 2; ++fam) {
      float p[8], p2[8];
      gram_vals(F, real ? f : 0, s0, fam, c[fam], ok[fam], p);
#pragma unroll
      for (int e = 0; e < 8; ++e) p2[e] = p[e] * p[e];
      acc.add(fam, p, p2, ok[fam], c[fam], s0, F.N);
      if (fam == 0) {
        uint4 h, l;
        const uint32_t o = tc::core_off(r, k0);
        split8(p, h, l);
        *reinterpret_cast<uint4 *>(base + o) = h;
        *reinterpret_cast<uint4 *>(base + 2 * gmt::A_PART + o) = l;
        split8(p2, h, l);
        *reinterpret_cast<uint4 *>(base + gmt::A_PART + o) = h;
        *reinterpret_cast<uint4 *>(base + 3 * gmt::A_PART + o) = l;
      }
    }
  }
  GramFeat tmp;
  acc.finish(sm, groups, c, ok, real ? gf + f : &tmp);
}

// The b-images are written a row group at a time: 8 rows x 32 samples of
// one chunk part are 512 contiguous bytes, one 16-byte piece per lane (lane
// = 8 k-group + row within the group), so every warp store is coalesced.
// A block takes one b-block and kBrowsCh chunks.  Per chunk the block first
// puts the centred values of its 6 b-features (both families) and the 16
// targets' values in shared memory, each computed or loaded once (the 8
// target lanes of a row group need the same values), then its warps take
// the row groups (H: b-feature g, family, half of the targets; G: two
// b-features' [q, q^2, q', q'^2]) and keep, per lane, the target sums of its
// H rows over the block's chunks.
constexpr int kBrowsCh = 16;  // chunks per k_gmt_brows block
constexpr int kHTypes = gmt::FB * 4;  // H row groups per b-block: g x family x half of the targets
static_assert(kHTypes == 3 * 8 && gmt::NTP == 16 && gmt::NG == 4 * 8, "row groups of the 8 warps");
static_assert(tc::KC == 32, "one chunk = 32 samples = 4 k-groups of 8");

// Per-block partial target sums: [b-block][chunk block][g][family][target]
// of (compensated pair s, c; sum of squares).
struct GmtPart {
  float s, c, q;
};

size_t gmt_part_count(int64_t n, int64_t N) {
  const int64_t nchunks = (N + tc::KC - 1) / tc::KC;
  const int64_t ncb = (nchunks + kBrowsCh - 1) / kBrowsCh;
  return (size_t)((n + gmt::FB - 1) / gmt::FB) * ncb * gmt::FB * 2 * gmt::NTP;
}

// Per screen: the b-image of b-block blockIdx.x, chunks kBrowsCh blockIdx.y
// .. + kBrowsCh - 1, and the block's partial target sums.  H rows: q y_t
// of x and of 1/x, y the FP32 targets t0 .. t0+T-1 (zero rows for t >= T
// and for feature slots past n); G rows: q, q^2 of x and of 1/x, and the
// zero rows after the last b-feature's.
__global__ void __launch_bounds__(256) k_gmt_brows(FeatTable F, int nchunks, const float *y32, int64_t ldy, int T,
                                                   const GramFeat *gf, unsigned char *bimg, GmtPart *part) {
  using namespace gmt;
  constexpr int KC = tc::KC;
  // double-buffered per-chunk values: [g][family][sample], [target][sample]
  // (rows padded to 36 floats: the 8 target rows a quarter-warp reads with
  // 16-byte loads fall in distinct banks)
  __shared__ __align__(16) float pv[2][FB][2][KC + 4];
  __shared__ __align__(16) float yv[2][NTP][KC + 4];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int kg = lane >> 3, r8 = lane & 7;
  const int64_t bb = blockIdx.x, cb = blockIdx.y;
  const int c0 = (int)cb * kBrowsCh, c1 = min(nchunks, c0 + kBrowsCh);
  const int64_t N = F.N;
  // the values thread x computes for every chunk: (g, family, sample) of
  // x < 2 FB KC = 384, then (target, sample) of x - 2 FB KC < NTP KC = 512
  // (x = threadIdx.x + 256 h, h = 0..3)
  static_assert(2 * FB * KC + NTP * KC <= 4 * 256, "four values per thread");
  auto fill = [&](int c, int buf) {
    const int64_t sb = (int64_t)c * KC;
#pragma unroll
    for (int h = 0; h < 4; ++h) {
      const int x = threadIdx.x + 256 * h;
      if (x < 2 * FB * KC) {
        const int g = x / (2 * KC), fam = (x / KC) & 1, e = x % KC;
        const int64_t f = bb * FB + g, sidx = sb + e;
        float v = 0.f;
        if (f < F.n) {
          const GramFeat G = gf[f];
          if (G.ok[fam] && sidx < N) {
            const float xv = F.v32[f * F.ld + sidx];
            v = (fam == 0 ? xv : __frcp_rn(xv)) - G.c[fam];
          }
        }
        pv[buf][g][fam][e] = v;
      } else if (x < 2 * FB * KC + NTP * KC) {
        const int t = (x - 2 * FB * KC) / KC, e = (x - 2 * FB * KC) % KC;
        const int64_t sidx = sb + e;
        yv[buf][t][e] = (t < T && sidx < N) ? y32[(int64_t)t * ldy + sidx] : 0.f;
      }
    }
  };
  // H row groups of this warp: types warp, warp + 8, warp + 16 (type =
  // 4 g + 2 family + half)
  Comp32 acc[3];
  float sq[3] = {0.f, 0.f, 0.f};
  if (c0 < c1) fill(c0, 0);
  for (int c = c0; c < c1; ++c) {
    const int buf = (c - c0) & 1;
    __syncthreads();  // this chunk's values are in; the other buffer is free
    if (c + 1 < c1) fill(c + 1, buf ^ 1);
    unsigned char *base = bimg + ((size_t)bb * nchunks + c) * B_IMG;
#pragma unroll
    for (int i = 0; i < 3; ++i) {
      const int type = warp + 8 * i;
      const int g = type >> 2, fam = (type >> 1) & 1, half = type & 1;
      const int t = half * 8 + r8;
      const float4 *pp = reinterpret_cast<const float4 *>(&pv[buf][g][fam][kg * 8]);
      const float4 *yp = reinterpret_cast<const float4 *>(&yv[buf][t][kg * 8]);
      const float4 pa = pp[0], pb = pp[1], ya = yp[0], yb = yp[1];
      const float p[8] = {pa.x, pa.y, pa.z, pa.w, pb.x, pb.y, pb.z, pb.w};
      const float y[8] = {ya.x, ya.y, ya.z, ya.w, yb.x, yb.y, yb.z, yb.w};
      float py[8];
      float part8 = 0.f;
#pragma unroll
      for (int e = 0; e < 8; ++e) {
        py[e] = p[e] * y[e];
        part8 += py[e];
        sq[i] = fmaf(py[e], py[e], sq[i]);
      }
      acc[i].add(part8);
      uint4 h, l;
      split8(py, h, l);
      const uint32_t o = tc::core_off(hrow(g, fam, t), kg * 8);
      *reinterpret_cast<uint4 *>(base + o) = h;
      *reinterpret_cast<uint4 *>(base + B_PART + o) = l;
    }
    if (warp < NG / 8) {
      // G row group `warp`: rows NH + 8 warp + r8 = b-feature 2 warp + r8 / 4,
      // type r8 % 4 (q, q^2 of x, then of 1/x)
      const int g = 2 * warp + (r8 >> 2), k = r8 & 3, fam = k >> 1;
      float v[8];
      if (g < FB) {
        const float4 *pp = reinterpret_cast<const float4 *>(&pv[buf][g][fam][kg * 8]);
        const float4 pa = pp[0], pb = pp[1];
        v[0] = pa.x, v[1] = pa.y, v[2] = pa.z, v[3] = pa.w, v[4] = pb.x, v[5] = pb.y, v[6] = pb.z, v[7] = pb.w;
        if (k & 1) {
#pragma unroll
          for (int e = 0; e < 8; ++e) v[e] = v[e] * v[e];
        }
      } else {
#pragma unroll
        for (int e = 0; e < 8; ++e) v[e] = 0.f;
      }
      uint4 h, l;
      split8(v, h, l);
      const uint32_t o = tc::core_off(NH + 8 * warp + r8, kg * 8);
      *reinterpret_cast<uint4 *>(base + o) = h;
      *reinterpret_cast<uint4 *>(base + B_PART + o) = l;
    }
  }
  // the four k-groups of each target meet in lanes 0..7
#pragma unroll
  for (int i = 0; i < 3; ++i) {
    Comp32 a = acc[i];
    float q = sq[i];
    for (int off = 8; off < 32; off <<= 1) {
      const float s = __shfl_xor_sync(0xffffffffu, a.s, off), c = __shfl_xor_sync(0xffffffffu, a.c, off);
      a.add(s);
      a.c += c;
      q += __shfl_xor_sync(0xffffffffu, q, off);
    }
    if (kg == 0) {
      const int type = warp + 8 * i;
      const int g = type >> 2, fam = (type >> 1) & 1, half = type & 1;
      const int t = half * 8 + r8;
      GmtPart o;
      o.s = a.s;
      o.c = a.c;
      o.q = q;
      part[(((size_t)bb * gridDim.y + cb) * FB + g) * 2 * NTP + fam * NTP + t] = o;
    }
  }
}

// The target sums of each feature from the blocks' partials: the pairs
// merged in FP32 (compensated), the sums of squares added in FP64.
__global__ void __launch_bounds__(64) k_gmt_tsum(int64_t n, int ncb, const GmtPart *part, int64_t groups,
                                                 GmtTgt *gt) {
  using namespace gmt;
  const int64_t f = blockIdx.x;
  const int x = threadIdx.x;  // family x NTP + target
  if (f >= n || x >= 2 * NTP) return;
  const int64_t bb = f / FB, g = f % FB;
  Comp32 a;
  double q = 0.0;
  for (int cb = 0; cb < ncb; ++cb) {
    const GmtPart p = part[(((size_t)bb * ncb + cb) * FB + g) * 2 * NTP + x];
    a.add(p.s);
    a.c += p.c;
    q += (double)p.q;
  }
  // the FP32 per-lane sums of squares are low by at most (terms per lane +
  // 2 shuffle levels + 4) u of themselves
  const double marg = 1.0 + ((double)kBrowsCh * 8.0 + 8.0) * 5.9604644775390625e-8;
  gt[f].sy[x / NTP][x % NTP] = (float)a.value();
  gt[f].ny[x / NTP][x % NTP] = __double2float_ru(sqrt(q * marg) * (1.0 + 1e-15));
  (void)groups;
}

// ------------------------------------------------------------------ kernel

struct GmtArgs {
  const unsigned char *aimg, *bimg;
  const GramFeat *gf;
  const GmtTgt *gt;
  const int2 *tiles;  // (a-block, b-block)
  int n_tiles;
  int nchunks, nblocks;
  float delta;
  int na, nb;  // a-blocks and b-blocks of the images
};

// The epilogue record of feature f (a-priori fields and sums).
__device__ __forceinline__ gram::EpiFeat gmt_rec(const ScreenArgs &A, const GramFeat *gf, int64_t f) {
  gram::EpiFeat c;
  c.fa = A.F.fa[f];
  c.fr = A.F.fr[f];
  c.flags = A.F.flags[f];
  c.cplx = A.F.cplx[f];
  c.uk[0] = A.F.ukey[2 * f];
  c.uk[1] = A.F.ukey[2 * f + 1];
  const GramFeat g = gf[f];
#pragma unroll
  for (int m = 0; m < 2; ++m) {
    c.c[m] = g.c[m];
    c.s1[m] = g.s1[m];
    c.s2[m] = g.s2[m];
    c.n1[m] = g.n1[m];
    c.n2[m] = g.n2[m];
    c.nu[m] = g.nu[m];
    c.sy[m] = 0.f;
    c.ny[m] = 0.f;
  }
  return c;
}

// A warp's pending pushes.  A lane stages a push with a shared-memory
// atomic (no global round trip in the scoring loop; a full stage falls back
// to a direct push); the whole warp writes the stage out: entries still at
// or above their list's current threshold, one global slot reservation per
// distinct list (the lanes holding one list's entries take consecutive
// slots), then the bound histograms.  Returns the lists written to.
struct GmtStage {
  uint64_t *id;
  float *s, *e;
  uint8_t *l;
  int *n;
};

__device__ __forceinline__ bool gmt_stage(const GmtStage &P, const CandBufs &B, int t0, int l, uint64_t id, float s,
                                          float e) {
  const int pos = atomicAdd(P.n, 1);
  if (pos < gmt::kStage) {
    P.id[pos] = id;
    P.s[pos] = s;
    P.e[pos] = e;
    P.l[pos] = (uint8_t)l;
    return true;
  }
  return push_one(B, t0 + l, id, s, e);
}

__device__ __forceinline__ uint32_t gmt_flush(const GmtStage &P, const CandBufs &B, int t0) {
  __syncwarp();
  const int lane = threadIdx.x & 31;
  const int n = min(*P.n, gmt::kStage);
  uint32_t lists = 0;
  for (int i0 = 0; i0 < n; i0 += 32) {
    const int i = i0 + lane;
    int l = -1;
    uint64_t id = 0;
    float s = 0.f, e = 0.f;
    if (i < n) {
      l = P.l[i];
      id = P.id[i];
      s = P.s[i];
      e = P.e[i];
      if (!(iv_hi(s, e) >= ld_relaxed(&B.theta[t0 + l]))) l = -1;  // below a threshold raised meanwhile
    }
    const unsigned grp = __match_any_sync(0xffffffffu, l);
    const int leader = __ffs(grp) - 1;
    unsigned base = 0;
    if (l >= 0 && lane == leader) base = atomicAdd(&B.count[t0 + l], (unsigned)__popc(grp));
    base = __shfl_sync(0xffffffffu, base, leader);
    if (l >= 0) {
      const unsigned pos = base + (unsigned)__popc(grp & ((1u << lane) - 1u));
      if ((int64_t)pos < B.cap) {
        const size_t x = (size_t)(t0 + l) * (size_t)B.cap + pos;
        B.id[x] = id;
        B.score[x] = s;
        B.eps[x] = e;
      }
      lists |= 1u << l;
    }
    // the bound histograms, one atomic per distinct (list, bin) of the batch
    // (entries near a threshold share bins)
    const bool act = l >= 0;
    const unsigned am = __ballot_sync(0xffffffffu, act);
    if (act) {
      const int bl = score_bin(iv_lo(s, e)), bh = score_bin(iv_hi(s, e)), bc = bl / kFine;
      const unsigned gl = __match_any_sync(am, l * kNumBins + bl), gc = __match_any_sync(am, l * kCoarse + bc),
                     gh = __match_any_sync(am, l * kNumBins + bh);
      const size_t lb = (size_t)(t0 + l);
      if (lane == __ffs(gl) - 1) atomicAdd(&B.hist[lb * kNumBins + bl], (unsigned)__popc(gl));
      if (lane == __ffs(gc) - 1) atomicAdd(&B.hist_c[lb * kCoarse + bc], (unsigned)__popc(gc));
      if (lane == __ffs(gh) - 1) atomicAdd(&B.hist_hi[lb * kNumBins + bh], (unsigned)__popc(gh));
    }
  }
  __syncwarp();
  if (lane == 0) *P.n = 0;
  __syncwarp();
  return __reduce_or_sync(0xffffffffu, lists);
}

// Common bookkeeping of one candidate once its interval part is known:
// realised decision, escalation, then every target's score, interval note
// and threshold push.  sy(t, &Sy, &dSy) gives target t's sum and bound;
// sy_bound bounds every |Sy| (a non-finite bound leaves the candidate to the
// FP64 escalation).  Returns the lists pushed to.
template <class SyFn>
__device__ __forceinline__ uint32_t gmt_targets(const ScreenArgs &A, LaneStats &ls, uint64_t gid, const GramVar &v,
                                                float invN, const float *ysum, const float *theta, float sy_bound,
                                                const GmtStage &P, SyFn sy) {
  if (v.realised == 0) {
    ls.r[DSE_R_REALISED]++;
    note_why(A, gid, DSE_R_REALISED);
    return 0;
  }
  if (v.realised != 1 || !(sy_bound < 1e30f)) {
    escalate(A, gid);
    ls.escalated++;
    return 0;
  }
  ls.r[DSE_VALID]++;
  ls.evaluated++;
  note_why(A, gid, DSE_VALID);
  uint32_t pushed = 0;
  const float u = 5.9604644775390625e-8f;
  // (a loop, not 16 unrolled copies: the epilogue's code stays small enough
  // for the instruction cache)
#pragma unroll 1
  for (int t = 0; t < gmt::NTP; ++t) {
    if (t >= A.T) break;
    float S, d, s, eps;
    sy(t, &S, &d);
    if (!A.ivl && v.q_lo > 0.f) {
      // cheap rejection: the pushed interval's upper edge is at most
      // 2 rhi (1 + 24u) + 4e-12 with rhi = (|P| + dP) / q_lo (gram_num's
      // numerator bound); most candidate-target pairs are far below the
      // list's threshold, and this test needs no division
      const float ys = ysum[t];
      const float P = fmaf(-v.S1, ys * invN, S);
      const float aP = fabsf(P), ays = fabsf(ys), aS1 = fabsf(v.S1);
      const float dP = (d + ays * invN * v.dS1 + 6.f * u * (fabsf(S) + aS1 * ays * invN) + v.E * (1.f + 2.f * u) +
                        2.f * u * v.q_hi + u * aP) *
                       1.01f;
      if ((aP + dP) * 2.0002f + 1e-10f * v.q_lo < theta[t] * v.q_lo) continue;
    }
    gram_num(v, S, d, invN, ysum[t], &s, &eps);
    eps *= 1.0f + 2.4e-7f;
    note_ivl(A, gid, A.t0 + t, s, eps);
    if (iv_hi(s, eps) >= theta[t] && gmt_stage(P, A.B, A.t0, t, gid, s, eps)) pushed |= 1u << t;
  }
  return pushed;
}

// Product-type slot v = u w of the ordered pair (i, j): u = x_i (family 0),
// w = family FW of x_j; entries G11, G12, G21, G22, and H of the 16 targets
// at run[HOFF ..] (an offset fixed at compile time, so that the running sums
// stay in registers); opc/ia/ib name the candidate (a/b of (i, j) or b/a of
// (j, i) for FW = 1, a*b of (i, j) for FW = 0).
template <int FW, int HOFF>
__device__ __forceinline__ uint32_t gmt_product(const ScreenArgs &A, const GmtArgs &GA, LaneStats &ls, int opc,
                                                int64_t ia, int64_t ib, int64_t i, int64_t j,
                                                const gram::EpiFeat &Fi, const gram::EpiFeat &Fj,
                                                const float (&run)[gmt::RUN], float G11, float G12, float G21,
                                                float G22, const float *ysum, const float *theta,
                                                const float (*py)[32], const GmtStage &P) {
  const int pos = A.slot_pos[opc - 6];
  if (pos < 0) return 0;
  const uint64_t pbase = A.G.um + (tri((uint64_t)ia) + (uint64_t)ib - A.G.tri_o) * (uint64_t)A.G.nb;
  const uint64_t gid = (uint64_t)A.n_stored + pbase + (uint64_t)pos;
  if (gid < A.id_begin || gid >= A.id_end) return 0;
  const gram::EpiFeat &Fa = ia == i ? Fi : Fj, &Fb = ia == i ? Fj : Fi;
  const int reason = gram_apriori(A, opc, ia, ib, Fa, Fb);
  if (reason != DSE_VALID) {
    ls.r[reason]++;
    note_why(A, gid, reason);
    return 0;
  }
  if (!((Fi.flags & Fj.flags) & F_FP32_SAFE)) {
    escalate(A, gid);
    ls.escalated++;
    return 0;
  }
  const float u = 5.9604644775390625e-8f;
  const float N = (float)A.N, invN = (float)A.invN, delta = GA.delta;
  const float cu = Fi.c[0], cw = Fj.c[FW];
  const float P1 = Fi.s1[0], P2 = Fi.s2[0];
  const float Q1 = Fj.s1[FW], Q2 = Fj.s2[FW];
  const float t1a = cu * Q1, t1b = cw * P1;
  const float S1 = t1a + t1b + G11;
  const float cucw = cu * cw;
  const float t2a = cu * cu * Q2, t2b = cw * cw * P2, t2c = 2.f * cucw * G11, t2d = 2.f * cu * G12,
              t2e = 2.f * cw * G21;
  const float S2 = t2a + t2b + G22 + t2c + t2d + t2e;
  const float acu = fabsf(cu), acw = fabsf(cw);
  const float n1u = Fi.n1[0], n2u = Fi.n2[0], n1w = Fj.n1[FW], n2w = Fj.n2[FW];
  const GramErr ge = gram_err(delta, G22, n1u, n2u, n1w, n2w, N);
  const float dG11 = ge.dG11, dG22 = ge.dG22, dG12 = ge.dG12, dG21 = ge.dG21;
  const float dS1 = (dG11 + 10.f * u * (fabsf(t1a) + fabsf(t1b) + fabsf(G11))) * 1.01f;
  const float dS2 = (dG22 + 2.f * acu * acw * dG11 + 2.f * acu * dG12 + 2.f * acw * dG21 +
                     12.f * u * (t2a + t2b + fabsf(G22) + fabsf(t2c) + fabsf(t2d) + fabsf(t2e))) *
                    1.01f;
  const float Z = S2 + 2.f * cucw * S1 + N * cucw * cucw;
  const float dZ = (dS2 + 2.f * fabsf(cucw) * dS1 + 10.f * u * (fabsf(S2) + 2.f * fabsf(cucw * S1) + N * cucw * cucw)) *
                   1.01f;
  const float Vhi = sqrtf(Z + dZ) * (1.f + 4.f * u);
  const float kappa = FW == 0 ? 4.01f : 5.01f;
  const float E = u * (kappa * Vhi + 1.01f * (acw * Fi.nu[0] + acu * Fj.nu[FW])) * 1.02f;
  const GramVar v = gram_var(S1, dS1, S2, dS2, Z, dZ, Vhi, E, N, invN, (float)A.fmin_std_rel64);
  const GmtTgt *tj = GA.gt + j;
  const int lane = threadIdx.x & 31;
  // the slot's H entries, copied out of the running sums with compile-time
  // indices (the target loop indexes this copy, so run[] stays in registers)
  float hv[gmt::NTP];
#pragma unroll
  for (int t = 0; t < gmt::NTP; ++t) hv[t] = run[HOFF + t];
  auto sy = [&](int t, float *S, float *d) {
    const float PY = py[t][lane], QY = __ldg(&tj->sy[FW][t]), nyw = __ldg(&tj->ny[FW][t]);
    const float tya = cu * QY, tyb = cw * PY, h = hv[t];
    *S = tya + tyb + h;
    *d = (delta * fminf(n1u * nyw, ge.h) + 10.f * u * (fabsf(tya) + fabsf(tyb) + fabsf(h)) +
          9.1f * u * (acu * n1w + acw * n1u)) *
         1.01f;
  };
  // |QY| <= |q|, |PY| <= |p| and |H| <= sqrt(G22) for a unit target
  const float bound = (acu * n1w + acw * n1u + ge.h) * 1.01f;
  return gmt_targets(A, ls, gid, v, invN, ysum, theta, bound, P, sy);
}

// a + b (sign 1) or a - b (sign -1) of the pair (i, j), i > j: family x of
// both features, shift k = c_i +- c_j; needs G11 of the x family.
__device__ __forceinline__ uint32_t gmt_addsub(const ScreenArgs &A, const GmtArgs &GA, LaneStats &ls, int opc,
                                               int64_t i, int64_t j, const gram::EpiFeat &Fi, const gram::EpiFeat &Fj,
                                               float G11, float G22, const float *ysum, const float *theta,
                                               const float (*py)[32], const GmtStage &P) {
  const int pos = A.slot_pos[opc - 6];
  if (pos < 0) return 0;
  const uint64_t pbase = A.G.um + (tri((uint64_t)i) + (uint64_t)j - A.G.tri_o) * (uint64_t)A.G.nb;
  const uint64_t gid = (uint64_t)A.n_stored + pbase + (uint64_t)pos;
  if (gid < A.id_begin || gid >= A.id_end) return 0;
  ls.seen++;
  const int reason = gram_apriori_add(A, opc, i, j, Fi, Fj);
  if (reason != DSE_VALID) {
    ls.r[reason]++;
    note_why(A, gid, reason);
    return 0;
  }
  if (!((Fi.flags & Fj.flags) & F_FP32_SAFE)) {
    escalate(A, gid);
    ls.escalated++;
    return 0;
  }
  const float u = 5.9604644775390625e-8f;
  const float N = (float)A.N, invN = (float)A.invN, delta = GA.delta;
  const float sign = opc == DSE_OP_ADD ? 1.f : -1.f;
  const float ca = Fi.c[0], cb = Fj.c[0], k = ca + sign * cb;
  const float P1 = Fi.s1[0], P2 = Fi.s2[0];
  const float Q1 = Fj.s1[0], Q2 = Fj.s2[0];
  const float S1 = P1 + sign * Q1;
  const float S2 = P2 + Q2 + sign * 2.f * G11;
  const float dG11 = gram_err(delta, G22, Fi.n1[0], Fi.n2[0], Fj.n1[0], Fj.n2[0], N).dG11;
  const float dS1 = 8.f * u * (fabsf(P1) + fabsf(Q1)) * 1.01f;
  const float dS2 = (2.f * dG11 + 8.f * u * (P2 + Q2 + 2.f * fabsf(G11))) * 1.01f;
  const float Z = S2 + 2.f * k * S1 + N * k * k;
  const float dZ = (dS2 + 2.f * fabsf(k) * dS1 + 10.f * u * (fabsf(S2) + 2.f * fabsf(k * S1) + N * k * k)) * 1.01f;
  const float Vhi = sqrtf(Z + dZ) * (1.f + 4.f * u);
  const float E = u * (2.01f * (Fi.nu[0] + Fj.nu[0]) + (fabsf(ca) + fabsf(cb)) * sqrtf(N) * (1.f + 4.f * u) + Vhi) *
                  1.02f;
  const GramVar v = gram_var(S1, dS1, S2, dS2, Z, dZ, Vhi, E, N, invN, (float)A.fmin_std_rel64);
  const GmtTgt *tj = GA.gt + j;
  const float n1s = Fi.n1[0] + Fj.n1[0];
  const int lane = threadIdx.x & 31;
  auto sy = [&](int t, float *S, float *d) {
    const float PY = py[t][lane], QY = __ldg(&tj->sy[0][t]);
    *S = PY + sign * QY;
    *d = (8.f * u * (fabsf(PY) + fabsf(QY)) + 9.1f * u * n1s) * 1.01f;
  };
  return gmt_targets(A, ls, gid, v, invN, ysum, theta, n1s * 1.01f, P, sy);
}

// Drain one accumulator set into the running sums: this warp's half HH of
// the H columns (3 b-features x 32) and its 12 columns of each G block.
template <int HH>
__device__ __forceinline__ void gmt_drain(uint32_t t, float (&run)[gmt::RUN], bool first) {
  using namespace gmt;
  float v[32];
#pragma unroll
  for (int c = 0; c < BPW; ++c) {
    tc::tmem_ld32(t + HH * BPW * HC + 32 * c, v);
#pragma unroll
    for (int k = 0; k < 32; ++k) run[32 * c + k] = first ? v[k] : run[32 * c + k] + v[k];
  }
  tc::tmem_ld32(t + NH, v);
#pragma unroll
  for (int k = 0; k < 4 * BPW; ++k) run[RG0 + k] = first ? v[4 * BPW * HH + k] : run[RG0 + k] + v[4 * BPW * HH + k];
  tc::tmem_ld32(t + N1, v);
#pragma unroll
  for (int k = 0; k < 4 * BPW; ++k) run[RG1 + k] = first ? v[4 * BPW * HH + k] : run[RG1 + k] + v[4 * BPW * HH + k];
}

// The candidates of the ordered pair (i, j), j the G-th b-feature of this
// warp's half: the quotient (w = 1/x_j) always, a*b, a+b, a-b when i > j.
template <int G>
__device__ __forceinline__ uint32_t gmt_pair(const ScreenArgs &A, const GmtArgs &GA, LaneStats &ls, int64_t i,
                                             int64_t j, const gram::EpiFeat &Fi, const float (&run)[gmt::RUN],
                                             const float *ysum, const float *theta, const float (*py)[32],
                                             const GmtStage &P) {
  const int64_t n = A.F.n;
  if (i >= n || j >= n || j == i) return 0;
  const bool igt = i > j;
  const int64_t hi = igt ? i : j, lo = igt ? j : i;
  if (hi < A.G.o) return 0;
  const gram::EpiFeat Fj = gmt_rec(A, GA.gf, j);
  constexpr int H0 = gmt::HC * G, G0 = gmt::RG0 + 4 * G, G1 = gmt::RG1 + 4 * G;
  uint32_t pushed = gmt_product<1, H0 + gmt::NTP>(A, GA, ls, igt ? DSE_OP_DIV : DSE_OP_RDIV, hi, lo, i, j, Fi, Fj,
                                                   run, run[G0 + 2], run[G0 + 3], run[G1 + 2], run[G1 + 3], ysum,
                                                   theta, py, P);
  if (igt) {
    pushed |= gmt_product<0, H0>(A, GA, ls, DSE_OP_MUL, i, j, i, j, Fi, Fj, run, run[G0], run[G0 + 1], run[G1],
                                 run[G1 + 1], ysum, theta, py, P);
    if (A.gram_addsub) {
      pushed |= gmt_addsub(A, GA, ls, DSE_OP_ADD, i, j, Fi, Fj, run[G0], run[G1 + 1], ysum, theta, py, P);
      pushed |= gmt_addsub(A, GA, ls, DSE_OP_SUB, i, j, Fi, Fj, run[G0], run[G1 + 1], ysum, theta, py, P);
    }
  }
  return pushed;
}

// Epilogue of warp part hh (b-features BPW hh .. BPW hh + BPW - 1 of every
// tile); one instance for every part (only the drain's TMEM columns depend
// on hh), so that the code stays small.
template <class WaitWarp, class Aborted>
__device__ __forceinline__ void gmt_epilogue(const ScreenArgs &A, const GmtArgs &GA, gmt::Shared &sh, uint32_t tmem,
                                             int q, int ew, int hh, WaitWarp wait_warp, Aborted aborted_warp) {
  using namespace gmt;
  const int lane = threadIdx.x & 31;
  const uint32_t lane_base = (uint32_t)(q * 32) << 16;
  LaneStats ls;
  ls.zero();
  float *theta = sh.theta[ew];
  int pend = 0;  // lane t: this warp's pushes to list t since it last raised its threshold
  const GmtStage P{sh.pid[ew], sh.ps[ew], sh.pe[ew], sh.pl[ew], &sh.pn[ew]};
  if (lane == 0) sh.pn[ew] = 0;
  __syncwarp();
  int lt = 0;
  for (int tile = blockIdx.x; tile < GA.n_tiles && !aborted_warp(); tile += gridDim.x, ++lt) {
    const int2 tl = GA.tiles[tile];
    float run[RUN];
    bool ok = true;
    for (int b = 0; b < GA.nblocks; ++b) {
      const uint32_t gb = (uint32_t)lt * GA.nblocks + b, set = gb & 1;
      if (!wait_warp(&sh.acc_full[set], (gb >> 1) & 1)) {
        ok = false;
        break;
      }
      tc::fence_after();
      const uint32_t ta = tmem + lane_base + set * SET;
      if (hh == 0)
        gmt_drain<0>(ta, run, b == 0);
      else if (hh == 1)
        gmt_drain<1>(ta, run, b == 0);
      else
        gmt_drain<2>(ta, run, b == 0);
      tc::fence_before();
      __syncwarp();
      if (lane == 0) tc::mbar_arrive(&sh.acc_empty[set]);
    }
    if (!ok) break;
    // this warp's copy of the thresholds (they only rise, so an older copy
    // is still a valid lower bound)
    for (int t = lane; t < NTP; t += 32) theta[t] = t < A.T ? ld_relaxed(&A.B.theta[A.t0 + t]) : 0.f;
    __syncwarp();
    const int64_t i = (int64_t)tl.x * FA + q * 32 + lane;
    const int64_t j0 = (int64_t)tl.y * FB + BPW * hh;
    const bool own = tl.x >= 0 && i < A.F.n;  // (tl.x < 0: the empty partner of a pair)
    gram::EpiFeat Fi;
    if (own) Fi = gmt_rec(A, GA.gf, i);
    // this lane's a-feature target sums (x family), target-major in shared
    // memory: read once per tile, not once per candidate and target
    float(*py)[32] = sh.py[ew];
    {
      const float4 *src = reinterpret_cast<const float4 *>(&GA.gt[own ? i : 0].sy[0][0]);
#pragma unroll
      for (int q4 = 0; q4 < NTP / 4; ++q4) {
        const float4 v4 = own ? src[q4] : make_float4(0.f, 0.f, 0.f, 0.f);
        py[4 * q4][lane] = v4.x;
        py[4 * q4 + 1][lane] = v4.y;
        py[4 * q4 + 2][lane] = v4.z;
        py[4 * q4 + 3][lane] = v4.w;
      }
      __syncwarp();
    }
    // after each b-feature the warp writes its staged pushes out, and the
    // lists it has pushed at least 16 entries to since it last raised them
    // get their thresholds raised and re-read (every warp of the first wave
    // of tiles scores with thresholds still at zero: without this, that
    // wave alone could fill the candidate buffers; later, pushes are rare
    // and a threshold scan per push would cost more than the scoring).
    // Lane t counts list t's pushes (staged or direct).
    auto raise = [&](uint32_t pushed) {
#pragma unroll
      for (int t = 0; t < NTP; ++t) {
        const int c = __popc(__ballot_sync(0xffffffffu, (pushed >> t) & 1u));
        if (lane == t) pend += c;
      }
      gmt_flush(P, A.B, A.t0);
      const uint32_t due = __ballot_sync(0xffffffffu, lane < NTP && pend >= 16);
      if (lane < NTP && pend >= 16) pend = 0;
      for (int t = 0; t < NTP; ++t)
        if (due & (1u << t)) refresh_theta(A.B, A.t0 + t, A.k);
      if (due) {
        for (int t = lane; t < NTP; t += 32) theta[t] = t < A.T ? ld_relaxed(&A.B.theta[A.t0 + t]) : 0.f;
        __syncwarp();
      }
    };
    raise(own ? gmt_pair<0>(A, GA, ls, i, j0, Fi, run, sh.ysum, theta, py, P) : 0u);
    raise(own ? gmt_pair<1>(A, GA, ls, i, j0 + 1, Fi, run, sh.ysum, theta, py, P) : 0u);
    static_assert(BPW == 2, "b-features per epilogue warp");
  }
  flush_stats(A, ls);
}

// CL = 2: the two CTAs of a cluster take the two tiles of a pair (the same
// b-block, two a-blocks): each copies its own a-image chunk and one half
// (BF16 hi or lo part) of the shared b-image chunk, multicast into both
// CTAs' stages, so the b-side is read from L2 once per pair; a stage is
// refilled once both CTAs' MMAs have released it (each MMA commit arrives on
// the empty barriers of both CTAs).  CL = 1: one CTA per tile.
template <int CL>
__global__ void __launch_bounds__(gmt::THREADS, 1) k_pair_gmt(const ScreenArgs A, const GmtArgs GA) {
  using namespace gmt;
  using namespace tc;
  static_assert(CL == 1 || CL == 2, "clusters of one or two CTAs");
  extern __shared__ __align__(1024) unsigned char smem[];
  Shared &sh = *reinterpret_cast<Shared *>(smem);
  unsigned char *stages = smem + shared_bytes();
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int nchunks = GA.nchunks, nblocks = GA.nblocks;
  const uint32_t crank = CL == 2 ? cluster_ctarank() : 0u;

  if (threadIdx.x == 0) {
    for (int s = 0; s < NS; ++s) {
      mbar_init(&sh.full[s], 1);
      mbar_init(&sh.empty[s], CL);
    }
    for (int b = 0; b < 2; ++b) {
      mbar_init(&sh.acc_full[b], 1);
      mbar_init(&sh.acc_empty[b], EPI);
    }
    mbar_init(&sh.drain, 1);
    sh.abort = 0;
    mbar_fence_init();
  }
  if (threadIdx.x < NTP) sh.ysum[threadIdx.x] = (int)threadIdx.x < A.T ? A.ysum32[A.t0 + threadIdx.x] : 0.f;
  if (warp == 1) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&sh.tmem_base)),
                 "r"((uint32_t)TMEM_COLS)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  fence_before();
  __syncthreads();
  fence_after();
  // (the peer's barriers are initialised before any copy or commit reaches them)
  if (CL == 2) cluster_sync_all();
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
        if (tl.x < 0) tl.x = 0;  // the empty partner of a pair: any a-block, nothing is scored
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
          const unsigned char *bsrc = GA.bimg + ((size_t)tl.y * nchunks + c) * B_IMG;
          if (CL == 2)
            bulk_g2s_mc(S + A_IMG + crank * B_PART, bsrc + crank * B_PART, B_PART, &sh.full[st], (uint16_t)3);
          else
            bulk_g2s(S + A_IMG, bsrc, B_IMG, &sh.full[st]);
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
      constexpr uint32_t IDESC1 = idesc_bf16(128, N1), IDESC2 = idesc_bf16(128, NG);
      int lt = 0;
      bool ok = true;
      for (int tile = blockIdx.x; ok && tile < GA.n_tiles && !*abort_flag; tile += gridDim.x, ++lt) {
        for (int b = 0; ok && b < nblocks; ++b) {
          const uint32_t gb = (uint32_t)lt * nblocks + b, set = gb & 1, ub = gb >> 1;
          if (ub >= 1 && !wait(&sh.acc_empty[set], (ub - 1) & 1)) {
            ok = false;
            break;
          }
          fence_after();
          const uint32_t d = tmem + set * SET;
          const int c0 = b * DB, c1 = min(nchunks, c0 + DB);
          for (int c = c0; c < c1; ++c) {
            const uint32_t gc = (uint32_t)lt * nchunks + c, st = gc % NS, u = gc / NS;
            if (!wait(&sh.full[st], u & 1)) {
              ok = false;
              break;
            }
            fence_after();
            const uint32_t S = smem_u32(stages + (size_t)st * STAGE);
            const uint32_t ph = S, p2h = S + A_PART, pl = S + 2 * A_PART, p2l = S + 3 * A_PART;
            const uint32_t bh = S + A_IMG, bl = bh + B_PART;
#pragma unroll
            for (int kk = 0; kk < KC / 16; ++kk) {
              const uint32_t koff = kk * 2 * LBO;
              const uint32_t acc = (c == c0 && kk == 0) ? 0u : 1u;
              mma_bf16(d, smem_desc(ph + koff), smem_desc(bh + koff), IDESC1, acc);
              mma_bf16(d + N1, smem_desc(p2h + koff), smem_desc(bh + G_OFF + koff), IDESC2, acc);
              mma_bf16(d, smem_desc(ph + koff), smem_desc(bl + koff), IDESC1, 1u);
              mma_bf16(d + N1, smem_desc(p2h + koff), smem_desc(bl + G_OFF + koff), IDESC2, 1u);
              mma_bf16(d, smem_desc(pl + koff), smem_desc(bh + koff), IDESC1, 1u);
              mma_bf16(d + N1, smem_desc(p2l + koff), smem_desc(bh + G_OFF + koff), IDESC2, 1u);
            }
            if (CL == 2)
              mma_commit_mc(&sh.empty[st], (uint16_t)3);
            else
              mma_commit(&sh.empty[st]);
          }
          if (!ok) break;
          mma_commit(&sh.acc_full[set]);
        }
      }
      // every MMA issued has completed before TMEM is freed
      mma_commit(&sh.drain);
      mbar_wait_bounded(&sh.drain, 0, kWait);
    }
  } else {
    // ------------------------------------------------------------ epilogue
    const int ew = warp - 2;  // 0 .. EPI-1
    const int q = warp & 3;   // TMEM lane quadrant = a-features 32 q .. 32 q + 31
    gmt_epilogue(A, GA, sh, tmem, q, ew, ew >> 2, wait_warp, aborted_warp);
  }
  fence_before();
  __syncthreads();
  fence_after();
  if (warp == 1)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"((uint32_t)TMEM_COLS) : "memory");
  // neither CTA leaves while the other's copies or commits may still reach it
  if (CL == 2) cluster_sync_all();
}

// ------------------------------------------------------------------- host

// Whether a per-target screen of T targets may take this path.
bool gmt_eligible(int T, int64_t N) { return T >= 2 && T <= gmt::NTP && N >= 16; }

static int64_t gmt_chunks(int64_t N) { return (N + tc::KC - 1) / tc::KC; }
static int64_t gmt_na(int64_t n) { return (n + gmt::FA - 1) / gmt::FA; }
static int64_t gmt_nb(int64_t n) { return (n + gmt::FB - 1) / gmt::FB; }

size_t gmt_space_bytes(int64_t n, int64_t N) {
  return (size_t)gmt_na(n) * gmt_chunks(N) * gmt::A_IMG + (size_t)n * sizeof(GramFeat) + 256;
}

size_t gmt_screen_bytes(int64_t n, int64_t N) {
  return (size_t)gmt_nb(n) * gmt_chunks(N) * gmt::B_IMG + (size_t)n * sizeof(GmtTgt) +
         gmt_part_count(n, N) * sizeof(GmtPart) + 512;
}

// Space part: a-images and feature sums, built once per space into `buf`
// (gmt_space_bytes).  Every byte of the images is written (zero rows for
// the slots past n), so no clearing pass is needed.
void gmt_build_space(const FeatTable &F, void *buf, cudaStream_t st) {
  const int64_t n = F.n, N = F.N;
  const int nchunks = (int)gmt_chunks(N);
  unsigned char *aimg = static_cast<unsigned char *>(buf);
  GramFeat *gf = reinterpret_cast<GramFeat *>(aimg + (size_t)gmt_na(n) * nchunks * gmt::A_IMG);
  note_launches(1);
  k_gmt_space<<<(unsigned)(gmt_na(n) * gmt::FA), 128, 0, st>>>(F, nchunks, aimg, gf);
}

// One screen's b-images and target sums into `scr` (gmt_screen_bytes):
// the images with the blocks' partial sums, then the sums.
void launch_gmt_brows(const ScreenArgs &A, const void *space_buf, void *scr, cudaStream_t st) {
  const int64_t n = A.F.n, N = A.N;
  const int nchunks = (int)gmt_chunks(N);
  const int ncb = (nchunks + kBrowsCh - 1) / kBrowsCh;
  const unsigned char *aimg = static_cast<const unsigned char *>(space_buf);
  const GramFeat *gf = reinterpret_cast<const GramFeat *>(aimg + (size_t)gmt_na(n) * nchunks * gmt::A_IMG);
  unsigned char *bimg = static_cast<unsigned char *>(scr);
  GmtTgt *gt = reinterpret_cast<GmtTgt *>(bimg + (size_t)gmt_nb(n) * nchunks * gmt::B_IMG);
  GmtPart *part = reinterpret_cast<GmtPart *>(reinterpret_cast<unsigned char *>(gt) +
                                              ((size_t)n * sizeof(GmtTgt) + 255) / 256 * 256);
  note_launches(2);
  k_gmt_brows<<<dim3((unsigned)gmt_nb(n), (unsigned)ncb), 256, 0, st>>>(A.F, nchunks, A.y32 + (int64_t)A.t0 * A.ldy,
                                                                      A.ldy, A.T, gf, bimg, part);
  k_gmt_tsum<<<(unsigned)n, 64, 0, st>>>(n, ncb, part, (int64_t)nchunks * (tc::KC / 8), gt);
}

// The tiles (a-block, b-block) holding an ordered pair (i, j), i != j, of a
// candidate of the binary block of rung k with an id in [id_begin, id_end),
// in groups of `group` consecutive a-blocks, b-block major within a group
// (the CTAs working at one time share b-images and sweep the group's
// a-images together).  The test is conservative: the pairs of a tile have
// max(i, j) in [max(a0, b0), max(a1, b1)].
void gmt_tiles(const dse_space *sp, uint64_t id_begin, uint64_t id_end, std::vector<int2> &out) {
  const RungGeom &g = sp->geom;
  const int64_t n = sp->n, o = g.o;
  out.clear();
  if (g.nb == 0 || n < 2) return;
  const uint64_t p_lo = id_begin > (uint64_t)sp->n ? id_begin - (uint64_t)sp->n : 0;
  const uint64_t p_hi = id_end > (uint64_t)sp->n ? id_end - (uint64_t)sp->n : 0;
  if (p_hi <= p_lo) return;
  auto pidx = [&](int64_t i, int64_t j) { return g.um + (tri((uint64_t)i) + (uint64_t)j - g.tri_o) * (uint64_t)g.nb; };
  const int64_t na = gmt_na(n), nb = gmt_nb(n);
  // (an even group: the tiles of a b-block within a group pair up for the
  // two CTAs of a cluster)
  int64_t group = std::max(1, tuning().gmt_group);
  group += group & 1;
  std::vector<int> as;
  for (int64_t ga = 0; ga < na; ga += group) {
    for (int64_t c = 0; c < nb; ++c) {
      const int64_t b0 = c * gmt::FB, b1 = std::min<int64_t>(b0 + gmt::FB, n) - 1;
      as.clear();
      for (int64_t a = ga; a < std::min(na, ga + group); ++a) {
        const int64_t a0 = a * gmt::FA, a1 = std::min<int64_t>(a0 + gmt::FA, n) - 1;
        const int64_t Ilo = std::max<int64_t>(std::max(a0, b0), std::max<int64_t>(o, 1));
        const int64_t Ihi = std::max(a1, b1);
        if (Ilo > Ihi) continue;
        if (a0 == b1 && a1 == b0) continue;  // a single feature on both sides: only i == j
        const uint64_t lo = pidx(Ilo, 0), hi = pidx(Ihi, Ihi - 1) + (uint64_t)g.nb;
        if (hi <= p_lo || lo >= p_hi) continue;
        as.push_back((int)a);
      }
      if (as.size() & 1) as.push_back(-1);  // an empty partner: the pair's second tile scores nothing
      for (int a : as) out.push_back(make_int2(a, (int)c));
    }
  }
}

// delta of the contraction entries for N samples: BF16x3 split, the
// tensor-core accumulation model of one block (2u per step x 4, steps = 3
// products x 2 k-steps x the block's chunks), one rounding of each squared
// or target-weighted row, and the FP32 sum of the block partials.
float gmt_delta(int64_t N) {
  const double u32 = 5.9604644775390625e-8;
  const int64_t nchunks = gmt_chunks(N);
  const int64_t per_block = std::min<int64_t>(nchunks, gmt::DB);
  const int64_t nblocks = (nchunks + gmt::DB - 1) / gmt::DB;
  const double steps = 3.0 * (tc::KC / 16) * (double)per_block;
  return (float)(4.0 * (2.0 * steps + 2.0) * u32 + 3.02 * 1.52587890625e-5 + 4.0 * u32 + 1.01 * (double)nblocks * u32);
}

// One screen's binary slots for T <= 16 targets: the kernel over `tiles`
// (device, n_tiles) after launch_gmt_brows.
dse_status launch_pair_gmt(const ScreenArgs &A, const void *space_buf, void *scr, const int2 *tiles, int n_tiles,
                           int sms, cudaStream_t st) {
  if (n_tiles <= 0) return DSE_OK;
  const int64_t n = A.F.n, N = A.N;
  const int nchunks = (int)gmt_chunks(N);
  const unsigned char *aimg = static_cast<const unsigned char *>(space_buf);
  const GramFeat *gf = reinterpret_cast<const GramFeat *>(aimg + (size_t)gmt_na(n) * nchunks * gmt::A_IMG);
  const unsigned char *bimg = static_cast<const unsigned char *>(scr);
  const GmtTgt *gt = reinterpret_cast<const GmtTgt *>(bimg + (size_t)gmt_nb(n) * nchunks * gmt::B_IMG);
  note_launches(1);
  // pairs of CTAs per cluster where the device co-schedules them (the count
  // of clusters that fit at once, per device)
  static int clusters[64] = {0};
  int dev = 0;
  cudaGetDevice(&dev);
  if (clusters[dev & 63] == 0) {
    DSE_CUDA(cudaFuncSetAttribute(k_pair_gmt<1>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)gmt::smem_total()));
    DSE_CUDA(cudaFuncSetAttribute(k_pair_gmt<2>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)gmt::smem_total()));
    cudaLaunchConfig_t q = {};
    cudaLaunchAttribute qa[1];
    qa[0].id = cudaLaunchAttributeClusterDimension;
    qa[0].val.clusterDim.x = 2;
    qa[0].val.clusterDim.y = 1;
    qa[0].val.clusterDim.z = 1;
    q.gridDim = dim3((unsigned)(sms - sms % 2));
    q.blockDim = dim3(gmt::THREADS);
    q.dynamicSmemBytes = gmt::smem_total();
    q.attrs = qa;
    q.numAttrs = 1;
    int nc = 0;
    if (cudaOccupancyMaxActiveClusters(&nc, k_pair_gmt<2>, &q) != cudaSuccess || nc < 1) {
      cudaGetLastError();
      nc = -1;  // no clusters: one CTA per tile
    }
    clusters[dev & 63] = nc;
  }
  GmtArgs GA{aimg, bimg, gf, gt, tiles, n_tiles, nchunks, (nchunks + gmt::DB - 1) / gmt::DB, gmt_delta(N),
             (int)gmt_na(n), (int)gmt_nb(n)};
  ScreenArgs B = A;
  B.group = 1;
  // (a spread sample of tiles launched first does not help here: a streaming
  // top-k over candidates in arbitrary order buffers about k (1 + ln(n / k))
  // entries per list whatever the start, and the sample's thresholds rise
  // no faster)
  const int nc = clusters[dev & 63];
  if (tuning().gmt_cluster == 2 && nc > 0 && n_tiles % 2 == 0) {
    // the tile list holds pairs (2p, 2p + 1) of one b-block; CTA x of the
    // grid takes tiles x, x + grid, ..., so both CTAs of a cluster take the
    // two tiles of the same pairs
    int grid = 2 * nc;
    if (grid > n_tiles) grid = n_tiles;
    cudaLaunchConfig_t cfg = {};
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeClusterDimension;
    at[0].val.clusterDim.x = 2;
    at[0].val.clusterDim.y = 1;
    at[0].val.clusterDim.z = 1;
    cfg.gridDim = dim3((unsigned)grid);
    cfg.blockDim = dim3(gmt::THREADS);
    cfg.dynamicSmemBytes = gmt::smem_total();
    cfg.stream = st;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    DSE_CUDA(cudaLaunchKernelEx(&cfg, k_pair_gmt<2>, B, GA));
    return DSE_OK;
  }
  const int grid = sms < n_tiles ? sms : n_tiles;
  k_pair_gmt<1><<<grid, gmt::THREADS, gmt::smem_total(), st>>>(B, GA);
  return DSE_OK;
}

}  // namespace dse
