// l0.cu -- exhaustive L0 search over a listed subspace (Eq. 1 solved exactly
// over the candidates SIS retained: SISSO's sparsifying step).
//
// For every D-subset {p_0 < .. < p_{D-1}} of the n listed candidates, the
// least-squares fit with intercept of y; the best subsets by RMSE.  With the
// candidates' centred columns X (n x N) and the centred target, the fit of a
// subset explains q = b_S^T G_SS^{-1} b_S of Syy (G = X X^T, b = X y), so
// the search is a scan of small Cholesky factorisations over the Gram
// matrix:
//   1. columns, centring, b and raw norms (one block per candidate);
//   2. the Gram matrix G (tiled, FP64; the dense contraction of the step);
//   3. the scan: D = 1 thread per candidate, D = 2 thread per pair, D = 3
//      warp per pair (p_0, p_1) with lanes over p_2 -- an incremental
//      Cholesky step per subset -- keeping each warp's 32 best (q, subset)
//      in registers across its lanes, then each block's 32 best;
//   4. the 32 best of all blocks (one block), then an explicit FP64 refit
//      of each (coefficients and the RMSE of the explicit residual) whose
//      order (RMSE, positions) decides.
// The rank rule is that of the refits: a pivot of the centred Cholesky at
// or below 1e-12 of the raw column's norm rejects the subset, with the
// pivots taken in position order (as a QR of [1, X_p0, X_p1, ...] would).
#include <math.h>
#include <string.h>

#include <algorithm>
#include <vector>

#include "dse_internal.cuh"
#include "eval64.cuh"
#include "plan.cuh"
#include "util.cuh"

namespace dse {

FeatTable table_of(const dse_space *S);

namespace {

constexpr int kTop = 32;        // subsets kept per warp / block / search
constexpr int kCol = 128;       // threads per column block
constexpr double kRank2 = 1e-24;  // (1e-12)^2: squared pivot / squared raw norm

__device__ __forceinline__ double col_value64(const FeatTable &F, const RungGeom &G, int64_t n_stored, uint64_t gid,
                                              int64_t s) {
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

template <int NV>
__device__ __forceinline__ void block_sum(double (&v)[NV], double *sm) {
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
#pragma unroll
  for (int i = 0; i < NV; ++i) v[i] = warp_sum64(v[i]);
  if (lane == 0)
#pragma unroll
    for (int i = 0; i < NV; ++i) sm[w * NV + i] = v[i];
  __syncthreads();
#pragma unroll
  for (int i = 0; i < NV; ++i) {
    double t = 0.0;
    for (int ww = 0; ww < (int)(blockDim.x >> 5); ++ww) t += sm[ww * NV + i];
    v[i] = t;
  }
  __syncthreads();
}

// Centred target and Syy (one block).
__global__ void __launch_bounds__(kCol) k_l0_target(const double *y, int64_t N, double *yc, double *syy,
                                                    double *ymean) {
  __shared__ double sm[(kCol / 32) * 2];
  double s[1] = {0.0};
  for (int64_t i = threadIdx.x; i < N; i += kCol) s[0] += y[i];
  block_sum<1>(s, sm);
  const double my = s[0] / (double)N;
  double q[1] = {0.0};
  for (int64_t i = threadIdx.x; i < N; i += kCol) {
    const double d = y[i] - my;
    yc[i] = d;
    q[0] = fma(d, d, q[0]);
  }
  block_sum<1>(q, sm);
  if (threadIdx.x == 0) {
    *syy = q[0];
    *ymean = my;
  }
}

// Column c: values, centred in X[c], raw sum of squares, b_c = X_c . yc, mean.
// An id outside the space gives a zero column (rejected by the rank rule).
__global__ void __launch_bounds__(kCol) k_l0_columns(FeatTable F, RungGeom G, int64_t n_stored, const uint64_t *ids,
                                                     int64_t n, const double *yc, double *X, double *nrm2, double *b,
                                                     double *mean) {
  __shared__ double sm[(kCol / 32) * 2];
  const int64_t c = blockIdx.x;
  if (c >= n) return;
  const int64_t N = F.N;
  const bool in_space = ids[c] < (uint64_t)n_stored + G.slots;
  double *x = X + c * N;
  double s[2] = {0.0, 0.0};
  for (int64_t i = threadIdx.x; i < N; i += kCol) {
    const double v = in_space ? col_value64(F, G, n_stored, ids[c], i) : 0.0;
    x[i] = v;
    s[0] += v;
    s[1] = fma(v, v, s[1]);
  }
  block_sum<2>(s, sm);
  const double m = s[0] / (double)N;
  double t[1] = {0.0};
  for (int64_t i = threadIdx.x; i < N; i += kCol) {
    const double d = x[i] - m;
    x[i] = d;
    t[0] = fma(d, yc[i], t[0]);
  }
  block_sum<1>(t, sm);
  if (threadIdx.x == 0) {
    nrm2[c] = s[1];
    b[c] = t[0];
    mean[c] = m;
  }
}

// Gram matrix of the centred columns: one 32 x 32 tile (bi <= bj) per block
// of 256 threads, 2 x 2 outputs per thread, samples staged in 32-sample
// slices through shared memory; both G[i][j] and G[j][i] are written.
constexpr int kGT = 32, kGS = 32;
__global__ void __launch_bounds__(256) k_l0_gram(const double *X, int64_t n, int64_t N, int64_t nt, double *Gm) {
  __shared__ double xi[kGT][kGS + 1], xj[kGT][kGS + 1];
  // tile index -> (bi, bj), bi <= bj, over the upper triangle of nt x nt tiles
  // tile t of the triangle with the diagonal: t = bj (bj + 1) / 2 + bi, bi <= bj
  const int64_t t = blockIdx.x;
  uint64_t bj = (uint64_t)((sqrt(8.0 * (double)t + 1.0) - 1.0) * 0.5);
  while ((bj + 1) * (bj + 2) / 2 <= (uint64_t)t) ++bj;
  while (bj * (bj + 1) / 2 > (uint64_t)t) --bj;
  const uint64_t bi = (uint64_t)t - bj * (bj + 1) / 2;
  const int64_t i0 = (int64_t)bi * kGT, j0 = (int64_t)bj * kGT;
  const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;  // 16 x 16 threads, 2 x 2 outputs each
  double acc[2][2] = {{0.0, 0.0}, {0.0, 0.0}};
  for (int64_t s0 = 0; s0 < N; s0 += kGS) {
    for (int e = threadIdx.x; e < kGT * kGS; e += 256) {
      const int r2 = e / kGS, k = e % kGS;
      const int64_t s = s0 + k;
      xi[r2][k] = (i0 + r2 < n && s < N) ? X[(i0 + r2) * N + s] : 0.0;
      xj[r2][k] = (j0 + r2 < n && s < N) ? X[(j0 + r2) * N + s] : 0.0;
    }
    __syncthreads();
#pragma unroll 8
    for (int k = 0; k < kGS; ++k) {
      const double a0 = xi[ty * 2][k], a1 = xi[ty * 2 + 1][k];
      const double b0 = xj[tx * 2][k], b1 = xj[tx * 2 + 1][k];
      acc[0][0] = fma(a0, b0, acc[0][0]);
      acc[0][1] = fma(a0, b1, acc[0][1]);
      acc[1][0] = fma(a1, b0, acc[1][0]);
      acc[1][1] = fma(a1, b1, acc[1][1]);
    }
    __syncthreads();
  }
#pragma unroll
  for (int a = 0; a < 2; ++a)
#pragma unroll
    for (int c2 = 0; c2 < 2; ++c2) {
      const int64_t i = i0 + ty * 2 + a, j = j0 + tx * 2 + c2;
      if (i < n && j < n) {
        Gm[i * n + j] = acc[a][c2];
        Gm[j * n + i] = acc[a][c2];
      }
    }
}

// (q, subset) ordering: larger explained q first, then positions ascending
// (packed 21 bits each, lexicographic as one integer).
struct Hit {
  double q;
  uint64_t key;
};
__device__ __forceinline__ bool better(double qa, uint64_t ka, double qb, uint64_t kb) {
  return qa > qb || (qa == qb && ka < kb);
}
__device__ __forceinline__ uint64_t pack3(int64_t p0, int64_t p1, int64_t p2) {
  return ((uint64_t)p0 << 42) | ((uint64_t)p1 << 21) | (uint64_t)p2;
}

// A warp's 32 best, one per lane: insert the lanes' candidates in `pass`.
struct WarpTop {
  double q;       // this lane's slot
  uint64_t key;
  double wq;      // the warp's worst slot (broadcast)
  uint64_t wkey;
  int wlane;
  __device__ void init() {
    q = -1.0;
    key = ~0ull;
    wq = -1.0;
    wkey = ~0ull;
    wlane = 0;
  }
  __device__ void worst() {
    // argmin over lanes of the ordering
    double mq = q;
    uint64_t mk = key;
    int ml = threadIdx.x & 31;
    for (int o = 16; o > 0; o >>= 1) {
      const double oq = __shfl_xor_sync(0xffffffffu, mq, o);
      const uint64_t ok = __shfl_xor_sync(0xffffffffu, mk, o);
      const int ol = __shfl_xor_sync(0xffffffffu, ml, o);
      if (better(mq, mk, oq, ok) || (mq == oq && mk == ok && ol < ml)) {
        mq = oq;
        mk = ok;
        ml = ol;
      }
    }
    wq = mq;
    wkey = mk;
    wlane = ml;
  }
  // every lane calls; cq/ck are this lane's candidate, valid if `has`
  __device__ void offer(bool has, double cq, uint64_t ck) {
    const int lane = threadIdx.x & 31;
    unsigned m = __ballot_sync(0xffffffffu, has && better(cq, ck, wq, wkey));
    while (m) {
      const int src = __ffs(m) - 1;
      m &= m - 1;
      const double sq = __shfl_sync(0xffffffffu, cq, src);
      const uint64_t sk = __shfl_sync(0xffffffffu, ck, src);
      if (better(sq, sk, wq, wkey)) {
        if (lane == wlane) {
          q = sq;
          key = sk;
        }
        worst();
      }
    }
  }
};

// Explained sum of squares of the subset, in position order (p0 < p1 < p2):
// incremental Cholesky of the centred Gram submatrix; -1 if a pivot fails
// the rank rule.
__device__ __forceinline__ double explained1(const double *Gm, const double *b, const double *nrm2, int64_t n,
                                             int64_t p0, double *L11, double *z1) {
  const double g = Gm[p0 * n + p0];
  if (!(g > kRank2 * nrm2[p0])) return -1.0;
  *L11 = sqrt(g);
  *z1 = b[p0] / *L11;
  return *z1 * *z1;
}

// Scan of every D-subset; each block writes its kTop best to out[block].
template <int D>
__global__ void __launch_bounds__(256) k_l0_scan(const double *Gm, const double *b, const double *nrm2, int64_t n,
                                                 Hit *out) {
  __shared__ Hit sh[8 * 32];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  WarpTop top;
  top.init();
  if (D == 1) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    const int64_t base0 = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    for (int64_t base = base0 - lane; base < n; base += stride) {
      const int64_t p = base + lane;
      double q = -1.0, L, z;
      if (p < n) q = explained1(Gm, b, nrm2, n, p, &L, &z);
      top.offer(q >= 0.0, q, pack3(p, 0, 0));
    }
  } else if (D == 2) {
    const uint64_t npairs = (uint64_t)n * (uint64_t)(n - 1) / 2;
    const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    const uint64_t base0 = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x - lane;
    for (uint64_t base = base0; base < npairs; base += stride) {
      const uint64_t idx = base + lane;
      double q = -1.0;
      uint64_t key = ~0ull;
      if (idx < npairs) {
        uint64_t hi, lo;
        pair_from_index(idx, &hi, &lo);  // lo < hi
        const int64_t p0 = (int64_t)lo, p1 = (int64_t)hi;
        double L11, z1;
        const double q1 = explained1(Gm, b, nrm2, n, p0, &L11, &z1);
        if (q1 >= 0.0) {
          const double L21 = Gm[p1 * n + p0] / L11;
          const double d = Gm[p1 * n + p1] - L21 * L21;
          if (d > kRank2 * nrm2[p1]) {
            const double z2 = (b[p1] - L21 * z1) / sqrt(d);
            q = q1 + z2 * z2;
            key = pack3(p0, p1, 0);
          }
        }
      }
      top.offer(q >= 0.0, q, key);
    }
  } else {
    // warp per pair (p0 < p1); lanes over p2 > p1
    const uint64_t npairs = (uint64_t)n * (uint64_t)(n - 1) / 2;
    const uint64_t warps = ((uint64_t)gridDim.x * blockDim.x) >> 5;
    for (uint64_t w = ((uint64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; w < npairs; w += warps) {
      uint64_t hi, lo;
      pair_from_index(w, &hi, &lo);
      const int64_t p0 = (int64_t)lo, p1 = (int64_t)hi;
      if (p1 + 1 >= n) continue;
      double L11, z1;
      const double q1 = explained1(Gm, b, nrm2, n, p0, &L11, &z1);
      if (q1 < 0.0) continue;
      const double L21 = Gm[p1 * n + p0] / L11;
      const double d2 = Gm[p1 * n + p1] - L21 * L21;
      if (!(d2 > kRank2 * nrm2[p1])) continue;
      const double L22 = sqrt(d2);
      const double z2 = (b[p1] - L21 * z1) / L22;
      const double q2 = q1 + z2 * z2;
      const double i11 = 1.0 / L11, i22 = 1.0 / L22;
      const double *g0 = Gm + p0 * n, *g1 = Gm + p1 * n;
      for (int64_t base = p1 + 1; base < n; base += 32) {
        const int64_t p2 = base + lane;
        double q = -1.0;
        if (p2 < n) {
          const double L31 = g0[p2] * i11;
          const double L32 = (g1[p2] - L31 * L21) * i22;
          const double d3 = Gm[p2 * n + p2] - L31 * L31 - L32 * L32;
          if (d3 > kRank2 * nrm2[p2]) {
            const double t = b[p2] - L31 * z1 - L32 * z2;
            q = q2 + t * t / d3;
          }
        }
        top.offer(q >= 0.0, q, pack3(p0, p1, p2));
      }
    }
  }
  // the block's kTop best: sort the 8 warps' 256 entries
  sh[warp * 32 + lane] = Hit{top.q, top.key};
  __syncthreads();
  for (int size = 2; size <= 256; size <<= 1)
    for (int stride = size >> 1; stride > 0; stride >>= 1) {
      const int i = threadIdx.x, j = i ^ stride;
      if (j > i) {
        const bool up = (i & size) == 0;
        const Hit a = sh[i], c = sh[j];
        const bool sw = up ? better(c.q, c.key, a.q, a.key) : better(a.q, a.key, c.q, c.key);
        if (sw) {
          sh[i] = c;
          sh[j] = a;
        }
      }
      __syncthreads();
    }
  if (threadIdx.x < kTop) out[(size_t)blockIdx.x * kTop + threadIdx.x] = sh[threadIdx.x];
}

// The kTop best of all blocks (one block; nb * kTop <= 8192 entries).
__global__ void __launch_bounds__(1024) k_l0_merge(Hit *in, int64_t m, Hit *best) {
  extern __shared__ Hit hs[];
  int64_t M = 1;
  while (M < m) M <<= 1;
  for (int64_t i = threadIdx.x; i < M; i += blockDim.x) hs[i] = i < m ? in[i] : Hit{-1.0, ~0ull};
  __syncthreads();
  for (int64_t size = 2; size <= M; size <<= 1)
    for (int64_t stride = size >> 1; stride > 0; stride >>= 1) {
      for (int64_t i = threadIdx.x; i < M; i += blockDim.x) {
        const int64_t j = i ^ stride;
        if (j > i) {
          const bool up = (i & size) == 0;
          const Hit a = hs[i], c = hs[j];
          const bool sw = up ? better(c.q, c.key, a.q, a.key) : better(a.q, a.key, c.q, c.key);
          if (sw) {
            hs[i] = c;
            hs[j] = a;
          }
        }
      }
      __syncthreads();
    }
  if (threadIdx.x < kTop) best[threadIdx.x] = hs[threadIdx.x];
}

// Explicit FP64 refit of each kept subset (one block each): coefficients
// from the centred Cholesky, RMSE of the explicit residual.
__global__ void __launch_bounds__(kCol) k_l0_refit(const Hit *best, int D, const double *X, const double *yc,
                                                   const double *mean, const double *Gm, const double *b,
                                                   const double *nrm2, int64_t n, int64_t N, double my,
                                                   double *rmse, double *coef) {
  __shared__ double sm[(kCol / 32) * 2];
  const Hit h = best[blockIdx.x];
  int64_t p[3];
  p[0] = (int64_t)((h.key >> 42) & 0x1FFFFF);
  p[1] = (int64_t)((h.key >> 21) & 0x1FFFFF);
  p[2] = (int64_t)(h.key & 0x1FFFFF);
  bool ok = h.q >= 0.0;
  double beta[4] = {0, 0, 0, 0};
  if (ok) {
    double L[3][3] = {}, z[3];
    for (int c = 0; c < D && ok; ++c) {
      double dsum = Gm[p[c] * n + p[c]];
      for (int k = 0; k < c; ++k) dsum -= L[c][k] * L[c][k];
      if (!(dsum > kRank2 * nrm2[p[c]])) {
        ok = false;
        break;
      }
      L[c][c] = sqrt(dsum);
      for (int r = c + 1; r < D; ++r) {
        double v = Gm[p[r] * n + p[c]];
        for (int k = 0; k < c; ++k) v -= L[r][k] * L[c][k];
        L[r][c] = v / L[c][c];
      }
    }
    if (ok) {
      for (int c = 0; c < D; ++c) {
        double v = b[p[c]];
        for (int k = 0; k < c; ++k) v -= L[c][k] * z[k];
        z[c] = v / L[c][c];
      }
      for (int c = D - 1; c >= 0; --c) {
        double v = z[c];
        for (int k = c + 1; k < D; ++k) v -= L[k][c] * beta[k + 1];
        beta[c + 1] = v / L[c][c];
      }
      double b0 = my;
      for (int c = 0; c < D; ++c) b0 -= beta[c + 1] * mean[p[c]];
      beta[0] = b0;
    }
  }
  double rss[1] = {0.0};
  if (ok)
    for (int64_t s = threadIdx.x; s < N; s += kCol) {
      double r = yc[s];
      for (int c = 0; c < D; ++c) r = fma(-beta[c + 1], X[p[c] * N + s], r);
      rss[0] = fma(r, r, rss[0]);
    }
  block_sum<1>(rss, sm);
  if (threadIdx.x == 0) {
    rmse[blockIdx.x] = ok ? sqrt(rss[0] / (double)N) : INFINITY;
    for (int c = 0; c < 4; ++c) coef[blockIdx.x * 4 + c] = ok ? beta[c] : 0.0;
  }
}

}  // namespace

dse_status l0_search_impl(dse_space *sp, const dse_l0_desc *d, int64_t *top_pos, double *top_rmse, double *top_coefs,
                          int32_t *n_found) {
  cudaStream_t st = (cudaStream_t)d->stream;
  const int64_t n = d->n_ids, N = sp->N;
  const int D = d->dim;
  const uint64_t total = (uint64_t)sp->n + sp->geom.slots;
  if (!d->ids_on_device)
    for (int64_t i = 0; i < n; ++i)
      if (d->ids[i] >= total) {
        set_error("candidate id %llu out of range", (unsigned long long)d->ids[i]);
        return DSE_ERANGE;
      }
  const int64_t nt = (n + kGT - 1) / kGT;
  const int sms = sm_count();
  const int nb = std::min<int64_t>(2 * sms, 8192 / kTop);  // scan blocks (their kTop bests fit the merge)
  // scratch
  double *yd = nullptr, *yc = nullptr, *syy = nullptr, *ym = nullptr, *X = nullptr, *nrm2 = nullptr, *bv = nullptr, *mean = nullptr,
         *Gm = nullptr, *rm = nullptr, *cf = nullptr;
  uint64_t *ids = nullptr;
  Hit *part = nullptr, *best = nullptr;
  Scratch sc;
  if (!d->y_on_device) sc.add(&yd, (size_t)N);
  if (!d->ids_on_device) sc.add(&ids, (size_t)n);
  sc.add(&yc, (size_t)N);
  sc.add(&syy, 1);
  sc.add(&ym, 1);
  sc.add(&X, (size_t)n * N);
  sc.add(&nrm2, (size_t)n);
  sc.add(&bv, (size_t)n);
  sc.add(&mean, (size_t)n);
  sc.add(&Gm, (size_t)n * n);
  sc.add(&part, (size_t)nb * kTop);
  sc.add(&best, kTop);
  sc.add(&rm, kTop);
  sc.add(&cf, (size_t)kTop * 4);
  void *base = nullptr;
  size_t bytes = 0;
  DSE_TRY(sc.alloc(&base, &bytes));
  struct Free {
    void *p;
    ~Free() { dfree(p); }
  } fr{base};
  const double *y = d->y;
  if (!d->y_on_device) {
    DSE_CUDA(cudaMemcpyAsync(yd, d->y, 8 * N, cudaMemcpyHostToDevice, st));
    y = yd;
  }
  const uint64_t *idp = d->ids;
  if (!d->ids_on_device) {
    DSE_CUDA(cudaMemcpyAsync(ids, d->ids, 8 * n, cudaMemcpyHostToDevice, st));
    idp = ids;
  }
  const FeatTable F = table_of(sp);
  note_launches(6);
  k_l0_target<<<1, kCol, 0, st>>>(y, N, yc, syy, ym);
  k_l0_columns<<<(unsigned)n, kCol, 0, st>>>(F, sp->geom, sp->n, idp, n, yc, X, nrm2, bv, mean);
  k_l0_gram<<<(unsigned)(nt * (nt + 1) / 2), 256, 0, st>>>(X, n, N, nt, Gm);
  if (D == 1) k_l0_scan<1><<<nb, 256, 0, st>>>(Gm, bv, nrm2, n, part);
  else if (D == 2) k_l0_scan<2><<<nb, 256, 0, st>>>(Gm, bv, nrm2, n, part);
  else k_l0_scan<3><<<nb, 256, 0, st>>>(Gm, bv, nrm2, n, part);
  {
    int64_t M = 1;
    while (M < (int64_t)nb * kTop) M <<= 1;
    const size_t sm = (size_t)M * sizeof(Hit);
    static bool attr = false;
    if (!attr) {
      DSE_CUDA(cudaFuncSetAttribute(k_l0_merge, cudaFuncAttributeMaxDynamicSharedMemorySize, 8192 * (int)sizeof(Hit)));
      attr = true;
    }
    k_l0_merge<<<1, 1024, sm, st>>>(part, (int64_t)nb * kTop, best);
  }
  k_l0_refit<<<kTop, kCol, 0, st>>>(best, D, X, yc, mean, Gm, bv, nrm2, n, N, 0.0, rm, cf);
  DSE_CUDA(cudaGetLastError());
  // reports: RMSEs, coefficients (intercept without the target's mean), the
  // subsets and the target's mean, one wait
  double *hs = static_cast<double *>(pinned_staging(8 * (kTop * 5 + 1) + sizeof(Hit) * kTop));
  if (!hs) return DSE_ENOMEM;
  Hit *hb = reinterpret_cast<Hit *>(hs + kTop * 5 + 1);
  DSE_CUDA(cudaMemcpyAsync(hs, rm, 8 * kTop, cudaMemcpyDeviceToHost, st));
  DSE_CUDA(cudaMemcpyAsync(hs + kTop, cf, 8 * kTop * 4, cudaMemcpyDeviceToHost, st));
  DSE_CUDA(cudaMemcpyAsync(hs + kTop * 5, ym, 8, cudaMemcpyDeviceToHost, st));
  DSE_CUDA(cudaMemcpyAsync(hb, best, sizeof(Hit) * kTop, cudaMemcpyDeviceToHost, st));
  DSE_CUDA(cudaStreamSynchronize(st));
  const double my = hs[kTop * 5];
  struct Row {
    double rmse;
    int64_t p[3];
    double c[4];
  };
  std::vector<Row> rows;
  for (int i = 0; i < kTop; ++i) {
    if (!(hb[i].q >= 0.0) || !(hs[i] < INFINITY)) continue;
    Row r;
    r.rmse = hs[i];
    r.p[0] = (int64_t)((hb[i].key >> 42) & 0x1FFFFF);
    r.p[1] = (int64_t)((hb[i].key >> 21) & 0x1FFFFF);
    r.p[2] = (int64_t)(hb[i].key & 0x1FFFFF);
    for (int c = 0; c < 4; ++c) r.c[c] = hs[kTop + i * 4 + c];
    r.c[0] += my;
    rows.push_back(r);
  }
  std::sort(rows.begin(), rows.end(), [&](const Row &a, const Row &c) {
    if (a.rmse != c.rmse) return a.rmse < c.rmse;
    for (int k = 0; k < D; ++k)
      if (a.p[k] != c.p[k]) return a.p[k] < c.p[k];
    return false;
  });
  const int nf = std::min<int>((int)rows.size(), d->n_top);
  for (int i = 0; i < nf; ++i) {
    if (top_pos)
      for (int k = 0; k < D; ++k) top_pos[i * D + k] = rows[i].p[k];
    if (top_rmse) top_rmse[i] = rows[i].rmse;
    if (top_coefs)
      for (int k = 0; k <= D; ++k) top_coefs[i * (D + 1) + k] = rows[i].c[k];
  }
  *n_found = nf;
  return DSE_OK;
}

}  // namespace dse

using namespace dse;

extern "C" dse_status dse_l0_search(dse_space *s, const dse_l0_desc *d, int64_t *top_pos, double *top_rmse,
                                    double *top_coefs, int32_t *n_found) {
  dse::NvtxRange nvtx_range_("dse_l0_search");
  clear_error();
  if (!s || !d || !d->y || !d->ids || !n_found || d->dim < 1 || d->dim > 3 || d->n_ids < d->dim ||
      d->n_ids > (1 << 16) || d->n_top < 1 || d->n_top > 32) {
    set_error("invalid L0 descriptor");
    return DSE_EINVAL;
  }
  *n_found = 0;
  DSE_TRY(check_device());
  AllocStream as((cudaStream_t)d->stream);
  return l0_search_impl(s, d, top_pos, top_rmse, top_coefs, n_found);
}
