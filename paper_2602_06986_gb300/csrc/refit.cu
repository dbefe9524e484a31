// refit.cu -- FP64 least-squares refits of the residual loop.
//
// Eq. 1 asks for the best linear model with at most D nonzero coefficients;
// the greedy loop (OMP is one of the strategies named in "Software
// Description") keeps the descriptors chosen so far fixed and, for every
// candidate retained by SIS, fits y on [fixed..., candidate] with an
// intercept, keeping the candidate with the smallest RMSE.  Each fit is a
// (D+1)-column problem solved in FP64 on the device: centred normal
// equations by Cholesky (a column whose Cholesky pivot falls below 1e-12 of
// its norm is rejected as collinear), the RMSE from the explicit residual.
#include <math.h>
#include <string.h>

#include "dse_internal.cuh"
#include "df32.cuh"
#include "eval64.cuh"
#include "util.cuh"

namespace dse {

FeatTable table_of(const dse_space *S);

__device__ __forceinline__ double col_value(const FeatTable &F, const RungGeom &G, int64_t n_stored, int op,
                                            int64_t a, int64_t b, int64_t s) {
  (void)G;
  (void)n_stored;
  return eval_op64(op, F.v64[a * F.ld + s], b >= 0 ? F.v64[b * F.ld + s] : 0.0);
}

__device__ __forceinline__ void decode_any(const RungGeom &G, int64_t n_stored, uint64_t gid, int *op, int64_t *a,
                                           int64_t *b) {
  if (gid < (uint64_t)n_stored) {
    *op = DSE_OP_PRIMARY;
    *a = (int64_t)gid;
    *b = -1;
  } else {
    decode_flat(G, gid - (uint64_t)n_stored, op, a, b);
  }
}

// Columns of the given ids into out[c][N]: block c (any block size),
// threads over samples, so that the FP64 evaluations of a column overlap.
__global__ void k_columns(FeatTable F, RungGeom G, int64_t n_stored, const uint64_t *ids, int n, double *out) {
  const int w = blockIdx.x;
  if (w >= n) return;
  if (ids[w] >= (uint64_t)n_stored + G.slots) {  // no such candidate (a failed step of a chained loop)
    for (int64_t s = threadIdx.x; s < F.N; s += blockDim.x) out[(int64_t)w * F.N + s] = 0.0;
    return;
  }
  int op;
  int64_t a, b;
  decode_any(G, n_stored, ids[w], &op, &a, &b);
  for (int64_t s = threadIdx.x; s < F.N; s += blockDim.x)
    out[(int64_t)w * F.N + s] = col_value(F, G, n_stored, op, a, b, s);
}

constexpr int kMaxP = 4;  // fixed columns + candidate

// One warp per candidate: fit, RMSE and coefficients (intercept first).
__global__ void k_refit(FeatTable F, RungGeom G, int64_t n_stored, const double *y, const double *fixed_cols, int nf,
                        const uint64_t *fixed_ids, const uint64_t *cand, int64_t n_cand, double *rmse_out,
                        double *beta_out) {
  const int lane = threadIdx.x & 31;
  const int64_t w = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  if (w >= n_cand) return;
  const int64_t N = F.N;
  const int p = nf + 1;
  const uint64_t gid = cand[w];
  bool dup = false;
  for (int j = 0; j < nf; ++j) dup |= fixed_ids[j] == gid;
  if (dup) {
    if (lane == 0) rmse_out[w] = INFINITY;
    return;
  }
  int op;
  int64_t a, b;
  decode_any(G, n_stored, gid, &op, &a, &b);
  auto xval = [&](int c, int64_t s) -> double {
    return c < nf ? fixed_cols[(int64_t)c * N + s] : col_value(F, G, n_stored, op, a, b, s);
  };
  // means
  double m[kMaxP] = {0, 0, 0, 0}, my = 0.0;
  for (int64_t s = lane; s < N; s += 32) {
    my += y[s];
    for (int c = 0; c < p; ++c) m[c] += xval(c, s);
  }
  my = warp_sum64(my) / (double)N;
  for (int c = 0; c < p; ++c) m[c] = warp_sum64(m[c]) / (double)N;
  // centred Gram, right-hand side and uncentred column norms
  double Gm[kMaxP][kMaxP] = {}, g[kMaxP] = {}, nrm[kMaxP] = {};
  for (int64_t s = lane; s < N; s += 32) {
    double xc[kMaxP];
    for (int c = 0; c < p; ++c) {
      double v = xval(c, s);
      xc[c] = v - m[c];
      nrm[c] = fma(v, v, nrm[c]);
    }
    double yc = y[s] - my;
    for (int c = 0; c < p; ++c) {
      g[c] = fma(xc[c], yc, g[c]);
      for (int d = 0; d <= c; ++d) Gm[c][d] = fma(xc[c], xc[d], Gm[c][d]);
    }
  }
  for (int c = 0; c < p; ++c) {
    g[c] = warp_sum64(g[c]);
    nrm[c] = sqrt(warp_sum64(nrm[c]));
    for (int d = 0; d <= c; ++d) Gm[c][d] = warp_sum64(Gm[c][d]);
  }
  // Cholesky G = L L^T (every lane computes the same small factorisation)
  double L[kMaxP][kMaxP] = {}, Li[kMaxP] = {};
  bool ok = true;
  for (int c = 0; c < p; ++c) {
    double dsum = Gm[c][c];
    for (int k = 0; k < c; ++k) dsum -= L[c][k] * L[c][k];
    if (!(dsum > 0.0)) {
      ok = false;
      break;
    }
    L[c][c] = sqrt(dsum);
    if (!(L[c][c] > 1e-12 * nrm[c])) {
      ok = false;
      break;
    }
    Li[c] = 1.0 / L[c][c];
    for (int r = c + 1; r < p; ++r) {
      double v = Gm[r][c];
      for (int k = 0; k < c; ++k) v -= L[r][k] * L[c][k];
      L[r][c] = v * Li[c];
    }
  }
  double beta[kMaxP + 1] = {};
  if (ok) {
    double z[kMaxP];
    for (int c = 0; c < p; ++c) {
      double v = g[c];
      for (int k = 0; k < c; ++k) v -= L[c][k] * z[k];
      z[c] = v * Li[c];
    }
    for (int c = p - 1; c >= 0; --c) {
      double v = z[c];
      for (int k = c + 1; k < p; ++k) v -= L[k][c] * beta[k + 1];
      beta[c + 1] = v * Li[c];
    }
    double b0 = my;
    for (int c = 0; c < p; ++c) b0 -= beta[c + 1] * m[c];
    beta[0] = b0;
  }
  double rss = 0.0;
  if (ok) {
    for (int64_t s = lane; s < N; s += 32) {
      double f = beta[0];
      for (int c = 0; c < p; ++c) f = fma(beta[c + 1], xval(c, s), f);
      double r = y[s] - f;
      rss = fma(r, r, rss);
    }
    rss = warp_sum64(rss);
  }
  if (lane == 0) {
    rmse_out[w] = ok ? sqrt(rss / (double)N) : INFINITY;
    for (int c = 0; c <= kMaxP; ++c) beta_out[w * (kMaxP + 1) + c] = ok && c <= p ? beta[c] : 0.0;
  }
}

// The same fit with one block of kWide threads per candidate (more warps in
// flight per SM than a warp per candidate when the candidate list is short).
constexpr int kWide = 128;

template <int NV, int THREADS = kWide>
__device__ __forceinline__ void block_sum_arr(double (&v)[NV], double *sm) {
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
#pragma unroll
    for (int ww = 0; ww < THREADS / 32; ++ww) t += sm[ww * NV + i];
    v[i] = t;
  }
  __syncthreads();
}

// The same over the entries `Live` marks (an entry known to be zero, such as
// a Gram entry of an unused fixed column, costs no FP64 reduction).
template <int NV, int THREADS, typename Live>
__device__ __forceinline__ void block_sum_live(double (&v)[NV], double *sm, Live live) {
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
#pragma unroll
  for (int i = 0; i < NV; ++i)
    if (live(i)) v[i] = warp_sum64(v[i]);
  if (lane == 0)
#pragma unroll
    for (int i = 0; i < NV; ++i)
      if (live(i)) sm[w * NV + i] = v[i];
  __syncthreads();
#pragma unroll
  for (int i = 0; i < NV; ++i) {
    if (!live(i)) continue;
    double t = 0.0;
#pragma unroll
    for (int ww = 0; ww < THREADS / 32; ++ww) t += sm[ww * NV + i];
    v[i] = t;
  }
  __syncthreads();
}

// Statistics of the fixed columns and the target, shared by every
// candidate's fit (one block): means, centred copies, their centred Gram
// matrix and products with the centred target, and the raw column norms
// (for the collinearity test).  pre layout: [0..kMaxP) means of the fixed
// columns, kMaxP: mean of y, then Gram lower triangle (kMaxP*kMaxP), then
// products with y (kMaxP), then raw norms (kMaxP).
constexpr int kPreMean = 0, kPreMy = kMaxP, kPreGram = kMaxP + 1, kPreG = kPreGram + kMaxP * kMaxP,
              kPreNorm = kPreG + kMaxP, kPreSize0 = kPreNorm + kMaxP;
// then the fit of y on the fixed columns alone (the Frisch-Waugh-Lovell
// form of every candidate's fit): Cholesky factor of the centred Gram
// matrix, coefficients, RSS of the explicit residual r = yc - Fc beta, sum r,
// sums of the centred fixed columns, and whether the fixed fit is full rank
constexpr int kPreL = kPreSize0, kPreBf = kPreL + kMaxP * kMaxP, kPreRss = kPreBf + kMaxP, kPreSr = kPreRss + 1,
              kPreSf = kPreSr + 1, kPreOk = kPreSf + kMaxP, kPreSize = kPreOk + 1;

// NF (the number of fixed columns) is a template argument so that every
// per-column array stays in registers.
constexpr int kPrep = kWide;  // threads of the (one-block) prep

template <int NF>
__global__ void __launch_bounds__(kPrep) k_refit_prep(const double *y, const double *fixed_cols, int64_t N,
                                                      double *fcc, double *ycc, double *rc, double *pre) {
  constexpr int nf = NF;
  __shared__ double sm[(kPrep / 32) * (kMaxP * kMaxP + 3 * kMaxP)];
  __shared__ double s_beta[kMaxP + 1];
  double mv[kMaxP + 1] = {0, 0, 0, 0, 0};
  for (int64_t s = threadIdx.x; s < N; s += kPrep) {
#pragma unroll
    for (int c = 0; c < nf; ++c) mv[c] += fixed_cols[(int64_t)c * N + s];
    mv[kMaxP] += y[s];
  }
  block_sum_live<kMaxP + 1, kPrep>(mv, sm, [](int i) { return i < NF || i == kMaxP; });
  double m[kMaxP];
#pragma unroll
  for (int c = 0; c < kMaxP; ++c) m[c] = mv[c] / (double)N;
  const double my = mv[kMaxP] / (double)N;
  double acc[kMaxP * kMaxP + 3 * kMaxP];
#pragma unroll
  for (int i = 0; i < kMaxP * kMaxP + 3 * kMaxP; ++i) acc[i] = 0.0;
  for (int64_t s = threadIdx.x; s < N; s += kPrep) {
    double xc[kMaxP] = {0, 0, 0, 0};
#pragma unroll
    for (int c = 0; c < nf; ++c) {
      const double v = fixed_cols[(int64_t)c * N + s];
      xc[c] = v - m[c];
      fcc[(int64_t)c * N + s] = xc[c];
      acc[kMaxP * kMaxP + kMaxP + c] = fma(v, v, acc[kMaxP * kMaxP + kMaxP + c]);
      acc[kMaxP * kMaxP + 2 * kMaxP + c] += xc[c];
    }
    const double yc = y[s] - my;
    ycc[s] = yc;
#pragma unroll
    for (int c = 0; c < nf; ++c) {
#pragma unroll
      for (int d = 0; d <= c; ++d) acc[c * kMaxP + d] = fma(xc[c], xc[d], acc[c * kMaxP + d]);
      acc[kMaxP * kMaxP + c] = fma(xc[c], yc, acc[kMaxP * kMaxP + c]);
    }
  }
  // live entries: the Gram lower triangle, products with y, norms and sums
  // of the nf used columns
  block_sum_live<kMaxP * kMaxP + 3 * kMaxP, kPrep>(acc, sm, [](int i) {
    return i < kMaxP * kMaxP ? (i / kMaxP < NF && i % kMaxP <= i / kMaxP) : ((i - kMaxP * kMaxP) % kMaxP < NF);
  });
  if (threadIdx.x == 0) {
#pragma unroll
    for (int c = 0; c < kMaxP; ++c) pre[kPreMean + c] = m[c];
    pre[kPreMy] = my;
#pragma unroll
    for (int i = 0; i < kMaxP * kMaxP; ++i) pre[kPreGram + i] = acc[i];
#pragma unroll
    for (int c = 0; c < kMaxP; ++c) pre[kPreG + c] = acc[kMaxP * kMaxP + c];
#pragma unroll
    for (int c = 0; c < kMaxP; ++c) pre[kPreNorm + c] = sqrt(acc[kMaxP * kMaxP + kMaxP + c]);
    // the fixed-only fit: Cholesky with the collinearity test on the pivots
    double L[kMaxP][kMaxP] = {}, Li[kMaxP] = {}, z[kMaxP] = {}, bf[kMaxP] = {};
    bool ok = true;
#pragma unroll
    for (int c = 0; c < nf; ++c) {
      double dsum = acc[c * kMaxP + c];
#pragma unroll
      for (int k = 0; k < c; ++k) dsum -= L[c][k] * L[c][k];
      const double piv = dsum > 0.0 ? sqrt(dsum) : 0.0;
      ok = ok && dsum > 0.0 && dsum > 1e-24 * acc[kMaxP * kMaxP + kMaxP + c];  // piv > 1e-12 |column|
      L[c][c] = ok ? piv : 1.0;
      Li[c] = 1.0 / L[c][c];  // one division per pivot (FP64 division is a long serial chain here)
#pragma unroll
      for (int r = c + 1; r < nf; ++r) {
        double v = acc[r * kMaxP + c];
#pragma unroll
        for (int k = 0; k < c; ++k) v -= L[r][k] * L[c][k];
        L[r][c] = v * Li[c];
      }
    }
#pragma unroll
    for (int c = 0; c < nf; ++c) {
      double v = acc[kMaxP * kMaxP + c];
#pragma unroll
      for (int k = 0; k < c; ++k) v -= L[c][k] * z[k];
      z[c] = v * Li[c];
    }
#pragma unroll
    for (int c = nf - 1; c >= 0; --c) {
      double v = z[c];
#pragma unroll
      for (int k = c + 1; k < nf; ++k) v -= L[k][c] * bf[k];
      bf[c] = v * Li[c];
    }
#pragma unroll
    for (int i = 0; i < kMaxP * kMaxP; ++i) pre[kPreL + i] = L[i / kMaxP][i % kMaxP];
#pragma unroll
    for (int c = 0; c < kMaxP; ++c) {
      pre[kPreBf + c] = ok ? bf[c] : 0.0;
      s_beta[c] = ok ? bf[c] : 0.0;
      pre[kPreSf + c] = acc[kMaxP * kMaxP + 2 * kMaxP + c];
    }
    pre[kPreOk] = ok ? 1.0 : 0.0;
  }
  __syncthreads();
  // the explicit residual of the fixed-only fit
  double bfr[kMaxP];
#pragma unroll
  for (int c = 0; c < kMaxP; ++c) bfr[c] = s_beta[c];
  double q[2] = {0.0, 0.0};
  for (int64_t s = threadIdx.x; s < N; s += kPrep) {
    double r = ycc[s];
#pragma unroll
    for (int c = 0; c < nf; ++c) r = fma(-bfr[c], fcc[(int64_t)c * N + s], r);
    rc[s] = r;
    q[0] = fma(r, r, q[0]);
    q[1] += r;
  }
  block_sum_arr<2, kPrep>(q, sm);
  if (threadIdx.x == 0) {
    pre[kPreRss] = q[0];
    pre[kPreSr] = q[1];
  }
}

// Column sums of the candidates whose record the re-score did not fill
// (out_x[w][7] == 0), one warp per candidate, with the same function and
// vectors as the re-score: {rc, fcc_0 ..} and their pair images xdf with
// scale exponents xexp.  A record is {c, sum (v - c), sum (v - c)^2,
// sum (v - c) rc, sum (v - c) fcc_j .., eps}, eps > 0 the relative error
// scale of its sums (pair or FP64 arithmetic).
template <int NF>
__global__ void __launch_bounds__(kColThreads) k_refit_fill(FeatTable F, RungGeom G, int64_t n_stored,
                                                            const uint64_t *cand, int64_t n_cand,
                                                            const int64_t *n_dev, const double *rc,
                                                            const double *fcc, const float2 *xdf, const int *xexp,
                                                            double *out_x, unsigned long long *minkey) {
  __shared__ ColShared sh;
  const int64_t w = blockIdx.x;
  if (w == 0 && threadIdx.x == 0) *minkey = ~0ull;  // the smallest RSS + err of this fit (below)
  if (w >= n_cand || (n_dev && w >= *n_dev)) return;
  double *x = out_x + w * 8;
  if (x[7] != 0.0) return;
  const int64_t N = F.N;
  const uint64_t gid = cand[w];
  if (gid >= (uint64_t)n_stored + G.slots) return;
  int op;
  int64_t a, b;
  decode_any(G, n_stored, gid, &op, &a, &b);
  ColVecs V;
  V.nv = 1 + NF;
#pragma unroll
  for (int m = 0; m < kColVec; ++m) {
    V.v64[m] = m == 0 ? rc : m <= NF ? fcc + (int64_t)(m - 1) * N : nullptr;
    V.vdf[m] = m <= NF ? xdf + (int64_t)m * N : nullptr;
    V.e[m] = m <= NF ? xexp[m] : 0;
  }
  ColSums cs;
  col_sums(F, op, a, b, N, V, cs, sh);
  if (threadIdx.x == 0) {
    x[0] = cs.c;
    x[1] = cs.acc[0];
    x[2] = cs.acc[1];
    for (int m = 0; m < 4; ++m) x[3 + m] = m < 1 + NF ? cs.acc[2 + m] : 0.0;
    x[7] = col_err_scale(cs, N);
  }
}

// The pair images of the refit vectors {rc, fcc_0 .. fcc_{NF-1}}: x 2^-e
// split into (RN(x 2^-e), RN(x 2^-e - hi)), e the scale exponent of the
// vector's 2-norm (RSS of the fixed-only fit, diagonal of the centred Gram
// matrix), so that every image has norm in [1/2, 1); xexp[m] = e.
template <int NF>
__global__ void k_refit_split(const double *rc, const double *fcc, const double *pre, int64_t N, float2 *xdf,
                              int *xexp) {
  const int64_t total = (int64_t)(1 + NF) * N;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < total; i += (int64_t)gridDim.x * blockDim.x) {
    const int m = (int)(i / N);
    const int64_t s = i - (int64_t)m * N;
    const double n2 = m == 0 ? pre[kPreRss] : pre[kPreGram + (m - 1) * kMaxP + (m - 1)];
    const int e = df::scale_exp(sqrt(n2 > 0.0 ? n2 : 0.0));
    const double x = __dmul_rn(m == 0 ? rc[s] : fcc[(int64_t)(m - 1) * N + s], df::pow2d(-e));
    const float h = __double2float_rn(x);
    xdf[i] = make_float2(h, __double2float_rn(__dsub_rn(x, (double)h)));
    if (s == 0) xexp[m] = e;
  }
}

// Order-preserving key of a double (unsigned comparison = numeric order).
__device__ __forceinline__ unsigned long long ord_key(double x) {
  const unsigned long long u = (unsigned long long)__double_as_longlong(x);
  return (u >> 63) ? ~u : (u | 0x8000000000000000ull);
}

// Every candidate's fit from its column sums (thread per candidate), in the
// Frisch-Waugh-Lovell form: with d the centred candidate column, e_j =
// sum d f_j, w = G^-1 e (G the centred Gram matrix of the fixed columns),
// |d_perp|^2 = sum d^2 - e.w and sum d_perp r = sum d r (r, the fixed-only
// residual, is orthogonal to the fixed columns), the candidate's coefficient
// is (sum d r) / |d_perp|^2 and RSS = RSS_fixed - (sum d r)^2 / |d_perp|^2.
// The pivot test is the full fit's (|d_perp| > 1e-12 |v|).  A fit that leaves
// less than 1e-6 of RSS_fixed (where the subtraction loses digits) is flagged
// for the explicit residual pass.  err_out gets a bound on the RSS error from
// the record's error scale eps: with the sums' errors at most eps sqrt(Sdd)
// |x|, (sum d r)^2 / |d_perp|^2 moves by at most 5 eps RSS_fixed Sdd /
// |d_perp|^2 (by Cauchy-Schwarz, (sum d r)^2 <= RSS_fixed |d_perp|^2); it is
// taken with a factor 8, and the smallest RSS + err of the fit is kept in
// *minkey (order key) for the near-best pass of k_refit_wide.
template <int NF>
__global__ void k_refit_solve(const double *out_x, const uint64_t *cand, int64_t n_cand, const int64_t *n_dev,
                              const uint64_t *fixed_ids, const double *pre, int64_t N, double *rmse_out,
                              double *beta_out, uint8_t *explicit_flag, double *err_out,
                              unsigned long long *minkey) {
  const int64_t w = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (w >= n_cand || (n_dev && w >= *n_dev)) return;
  constexpr int nf = NF;
  const uint64_t gid = cand[w];
  bool dup = false;
#pragma unroll
  for (int j = 0; j < nf; ++j) dup |= fixed_ids[j] == gid;
  explicit_flag[w] = 0;
  err_out[w] = 0.0;
  const double *x = out_x + w * 8;
  if (dup || x[7] == 0.0 || pre[kPreOk] == 0.0) {
    rmse_out[w] = INFINITY;
#pragma unroll
    for (int c = 0; c <= kMaxP; ++c) beta_out[w * (kMaxP + 1) + c] = 0.0;
    return;
  }
  const double Nd = (double)N;
  const double c0 = x[0], S1 = x[1], S2 = x[2];
  const double mS = S1 / Nd;  // vbar - c
  const double Sdd = S2 - S1 * mS;
  const double Sdr = x[3] - mS * pre[kPreSr];
  double e[kMaxP] = {}, z[kMaxP] = {}, wv[kMaxP] = {};
#pragma unroll
  for (int j = 0; j < nf; ++j) e[j] = x[4 + j] - mS * pre[kPreSf + j];
  // w = G^-1 e with G = L L^T
#pragma unroll
  for (int c = 0; c < nf; ++c) {
    double v = e[c];
#pragma unroll
    for (int k = 0; k < c; ++k) v -= pre[kPreL + c * kMaxP + k] * z[k];
    z[c] = v / pre[kPreL + c * kMaxP + c];
  }
#pragma unroll
  for (int c = nf - 1; c >= 0; --c) {
    double v = z[c];
#pragma unroll
    for (int k = c + 1; k < nf; ++k) v -= pre[kPreL + k * kMaxP + c] * wv[k];
    wv[c] = v / pre[kPreL + c * kMaxP + c];
  }
  double ew = 0.0;
#pragma unroll
  for (int j = 0; j < nf; ++j) ew += e[j] * wv[j];
  const double den = Sdd - ew;
  const double raw2 = S2 + 2.0 * c0 * S1 + Nd * c0 * c0;  // sum v^2
  const bool ok = den > 0.0 && sqrt(den) > 1e-12 * sqrt(raw2 > 0.0 ? raw2 : 0.0);
  double *bo = beta_out + w * (kMaxP + 1);
  if (!ok) {
    rmse_out[w] = INFINITY;
#pragma unroll
    for (int c = 0; c <= kMaxP; ++c) bo[c] = 0.0;
    return;
  }
  const double bc = Sdr / den;
  const double rss_f = pre[kPreRss];
  const double rss = rss_f - Sdr * bc;
  double b0 = pre[kPreMy] - bc * (c0 + mS);
#pragma unroll
  for (int j = 0; j < nf; ++j) {
    const double bj = pre[kPreBf + j] - wv[j] * bc;
    bo[j + 1] = bj;
    b0 -= bj * pre[kPreMean + j];
  }
  bo[0] = b0;
  bo[nf + 1] = bc;
#pragma unroll
  for (int c = nf + 2; c <= kMaxP; ++c) bo[c] = 0.0;
  if (rss < 1e-6 * rss_f) {
    explicit_flag[w] = 1;
    rmse_out[w] = INFINITY;
  } else {
    rmse_out[w] = sqrt(rss / Nd);
    const double err = 40.0 * x[7] * rss_f * (Sdd / den);
    err_out[w] = err;
    atomicMin(minkey, ord_key(rss + err));
  }
}

// One block of kWide threads per candidate v: the fit of the centred target
// on the centred [fixed..., v] (Cholesky of the centred normal equations,
// collinearity test on the pivots against the raw column norms), then the
// residual sum of squares explicitly.  Per sample and candidate only the
// terms that involve v are accumulated: Σv, Σv², then Σd², Σd·f_j, Σd·y with
// d = v - mean(v), then the residual.  CACHE: v is evaluated once into
// shared memory (N doubles); FP64 arithmetic is the cost on this part.
// In `near` mode (the refit chain) a block does the fits flagged by
// k_refit_solve (`only`) and every fit whose RSS, within its error bound,
// could be the smallest of the unflagged ones: a fit left out has a true
// RSS above that of the best unflagged fit, which is done here, so the pick
// and its RMSE are those of an FP64 fit (err 0 marks a fit done here).
constexpr int64_t kRefitCacheMax = 6144;  // samples (48 KiB)

template <bool CACHE, int NF>
__global__ void __launch_bounds__(kWide) k_refit_wide(FeatTable F, RungGeom G, int64_t n_stored, const double *fcc,
                                                      const double *ycc, const double *pre,
                                                      const uint64_t *fixed_ids, const uint64_t *cand, int64_t n_cand,
                                                      const int64_t *n_dev, double *rmse_out, double *beta_out,
                                                      const uint8_t *only, double *err_out,
                                                      unsigned long long *minkey, bool near) {
  constexpr int nf = NF;
  __shared__ double sm[(kWide / 32) * 20];
  __shared__ double s_bc[kMaxP + 2];
  extern __shared__ double col[];
  const int64_t w = blockIdx.x;
  if (w >= n_cand || (n_dev && w >= *n_dev)) return;
  const int64_t N = F.N;
  const bool flagged = only && only[w];
  if (near && !flagged) {
    // a fit whose RSS, within its error bound, could be the smallest:
    // RSS_w - err_w <= min_j (RSS_j + err_j) over the unflagged fits (the
    // flagged ones are done here anyway)
    const double r = rmse_out[w], e = err_out[w];
    if (!(r < INFINITY) || !(e > 0.0) || ord_key(r * r * (double)N - e) > *minkey) return;
  } else if (!near && only && !flagged) {
    return;
  }
  constexpr int p = nf + 1;
  const uint64_t gid = cand[w];
  bool dup = false;
  for (int j = 0; j < nf; ++j) dup |= fixed_ids[j] == gid;
  if (threadIdx.x == 0) err_out[w] = 0.0;  // the value written here is the FP64 fit's
  if (dup) {
    if (threadIdx.x == 0) rmse_out[w] = INFINITY;
    return;
  }
  int op;
  int64_t a, b;
  decode_any(G, n_stored, gid, &op, &a, &b);
  auto vval = [&](int64_t s) -> double { return CACHE ? col[s] : col_value(F, G, n_stored, op, a, b, s); };
  double s1[2] = {0.0, 0.0};  // sum v, sum v^2
  for (int64_t s = threadIdx.x; s < N; s += kWide) {
    const double v = col_value(F, G, n_stored, op, a, b, s);
    if (CACHE) col[s] = v;
    s1[0] += v;
    s1[1] = fma(v, v, s1[1]);
  }
  block_sum_arr<2>(s1, sm);
  const double mvv = s1[0] / (double)N;
  double s2[kMaxP + 2] = {0, 0, 0, 0, 0, 0};  // sum d f_j (j < nf), sum d^2, sum d y
  for (int64_t s = threadIdx.x; s < N; s += kWide) {
    const double dv = vval(s) - mvv;
#pragma unroll
    for (int c = 0; c < nf; ++c) s2[c] = fma(dv, fcc[(int64_t)c * N + s], s2[c]);
    s2[kMaxP] = fma(dv, dv, s2[kMaxP]);
    s2[kMaxP + 1] = fma(dv, ycc[s], s2[kMaxP + 1]);
  }
  block_sum_live<kMaxP + 2, kWide>(s2, sm, [](int i) { return i < NF || i >= kMaxP; });
  if (threadIdx.x == 0) {
    double Gm[kMaxP][kMaxP] = {}, g[kMaxP] = {}, nrm[kMaxP] = {};
#pragma unroll
    for (int c = 0; c < nf; ++c) {
#pragma unroll
      for (int d = 0; d <= c; ++d) Gm[c][d] = pre[kPreGram + c * kMaxP + d];
      g[c] = pre[kPreG + c];
      nrm[c] = pre[kPreNorm + c];
      Gm[nf][c] = s2[c];
    }
    Gm[nf][nf] = s2[kMaxP];
    g[nf] = s2[kMaxP + 1];
    nrm[nf] = sqrt(s1[1]);
    double L[kMaxP][kMaxP] = {}, Li[kMaxP] = {};
    bool ok = true;
#pragma unroll
    for (int c = 0; c < p; ++c) {
      double dsum = Gm[c][c];
#pragma unroll
      for (int k = 0; k < c; ++k) dsum -= L[c][k] * L[c][k];
      // a non-positive or tiny pivot (collinear column) rejects the fit; the
      // remaining steps run on a harmless pivot so that the loops stay
      // branch-free and fully unrolled
      const double piv = dsum > 0.0 ? sqrt(dsum) : 0.0;
      ok = ok && dsum > 0.0 && piv > 1e-12 * nrm[c];
      L[c][c] = ok ? piv : 1.0;
      Li[c] = 1.0 / L[c][c];  // one division per pivot (FP64 division is a long serial chain here)
#pragma unroll
      for (int r = c + 1; r < p; ++r) {
        double v = Gm[r][c];
#pragma unroll
        for (int k = 0; k < c; ++k) v -= L[r][k] * L[c][k];
        L[r][c] = v * Li[c];
      }
    }
    double beta[kMaxP + 1] = {};
    if (ok) {
      double z[kMaxP];
#pragma unroll
      for (int c = 0; c < p; ++c) {
        double v = g[c];
#pragma unroll
        for (int k = 0; k < c; ++k) v -= L[c][k] * z[k];
        z[c] = v * Li[c];
      }
#pragma unroll
      for (int c = p - 1; c >= 0; --c) {
        double v = z[c];
#pragma unroll
        for (int k = c + 1; k < p; ++k) v -= L[k][c] * beta[k + 1];
        beta[c + 1] = v * Li[c];
      }
      double b0 = pre[kPreMy];
#pragma unroll
      for (int c = 0; c < nf; ++c) b0 -= beta[c + 1] * pre[kPreMean + c];
      b0 -= beta[p] * mvv;
      beta[0] = b0;
    }
#pragma unroll
    for (int c = 0; c <= kMaxP; ++c) beta_out[w * (kMaxP + 1) + c] = ok && c <= p ? beta[c] : 0.0;
#pragma unroll
    for (int c = 0; c < p; ++c) s_bc[c] = beta[c + 1];
    s_bc[kMaxP + 1] = ok ? 1.0 : 0.0;
  }
  __syncthreads();
  const bool ok = s_bc[kMaxP + 1] != 0.0;
  double rss[1] = {0.0};
  if (ok) {
    double bc[kMaxP];
#pragma unroll
    for (int c = 0; c < p; ++c) bc[c] = s_bc[c];
    for (int64_t s = threadIdx.x; s < N; s += kWide) {
      double r = ycc[s];
#pragma unroll
      for (int c = 0; c < nf; ++c) r = fma(-bc[c], fcc[(int64_t)c * N + s], r);
      r = fma(-bc[nf], vval(s) - mvv, r);
      rss[0] = fma(r, r, rss[0]);
    }
  }
  block_sum_arr<1>(rss, sm);
  if (threadIdx.x == 0) rmse_out[w] = ok ? sqrt(rss[0] / (double)N) : INFINITY;
}

__global__ void k_argmin(const double *rmse, const uint64_t *cand, int64_t n, int64_t *best, const double *beta,
                         double *report, const int64_t *n_dev, uint64_t *chosen);
__global__ void k_residual(FeatTable F, RungGeom G, int64_t n_stored, const double *y, const double *fixed_cols,
                           int nf, const uint64_t *cand, const int64_t *best, const double *beta_all, double *res);

// Buffers of one refit step, carved from one scratch block: fixed columns,
// their centred copies, centred y, the fixed-only residual, the shared
// statistics, and per candidate its column sums, RMSE, coefficients and the
// explicit-pass flag.
struct RefitBufs {
  double *fc, *fcc, *ycc, *rc, *pre, *outx, *rm, *beta, *err;
  uint8_t *flag;
  int64_t *best;
  unsigned long long *minkey;  // order key of the smallest RSS + err of the current fit
  float2 *xdf;  // [kMaxP][N] pair images of {rc, fcc_0 ..}
  int *xexp;    // [kMaxP] their scale exponents
};

static size_t rnd256(size_t b) { return (b + 255) / 256 * 256; }

size_t refit_chain_bytes(int64_t N, int64_t cap) {
  return rnd256(8 * (size_t)N * kMaxP) * 2 + rnd256(8 * N) * 2 + rnd256(8 * kPreSize) + rnd256(64 * (size_t)cap) +
         rnd256(8 * cap) + rnd256(8 * (size_t)cap * (kMaxP + 1)) + rnd256(cap) + rnd256(8) + rnd256(8 * cap) +
         rnd256(8) + rnd256(8 * (size_t)N * kMaxP) + rnd256(4 * kMaxP);
}

static RefitBufs carve(void *scratch, int64_t N, int64_t cap) {
  char *p = static_cast<char *>(scratch);
  RefitBufs b;
  auto take = [&](size_t bytes) {
    char *q = p;
    p += rnd256(bytes);
    return q;
  };
  b.fc = reinterpret_cast<double *>(take(8 * (size_t)N * kMaxP));
  b.fcc = reinterpret_cast<double *>(take(8 * (size_t)N * kMaxP));
  b.ycc = reinterpret_cast<double *>(take(8 * N));
  b.rc = reinterpret_cast<double *>(take(8 * N));
  b.pre = reinterpret_cast<double *>(take(8 * kPreSize));
  b.outx = reinterpret_cast<double *>(take(64 * (size_t)cap));
  b.rm = reinterpret_cast<double *>(take(8 * cap));
  b.beta = reinterpret_cast<double *>(take(8 * (size_t)cap * (kMaxP + 1)));
  b.flag = reinterpret_cast<uint8_t *>(take(cap));
  b.best = reinterpret_cast<int64_t *>(take(8));
  b.err = reinterpret_cast<double *>(take(8 * cap));
  b.minkey = reinterpret_cast<unsigned long long *>(take(8));
  b.xdf = reinterpret_cast<float2 *>(take(8 * (size_t)N * kMaxP));
  b.xexp = reinterpret_cast<int *>(take(4 * kMaxP));
  return b;
}

template <int NF>
static void prep_nf(const dse_space *S, const double *y, const RefitBufs &b, cudaStream_t st) {
  k_refit_prep<NF><<<1, kPrep, 0, st>>>(y, b.fc, S->N, b.fcc, b.ycc, b.rc, b.pre);
  const int64_t total = (int64_t)(1 + NF) * S->N;
  k_refit_split<NF><<<(unsigned)std::min<int64_t>(256, (total + 255) / 256), 256, 0, st>>>(b.rc, b.fcc, b.pre, S->N,
                                                                                         b.xdf, b.xexp);
}

// Fill the missing column sums, solve every fit, redo the flagged ones
// explicitly (one block per flagged candidate).
template <int NF>
static void fit_nf(const FeatTable &F, const dse_space *S, const uint64_t *fid, const uint64_t *cand, int64_t cap,
                   const int64_t *n_dev, const RefitBufs &b, cudaStream_t st) {
  const int64_t N = S->N;
  k_refit_fill<NF><<<(unsigned)cap, kColThreads, 0, st>>>(F, S->geom, S->n, cand, cap, n_dev, b.rc, b.fcc, b.xdf,
                                                          b.xexp, b.outx, b.minkey);
  k_refit_solve<NF><<<(unsigned)((cap + 127) / 128), 128, 0, st>>>(b.outx, cand, cap, n_dev, fid, b.pre, N, b.rm,
                                                                    b.beta, b.flag, b.err, b.minkey);
  auto wide = [&](const uint8_t *only, bool near) {
    if (N <= kRefitCacheMax)
      k_refit_wide<true, NF><<<(unsigned)cap, kWide, (size_t)N * sizeof(double), st>>>(
          F, S->geom, S->n, b.fcc, b.ycc, b.pre, fid, cand, cap, n_dev, b.rm, b.beta, only, b.err, b.minkey, near);
    else
      k_refit_wide<false, NF><<<(unsigned)cap, kWide, 0, st>>>(F, S->geom, S->n, b.fcc, b.ycc, b.pre, fid, cand, cap,
                                                                n_dev, b.rm, b.beta, only, b.err, b.minkey, near);
  };
  // in FP64: the fits the sums cannot resolve (near-perfect ones) and every
  // fit that could still be the best within its error bound
  wide(b.flag, true);
}

// The fixed columns' statistics and residual (before the screen whose
// re-score takes the candidates' sums against them).
void refit_chain_prep(dse_space *S, const double *y, const uint64_t *fid, int nf, void *scratch, int64_t cap,
                      cudaStream_t st) {
  const RefitBufs b = carve(scratch, S->N, cap);
  const FeatTable F = table_of(S);
  note_launches(2 + (nf ? 1 : 0));
  if (nf) k_columns<<<(unsigned)nf, 256, 0, st>>>(F, S->geom, S->n, fid, nf, b.fc);
  switch (nf) {
    case 0: prep_nf<0>(S, y, b, st); break;
    case 1: prep_nf<1>(S, y, b, st); break;
    case 2: prep_nf<2>(S, y, b, st); break;
    default: prep_nf<3>(S, y, b, st); break;
  }
}

// What a re-score needs to take the refit sums: the vectors {rc, fcc_0 ..}
// (1 + nf of them), their pair images and scale exponents, and the
// per-candidate record array.
void refit_chain_vectors(void *scratch, int64_t N, int64_t cap, const double **vec, const float2 **vdf,
                         const int **vexp, double **outx) {
  const RefitBufs b = carve(scratch, N, cap);
  vec[0] = b.rc;
  vdf[0] = b.xdf;
  for (int j = 0; j < 3; ++j) {
    vec[1 + j] = b.fcc + (size_t)j * N;
    vdf[1 + j] = b.xdf + (size_t)(1 + j) * N;
  }
  *vexp = b.xexp;
  *outx = b.outx;
}

// The fits of candidates cand[0..*n_dev) (at most cap) after refit_chain_prep;
// have_sums: the re-score filled the records (else every record is taken
// here).  Writes the winner's report, its id to *chosen and the residual.
void refit_chain_fit(dse_space *S, const double *y, const uint64_t *fid, int nf, const uint64_t *cand, int64_t cap,
                     const int64_t *n_dev, void *scratch, bool have_sums, double *res, double *report,
                     uint64_t *chosen, cudaStream_t st) {
  const RefitBufs b = carve(scratch, S->N, cap);
  const FeatTable F = table_of(S);
  if (!have_sums) cudaMemsetAsync(b.outx, 0, 64 * (size_t)cap, st);
  note_launches(5);
  switch (nf) {
    case 0: fit_nf<0>(F, S, fid, cand, cap, n_dev, b, st); break;
    case 1: fit_nf<1>(F, S, fid, cand, cap, n_dev, b, st); break;
    case 2: fit_nf<2>(F, S, fid, cand, cap, n_dev, b, st); break;
    default: fit_nf<3>(F, S, fid, cand, cap, n_dev, b, st); break;
  }
  k_argmin<<<1, 1024, 0, st>>>(b.rm, cand, cap, b.best, b.beta, report, n_dev, chosen);
  k_residual<<<64, 256, 0, st>>>(F, S->geom, S->n, y, b.fc, nf, cand, b.best, b.beta, res);
}

// Index of the smallest RMSE (ties: lower id); one block.  report (when not
// null) gets {index, id, rmse, beta[kMaxP + 1]} of the winner as doubles /
// bit patterns, for one small copy to the host.
// n_dev (when not null) caps n with a count on the device; chosen (when not
// null) gets the winner's id (2^64-1 if none), for fits chained on the device.
__global__ void k_argmin(const double *rmse, const uint64_t *cand, int64_t n, int64_t *best, const double *beta,
                         double *report, const int64_t *n_dev, uint64_t *chosen) {
  if (n_dev && *n_dev < n) n = *n_dev;
  // comparisons on order-preserving integer keys of the RMSEs (the integer
  // pipe instead of the slow FP64 one); a NaN ranks with +inf
  const unsigned long long kinf = ord_key(INFINITY);
  auto key = [&](double r) {
    const unsigned long long b = (unsigned long long)__double_as_longlong(r);
    const bool nan = (b & 0x7FF0000000000000ull) == 0x7FF0000000000000ull && (b & 0x000FFFFFFFFFFFFFull) != 0ull;
    return nan ? kinf : ord_key(r);
  };
  __shared__ unsigned long long bv[1024];
  __shared__ uint64_t bid[1024];
  __shared__ int64_t bix[1024];
  unsigned long long v = kinf;
  uint64_t id = ~0ull;
  int64_t ix = -1;
  for (int64_t i = threadIdx.x; i < n; i += blockDim.x) {
    const unsigned long long r = key(rmse[i]);
    if (r < v || (r == v && cand[i] < id)) {
      v = r;
      id = cand[i];
      ix = i;
    }
  }
  bv[threadIdx.x] = v;
  bid[threadIdx.x] = id;
  bix[threadIdx.x] = ix;
  __syncthreads();
  for (int o = blockDim.x / 2; o > 0; o >>= 1) {
    if ((int)threadIdx.x < o) {
      const unsigned long long r = bv[threadIdx.x + o];
      uint64_t i2 = bid[threadIdx.x + o];
      if (r < bv[threadIdx.x] || (r == bv[threadIdx.x] && i2 < bid[threadIdx.x])) {
        bv[threadIdx.x] = r;
        bid[threadIdx.x] = i2;
        bix[threadIdx.x] = bix[threadIdx.x + o];
      }
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    const int64_t b = bv[0] < kinf ? bix[0] : -1;
    *best = b;
    if (chosen) *chosen = b >= 0 ? cand[b] : ~0ull;
    if (report) {
      report[0] = __longlong_as_double(b);
      report[1] = __longlong_as_double(b >= 0 ? (long long)cand[b] : -1ll);
      report[2] = b >= 0 ? rmse[b] : INFINITY;
      for (int c = 0; c <= kMaxP; ++c) report[3 + c] = b >= 0 ? beta[b * (kMaxP + 1) + c] : 0.0;
    }
  }
}

// Residual y - fit of the chosen candidate.
__global__ void k_residual(FeatTable F, RungGeom G, int64_t n_stored, const double *y, const double *fixed_cols,
                           int nf, const uint64_t *cand, const int64_t *best, const double *beta_all, double *res) {
  const int64_t bi = *best;
  if (bi < 0) return;
  const double *beta = beta_all + bi * (kMaxP + 1);
  int op;
  int64_t a, b;
  decode_any(G, n_stored, cand[bi], &op, &a, &b);
  for (int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; s < F.N; s += (int64_t)gridDim.x * blockDim.x) {
    double f = beta[0];
    for (int c = 0; c < nf; ++c) f = fma(beta[c + 1], fixed_cols[(int64_t)c * F.N + s], f);
    f = fma(beta[nf + 1], col_value(F, G, n_stored, op, a, b, s), f);
    res[s] = y[s] - f;
  }
}

// ------------------------------------------------ refits chained on the device
// (refit_chain_prep / refit_chain_fit above)

static inline long long __double_as_longlong_host(double x) {
  long long v;
  memcpy(&v, &x, sizeof(v));
  return v;
}

dse_status refit_impl(dse_space *S, const dse_refit_desc *d, uint64_t *best_id, double *best_rmse, double *coefs,
                      double *residual) {
  cudaStream_t st = (cudaStream_t)d->stream;
  const int64_t N = S->N, nc = d->n_cand;
  const int nf = d->n_fixed;
  const uint64_t total = (uint64_t)S->n + S->geom.slots;
  for (int j = 0; j < nf; ++j)
    if (d->fixed[j] >= total) {
      set_error("fixed id out of range");
      return DSE_ERANGE;
    }
  if (!d->cand_on_device)
    for (int64_t i = 0; i < nc; ++i)
      if (d->cand[i] >= total) {
        set_error("candidate id out of range");
        return DSE_ERANGE;
      }
  // one scratch block: the refit step's buffers, then y, fixed ids,
  // candidates, the report and the residual
  size_t off = 0;
  auto take = [&](size_t bytes) {
    size_t o = off;
    off += (bytes + 255) / 256 * 256;
    return o;
  };
  // inputs already on the device are read in place; a device residual
  // buffer is written in place (the call waits before it returns)
  const bool res_dev = residual && is_device_pointer(residual);
  const int64_t cap = nc > 0 ? nc : 1;
  size_t o_chain = take(refit_chain_bytes(N, cap)), o_y = take(d->y_on_device ? 0 : 8 * N), o_fid = take(8 * 4),
         o_c = take(d->cand_on_device ? 0 : 8 * nc), o_rep = take(8 * (kMaxP + 4)),
         o_res = take(res_dev ? 0 : 8 * N);
  char *base = nullptr;
  DSE_TRY(dmalloc(reinterpret_cast<void **>(&base), off, "refit scratch"));
  const double *y = d->y_on_device ? d->y : reinterpret_cast<double *>(base + o_y);
  uint64_t *fid = reinterpret_cast<uint64_t *>(base + o_fid);
  const uint64_t *cand = d->cand_on_device ? d->cand : reinterpret_cast<uint64_t *>(base + o_c);
  double *rep = reinterpret_cast<double *>(base + o_rep);
  double *res = res_dev ? residual : reinterpret_cast<double *>(base + o_res);
  cudaError_t e = cudaSuccess;
  if (!d->y_on_device)
    e = cudaMemcpyAsync(const_cast<double *>(y), d->y, 8 * N, cudaMemcpyHostToDevice, st);
  if (!e && nf) e = cudaMemcpyAsync(fid, d->fixed, 8 * nf, cudaMemcpyHostToDevice, st);
  if (!e && !d->cand_on_device)
    e = cudaMemcpyAsync(const_cast<uint64_t *>(cand), d->cand, 8 * nc, cudaMemcpyHostToDevice, st);
  if (e) {
    dfree(base);
    return cuda_status(e, "refit upload");
  }
  refit_chain_prep(S, y, fid, nf, base + o_chain, cap, st);
  refit_chain_fit(S, y, fid, nf, cand, nc, nullptr, base + o_chain, false, res, rep, nullptr, st);
  // one asynchronous copy of the winner's report (and of a host residual), one sync
  double *h = static_cast<double *>(pinned_staging(8 * (kMaxP + 4)));
  if (!h) {
    dfree(base);
    return DSE_ENOMEM;
  }
  e = cudaMemcpyAsync(h, rep, 8 * (kMaxP + 4), cudaMemcpyDeviceToHost, st);
  if (!e && residual && !res_dev) e = cudaMemcpyAsync(residual, res, 8 * N, cudaMemcpyDeviceToHost, st);
  if (!e) e = cudaStreamSynchronize(st);
  dfree(base);
  if (e) return cuda_status(e, "refit");
  const int64_t hb = (int64_t)__double_as_longlong_host(h[0]);
  if (hb < 0) {
    set_error("no candidate gives a full-rank fit");
    return DSE_EINVAL;
  }
  *best_id = (uint64_t)__double_as_longlong_host(h[1]);
  *best_rmse = h[2];
  if (coefs)
    for (int c = 0; c < nf + 2; ++c) coefs[c] = h[3 + c];
  return DSE_OK;
}

}  // namespace dse
