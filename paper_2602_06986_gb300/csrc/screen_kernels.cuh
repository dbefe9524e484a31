// screen_kernels.cuh -- launchers of the screening and selection kernels.
#pragma once

#include "dse_internal.cuh"

namespace dse {

enum { KIND_MUL = 0, KIND_ADD = 1 };

void launch_targets(const double *Y, int64_t ldY, int T, int64_t N, int32_t ldy, double *y64, float *y32,
                    float2 *ydf, float *ysum32, int *err, cudaStream_t st);
void launch_feature(int prec64, int nt, const ScreenArgs &A, uint64_t id0, uint64_t id1, uint64_t p0, uint64_t p1,
                    float gamma, int sms, cudaStream_t st);
dse_status launch_pair(int prec64, int kind, int nt, const ScreenArgs &A, int block_len, int sms, cudaStream_t st);
void launch_escalate(const ScreenArgs &A, int sms, cudaStream_t st, const ScreenArgs *batch = nullptr);
// With A.why: the reason of the candidates no kernel visits (additive slots
// of pairs with unequal units).
void launch_why_fixup(const ScreenArgs &A, int sms, cudaStream_t st);
void launch_pairlist(int prec64, int nt, const ScreenArgs &A, const int2 *pairs, int64_t n_pairs, float gamma,
                     int sms, cudaStream_t st);

// Batched screens (one problem per list; problem arguments in device array
// `args`; work in jobs taken from a device counter).
void launch_targets_batched(const double *Y, const int64_t *yoff, const ScreenArgs *args, int n, int32_t ldy,
                            double *y64, float *y32, float *ysum32, int *err, cudaStream_t st);
void launch_feature_batched(int prec64, const ScreenArgs *args, const Job *jobs, int n_jobs, unsigned int *counter,
                            int sms, cudaStream_t st);
dse_status launch_pair_batched(int prec64, int kind, const ScreenArgs &A0, const ScreenArgs *args, int sms,
                               cudaStream_t st);
void launch_pairlist_batched(int prec64, const ScreenArgs *args, const int2 *pairs, const Job *jobs, int n_jobs,
                             unsigned int *counter, int sms, cudaStream_t st);

// Per-list selection state.
struct SelState {
  unsigned n;               // buffered entries (capped)
  int all_in;               // n <= k: every entry is retained
  int binL, binH;           // bins holding L and H
  unsigned rankL, rankH;    // their ranks within those bins
  unsigned nL, nH;          // entries collected from those bins
  float L, H;
};

// Selection of the exact top-k of every list from its candidate buffer.
struct SelectArgs {
  SelState *state;          // [lists]
  float *colL, *colH;       // [lists][cap] bounds collected from the L / H bins
  CandBufs B;
  int32_t n_lists;
  int64_t k;
  int32_t all64;            // re-score every retained entry in FP64
  // retained set R per list
  uint64_t *r_id;           // [lists][cap]
  float *r_s32, *r_e32;     // [lists][cap]
  double *r_s64, *r_e64;    // [lists][cap]
  uint64_t *r_key;          // [lists][cap] ordering key of the final score
  uint8_t *r_need;          // [lists][cap]
  unsigned int *r_count;    // [lists]
  unsigned int *overflow;   // [lists]
  // re-score jobs: the pair / FP64 re-score's (count n_jobs[0]) and, with
  // rescore32, the FP32 re-score's (job32, job32_list, count n_jobs[1])
  uint32_t *job;            // [lists * cap] packed (list << 24 | pos) is not enough: two arrays
  uint32_t *job_list;
  unsigned int *n_jobs;     // [2]
  uint32_t *job32 = nullptr;       // [lists * cap]
  uint32_t *job32_list = nullptr;  // [lists * cap]
  int32_t rescore32 = 0;    // set by launch_select where the FP32 re-score applies
  // outputs
  uint64_t *out_id;
  double *out_score, *out_eps;
  int64_t *out_n;
  double *max_eps;          // [lists] largest returned bound
  unsigned int *r_rank;     // [lists][cap] rank of each retained entry
  // optional column sums for refits that follow the screen (one target,
  // N <= 4096): the re-score of each entry also accumulates its shifted
  // column against nx vectors (FP64 rows xv, pair images xdf with scale
  // exponents xexp[0..nx)); r_x [lists][cap][8] = {c, S1, S2, E_0.., eps},
  // out_x [lists][k][8] the same in rank order (last field, the sums'
  // relative error scale, 0 when the entry was not re-scored)
  const double *xv[4];
  const float2 *xdf[4];
  const int *xexp;
  int32_t nx;
  double *r_x, *out_x;
  unsigned long long *stats;
};

dse_status launch_select(const SelectArgs &S, const ScreenArgs &A, int sms, cudaStream_t st,
                         const ScreenArgs *batch = nullptr);

}  // namespace dse
