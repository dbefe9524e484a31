// plan.cuh -- host-side planning helpers shared by the single and batched
// screens: scratch layout, pair tile lists, equal-unit pair lists, error
// factors.
#pragma once

#include <utility>
#include <vector>

#include "dse_internal.cuh"
#include "util.cuh"

namespace dse {

// One device allocation carved into 256-byte-aligned pieces.
struct Scratch {
  std::vector<std::pair<void **, size_t>> items;
  template <typename T>
  void add(T **p, size_t count) {
    items.push_back({reinterpret_cast<void **>(p), (count ? count : 1) * sizeof(T)});
  }
  dse_status alloc(void **base, size_t *bytes) {
    size_t tot = 0;
    for (auto &it : items) tot += (it.second + 255) / 256 * 256;
    DSE_TRY(dmalloc(base, tot, "screen scratch"));
    *bytes = tot;
    size_t off = 0;
    for (auto &it : items) {
      *it.first = reinterpret_cast<char *>(*base) + off;
      off += (it.second + 255) / 256 * 256;
    }
    return DSE_OK;
  }
};

int sm_count();
dse_status check_device();

// Pair tiles over the positions of rows grouped in consecutive classes
// (class c = positions [cb[c], cb[c+1])), pairs position_i > position_j.
void class_tiles(const std::vector<int64_t> &cb, int64_t npos, int BI, int BJ, int64_t i_from,
                 std::vector<Tile> &out);
// Triangle tiles over ids: i in [ia, ib], j < i.
void triangle_tiles(int64_t ia, int64_t ib, int BI, int BJ, std::vector<Tile> &out);
// The pairs (i > j, i in the newest stored rung) of equal unit vectors, built
// once per space and kept on the device (synchronises the stream).
dse_status equal_unit_pairs(dse_space *sp, cudaStream_t st);
// Number of p' in [0, x) with p' mod nb in posset.
uint64_t count_slots_mod(uint64_t x, int nb, const std::vector<int> &posset);
// Exhaustive L0 search (l0.cu).
dse_status l0_search_impl(dse_space *sp, const dse_l0_desc *d, int64_t *top_pos, double *top_rmse, double *top_coefs,
                          int32_t *n_found);
// Accumulation error factors of the CUDA-core kernels for N samples.
void accum_factors(int64_t N, int prec64, float *gamma_lane, float *gamma_pair, int *block_len);

}  // namespace dse
