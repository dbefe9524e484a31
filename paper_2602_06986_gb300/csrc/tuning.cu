// tuning.cu -- the planner's launch and tile parameters (dse_set_tuning).
//
// The values are process-wide; an autotuner times candidate settings on the
// device and installs the fastest.  Zero fields mean the built-in default.
#include <mutex>

#include "dse_internal.cuh"
#include "util.cuh"

namespace dse {

namespace {
std::mutex g_mu;
dse_tuning g_tuning = {};  // all zero: defaults
}  // namespace

// The active value of each parameter (defaults filled in).
Tuning tuning() {
  dse_tuning t;
  {
    std::lock_guard<std::mutex> lk(g_mu);
    t = g_tuning;
  }
  Tuning o;
  o.tile_group_tc = t.tile_group > 0 ? t.tile_group : 8;
  o.tile_group_cc = t.tile_group > 0 ? t.tile_group : 4;
  o.seed_stride = t.seed_stride > 0 ? t.seed_stride : 64;
  o.gram_max_n = t.gram_max_n > 0 ? t.gram_max_n : 2048;
  o.tc_min_targets = t.tc_min_targets > 0 ? t.tc_min_targets : 8;
  o.batch_job_samples = t.batch_job_samples > 0 ? t.batch_job_samples : (1 << 14);
  o.gmt_group = t.gmt_group > 0 ? t.gmt_group : 2;
  o.gmt_cluster = t.gmt_cluster > 0 ? t.gmt_cluster : 2;
  return o;
}

}  // namespace dse

extern "C" dse_status dse_set_tuning(const dse_tuning *t) {
  using namespace dse;
  clear_error();
  dse_tuning v = {};
  if (t) {
    v = *t;
    const bool ok = (v.tile_group == 0 || (v.tile_group >= 1 && v.tile_group <= 64)) &&
                    (v.seed_stride == 0 || (v.seed_stride >= 2 && v.seed_stride <= 4096)) &&
                    (v.gram_max_n == 0 || (v.gram_max_n >= 16 && v.gram_max_n <= 2048)) &&
                    (v.tc_min_targets == 0 || (v.tc_min_targets >= 1 && v.tc_min_targets <= 4096)) &&
                    (v.batch_job_samples == 0 || (v.batch_job_samples >= 1024 && v.batch_job_samples <= (1 << 20))) &&
                    (v.gmt_group == 0 || (v.gmt_group >= 1 && v.gmt_group <= 4096)) &&
                    (v.gmt_cluster == 0 || v.gmt_cluster == 1 || v.gmt_cluster == 2);
    if (!ok) {
      set_error("tuning value outside its range");
      return DSE_EINVAL;
    }
  }
  std::lock_guard<std::mutex> lk(g_mu);
  g_tuning = v;
  return DSE_OK;
}

extern "C" dse_status dse_get_tuning(dse_tuning *t) {
  using namespace dse;
  clear_error();
  if (!t) {
    set_error("null argument");
    return DSE_EINVAL;
  }
  const Tuning a = tuning();
  dse_tuning o = {};
  o.tile_group = a.tile_group_tc == a.tile_group_cc ? a.tile_group_tc : 0;
  o.seed_stride = a.seed_stride;
  o.gram_max_n = a.gram_max_n;
  o.tc_min_targets = a.tc_min_targets;
  o.batch_job_samples = a.batch_job_samples;
  o.gmt_group = a.gmt_group;
  o.gmt_cluster = a.gmt_cluster;
  *t = o;
  return DSE_OK;
}
