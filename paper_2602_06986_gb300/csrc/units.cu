// units.cu -- dse_candidate_units: the unit vector each candidate carries.
//
// "Physics-Informed Constraints": expressions carry physical units and the
// dimensionally invalid ones are excluded.  Stored features keep their scaled
// exponent vectors in the table; a candidate of the last rung gets its vector
// from its op's rule applied to its operands' vectors, by the same device
// functions (flat-index decode, unit_rule) the screen uses.
#include <vector>

#include "dse_internal.cuh"
#include "eval64.cuh"
#include "util.cuh"

namespace dse {

FeatTable table_of(const dse_space *S);
dse_status check_device();

__global__ void k_candidate_units(FeatTable F, RungGeom G, int D, int check_addsub, int explog_dimless,
                                  const uint64_t *ids, int64_t n, int64_t *units, int8_t *ok) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const uint64_t id = ids[i];
    int32_t u[kMaxDims] = {0};
    bool good = true;
    if (id < (uint64_t)F.n) {
      for (int d = 0; d < D; ++d) u[d] = F.units[id * kMaxDims + d];
    } else {
      int op;
      int64_t a, b;
      good = decode_flat(G, id - (uint64_t)F.n, &op, &a, &b);
      int bad = 0;
      if (good)
        good = unit_rule(op, F.units + a * kMaxDims, b >= 0 ? F.units + b * kMaxDims : nullptr, D, check_addsub,
                         explog_dimless, u, &bad);
    }
    for (int d = 0; d < D; ++d) units[i * D + d] = good ? (int64_t)u[d] : 0;
    ok[i] = good ? 1 : 0;
  }
}

}  // namespace dse

extern "C" dse_status dse_candidate_units(dse_space *s, const uint64_t *ids, int64_t n, int64_t *units,
                                          int8_t *unit_ok) {
  using namespace dse;
  clear_error();
  if (!s || n < 0 || (n > 0 && (!ids || !unit_ok || (s->D > 0 && !units)))) {
    set_error("invalid argument");
    return DSE_EINVAL;
  }
  if (n == 0) return DSE_OK;
  const uint64_t total = (uint64_t)s->n + s->geom.slots;
  for (int64_t i = 0; i < n; ++i)
    if (ids[i] >= total) {
      set_error("candidate id %llu outside [0, %llu)", (unsigned long long)ids[i], (unsigned long long)total);
      return DSE_ERANGE;
    }
  DSE_TRY(check_device());
  cudaStream_t st = s->stream;
  AllocStream as(st);
  const int D = s->D;
  const size_t bi = (size_t)n * 8, bu = (size_t)n * (D > 0 ? D : 1) * 8, bo = (size_t)n;
  char *buf = nullptr;
  DSE_TRY(dmalloc(reinterpret_cast<void **>(&buf), bi + bu + bo, "candidate units"));
  uint64_t *d_ids = reinterpret_cast<uint64_t *>(buf);
  int64_t *d_u = reinterpret_cast<int64_t *>(buf + bi);
  int8_t *d_ok = reinterpret_cast<int8_t *>(buf + bi + bu);
  cudaError_t e = cudaMemcpyAsync(d_ids, ids, bi, cudaMemcpyHostToDevice, st);
  if (!e) {
    const int64_t blocks = std::min<int64_t>((n + 255) / 256, 1024);
    note_launches(1);
    k_candidate_units<<<(unsigned)blocks, 256, 0, st>>>(table_of(s), s->geom, D, s->unit_check_addsub,
                                                         s->explog_dimensionless, d_ids, n, d_u, d_ok);
    e = cudaGetLastError();
  }
  if (!e && D > 0) e = cudaMemcpyAsync(units, d_u, (size_t)n * D * 8, cudaMemcpyDeviceToHost, st);
  if (!e) e = cudaMemcpyAsync(unit_ok, d_ok, bo, cudaMemcpyDeviceToHost, st);
  if (!e) e = cudaStreamSynchronize(st);
  dfree(buf);
  if (e) return cuda_status(e, "candidate units");
  return DSE_OK;
}
