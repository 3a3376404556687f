// mp_run_noalloc: a whole multipath run for callers that cannot allocate
// device memory.
//
// Some callers cannot call cudaMalloc: code running inside a host framework
// that owns every device allocation (a fixed memory pool or arena), code
// restricted from growing the device heap after start-up, or a plugin whose
// host forbids allocator calls on its threads.  They can still hand over
// their inputs (host memory) and an output buffer they already own.
//
// This file keeps everything else a run needs -- the per-path records that
// pass from the sweep kernel to the reduction kernel, the work-queue counter,
// and the device copies of the system, work-item and column-walk unit tables
// -- in one file-scope __device__ array of fixed size.  Every GPU that loads
// the library holds that array (about 3.4 MB) until the process exits.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <mutex>

#include "kernels.h"
#include "mp.h"

namespace {

using mpk::DevSystem;
using mpk::WorkItem;

constexpr int kMaxDevices = 64;

// Column-walk units: one table per lattice size of a call (the threads per
// path and so the segment count depend on L alone here), at most L^3/2
// entries for each even L up to the largest size shared memory holds.
constexpr int kMaxUnits = [] {
  int n = 0;
  for (int L = 2; L <= 26; L += 2) n += L * L * L / 2;
  return n;
}();

struct NoallocScratch {
  double records[static_cast<size_t>(MP_NOALLOC_MAX_PATHS) * MP_NREC];
  WorkItem items[MP_NOALLOC_MAX_PATHS];
  DevSystem systems[MP_NOALLOC_MAX_SYSTEMS];
  int4 units[kMaxUnits];
  int queue[64];  // queue[0]: the work counter, queue[1]: the kernels' error word
};

// The shared scratch.  In host code this name is a host-side stand-in, not a
// device address: the kernels get the address from cudaGetSymbolAddress.
static __device__ __align__(256) NoallocScratch g_noalloc_scratch;

std::mutex g_mu;                                  // serialises host-side set-up
NoallocScratch* g_addr[kMaxDevices] = {nullptr};  // device address, per device
WorkItem g_items[MP_NOALLOC_MAX_PATHS];           // host staging of the tables
DevSystem g_systems[MP_NOALLOC_MAX_SYSTEMS];
int4 g_units[kMaxUnits];

int round_up(int v, int m) { return (v + m - 1) / m * m; }

}  // namespace

extern "C" int mp_run_noalloc(const mp_system* systems, int n_systems, int precision,
                              int64_t n_therm, int64_t n_meas, uint64_t seed, double* d_estimates,
                              void* stream) {
  if (!systems || !d_estimates || n_systems < 1 || n_systems > MP_NOALLOC_MAX_SYSTEMS)
    return MP_EINVAL;
  if (precision != MP_FP32 && precision != MP_FP64) return MP_EINVAL;
  if (n_therm < 0 || n_meas < 1 || n_therm + n_meas > 0xffffffffLL) return MP_EINVAL;
  int64_t total = 0;
  for (int k = 0; k < n_systems; ++k) {
    const mp_system& s = systems[k];
    if (s.lattice != MP_LATTICE_SC && s.lattice != MP_LATTICE_CHAIN) return MP_EINVAL;
    if (!(s.T > 0.0) || !std::isfinite(s.T) || !std::isfinite(s.J) || !std::isfinite(s.h))
      return MP_EINVAL;
    if (s.n_paths < 1 || s.path_begin < 0 || s.path_begin + s.n_paths > 0x100000000LL) return MP_EINVAL;
    if (s.lattice == MP_LATTICE_SC && (s.L < 2 || (s.L & 1) || !mpk::sweep_supports_L(precision, s.L)))
      return MP_EINVAL;
    if (s.lattice == MP_LATTICE_CHAIN && (s.L < 2 || s.L > 8192)) return MP_EINVAL;
    total += s.n_paths;
    if (total > MP_NOALLOC_MAX_PATHS) return MP_EINVAL;  // beyond the static scratch
  }

  std::lock_guard<std::mutex> lock(g_mu);
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) {
    cudaGetLastError();
    return MP_ECUDA;
  }
  // Set-up, once per device, with that device current.
  if (!g_addr[dev]) {
    void* p = nullptr;
    if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess || !p) {
      cudaGetLastError();
      return MP_ECUDA;
    }
    g_addr[dev] = static_cast<NoallocScratch*>(p);
  }
  NoallocScratch* d = g_addr[dev];
  cudaStream_t st = static_cast<cudaStream_t>(stream);

  // Launch shape: one kernel variant for the batch, one path per work item.
  int variant = systems[0].lattice == MP_LATTICE_CHAIN ? -1 : systems[0].L;
  for (int k = 1; k < n_systems; ++k) {
    const int v = systems[k].lattice == MP_LATTICE_CHAIN ? -1 : systems[k].L;
    if (v != variant) variant = 0;
  }
  int smem_max = 0, cta_max = 0, sms = 0;
  if (mpk::sweep_prepare(precision, variant, dev, &smem_max, &cta_max) != cudaSuccess ||
      mpk::reduce_prepare() != cudaSuccess ||
      cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) {
    cudaGetLastError();
    return MP_ECUDA;
  }
  const int real = precision == MP_FP64 ? 8 : 4;
  int cta = 32, smem = 0, n_items = 0, n_units = 0;
  int unit_of_L[27];  // first unit-table entry of each size, -1 = none yet
  std::fill(unit_of_L, unit_of_L + 27, -1);
  int64_t rec = 0, max_paths = 0;
  for (int k = 0; k < n_systems; ++k) {
    const mp_system& s = systems[k];
    const int N = s.lattice == MP_LATTICE_SC ? s.L * s.L * s.L : s.L;
    const int NH = (N + 1) / 2;
    const int tp = std::min(cta_max, std::max(32, round_up((NH + 7) / 8, 32)));
    const int slice = round_up(mpk::slice_spin_offset(tp, 1) + 6 * round_up(NH, 2) * real, 128);
    if (slice > smem_max) return MP_EINVAL;
    DevSystem& ds = g_systems[k];
    std::memset(&ds, 0, sizeof(ds));
    ds.lattice = s.lattice;
    ds.L = s.L;
    ds.N = N;
    ds.NH = NH;
    ds.tp = tp;
    ds.g = 1;
    ds.slice_bytes = slice;
    ds.ring = 1;
    ds.T = s.T;
    ds.J = s.J;
    ds.h = s.h;
    ds.beta = 1.0 / s.T;
    ds.rec_offset = rec;
    ds.n_paths = s.n_paths;
    ds.path_begin = s.path_begin;
    ds.unit_off = -1;
    if (s.lattice == MP_LATTICE_SC) {  // the column walk's units (column_unit)
      const int U = mpk::column_chunk(real, s.L, variant == 0);
      const int K = mpk::column_segments(s.L, U, tp);
      const int cnt = s.L * s.L / 2 * K;
      if (s.L > 26 || (unit_of_L[s.L] < 0 && n_units + cnt > kMaxUnits)) return MP_EINVAL;
      if (unit_of_L[s.L] < 0) {
        unit_of_L[s.L] = n_units;
        for (int u = 0; u < cnt; ++u) g_units[n_units++] = mpk::column_unit(s.L, K, u);
      }
      ds.unit_off = unit_of_L[s.L];
      ds.unit_K = K;
      ds.unit_U = U;
    }
    for (int64_t p = 0; p < s.n_paths; ++p) g_items[n_items++] = WorkItem{k, 1, p};
    rec += s.n_paths;
    cta = std::max(cta, tp);
    smem = std::max(smem, slice);
    max_paths = std::max<int64_t>(max_paths, s.n_paths);
  }
  int per_sm = 0;
  if (mpk::sweep_occupancy(precision, variant, cta, smem, &per_sm) != cudaSuccess || per_sm < 1) {
    cudaGetLastError();
    return MP_EINVAL;
  }
  const int grid = static_cast<int>(std::min<int64_t>(n_items, static_cast<int64_t>(sms) * per_sm));

  if (cudaMemcpyAsync(d->systems, g_systems, sizeof(DevSystem) * n_systems, cudaMemcpyHostToDevice,
                      st) != cudaSuccess ||
      cudaMemcpyAsync(d->items, g_items, sizeof(WorkItem) * n_items, cudaMemcpyHostToDevice, st) !=
          cudaSuccess ||
      (n_units > 0 &&
       cudaMemcpyAsync(d->units, g_units, sizeof(int4) * n_units, cudaMemcpyHostToDevice, st) != cudaSuccess) ||
      cudaMemsetAsync(d->queue, 0, 2 * sizeof(int), st) != cudaSuccess) {
    cudaGetLastError();
    return MP_ECUDA;
  }
  mpk::SweepParams p{};
  p.systems = d->systems;
  p.items = d->items;
  p.queue = d->queue;
  p.records = d->records;
  p.spins = nullptr;
  p.spin_offset = nullptr;
  p.n_items = n_items;
  p.init_mode = MP_INIT_SPHERE;
  p.n_therm = n_therm;
  p.n_meas = n_meas;
  p.s_begin = 0;
  p.s_end = n_therm + n_meas;
  p.key = mpk::philox_round_keys(seed);
  p.error = d->queue + 1;  // where a kernel would report a path that stopped early
  p.units = d->units;
  mpk::ReduceParams r{};
  r.systems = d->systems;
  r.records = d->records;
  r.est = d_estimates;
  r.n_therm = n_therm;
  r.n_meas = n_meas;
  if (mpk::launch_sweep(precision, variant, p, grid, cta, smem, st) != cudaSuccess ||
      mpk::launch_reduce(r, n_systems, max_paths, st) != cudaSuccess) {
    cudaGetLastError();
    return MP_ECUDA;
  }
  // The host staging tables were copied from pageable memory, which completes
  // before cudaMemcpyAsync returns, so the next call may reuse them.
  return MP_OK;
}
