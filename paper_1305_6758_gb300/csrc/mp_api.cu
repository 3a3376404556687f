// C ABI of the multipath Metropolis library (declared in include/mp.h).
//
// A handle owns the plan of one batch of systems: the per-system launch shape
// (threads per path, paths per CTA, shared-memory slice), the persistent work
// queue, the device buffers (per-path records, estimates, optional final
// spins) and, with MP_FLAG_GRAPH, a CUDA graph of one run: zero the queue,
// the sweep kernel, the reduction kernel, with timing events between them.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <map>
#include <mutex>
#include <string>
#include <tuple>
#include <vector>

#include "kernels.h"
#include "mp.h"

namespace mpk {

bool sweep_supports_L_fp32(int L);
bool sweep_supports_L_fp64(int L);
cudaError_t sweep_prepare_fp32(int variant, int device, int* max_dynamic, int* max_threads);
cudaError_t sweep_prepare_fp64(int variant, int device, int* max_dynamic, int* max_threads);
cudaError_t sweep_occupancy_fp32(int variant, int cta, int smem, int* blocks);
cudaError_t sweep_occupancy_fp64(int variant, int cta, int smem, int* blocks);
cudaError_t launch_sweep_fp32(int variant, const SweepParams& p, int grid, int cta, int smem,
                              cudaStream_t st);
cudaError_t launch_sweep_fp64(int variant, const SweepParams& p, int grid, int cta, int smem,
                              cudaStream_t st);
cudaError_t sweep_cluster_occupancy_fp32(int variant, int cta, int smem, int* clusters);
cudaError_t sweep_cluster_occupancy_fp64(int variant, int cta, int smem, int* clusters);

bool sweep_supports_L(int precision, int L) {
  return precision == MP_FP64 ? sweep_supports_L_fp64(L) : sweep_supports_L_fp32(L);
}
cudaError_t sweep_prepare(int precision, int variant, int device, int* max_dynamic,
                          int* max_threads) {
  if (is_ising_variant(variant)) return ising_prepare(variant, device, max_dynamic, max_threads);
  return precision == MP_FP64 ? sweep_prepare_fp64(variant, device, max_dynamic, max_threads)
                              : sweep_prepare_fp32(variant, device, max_dynamic, max_threads);
}
cudaError_t sweep_occupancy(int precision, int variant, int cta, int smem, int* blocks) {
  if (is_ising_variant(variant)) return ising_occupancy(variant, cta, smem, blocks);
  return precision == MP_FP64 ? sweep_occupancy_fp64(variant, cta, smem, blocks)
                              : sweep_occupancy_fp32(variant, cta, smem, blocks);
}
cudaError_t sweep_cluster_occupancy(int precision, int variant, int cta, int smem, int* clusters) {
  return precision == MP_FP64 ? sweep_cluster_occupancy_fp64(variant, cta, smem, clusters)
                              : sweep_cluster_occupancy_fp32(variant, cta, smem, clusters);
}
cudaError_t launch_sweep(int precision, int variant, const SweepParams& p, int grid, int cta,
                         int smem, cudaStream_t st) {
  if (is_ising_variant(variant)) return launch_ising(variant, p, grid, cta, smem, st);
  return precision == MP_FP64 ? launch_sweep_fp64(variant, p, grid, cta, smem, st)
                              : launch_sweep_fp32(variant, p, grid, cta, smem, st);
}

}  // namespace mpk

using namespace mpk;

namespace {

thread_local std::string g_create_error;

int64_t sites_of(const mp_system& s) {
  if (s.lattice == MP_LATTICE_ISING) return static_cast<int64_t>(s.L) * s.L;
  return s.lattice == MP_LATTICE_SC ? static_cast<int64_t>(s.L) * s.L * s.L : s.L;
}

// Shared-memory bytes of one path's spins (both colours) in the sweep kernels.
int64_t lattice_bytes(const mp_system& s, int real) {
  const int64_t NH = (sites_of(s) + 1) / 2;
  if (s.lattice == MP_LATTICE_ISING) return kIsingThrBytes + 2 * NH;
  return 6 * ((NH + 1) & ~int64_t{1}) * real;  // per colour: (x, y) pairs then z, even length
}

// Ising acceptance as an integer test on a Philox word r (Appendix A kernel):
// accept iff r < t with t = #{r : (r + 1/2) 2^-32 < exp(-beta dE)}, for
// dE = 2 s (J k + h), s = +1 (entries 0..4) and -1 (5..9), neighbour sum
// k = -4, -2, 0, 2, 4; dE <= 0 is always accepted (t = 2^32).  (r + 1/2) 2^-32
// and p 2^32 are exact in FP64, so r + 1/2 < p 2^32 <=> r < ceil(p 2^32 - 1/2).
void ising_thresholds(const mp_system& s, unsigned long long* t) {
  const double beta = 1.0 / s.T;
  for (int a = 0; a < 2; ++a) {
    const double sg = a == 0 ? 1.0 : -1.0;
    for (int k = 0; k < 5; ++k) {
      const double dE = 2.0 * sg * (s.J * static_cast<double>(2 * k - 4) + s.h);
      unsigned long long v = 1ull << 32;
      if (dE > 0.0) {
        const double y = std::exp(-beta * dE) * 4294967296.0 - 0.5;
        v = y <= 0.0 ? 0ull : std::min<unsigned long long>(static_cast<unsigned long long>(std::ceil(y)), 1ull << 32);
      }
      t[a * 5 + k] = v;
    }
  }
}

int round_up(int v, int m) { return (v + m - 1) / m * m; }

// Streamed lattices: one half-plane (one colour of one z-plane, 3 L^2/2 values)
// padded to 16 bytes, in bytes.
int half_plane_bytes(int L, int real) { return round_up(3 * (L * L / 2) * real, 16); }

// Lattices held in the shared memory of the two CTAs of a cluster: the FP32
// simple cubic L = 32 (393 KB of spins, too large for one SM, not for two),
// unless every lattice is to stream from HBM.
bool paired(const mp_system& s, int precision, uint32_t flags) {
  return s.lattice == MP_LATTICE_SC && s.L == kPairL && precision == MP_FP32 &&
         !(flags & (MP_FLAG_STREAM | MP_FLAG_RANDOM_SITE));
}

bool streamed(const mp_system& s, int precision, uint32_t flags) {
  // the plane wavefront needs at least four planes
  return s.lattice == MP_LATTICE_SC && s.L >= 4 && !paired(s, precision, flags) &&
         ((flags & MP_FLAG_STREAM) || !sweep_supports_L(precision, s.L));
}

// Lattices to stream whose ring of nine half-planes does not fit one SM's
// shared memory (FP64 L >= 46, FP32 L >= 66; `optin` is the device's largest
// shared memory per CTA, of which the kernels' static data take under 4 KB)
// are updated in place in HBM instead: every site decoded from its index,
// neighbours read from global memory, one barrier per half-sweep.
bool in_place(const mp_system& s, int precision, uint32_t flags, int optin) {
  if (!streamed(s, precision, flags)) return false;
  const int real = precision == MP_FP64 ? 8 : 4;
  return 128 + 9 * half_plane_bytes(s.L, real) + slice_spin_offset(32, 1) > optin - 4096;
}

}  // namespace

struct mp_state {
  int device = 0;
  int precision = MP_FP32;
  int init_mode = MP_INIT_SPHERE;
  uint32_t flags = 0;
  int64_t n_therm = 0, n_meas = 1;
  uint64_t seed = 0;
  cudaStream_t stream = nullptr;
  bool own_stream = false;
  mp_alloc_fn alloc_fn = nullptr;
  mp_free_fn free_fn = nullptr;
  void* alloc_ctx = nullptr;

  std::vector<mp_system> systems;
  std::vector<DevSystem> hsys;
  std::vector<WorkItem> items;
  std::vector<WorkItem> pair_items;  // one path each, for two-CTA clusters (after items in d_items)
  std::vector<int64_t> spin_offset;
  int64_t total_paths = 0, max_paths = 0, total_spins = 0;

  int cta = 0, grid = 0, smem = 0;
  int variant = 0;  // sweep kernel variant (see kernels.h)

  DevSystem* d_sys = nullptr;
  WorkItem* d_items = nullptr;
  int* d_queue = nullptr;
  double* d_rec = nullptr;
  double* d_est = nullptr;
  double* d_spins = nullptr;
  int64_t* d_spin_offset = nullptr;
  unsigned long long* d_thr = nullptr;  // Ising acceptance thresholds, 10 per system
  int4* d_units = nullptr;         // column-walk unit tables (column_unit), one per (L, K, U)
  int64_t units_capacity = 0;      // entries allocated at d_units
  int64_t upload_bytes = 0;        // bytes the last upload_tables copied to the device
  double* d_sort = nullptr;        // sort space of the distribution coefficient (systems > 16384 paths)
  int* d_error = nullptr;          // nonzero when a bounded wait in a kernel gave up
  void* d_lattice = nullptr;       // HBM lattices of streamed paths
  size_t lattice_capacity = 0;     // bytes allocated at d_lattice
  std::vector<int> tp_override;    // per system threads per path (autotuner), 0 = planner
  // resumable runs (mp_run_sweeps / mp_checkpoint / mp_restore)
  unsigned char* d_state = nullptr;
  int64_t state_bytes = 0;
  std::vector<int64_t> state_offset, state_stride;  // bytes, per system
  int64_t* d_state_offset = nullptr;
  int64_t* d_state_stride = nullptr;
  int64_t sweeps_done = 0;         // progress of the resumable schedule
  int* h_cancel = nullptr;         // host-mapped cancel flag
  int* d_cancel = nullptr;
  int64_t lattice_stride = 0;      // bytes per (CTA, group) lattice buffer
  int lattice_groups = 0;          // buffers per CTA
  std::vector<void*> owned;

  cudaGraphExec_t gexec = nullptr;
  bool graph_dirty = true;
  cudaEvent_t ev[3] = {nullptr, nullptr, nullptr};
  bool ran = false;
  std::string err;
};

namespace {

int fail(mp_state* h, int code, const char* fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof(buf), fmt, ap);
  va_end(ap);
  if (h) h->err = buf;
  else g_create_error = buf;
  return code;
}

int cuda_fail(mp_state* h, cudaError_t e, const char* what) {
  return fail(h, MP_ECUDA, "%s: %s", what, cudaGetErrorString(e));
}

#define MP_CUDA(h, call)                                  \
  do {                                                    \
    cudaError_t e_ = (call);                              \
    if (e_ != cudaSuccess) return cuda_fail((h), e_, #call); \
  } while (0)

// Makes the handle's device current for the scope and restores the caller's.
struct DeviceGuard {
  int prev = -1;
  explicit DeviceGuard(int dev) {
    if (cudaGetDevice(&prev) == cudaSuccess && prev != dev) cudaSetDevice(dev);
    else prev = -1;
  }
  ~DeviceGuard() {
    if (prev >= 0) cudaSetDevice(prev);
  }
};

void* dev_alloc(mp_state* h, size_t bytes) {
  bytes = (bytes + 255) / 256 * 256;
  void* p = nullptr;
  if (h->alloc_fn) {
    p = h->alloc_fn(h->alloc_ctx, bytes);
  } else if (cudaMalloc(&p, bytes) != cudaSuccess) {
    cudaGetLastError();
    p = nullptr;
  }
  if (p) h->owned.push_back(p);
  return p;
}

void dev_free(mp_state* h, void* p) {
  if (!p) return;
  for (size_t i = 0; i < h->owned.size(); ++i) {
    if (h->owned[i] == p) {
      h->owned.erase(h->owned.begin() + static_cast<long>(i));
      break;
    }
  }
  if (h->alloc_fn) h->free_fn(h->alloc_ctx, p);
  else cudaFree(p);
}

void release(mp_state* h) {
  if (h->stream) cudaStreamSynchronize(h->stream);
  if (h->gexec) cudaGraphExecDestroy(h->gexec);
  for (auto& e : h->ev)
    if (e) cudaEventDestroy(e);
  for (void* p : h->owned) {
    if (h->alloc_fn) h->free_fn(h->alloc_ctx, p);
    else cudaFree(p);
  }
  h->owned.clear();
  if (h->h_cancel) cudaFreeHost(h->h_cancel);
  if (h->own_stream && h->stream) cudaStreamDestroy(h->stream);
}

// Every system of a batch: lattice kind, size, temperature, couplings, paths.
int validate_systems(const mp_system* systems, int n, uint32_t flags) {
  for (int k = 0; k < n; ++k) {
    const mp_system& s = systems[k];
    if (s.lattice != MP_LATTICE_SC && s.lattice != MP_LATTICE_CHAIN && s.lattice != MP_LATTICE_ISING)
      return fail(nullptr, MP_EINVAL, "system %d: unknown lattice %d", k, s.lattice);
    if ((s.lattice == MP_LATTICE_ISING) != (systems[0].lattice == MP_LATTICE_ISING))
      return fail(nullptr, MP_EINVAL, "Ising and Heisenberg systems cannot share a batch");
    if (s.lattice == MP_LATTICE_ISING && (flags & MP_FLAG_RANDOM_SITE))
      return fail(nullptr, MP_EINVAL, "the random-site order is built for Heisenberg systems only");
    if (!(s.T > 0.0) || !std::isfinite(s.T) || !std::isfinite(s.J) || !std::isfinite(s.h))
      return fail(nullptr, MP_EINVAL, "system %d: need finite T > 0, J, h", k);
    if (s.n_paths < 1 || s.n_paths > 0x7fffffffLL)
      return fail(nullptr, MP_EINVAL, "system %d: n_paths must be in 1..2^31-1", k);
    if (s.path_begin < 0 || s.path_begin + s.n_paths > 0x100000000LL)
      return fail(nullptr, MP_EINVAL, "system %d: path ids path_begin .. path_begin + n_paths - 1 "
                  "must lie in 0..2^32-1", k);
    if (s.lattice == MP_LATTICE_SC) {
      if (s.L < 2 || (s.L & 1))
        return fail(nullptr, MP_EINVAL, "system %d: simple cubic L must be even and >= 2", k);
      if (s.L > 1024) return fail(nullptr, MP_EINVAL, "system %d: L=%d above 1024", k, s.L);
    } else if (s.lattice == MP_LATTICE_ISING) {
      if (s.L < 2 || (s.L & 1) || s.L > MP_ISING_MAX_L)
        return fail(nullptr, MP_EINVAL, "system %d: Ising L must be even in 2..%d", k, MP_ISING_MAX_L);
    } else if (s.L < 2 || s.L > 8192) {
      return fail(nullptr, MP_EINVAL, "system %d: chain length must be in 2..8192", k);
    }
  }
  return MP_OK;
}

int validate(const mp_config* cfg) {
  if (!cfg) return fail(nullptr, MP_EINVAL, "config is NULL");
  if (cfg->precision != MP_FP32 && cfg->precision != MP_FP64)
    return fail(nullptr, MP_EINVAL, "unknown precision %d", cfg->precision);
  if (cfg->init_mode < MP_INIT_SPHERE || cfg->init_mode > MP_INIT_ORDERED)
    return fail(nullptr, MP_EINVAL, "unknown init mode %d", cfg->init_mode);
  if (cfg->n_systems < 1 || cfg->n_systems > 65535 || !cfg->systems)
    return fail(nullptr, MP_EINVAL, "n_systems must be in 1..65535 with a systems array");
  if (cfg->n_therm < 0 || cfg->n_meas < 1)
    return fail(nullptr, MP_EINVAL, "need n_therm >= 0 and n_meas >= 1");
  if (cfg->n_therm + cfg->n_meas > 0xffffffffLL)
    return fail(nullptr, MP_EINVAL, "more than 2^32-1 sweeps");
  if (cfg->alloc_fn && !cfg->free_fn) return fail(nullptr, MP_EINVAL, "alloc_fn without free_fn");
  if (cfg->cta_threads != 0 &&
      (cfg->cta_threads < 32 || cfg->cta_threads > kMaxCta || cfg->cta_threads % 32))
    return fail(nullptr, MP_EINVAL, "cta_threads must be a multiple of 32 in 32..1024");
  if (cfg->threads_per_path != 0 &&
      (cfg->threads_per_path < 32 || cfg->threads_per_path > kMaxCta || cfg->threads_per_path % 32))
    return fail(nullptr, MP_EINVAL, "threads_per_path must be a multiple of 32 in 32..1024");
  return validate_systems(cfg->systems, cfg->n_systems, cfg->flags);
}

// Launch shape: threads per path from the sites per colour (about 8 sites per
// thread per half-sweep), paths per CTA from the CTA size, the named-barrier
// budget and shared memory; the CTA shrinks while there are too few work
// items to cover every SM twice.
int plan_random_site(mp_state* h);

int plan(mp_state* h, const mp_config* cfg) {
  if (h->flags & MP_FLAG_RANDOM_SITE) return plan_random_site(h);
  const int real = h->precision == MP_FP64 ? 8 : 4;
  const int n = static_cast<int>(h->systems.size());
  h->lattice_groups = 0;
  h->lattice_stride = 0;
  h->max_paths = 0;
  // one kernel per lattice size when the batch has a single size; lattices
  // too large for shared memory are streamed from HBM (any size, one kernel)
  int optin = 0;
  MP_CUDA(h, cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, h->device));
  auto global = [&](const mp_system& sy) { return in_place(sy, h->precision, h->flags, optin); };
  // lattices held by two-CTA clusters run in the mixed-size kernel
  auto variant_of = [&](const mp_system& sy) {
    if (sy.lattice == MP_LATTICE_ISING) return ising_compiled_L(sy.L) ? ising_variant(sy.L) : kIsingKernel;
    if (sy.lattice == MP_LATTICE_CHAIN) return -1;
    if (paired(sy, h->precision, h->flags)) return 0;  // the mixed-size kernel
    if (!streamed(sy, h->precision, h->flags)) return sy.L;
    if (global(sy)) return kGlobalKernel;
    // L = 32 and 64 have kernels compiled for their size
    return sy.L == 64 ? kStreamL64 : (sy.L == 32 ? kStreamL32 : -2);
  };
  int variant = variant_of(h->systems[0]);
  bool all_streamed = true;
  for (int k = 0; k < n; ++k) {
    const int v = variant_of(h->systems[k]);
    all_streamed = all_streamed && (v == -2 || v == kStreamL64 || v == kStreamL32 || v == kGlobalKernel);
    if (v != variant) variant = 0;
  }
  // streamed sizes mixed, or streamed with in-place ones: the streamed kernel runs both
  if (variant == 0 && all_streamed) variant = -2;
  // Ising sizes mixed (batches are all Ising or all Heisenberg): the kernel for any L
  if (variant == 0 && h->systems[0].lattice == MP_LATTICE_ISING) variant = kIsingKernel;
  h->variant = variant;
  int sms = 0, smem_max = 0, cta_max = 0;
  MP_CUDA(h, cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, h->device));
  MP_CUDA(h, sweep_prepare(h->precision, variant, h->device, &smem_max, &cta_max));
  // kernels with room for more registers per thread take more sites per thread
  const double target = cta_max <= 512 ? 16.0 : 8.0;
  MP_CUDA(h, reduce_prepare());
  std::vector<int> tp(n), slice(n), ring(n);
  // The partial-sum ring (sweeps per half): the largest power of two up to 16
  // among those that fit the most paths into one CTA -- shared memory, the
  // CTA size and the named barriers permit (a shorter ring only flushes to
  // the FP64 accumulators more often).
  auto pick_ring = [&](int& r, int& sl, auto need, int threads) {
    const int cap = std::max(1, threads > 32 ? std::min(15, cta_max / threads) : cta_max / threads);
    int best_r = 0, best_sl = 0, best_fit = -1;
    for (r = 16; r >= 1; r /= 2) {
      const int s = need();
      const int fit = s <= smem_max ? std::min(cap, smem_max / s) : 0;
      if (fit > best_fit) {
        best_fit = fit;
        best_r = r;
        best_sl = s;
      }
    }
    r = best_r;
    sl = best_sl;
  };
  int max_tp = 32;
  for (int k = 0; k < n; ++k) {
    const int64_t N = sites_of(h->systems[k]);
    const int NH = static_cast<int>((N + 1) / 2);
    int t = (static_cast<int>(h->tp_override.size()) > k && h->tp_override[k] > 0) ? h->tp_override[k]
                                                                                  : cfg->threads_per_path;
    if (paired(h->systems[k], h->precision, h->flags)) {
      // one CTA of cta_max threads on each half: one column of L/2 planes per thread
      if (t != 0 && t != cta_max)
        return fail(h, MP_EINVAL, "system %d: L=%d runs on two-CTA clusters of %d threads each", k,
                    h->systems[k].L, cta_max);
      tp[k] = cta_max;
      ring[k] = 16;
      // the ring of the CTA that owns the path holds both CTAs' warps
      auto need = [&]() {
        return round_up(slice_spin_offset(2 * cta_max, ring[k]) + pair_spin_bytes(kPairL, real), 128);
      };
      pick_ring(ring[k], slice[k], need, cta_max);
      if (slice[k] > smem_max)
        return fail(h, MP_EINVAL, "system %d: L=%d needs %d bytes of shared memory per CTA (max %d)", k,
                    h->systems[k].L, slice[k], smem_max);
      max_tp = std::max(max_tp, cta_max);
      continue;
    }
    if (global(h->systems[k])) {
      // in place in HBM: one CTA's worth of threads per path by default
      if (t == 0) t = cta_max;
      if (t > cta_max) return fail(h, MP_EINVAL, "threads_per_path %d above %d", t, cta_max);
      tp[k] = t;
      ring[k] = 16;
      pick_ring(ring[k], slice[k], [&]() { return round_up(slice_spin_offset(t, ring[k]), 128); }, t);
      max_tp = std::max(max_tp, t);
      continue;
    }
    if (streamed(h->systems[k], h->precision, h->flags)) {
      // one thread per column x/2 of a z-plane and about L/4 rows per thread
      const int L = h->systems[k].L, HL = L / 2;
      if (t == 0) t = std::min(cta_max, round_up(HL * ((L + 3) / 4), 32));
      if (t > cta_max || t < HL)
        return fail(h, MP_EINVAL, "system %d: threads_per_path %d outside %d..%d", k, t, HL, cta_max);
      tp[k] = t;
      ring[k] = 16;
      auto need = [&]() {
        return round_up(slice_spin_offset(t, ring[k]) + 128 + 9 * half_plane_bytes(L, real), 128);
      };
      pick_ring(ring[k], slice[k], need, t);
      if (slice[k] > smem_max)
        return fail(h, MP_EINVAL, "system %d: L=%d needs %d bytes of shared memory for its "
                    "half-plane ring (max %d)", k, L, slice[k], smem_max);
      max_tp = std::max(max_tp, t);
      continue;
    }
    if (t == 0 && h->systems[k].lattice == MP_LATTICE_SC) {
      // a divisor of the sites per colour lets each thread walk a block of
      // columns; pick the one closest to the target sites per thread
      double best = 1e30;
      for (int c = 32; c <= std::min(cta_max, NH); c += 32) {
        if (NH % c) continue;
        const double d = std::fabs(static_cast<double>(NH) / c - target);
        if (d < best) {
          best = d;
          t = c;
        }
      }
    }
    if (t == 0)
      t = std::min(cta_max, std::max(32, round_up(static_cast<int>(std::ceil(NH / target)), 32)));
    if (t > cta_max) return fail(h, MP_EINVAL, "threads_per_path %d above %d", t, cta_max);
    tp[k] = t;
    // partial-sum ring: the largest power of two up to 16 sweeps that fits
    ring[k] = 16;
    // shared-memory bytes of the lattice (Ising: with a copy of each boundary row)
    const int64_t lat = h->systems[k].lattice == MP_LATTICE_ISING ? ising_slice_spin_bytes(h->systems[k].L)
                                                                   : lattice_bytes(h->systems[k], real);
    pick_ring(ring[k], slice[k], [&]() {
      return static_cast<int>(std::min<int64_t>(INT32_MAX / 2, round_up(slice_spin_offset(t, ring[k]) + lat, 128)));
    }, t);
    if (slice[k] > smem_max)
      return fail(h, MP_EINVAL, "system %d needs %d bytes of shared memory per path (max %d)", k,
                  slice[k], smem_max);
    max_tp = std::max(max_tp, t);
  }
  auto paths_per_cta = [&](int k, int cta) {
    if (paired(h->systems[k], h->precision, h->flags)) return 1;  // one path per cluster
    int g = cta / tp[k];
    if (tp[k] > 32) g = std::min(g, 15);  // named barriers 1..15
    g = std::min<int64_t>(g, smem_max / slice[k]);
    g = static_cast<int>(std::min<int64_t>(g, h->systems[k].n_paths));
    return std::max(g, 1);
  };
  auto count_items = [&](int cta) {
    int64_t items = 0;
    for (int k = 0; k < n; ++k) {
      const int g = paths_per_cta(k, cta);
      items += (h->systems[k].n_paths + g - 1) / g;
    }
    return items;
  };
  int cta = cfg->cta_threads;
  if (cta > cta_max) return fail(h, MP_EINVAL, "cta_threads %d above %d for this precision", cta, cta_max);
  if (cta == 0) {
    cta = cta_max;
    while (cta / 2 >= std::max(max_tp, 128) && count_items(cta) < 2LL * sms) cta /= 2;
  }
  if (cta < max_tp) return fail(h, MP_EINVAL, "cta_threads %d below threads per path %d", cta, max_tp);

  if (cta < cta_max) {
    for (int k = 0; k < n; ++k)
      if (paired(h->systems[k], h->precision, h->flags))
        return fail(h, MP_EINVAL, "cta_threads %d: L=%d runs on two-CTA clusters of %d threads each", cta,
                    h->systems[k].L, cta_max);
  }

  h->hsys.resize(n);
  h->items.clear();
  h->pair_items.clear();
  h->spin_offset.assign(n, 0);
  int smem = 0;
  int64_t rec = 0, spins = 0;
  for (int k = 0; k < n; ++k) {
    const mp_system& s = h->systems[k];
    DevSystem& d = h->hsys[k];
    d.lattice = s.lattice;
    d.L = s.L;
    d.N = static_cast<int32_t>(sites_of(s));
    d.NH = (d.N + 1) / 2;
    d.tp = tp[k];
    d.g = paths_per_cta(k, cta);
    d.slice_bytes = slice[k];
    d.ring = ring[k];
    d.T = s.T;
    d.J = s.J;
    d.h = s.h;
    d.beta = 1.0 / s.T;
    d.rec_offset = rec;
    d.n_paths = s.n_paths;
    d.path_begin = s.path_begin;
    d.mode = paired(s, h->precision, h->flags) ? kModePair
             : global(s)                         ? kModeGlobal
             : streamed(s, h->precision, h->flags) ? kModeStreamed : kModeShared;
    d.unit_K = 0;  // unit tables are made when the plan's tables are uploaded
    d.unit_off = -1;
    d.unit_U = 0;
    if (d.mode == kModeStreamed) {
      h->lattice_groups = std::max(h->lattice_groups, d.g);
      h->lattice_stride = std::max<int64_t>(
          h->lattice_stride, static_cast<int64_t>(2) * s.L * half_plane_bytes(s.L, real));
    } else if (d.mode == kModeGlobal) {  // the shared-memory layout, in HBM
      h->lattice_groups = std::max(h->lattice_groups, d.g);
      h->lattice_stride = std::max<int64_t>(h->lattice_stride, lattice_bytes(s, real));
    }
    rec += s.n_paths;
    h->spin_offset[k] = spins;
    spins += s.n_paths * 3 * static_cast<int64_t>(d.N);
    smem = std::max(smem, d.g * d.slice_bytes);
    if (d.mode == kModePair) {
      for (int64_t p0 = 0; p0 < s.n_paths; ++p0) h->pair_items.push_back(WorkItem{k, 1, p0});
    } else {
      for (int64_t p0 = 0; p0 < s.n_paths; p0 += d.g)
        h->items.push_back(WorkItem{k, static_cast<int32_t>(std::min<int64_t>(d.g, s.n_paths - p0)), p0});
    }
    h->max_paths = std::max(h->max_paths, s.n_paths);
  }
  // largest lattices first, so the persistent CTAs finish together
  std::stable_sort(h->items.begin(), h->items.end(), [&](const WorkItem& a, const WorkItem& b) {
    return h->hsys[a.sys].N > h->hsys[b.sys].N;
  });
  if (h->items.size() > 0x7fffffffULL) return fail(h, MP_EINVAL, "too many work items");
  h->total_paths = rec;
  h->total_spins = spins;
  h->cta = cta;
  h->smem = smem;
  int per_sm = 0;
  MP_CUDA(h, sweep_occupancy(h->precision, variant, cta, smem, &per_sm));
  if (per_sm < 1) return fail(h, MP_EINVAL, "launch shape %d threads x %d bytes does not fit an SM", cta, smem);
  h->grid = static_cast<int>(std::min<int64_t>(static_cast<int64_t>(h->items.size()),
                                               static_cast<int64_t>(sms) * per_sm));
  if (!h->pair_items.empty()) {
    // a launch in clusters of two CTAs: as many clusters as can be resident
    int clusters = 0;
    MP_CUDA(h, sweep_cluster_occupancy(h->precision, variant, cta, smem, &clusters));
    if (clusters < 1)
      return fail(h, MP_EINVAL, "no two-CTA cluster of %d threads x %d bytes fits the device", cta, smem);
    h->grid = 2 * clusters;
  }
  return MP_OK;
}

// The random-site order: one thread per path (128-thread CTAs), every path's
// lattice in HBM; no work items.
int plan_random_site(mp_state* h) {
  const int n = static_cast<int>(h->systems.size());
  h->variant = kRandomSiteKernel;
  h->hsys.resize(n);
  h->items.clear();
  h->spin_offset.assign(n, 0);
  h->max_paths = 0;
  int64_t rec = 0, spins = 0;
  for (int k = 0; k < n; ++k) {
    const mp_system& s = h->systems[k];
    DevSystem& d = h->hsys[k];
    d = DevSystem{};
    d.lattice = s.lattice;
    d.L = s.L;
    d.N = static_cast<int32_t>(sites_of(s));
    d.NH = (d.N + 1) / 2;
    d.tp = 1;
    d.g = 1;
    d.ring = 1;
    d.T = s.T;
    d.J = s.J;
    d.h = s.h;
    d.beta = 1.0 / s.T;
    d.rec_offset = rec;
    d.n_paths = s.n_paths;
    d.path_begin = s.path_begin;
    d.mode = kModeShared;
    rec += s.n_paths;
    h->spin_offset[k] = spins;
    spins += s.n_paths * 3 * static_cast<int64_t>(d.N);
    h->max_paths = std::max(h->max_paths, s.n_paths);
  }
  h->total_paths = rec;
  h->total_spins = spins;
  h->cta = 128;
  h->smem = 0;
  const int64_t grid = (rec + 127) / 128;
  if (grid > 0x7fffffffLL) return fail(h, MP_EINVAL, "too many paths");
  h->grid = static_cast<int>(grid);
  h->lattice_groups = 0;
  h->lattice_stride = 0;
  MP_CUDA(h, reduce_prepare());
  return MP_OK;
}

// One run of sweeps [s_begin, s_end) of the schedule, then the reduction.
int enqueue_run(mp_state* h, int64_t s_begin, int64_t s_end, bool resume, bool save,
                bool capturing = false) {
  SweepParams p{};
  p.systems = h->d_sys;
  p.items = h->d_items;
  p.queue = h->d_queue;
  p.records = h->d_rec;
  p.spins = h->d_spins;
  p.spin_offset = h->d_spin_offset;
  p.n_items = static_cast<int32_t>(h->items.size());
  p.pair_items = h->d_items + h->items.size();
  p.n_pair_items = static_cast<int32_t>(h->pair_items.size());
  p.pair_queue = h->d_queue + 1;
  p.init_mode = h->init_mode | ((h->flags & MP_FLAG_TWO_START) ? kTwoStart : 0);
  p.key = philox_round_keys(h->seed);
  p.lattice = h->d_lattice;
  p.lattice_stride = h->lattice_stride;
  p.lattice_groups = h->lattice_groups;
  p.error = h->d_error;
  p.ising_thr = h->d_thr;
  p.units = h->d_units;
  p.test_stall = (h->flags & MP_FLAG_TEST_STALL) ? 1u : 0u;
  p.s_begin = s_begin;
  p.s_end = s_end;
  p.state = save || resume ? h->d_state : nullptr;
  p.state_offset = h->d_state_offset;
  p.state_stride = h->d_state_stride;
  p.resume = resume ? 1 : 0;
  p.save = save ? 1 : 0;
  p.cancel = h->d_cancel;
  p.n_therm = h->n_therm;
  p.n_meas = h->n_meas;
  ReduceParams r{};
  r.systems = h->d_sys;
  r.records = h->d_rec;
  r.est = h->d_est;
  r.n_therm = std::min(s_end, h->n_therm);
  r.n_meas = std::max<int64_t>(0, s_end - h->n_therm);
  r.sort_buf = h->d_sort;
  const unsigned evflag = capturing ? cudaEventRecordExternal : cudaEventRecordDefault;
  MP_CUDA(h, cudaMemsetAsync(h->d_queue, 0, 2 * sizeof(int), h->stream));
  MP_CUDA(h, cudaMemsetAsync(h->d_error, 0, sizeof(int), h->stream));
  MP_CUDA(h, cudaEventRecordWithFlags(h->ev[0], h->stream, evflag));
  if (h->variant == kRandomSiteKernel)
    MP_CUDA(h, launch_random_site(h->precision, p, static_cast<int>(h->hsys.size()), h->total_paths,
                                  h->d_lattice, h->total_spins / 3, h->stream));
  else
    MP_CUDA(h, launch_sweep(h->precision, h->variant, p, h->grid, h->cta, h->smem, h->stream));
  MP_CUDA(h, cudaEventRecordWithFlags(h->ev[1], h->stream, evflag));
  MP_CUDA(h, launch_reduce(r, static_cast<int>(h->hsys.size()), h->max_paths, h->stream));
  MP_CUDA(h, cudaEventRecordWithFlags(h->ev[2], h->stream, evflag));
  return MP_OK;
}

}  // namespace

// The HBM lattice buffers of the current plan (streamed paths), grown on demand.
int ensure_lattice(mp_state* h) {
  size_t need = 0;
  if (h->variant == kRandomSiteKernel) {  // every path's lattice
    need = static_cast<size_t>(h->total_spins / 3) * random_site_bytes_per_site(h->precision);
  } else {
    if (h->lattice_groups == 0) return MP_OK;
    h->lattice_stride = (h->lattice_stride + 255) / 256 * 256;
    need = static_cast<size_t>(h->grid) * h->lattice_groups * h->lattice_stride;
  }
  if (need <= h->lattice_capacity) return MP_OK;
  MP_CUDA(h, cudaStreamSynchronize(h->stream));
  dev_free(h, h->d_lattice);
  h->d_lattice = dev_alloc(h, need);
  h->lattice_capacity = h->d_lattice ? need : 0;
  if (!h->d_lattice) return fail(h, MP_ENOMEM, "lattice buffer allocation failed");
  return MP_OK;
}

// Tables of a launch: systems, the given work items and, after them, the
// paths for two-CTA clusters (with_pairs).
int upload_tables(mp_state* h, const std::vector<WorkItem>& items, bool with_pairs) {
  const int n = static_cast<int>(h->hsys.size());
  // The column-walk units of the simple cubic lattices in shared memory, one
  // table per (L, K, U) shared by every system with those values: the host
  // decodes each unit once instead of every thread at every half-sweep.  U is
  // the chunk of the kernel the plan launches (the mixed-size kernel's for a
  // batch of uneven sizes).
  std::vector<int4> units;
  std::map<std::tuple<int, int, int>, int> unit_at;
  const bool mixed = h->variant == 0;
  const int real = h->precision == MP_FP64 ? 8 : 4;
  for (int k = 0; k < n; ++k) {
    DevSystem& d = h->hsys[k];
    d.unit_off = -1;
    d.unit_K = 0;
    d.unit_U = 0;
    if ((h->flags & MP_FLAG_DEVICE_UNITS) || h->variant == kRandomSiteKernel || d.lattice != MP_LATTICE_SC ||
        d.mode != kModeShared)
      continue;
    const int U = column_chunk(real, d.L, mixed);
    const int K = column_segments(d.L, U, d.tp);
    const int n_units = d.L * d.L / 2 * K;
    auto it = unit_at.find(std::make_tuple(d.L, K, U));
    if (it == unit_at.end()) {
      if (static_cast<int64_t>(units.size()) + n_units > h->units_capacity)
        return fail(h, MP_ENOMEM, "system %d: no room for its column-walk unit table", k);
      it = unit_at.emplace(std::make_tuple(d.L, K, U), static_cast<int>(units.size())).first;
      for (int u = 0; u < n_units; ++u) units.push_back(column_unit(d.L, K, u));
    }
    d.unit_off = it->second;
    d.unit_K = K;
    d.unit_U = U;
  }
  int64_t bytes = 0;
  auto copy = [&](void* dst, const void* src, size_t b) {
    bytes += static_cast<int64_t>(b);
    return cudaMemcpyAsync(dst, src, b, cudaMemcpyHostToDevice, h->stream);
  };
  MP_CUDA(h, copy(h->d_sys, h->hsys.data(), sizeof(DevSystem) * n));
  if (!items.empty()) MP_CUDA(h, copy(h->d_items, items.data(), sizeof(WorkItem) * items.size()));
  if (with_pairs && !h->pair_items.empty())
    MP_CUDA(h, copy(h->d_items + items.size(), h->pair_items.data(), sizeof(WorkItem) * h->pair_items.size()));
  MP_CUDA(h, copy(h->d_spin_offset, h->spin_offset.data(), sizeof(int64_t) * n));
  std::vector<unsigned long long> thr(10 * static_cast<size_t>(n), 0ull);
  for (int k = 0; k < n; ++k)
    if (h->systems[k].lattice == MP_LATTICE_ISING) ising_thresholds(h->systems[k], &thr[10 * k]);
  MP_CUDA(h, copy(h->d_thr, thr.data(), sizeof(unsigned long long) * thr.size()));
  if (!units.empty()) MP_CUDA(h, copy(h->d_units, units.data(), sizeof(int4) * units.size()));
  MP_CUDA(h, cudaStreamSynchronize(h->stream));
  h->upload_bytes = bytes;
  return MP_OK;
}

// Throughput (attempts per ms) of system k under the current plan: one wave
// of its work items through the real sweep kernel, timed for s and for 2 s
// sweeps (about 1e8 attempts per s); the difference leaves out what does not
// scale with the sweeps (launch, initial state, records), which would
// otherwise favour layouts whose wave holds fewer paths.  Returns < 0 on
// error.
double calibrate(mp_state* h, int k) {
  std::vector<WorkItem> sub;
  int64_t paths = 0;
  for (const WorkItem& it : h->items) {
    if (it.sys != k) continue;
    sub.push_back(it);
    paths += it.count;
    if (static_cast<int>(sub.size()) >= h->grid) break;
  }
  if (sub.empty() || upload_tables(h, sub, false) != MP_OK || ensure_lattice(h) != MP_OK) return -1.0;
  const double per_sweep = static_cast<double>(paths) * h->hsys[k].N;
  const int64_t s1 = std::max<int64_t>(2, std::min<int64_t>(256, static_cast<int64_t>(1e8 / per_sweep)));
  SweepParams p{};
  p.systems = h->d_sys;
  p.items = h->d_items;
  p.queue = h->d_queue;
  p.records = h->d_rec;
  p.n_items = static_cast<int32_t>(sub.size());
  p.init_mode = h->init_mode | ((h->flags & MP_FLAG_TWO_START) ? kTwoStart : 0);
  p.s_begin = 0;
  p.key = philox_round_keys(h->seed);
  p.lattice = h->d_lattice;
  p.lattice_stride = h->lattice_stride;
  p.lattice_groups = h->lattice_groups;
  p.error = h->d_error;
  p.ising_thr = h->d_thr;
  p.units = h->d_units;
  // the faster of two timed launches of `sweeps` sweeps (half thermalisation,
  // half measurement, like a typical run); < 0 on error
  auto timed = [&](int64_t sweeps) -> float {
    p.n_therm = sweeps / 2;
    p.n_meas = sweeps - sweeps / 2;
    p.s_end = sweeps;
    float best = -1.f;
    for (int rep = 0; rep < 2; ++rep) {
      float ms = 0.f;
      if (cudaMemsetAsync(h->d_queue, 0, sizeof(int), h->stream) != cudaSuccess ||
          cudaMemsetAsync(h->d_error, 0, sizeof(int), h->stream) != cudaSuccess ||
          cudaEventRecord(h->ev[0], h->stream) != cudaSuccess ||
          launch_sweep(h->precision, h->variant, p, std::min<int>(h->grid, static_cast<int>(sub.size())),
                       h->cta, h->smem, h->stream) != cudaSuccess ||
          cudaEventRecord(h->ev[1], h->stream) != cudaSuccess ||
          cudaEventSynchronize(h->ev[1]) != cudaSuccess ||
          cudaEventElapsedTime(&ms, h->ev[0], h->ev[1]) != cudaSuccess) {
        cudaGetLastError();
        return -1.f;
      }
      if (best < 0.f || ms < best) best = ms;
    }
    return best;
  };
  const float t1 = timed(s1), t2 = timed(2 * s1);
  if (t1 < 0.f || t2 < 0.f) return -1.0;
  if (t2 <= t1) return per_sweep * 2 * s1 / std::max(t2, 1e-3f);  // too short to separate
  return per_sweep * s1 / (t2 - t1);
}

// Threads-per-path candidates of system k for the autotuner.
std::vector<int> tp_candidates(mp_state* h, int k, int cta_max) {
  const mp_system& sy = h->systems[k];
  std::vector<int> c;
  auto add = [&](int t) {
    t = round_up(std::max(t, 32), 32);
    if (t <= cta_max && std::find(c.begin(), c.end(), t) == c.end()) c.push_back(t);
  };
  const int64_t N = sites_of(sy);
  const int NH = static_cast<int>((N + 1) / 2);
  if (paired(sy, h->precision, h->flags)) return c;  // one fixed layout
  if (streamed(sy, h->precision, h->flags)) {
    const int HL = sy.L / 2;
    for (int r : {2, 4, 8}) add(std::max(HL, HL * ((sy.L + r - 1) / r)));
    return c;
  }
  // every multiple of 32 with 2 .. 48 sites per thread: the column-segment
  // walk runs any of them, and how well a count splits the columns is easier
  // to measure than to model.  Ising paths also try up to 64 sites per thread:
  // their lattices are bytes, so one warp per path (synchronised by
  // __syncwarp instead of a named barrier) fits 32 paths into a CTA, which at
  // L = 60 beats every wider layout.
  const double max_sites = sy.lattice == MP_LATTICE_ISING ? 64.0 : 48.0;
  for (int t = 32; t <= std::min(cta_max, NH); t += 32) {
    const double sites = static_cast<double>(NH) / t;
    if (sites >= 2.0 && sites <= max_sites) add(t);
  }
  return c;
}

// The autotuner's choices, remembered for the life of the process: a later
// handle whose batch has the same shape on the same device (the key below)
// takes the measured layout without timing it again.  Temperatures, fields
// and seeds are not part of the key: they do not change the launch shape.
std::mutex g_tune_mu;
std::map<std::string, std::vector<int>> g_tune_memo;

std::string tune_key(const mp_state* h, const mp_config* cfg) {
  std::string k = std::to_string(h->device) + "/" + std::to_string(h->precision) + "/" +
                  std::to_string(h->flags & (MP_FLAG_STREAM | MP_FLAG_TWO_START | MP_FLAG_DEVICE_UNITS)) + "/" +
                  std::to_string(h->init_mode) + "/" + std::to_string(cfg->cta_threads);
  for (const mp_system& s : h->systems)
    k += "/" + std::to_string(s.lattice) + ":" + std::to_string(s.L) + ":" + std::to_string(s.n_paths);
  return k;
}

// Pick each system's threads per path by measuring the candidates in the
// batch's own kernel; leaves the handle planned with the choice.
int autotune(mp_state* h, const mp_config* cfg) {
  const int n = static_cast<int>(h->systems.size());
  const std::string key = tune_key(h, cfg);
  {
    std::lock_guard<std::mutex> lock(g_tune_mu);
    auto it = g_tune_memo.find(key);
    if (it != g_tune_memo.end() && static_cast<int>(it->second.size()) == n) {
      h->tp_override = it->second;
      return plan(h, cfg);
    }
  }
  h->tp_override.assign(n, 0);
  int smem_max = 0, cta_max = 0;
  MP_CUDA(h, sweep_prepare(h->precision, h->variant, h->device, &smem_max, &cta_max));
  for (int k = 0; k < n; ++k) {
    // systems of the same lattice kind and size share the choice
    int same = -1;
    for (int j = 0; j < k && same < 0; ++j)
      if (h->systems[j].lattice == h->systems[k].lattice && h->systems[j].L == h->systems[k].L) same = j;
    if (same >= 0) {
      h->tp_override[k] = h->tp_override[same];
      continue;
    }
    const std::vector<int> cands = tp_candidates(h, k, cta_max);
    if (cands.size() < 2) continue;
    double best = -1.0;
    int best_t = 0;
    for (int t : cands) {
      h->tp_override[k] = t;
      if (plan(h, cfg) != MP_OK) continue;
      // the one-wave rate, times the fraction of the persistent grid's work
      // the batch's items fill (few large items leave CTAs idle at the end)
      const int64_t items = static_cast<int64_t>(h->items.size());
      const int64_t waves = (items + h->grid - 1) / h->grid;
      const double fill = waves > 0 ? static_cast<double>(items) / static_cast<double>(waves * h->grid) : 1.0;
      const double rate = calibrate(h, k) * fill;
      if (rate > best) {
        best = rate;
        best_t = t;
      }
    }
    h->tp_override[k] = best_t;
  }
  h->err.clear();
  const int rc = plan(h, cfg);
  if (rc == MP_OK) {
    std::lock_guard<std::mutex> lock(g_tune_mu);
    g_tune_memo[key] = h->tp_override;
  }
  return rc;
}

// After the stream has drained: MP_ETIMEOUT if a kernel's bounded wait gave up.
int check_error_flag(mp_state* h) {
  int flag = 0;
  MP_CUDA(h, cudaMemcpy(&flag, h->d_error, sizeof(int), cudaMemcpyDeviceToHost));
  if (flag == kErrCanceled) return fail(h, MP_ECANCELED, "the run was canceled; results invalid");
  if (flag == kErrLaunch) return fail(h, MP_ECUDA, "two-CTA cluster paths ran without a cluster launch");
  if (flag) return fail(h, MP_ETIMEOUT, "a bulk copy did not complete in time; results invalid");
  return MP_OK;
}

extern "C" {

int mp_create(int L, double T, double J, double h, int64_t n_paths, int64_t n_therm, int64_t n_meas,
              uint64_t seed, mp_handle* out) {
  mp_system s{MP_LATTICE_SC, L, T, J, h, n_paths};
  mp_config cfg{};
  cfg.precision = MP_FP32;
  cfg.init_mode = MP_INIT_SPHERE;
  cfg.n_systems = 1;
  cfg.flags = MP_FLAG_GRAPH;
  cfg.systems = &s;
  cfg.n_therm = n_therm;
  cfg.n_meas = n_meas;
  cfg.seed = seed;
  return mp_create_ex(&cfg, out);
}

int mp_create_ex(const mp_config* cfg, mp_handle* out) {
  g_create_error.clear();
  if (!out) return fail(nullptr, MP_EINVAL, "out is NULL");
  *out = nullptr;
  int rc = validate(cfg);
  if (rc != MP_OK) return rc;
  mp_state* h = new mp_state();
  if (cudaGetDevice(&h->device) != cudaSuccess) {
    cudaGetLastError();
    delete h;
    return fail(nullptr, MP_ECUDA, "no CUDA device");
  }
  h->precision = cfg->precision;
  h->init_mode = cfg->init_mode;
  h->flags = cfg->flags;
  h->n_therm = cfg->n_therm;
  h->n_meas = cfg->n_meas;
  h->seed = cfg->seed;
  h->alloc_fn = cfg->alloc_fn;
  h->free_fn = cfg->free_fn;
  h->alloc_ctx = cfg->alloc_ctx;
  h->systems.assign(cfg->systems, cfg->systems + cfg->n_systems);
  auto bail = [&](int code) {
    g_create_error = h->err;
    release(h);
    delete h;
    return code;
  };
  if (cfg->stream) {
    h->stream = static_cast<cudaStream_t>(cfg->stream);
  } else {
    cudaError_t e = cudaStreamCreateWithFlags(&h->stream, cudaStreamNonBlocking);
    if (e != cudaSuccess) return bail(cuda_fail(h, e, "cudaStreamCreateWithFlags"));
    h->own_stream = true;
  }
  rc = plan(h, cfg);
  if (rc != MP_OK) return bail(rc);
  for (auto& e : h->ev) {
    cudaError_t ce = cudaEventCreate(&e);
    if (ce != cudaSuccess) return bail(cuda_fail(h, ce, "cudaEventCreate"));
  }
  {  // the cancel flag: host memory the kernels can read while they run
    cudaError_t ce = cudaHostAlloc(reinterpret_cast<void**>(&h->h_cancel), sizeof(int), cudaHostAllocMapped);
    if (ce != cudaSuccess) return bail(cuda_fail(h, ce, "cudaHostAlloc"));
    *h->h_cancel = 0;
    ce = cudaHostGetDevicePointer(reinterpret_cast<void**>(&h->d_cancel), h->h_cancel, 0);
    if (ce != cudaSuccess) return bail(cuda_fail(h, ce, "cudaHostGetDevicePointer"));
  }
  const int n = static_cast<int>(h->hsys.size());
  h->d_sys = static_cast<DevSystem*>(dev_alloc(h, sizeof(DevSystem) * n));
  h->d_items = static_cast<WorkItem*>(dev_alloc(h, sizeof(WorkItem) * h->total_paths));  // any plan fits
  h->d_queue = static_cast<int*>(dev_alloc(h, 256));
  h->d_rec = static_cast<double*>(dev_alloc(h, sizeof(double) * MP_NREC * h->total_paths));
  h->d_est = static_cast<double*>(dev_alloc(h, sizeof(double) * MP_NEST * n));
  h->d_spin_offset = static_cast<int64_t*>(dev_alloc(h, sizeof(int64_t) * n));
  h->d_thr = static_cast<unsigned long long*>(dev_alloc(h, sizeof(unsigned long long) * 10 * n));
  // unit tables: at most L^3/2 units per simple cubic size that fits shared memory
  h->units_capacity = 0;
  for (const mp_system& s : h->systems)
    if (s.lattice == MP_LATTICE_SC && s.L <= 26) h->units_capacity += static_cast<int64_t>(s.L) * s.L * s.L / 2;
  h->d_units = h->units_capacity > 0 ? static_cast<int4*>(dev_alloc(h, sizeof(int4) * h->units_capacity)) : nullptr;
  if (!h->d_sys || !h->d_items || !h->d_queue || !h->d_rec || !h->d_est || !h->d_spin_offset ||
      !h->d_thr || (h->units_capacity > 0 && !h->d_units))
    return bail(fail(h, MP_ENOMEM, "device allocation failed"));
  h->d_error = static_cast<int*>(dev_alloc(h, 256));
  if (!h->d_error) return bail(fail(h, MP_ENOMEM, "device allocation failed"));
  if (h->max_paths > MP_R_MAX_PATHS) {  // sorting space for r beyond shared memory
    h->d_sort = static_cast<double*>(dev_alloc(h, sizeof(double) * 2 * h->total_paths));
    if (!h->d_sort) return bail(fail(h, MP_ENOMEM, "sort buffer allocation failed"));
  }
  if (h->flags & MP_FLAG_KEEP_SPINS) {
    h->d_spins = static_cast<double*>(dev_alloc(h, sizeof(double) * h->total_spins));
    if (!h->d_spins) return bail(fail(h, MP_ENOMEM, "spin buffer allocation failed"));
  }
  if ((h->flags & MP_FLAG_AUTOTUNE) && cfg->threads_per_path == 0 && !(h->flags & MP_FLAG_RANDOM_SITE)) {
    rc = autotune(h, cfg);
    if (rc != MP_OK) return bail(rc);
  }
  rc = ensure_lattice(h);
  if (rc != MP_OK) return bail(rc);
  rc = upload_tables(h, h->items, true);
  if (rc != MP_OK) return bail(rc);
  *out = h;
  return MP_OK;
}

int mp_run(mp_handle h) {
  if (!h) return fail(nullptr, MP_EINVAL, "handle is NULL");
  DeviceGuard dg(h->device);
  if (!(h->flags & MP_FLAG_GRAPH)) {
    *h->h_cancel = 0;
    int rc = enqueue_run(h, 0, h->n_therm + h->n_meas, false, false);
    if (rc != MP_OK) return rc;
    h->ran = true;
    return MP_OK;
  }
  if (h->graph_dirty || !h->gexec) {
    if (h->gexec) {
      cudaGraphExecDestroy(h->gexec);
      h->gexec = nullptr;
    }
    MP_CUDA(h, cudaStreamBeginCapture(h->stream, cudaStreamCaptureModeThreadLocal));
    int rc = enqueue_run(h, 0, h->n_therm + h->n_meas, false, false, true);
    cudaGraph_t graph = nullptr;
    cudaError_t e = cudaStreamEndCapture(h->stream, &graph);
    if (rc != MP_OK) {
      if (graph) cudaGraphDestroy(graph);
      return rc;
    }
    if (e != cudaSuccess) return cuda_fail(h, e, "cudaStreamEndCapture");
    e = cudaGraphInstantiate(&h->gexec, graph, 0);
    cudaGraphDestroy(graph);
    if (e != cudaSuccess) return cuda_fail(h, e, "cudaGraphInstantiate");
    h->graph_dirty = false;
  }
  *h->h_cancel = 0;
  MP_CUDA(h, cudaGraphLaunch(h->gexec, h->stream));
  h->ran = true;
  return MP_OK;
}

int mp_set_seed(mp_handle h, uint64_t seed) {
  if (!h) return fail(nullptr, MP_EINVAL, "handle is NULL");
  if (seed != h->seed) {
    h->seed = seed;
    h->graph_dirty = true;
  }
  return MP_OK;
}

int mp_estimates(mp_handle h, int system, mp_estimates_t* out) {
  if (!h) return fail(nullptr, MP_EINVAL, "handle is NULL");
  if (!out || system < 0 || system >= static_cast<int>(h->hsys.size()))
    return fail(h, MP_EINVAL, "bad system index %d or NULL output", system);
  if (!h->ran) return fail(h, MP_ESTATE, "no run yet");
  DeviceGuard dg(h->device);
  MP_CUDA(h, cudaMemcpyAsync(out, h->d_est + static_cast<int64_t>(system) * MP_NEST,
                             sizeof(mp_estimates_t), cudaMemcpyDeviceToHost, h->stream));
  MP_CUDA(h, cudaStreamSynchronize(h->stream));
  float ms = 0.f;  // sweep and reduction kernels of the last run
  out->elapsed_s = cudaEventElapsedTime(&ms, h->ev[0], h->ev[2]) == cudaSuccess ? 1e-3 * ms : NAN;
  cudaGetLastError();
  return check_error_flag(h);
}

int mp_paths(mp_handle h, int system, double* host_out, int64_t cap) {
  if (!h) return fail(nullptr, MP_EINVAL, "handle is NULL");
  if (!host_out || system < 0 || system >= static_cast<int>(h->hsys.size()))
    return fail(h, MP_EINVAL, "bad system index %d or NULL output", system);
  const DevSystem& d = h->hsys[system];
  if (cap < d.n_paths * MP_NREC) return fail(h, MP_EINVAL, "capacity %lld below %lld", (long long)cap,
                                            (long long)(d.n_paths * MP_NREC));
  if (!h->ran) return fail(h, MP_ESTATE, "no run yet");
  DeviceGuard dg(h->device);
  MP_CUDA(h, cudaMemcpyAsync(host_out, h->d_rec + d.rec_offset * MP_NREC,
                             sizeof(double) * MP_NREC * d.n_paths, cudaMemcpyDeviceToHost, h->stream));
  MP_CUDA(h, cudaStreamSynchronize(h->stream));
  return check_error_flag(h);
}

int mp_device_buffers(mp_handle h, double** d_records, double** d_estimates) {
  if (!h) return fail(nullptr, MP_EINVAL, "handle is NULL");
  if (d_records) *d_records = h->d_rec;
  if (d_estimates) *d_estimates = h->d_est;
  return MP_OK;
}

int mp_spins(mp_handle h, int system, int64_t path, double* host_out, int64_t cap) {
  if (!h) return fail(nullptr, MP_EINVAL, "handle is NULL");
  if (!(h->flags & MP_FLAG_KEEP_SPINS)) return fail(h, MP_ESTATE, "created without MP_FLAG_KEEP_SPINS");
  if (!host_out || system < 0 || system >= static_cast<int>(h->hsys.size()))
    return fail(h, MP_EINVAL, "bad system index %d or NULL output", system);
  const DevSystem& d = h->hsys[system];
  if (path < 0 || path >= d.n_paths) return fail(h, MP_EINVAL, "path %lld out of range", (long long)path);
  const int64_t n = 3 * static_cast<int64_t>(d.N);
  if (cap < n) return fail(h, MP_EINVAL, "capacity %lld below %lld", (long long)cap, (long long)n);
  if (!h->ran) return fail(h, MP_ESTATE, "no run yet");
  DeviceGuard dg(h->device);
  MP_CUDA(h, cudaMemcpyAsync(host_out, h->d_spins + h->spin_offset[system] + path * n,
                             sizeof(double) * n, cudaMemcpyDeviceToHost, h->stream));
  MP_CUDA(h, cudaStreamSynchronize(h->stream));
  return MP_OK;
}

int mp_backward(mp_handle h, const double* d_g_e, const double* d_g_m, double* d_grad_beta,
                double* d_grad_h) {
  if (!h) return fail(nullptr, MP_EINVAL, "handle is NULL");
  if (!d_g_e || !d_g_m || !d_grad_beta || !d_grad_h) return fail(h, MP_EINVAL, "NULL gradient buffer");
  if (!h->ran) return fail(h, MP_ESTATE, "no run yet");
  DeviceGuard dg(h->device);
  BackwardParams p{h->d_sys, h->d_rec, d_g_e, d_g_m, d_grad_beta, d_grad_h};
  MP_CUDA(h, launch_backward(p, static_cast<int>(h->hsys.size()), h->stream));
  return MP_OK;
}

int mp_timing(mp_handle h, double* sweep_ms, double* reduce_ms) {
  if (!h) return fail(nullptr, MP_EINVAL, "handle is NULL");
  if (!h->ran) return fail(h, MP_ESTATE, "no run yet");
  DeviceGuard dg(h->device);
  MP_CUDA(h, cudaStreamSynchronize(h->stream));
  float a = 0.f, b = 0.f;
  MP_CUDA(h, cudaEventElapsedTime(&a, h->ev[0], h->ev[1]));
  MP_CUDA(h, cudaEventElapsedTime(&b, h->ev[1], h->ev[2]));
  if (sweep_ms) *sweep_ms = a;
  if (reduce_ms) *reduce_ms = b;
  return MP_OK;
}

int mp_plan(mp_handle h, int* cta_threads, int* grid, int* smem_bytes, int* n_items) {
  if (!h) return fail(nullptr, MP_EINVAL, "handle is NULL");
  if (cta_threads) *cta_threads = h->cta;
  if (grid) *grid = h->grid;
  if (smem_bytes) *smem_bytes = h->smem;
  if (n_items) *n_items = static_cast<int>(h->items.size() + h->pair_items.size());
  return MP_OK;
}

int mp_upload_bytes(mp_handle h, int64_t* bytes) {
  if (!h || !bytes) return fail(h, MP_EINVAL, "handle or output is NULL");
  *bytes = h->upload_bytes;
  return MP_OK;
}

}  // extern "C"

namespace {

// Per-path resumable state: kStateHeader bytes of accumulators, then the spins
// in the kernel's own layout (colour-split SoA for shared-memory paths, the
// padded half-plane layout for streamed ones).
int ensure_state(mp_state* h) {
  if (h->d_state) return MP_OK;
  const int n = static_cast<int>(h->hsys.size());
  const int real = h->precision == MP_FP64 ? 8 : 4;
  h->state_offset.assign(n, 0);
  h->state_stride.assign(n, 0);
  int64_t off = 0;
  for (int k = 0; k < n; ++k) {
    const DevSystem& d = h->hsys[k];
    const int64_t spins = d.mode == kModeStreamed
                              ? static_cast<int64_t>(2) * d.L * half_plane_bytes(d.L, real)
                              : lattice_bytes(h->systems[k], real);
    h->state_stride[k] = (kStateHeader + spins + 255) / 256 * 256;
    h->state_offset[k] = off;
    off += h->state_stride[k] * d.n_paths;
  }
  h->state_bytes = off;
  h->d_state = static_cast<unsigned char*>(dev_alloc(h, static_cast<size_t>(off)));
  h->d_state_offset = static_cast<int64_t*>(dev_alloc(h, sizeof(int64_t) * n));
  h->d_state_stride = static_cast<int64_t*>(dev_alloc(h, sizeof(int64_t) * n));
  if (!h->d_state || !h->d_state_offset || !h->d_state_stride)
    return fail(h, MP_ENOMEM, "state allocation failed (%lld bytes)", static_cast<long long>(off));
  MP_CUDA(h, cudaMemcpyAsync(h->d_state_offset, h->state_offset.data(), sizeof(int64_t) * n,
                             cudaMemcpyHostToDevice, h->stream));
  MP_CUDA(h, cudaMemcpyAsync(h->d_state_stride, h->state_stride.data(), sizeof(int64_t) * n,
                             cudaMemcpyHostToDevice, h->stream));
  MP_CUDA(h, cudaStreamSynchronize(h->stream));
  return MP_OK;
}

// Version 2: spins stored as (x, y) pairs then z per colour (or half-plane).
constexpr uint64_t kCheckpointVersion = 2;

struct CheckpointHeader {
  char magic[8];
  uint64_t version;
  uint64_t config_hash;
  int64_t sweeps_done;
  int64_t state_bytes;
  int64_t reserved[3];
};

// FNV-1a over everything the state depends on: systems, precision, seed,
// schedule, init mode and each system's lattice mode.
uint64_t config_hash(const mp_state* h) {
  uint64_t x = 1469598103934665603ull;
  auto mix = [&](const void* p, size_t n) {
    const unsigned char* b = static_cast<const unsigned char*>(p);
    for (size_t i = 0; i < n; ++i) x = (x ^ b[i]) * 1099511628211ull;
  };
  for (const mp_system& s : h->systems) {
    mix(&s.lattice, sizeof(s.lattice));
    mix(&s.L, sizeof(s.L));
    mix(&s.T, sizeof(s.T));
    mix(&s.J, sizeof(s.J));
    mix(&s.h, sizeof(s.h));
    mix(&s.n_paths, sizeof(s.n_paths));
    mix(&s.path_begin, sizeof(s.path_begin));
  }
  for (const DevSystem& d : h->hsys) mix(&d.mode, sizeof(d.mode));
  mix(&h->precision, sizeof(h->precision));
  mix(&h->init_mode, sizeof(h->init_mode));
  mix(&h->seed, sizeof(h->seed));
  mix(&h->n_therm, sizeof(h->n_therm));
  mix(&h->n_meas, sizeof(h->n_meas));
  return x;
}

}  // namespace

extern "C" {

int mp_run_sweeps(mp_handle h, int64_t n_sweeps) {
  if (!h) return fail(nullptr, MP_EINVAL, "handle is NULL");
  if (h->flags & MP_FLAG_RANDOM_SITE) return fail(h, MP_EINVAL, "random-site runs are not resumable");
  const int64_t total = h->n_therm + h->n_meas;
  if (n_sweeps < 1) return fail(h, MP_EINVAL, "n_sweeps must be >= 1");
  if (h->sweeps_done >= total) return fail(h, MP_ESTATE, "the schedule of %lld sweeps is complete",
                                           static_cast<long long>(total));
  DeviceGuard dg(h->device);
  int rc = ensure_state(h);
  if (rc != MP_OK) return rc;
  const int64_t s_end = std::min(total, h->sweeps_done + n_sweeps);
  *h->h_cancel = 0;
  rc = enqueue_run(h, h->sweeps_done, s_end, h->sweeps_done > 0, true);
  if (rc != MP_OK) return rc;
  MP_CUDA(h, cudaStreamSynchronize(h->stream));
  rc = check_error_flag(h);
  if (rc != MP_OK) return rc;  // canceled or timed out: the saved state is unchanged
  h->sweeps_done = s_end;
  if (s_end > h->n_therm) h->ran = true;
  return MP_OK;
}

int mp_progress(mp_handle h, int64_t* sweeps_done) {
  if (!h || !sweeps_done) return fail(h, MP_EINVAL, "NULL argument");
  *sweeps_done = h->sweeps_done;
  return MP_OK;
}

int mp_checkpoint(mp_handle h, void* buf, size_t* nbytes) {
  if (!h || !nbytes) return fail(h, MP_EINVAL, "NULL argument");
  if (h->flags & MP_FLAG_RANDOM_SITE) return fail(h, MP_EINVAL, "random-site runs are not resumable");
  if (h->sweeps_done == 0 || !h->d_state) return fail(h, MP_ESTATE, "nothing to checkpoint (no mp_run_sweeps yet)");
  const size_t need = sizeof(CheckpointHeader) + static_cast<size_t>(h->state_bytes);
  if (!buf) {
    *nbytes = need;
    return MP_OK;
  }
  if (*nbytes < need) return fail(h, MP_EINVAL, "buffer of %zu bytes, need %zu", *nbytes, need);
  DeviceGuard dg(h->device);
  CheckpointHeader hd{};
  std::memcpy(hd.magic, "MPCKPT01", 8);
  hd.version = kCheckpointVersion;
  hd.config_hash = config_hash(h);
  hd.sweeps_done = h->sweeps_done;
  hd.state_bytes = h->state_bytes;
  std::memcpy(buf, &hd, sizeof(hd));
  MP_CUDA(h, cudaMemcpyAsync(static_cast<unsigned char*>(buf) + sizeof(hd), h->d_state,
                             static_cast<size_t>(h->state_bytes), cudaMemcpyDeviceToHost, h->stream));
  MP_CUDA(h, cudaStreamSynchronize(h->stream));
  *nbytes = need;
  return MP_OK;
}

int mp_restore(mp_handle h, const void* buf, size_t nbytes) {
  if (!h || !buf) return fail(h, MP_EINVAL, "NULL argument");
  if (h->flags & MP_FLAG_RANDOM_SITE) return fail(h, MP_EINVAL, "random-site runs are not resumable");
  if (nbytes < sizeof(CheckpointHeader)) return fail(h, MP_EINVAL, "checkpoint too short");
  CheckpointHeader hd;
  std::memcpy(&hd, buf, sizeof(hd));
  if (std::memcmp(hd.magic, "MPCKPT01", 8) != 0 || hd.version != kCheckpointVersion)
    return fail(h, MP_EINVAL, "not a checkpoint of this library");
  if (hd.config_hash != config_hash(h))
    return fail(h, MP_EINVAL, "checkpoint of a different configuration");
  DeviceGuard dg(h->device);
  int rc = ensure_state(h);
  if (rc != MP_OK) return rc;
  if (hd.state_bytes != h->state_bytes || nbytes < sizeof(hd) + static_cast<size_t>(hd.state_bytes))
    return fail(h, MP_EINVAL, "checkpoint size does not match");
  MP_CUDA(h, cudaMemcpyAsync(h->d_state, static_cast<const unsigned char*>(buf) + sizeof(hd),
                             static_cast<size_t>(hd.state_bytes), cudaMemcpyHostToDevice, h->stream));
  MP_CUDA(h, cudaStreamSynchronize(h->stream));
  h->sweeps_done = hd.sweeps_done;
  return MP_OK;
}

int mp_cancel(mp_handle h) {
  if (!h) return fail(nullptr, MP_EINVAL, "handle is NULL");
  *reinterpret_cast<volatile int*>(h->h_cancel) = 1;
  return MP_OK;
}

int mp_system_plan(mp_handle h, int system, int* threads_per_path, int* paths_per_cta,
                   int* streamed_from_hbm) {
  if (!h) return fail(nullptr, MP_EINVAL, "handle is NULL");
  if (system < 0 || system >= static_cast<int>(h->hsys.size()))
    return fail(h, MP_EINVAL, "bad system index %d", system);
  const DevSystem& d = h->hsys[system];
  if (threads_per_path) *threads_per_path = d.tp;
  if (paths_per_cta) *paths_per_cta = d.g;
  // 0 shared memory, 1 streamed from HBM, 2 two-CTA cluster, 3 in place in HBM
  if (streamed_from_hbm) *streamed_from_hbm = d.mode;
  return MP_OK;
}

int mp_reduce(const mp_system* systems, int n_systems, int64_t n_therm, int64_t n_meas,
              const double* d_records, double* d_estimates, void* stream) {
  g_create_error.clear();
  if (!systems || !d_records || !d_estimates || n_systems < 1 || n_systems > 65535)
    return fail(nullptr, MP_EINVAL, "NULL pointer or n_systems outside 1..65535");
  if (n_therm < 0 || n_meas < 0) return fail(nullptr, MP_EINVAL, "negative sweep counts");
  int rc = validate_systems(systems, n_systems, 0);
  if (rc != MP_OK) return rc;
  std::vector<DevSystem> table(n_systems);
  int64_t rec = 0, max_paths = 0;
  for (int k = 0; k < n_systems; ++k) {
    const mp_system& s = systems[k];
    DevSystem& d = table[k];
    d = DevSystem{};
    d.lattice = s.lattice;
    d.L = s.L;
    d.N = static_cast<int32_t>(sites_of(s));
    d.NH = (d.N + 1) / 2;
    d.T = s.T;
    d.J = s.J;
    d.h = s.h;
    d.beta = 1.0 / s.T;
    d.rec_offset = rec;
    d.n_paths = s.n_paths;
    d.path_begin = s.path_begin;
    rec += s.n_paths;
    max_paths = std::max(max_paths, s.n_paths);
  }
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  DevSystem* d_sys = nullptr;
  double* d_sort = nullptr;
  auto done = [&](int code) {
    if (d_sys) cudaFree(d_sys);
    if (d_sort) cudaFree(d_sort);
    cudaGetLastError();
    return code;
  };
  if (cudaMalloc(&d_sys, sizeof(DevSystem) * n_systems) != cudaSuccess ||
      (max_paths > MP_R_MAX_PATHS && cudaMalloc(&d_sort, sizeof(double) * 2 * rec) != cudaSuccess))
    return done(fail(nullptr, MP_ENOMEM, "device allocation failed"));
  cudaError_t e = reduce_prepare();
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(d_sys, table.data(), sizeof(DevSystem) * n_systems, cudaMemcpyHostToDevice, st);
  ReduceParams r{};
  r.systems = d_sys;
  r.records = d_records;
  r.est = d_estimates;
  r.n_therm = n_therm;
  r.n_meas = n_meas;
  r.sort_buf = d_sort;
  if (e == cudaSuccess) e = launch_reduce(r, n_systems, max_paths, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess)
    return done(fail(nullptr, MP_ECUDA, "mp_reduce: %s", cudaGetErrorString(e)));
  return done(MP_OK);
}

int mp_philox(const uint32_t* d_ctr, int64_t n, uint64_t seed, uint32_t* d_out, void* stream) {
  if (n < 0 || (n > 0 && (!d_ctr || !d_out))) return fail(nullptr, MP_EINVAL, "bad Philox arguments");
  cudaError_t e = launch_philox(d_ctr, n, seed, d_out, static_cast<cudaStream_t>(stream));
  if (e != cudaSuccess) return cuda_fail(nullptr, e, "philox kernel");
  return MP_OK;
}

void mp_destroy(mp_handle h) {
  if (!h) return;
  DeviceGuard dg(h->device);
  release(h);
  delete h;
}

const char* mp_last_error(mp_handle h) { return h ? h->err.c_str() : g_create_error.c_str(); }

const char* mp_status_string(int status) {
  switch (status) {
    case MP_OK: return "MP_OK";
    case MP_EINVAL: return "MP_EINVAL";
    case MP_ENOMEM: return "MP_ENOMEM";
    case MP_ECUDA: return "MP_ECUDA";
    case MP_ESTATE: return "MP_ESTATE";
    case MP_ECANCELED: return "MP_ECANCELED";
    case MP_ETIMEOUT: return "MP_ETIMEOUT";
    default: return "MP_E?";
  }
}

}  // extern "C"
