// Host-side launchers of the library's kernels (internal interface between the
// C ABI in mp_api.cu and the kernel translation units).
#pragma once
#include <cuda_runtime.h>

#include <cstdint>

#include "common.cuh"

namespace mpk {

struct ReduceParams {
  const DevSystem* systems;
  const double* records;
  double* est;  // MP_NEST doubles per system
  int64_t n_therm, n_meas;
  // Sort space for the distribution coefficient of systems with more than
  // MP_R_MAX_PATHS paths: 2 n_paths doubles at 2 rec_offset per system
  // (nullptr when no system is that large).
  double* sort_buf;
};

struct BackwardParams {
  const DevSystem* systems;
  const double* records;
  const double* g_e;
  const double* g_m;
  double* grad_beta;
  double* grad_h;
};

// Shared-memory sweep kernels.  `variant` selects the kernel: L > 0 a batch
// of simple cubic lattices of that one size, -1 open chains only, 0 a batch
// of uneven sizes (the kernel switches per work item).
bool sweep_supports_L(int precision, int L);
cudaError_t sweep_prepare(int precision, int variant, int device, int* max_dynamic,
                          int* max_threads);
cudaError_t sweep_occupancy(int precision, int variant, int cta, int smem, int* blocks_per_sm);
cudaError_t launch_sweep(int precision, int variant, const SweepParams& p, int grid, int cta,
                         int smem, cudaStream_t st);

// The streamed kernels compiled for simple cubic L = 32 and L = 64 (all
// systems of the batch streamed at that size).
constexpr int kStreamL32 = -1032;
constexpr int kStreamL64 = -1064;

// The square-lattice Ising kernels: variant kIsingKernel runs any even L;
// ising_variant(L) a batch whose systems all have the size L, compiled for it
// (L in 20, 40, 50, 60: ising_compiled_L).
constexpr int kIsingKernel = -3;
constexpr int ising_variant(int L) { return -3000 - L; }
constexpr int ising_variant_L(int v) { return v <= -3000 ? -3000 - v : 0; }
constexpr bool is_ising_variant(int v) { return v == kIsingKernel || v <= -3000; }
bool ising_compiled_L(int L);
cudaError_t ising_prepare(int variant, int device, int* max_dynamic, int* max_threads);
cudaError_t ising_occupancy(int variant, int cta, int smem, int* blocks);
cudaError_t launch_ising(int variant, const SweepParams& p, int grid, int cta, int smem, cudaStream_t st);
// Slice bytes of an Ising path: thresholds (128 bytes), then per colour L + 2
// rows of L/2 bytes (the lattice's rows and a copy of each boundary row).
constexpr int kIsingThrBytes = 128;
constexpr int ising_slice_spin_bytes(int L) { return kIsingThrBytes + 2 * (L / 2) * (L + 2); }

// The random-site order (MP_FLAG_RANDOM_SITE, variant kRandomSiteKernel): one
// thread per path, lattices in HBM (random_site_bytes_per_site bytes per site
// and path).
constexpr int kRandomSiteKernel = -4;
int random_site_bytes_per_site(int precision);
cudaError_t launch_random_site(int precision, const SweepParams& p, int n_systems, int64_t total_paths,
                               void* lattice, int64_t elements, cudaStream_t st);

cudaError_t reduce_prepare();  // raise the dynamic shared memory limit
cudaError_t launch_reduce(const ReduceParams& p, int n_systems, int64_t max_paths, cudaStream_t st);
cudaError_t launch_backward(const BackwardParams& p, int n_systems, cudaStream_t st);
cudaError_t launch_philox(const uint32_t* ctr, int64_t n, uint64_t seed, uint32_t* out,
                          cudaStream_t st);

}  // namespace mpk
