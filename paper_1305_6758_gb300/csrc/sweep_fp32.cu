// FP32 form of the shared-memory sweep: FP32 spins, energy differences and
// Boltzmann factors; FP64 per-path accumulators.
// This file holds part a (the smallest shared-memory lattice sizes) and the
// host entry points; parts b, c and d are sweep_fp32_b.cu, _c.cu and _d.cu.
#define REAL float
#define SUFFIX(f) f##_fp32
#define MPK_FOR_EACH_L MPK_FOR_EACH_L_FP32
#include "sweep_inst.cuh"

namespace mpk {

const void* SUFFIX(sweep_part_a)(int variant) {
  switch (variant) {
    MPK_PART_CASE(2)
    MPK_PART_CASE(4)
    MPK_PART_CASE(6)
    MPK_PART_CASE(8)
    MPK_PART_CASE(10)
    MPK_PART_CASE(12)
    default: return nullptr;
  }
}
const void* SUFFIX(sweep_part_b)(int variant);
const void* SUFFIX(sweep_part_c)(int variant);
const void* SUFFIX(sweep_part_d)(int variant);

// kernel of a variant (simple cubic L, chain, streamed or mixed); nullptr if not built
static const void* kernel_of(int variant) {
  const void* k = SUFFIX(sweep_part_a)(variant);
  if (!k) k = SUFFIX(sweep_part_b)(variant);
  if (!k) k = SUFFIX(sweep_part_c)(variant);
  if (!k) k = SUFFIX(sweep_part_d)(variant);
  return k;
}

bool SUFFIX(sweep_supports_L)(int L) { return L > 0 && kernel_of(L) != nullptr; }

// Raises a variant's dynamic shared-memory limit to what the device allows
// beside the kernel's static shared memory; returns that limit in
// *max_dynamic and the kernel's largest CTA in *max_threads.
cudaError_t SUFFIX(sweep_prepare)(int variant, int device, int* max_dynamic, int* max_threads) {
  const void* k = kernel_of(variant);
  if (!k) return cudaErrorInvalidValue;
  int optin = 0;
  cudaError_t e = cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, device);
  if (e != cudaSuccess) return e;
  cudaFuncAttributes fa;
  e = cudaFuncGetAttributes(&fa, k);
  if (e != cudaSuccess) return e;
  *max_dynamic = optin - static_cast<int>(fa.sharedSizeBytes);
  *max_threads = fa.maxThreadsPerBlock;
  return cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, *max_dynamic);
}

cudaError_t SUFFIX(sweep_occupancy)(int variant, int cta, int smem, int* blocks) {
  const void* k = kernel_of(variant);
  if (!k) return cudaErrorInvalidValue;
  return cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks, k, cta, smem);
}

// Launch of a variant; with paths for two-CTA clusters (p.n_pair_items > 0)
// the grid (then even) runs as clusters of two CTAs.
cudaError_t SUFFIX(launch_sweep)(int variant, const SweepParams& p, int grid, int cta, int smem,
                                 cudaStream_t st) {
  const void* k = kernel_of(variant);
  if (!k) return cudaErrorInvalidValue;
  void* args[] = {const_cast<SweepParams*>(&p)};
  if (p.n_pair_items <= 0)
    return cudaLaunchKernel(k, dim3(grid), dim3(cta), args, static_cast<size_t>(smem), st);
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(grid);
  cfg.blockDim = dim3(cta);
  cfg.dynamicSmemBytes = static_cast<size_t>(smem);
  cfg.stream = st;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeClusterDimension;
  at[0].val.clusterDim.x = 2;
  at[0].val.clusterDim.y = 1;
  at[0].val.clusterDim.z = 1;
  cfg.attrs = at;
  cfg.numAttrs = 1;
  return cudaLaunchKernelExC(&cfg, k, args);
}

// Two-CTA clusters of a variant that can be resident at once.
cudaError_t SUFFIX(sweep_cluster_occupancy)(int variant, int cta, int smem, int* clusters) {
  const void* k = kernel_of(variant);
  if (!k) return cudaErrorInvalidValue;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(2);
  cfg.blockDim = dim3(cta);
  cfg.dynamicSmemBytes = static_cast<size_t>(smem);
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeClusterDimension;
  at[0].val.clusterDim.x = 2;
  at[0].val.clusterDim.y = 1;
  at[0].val.clusterDim.z = 1;
  cfg.attrs = at;
  cfg.numAttrs = 1;
  return cudaOccupancyMaxActiveClusters(clusters, k, &cfg);
}

}  // namespace mpk
