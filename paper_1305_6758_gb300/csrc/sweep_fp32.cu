// FP32 form of the shared-memory sweep: FP32 spins, energy differences and
// Boltzmann factors; FP64 per-path accumulators.
#include "kernels.h"
#include "sweep.cuh"

namespace mpk {

template <>
__device__ __forceinline__ void dispatch_path<float>(const DevSystem& sy, int sys_idx, int64_t path,
                                                     const SweepParams& P, unsigned char* slice,
                                                     int tid, int tp, int bar) {
  if (sy.lattice == MP_LATTICE_CHAIN) {
    run_path<float>(GeomChain{sy.N}, sy, sys_idx, path, P, slice, tid, tp, bar);
    return;
  }
  switch (sy.L) {
#define MPK_CASE(LL)                                                             \
  case LL:                                                                       \
    run_path<float>(GeomSC<LL>{}, sy, sys_idx, path, P, slice, tid, tp, bar);    \
    break;
    MPK_FOR_EACH_L_FP32(MPK_CASE)
#undef MPK_CASE
    default:
      break;
  }
}

bool sweep_supports_L_fp32(int L) {
  switch (L) {
#define MPK_CASE(LL) case LL:
    MPK_FOR_EACH_L_FP32(MPK_CASE)
#undef MPK_CASE
    return true;
    default:
      return false;
  }
}

cudaError_t sweep_prepare_fp32() {
  return cudaFuncSetAttribute(sweep_kernel<float>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                              kSmemMax);
}

cudaError_t sweep_occupancy_fp32(int cta, int smem, int* blocks) {
  return cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks, sweep_kernel<float>, cta, smem);
}

cudaError_t launch_sweep_fp32(const SweepParams& p, int grid, int cta, int smem, cudaStream_t st) {
  sweep_kernel<float><<<grid, cta, smem, st>>>(p);
  return cudaGetLastError();
}

}  // namespace mpk
