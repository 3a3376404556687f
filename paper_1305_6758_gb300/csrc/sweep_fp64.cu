// FP64 form of the shared-memory sweep (the plain FP64 GPU form): FP64 spins,
// energy differences, Boltzmann factors and accumulators.
#include "kernels.h"
#include "sweep.cuh"

namespace mpk {

template <>
__device__ __forceinline__ void dispatch_path<double>(const DevSystem& sy, int sys_idx, int64_t path,
                                                     const SweepParams& P, unsigned char* slice,
                                                     int tid, int tp, int bar) {
  if (sy.lattice == MP_LATTICE_CHAIN) {
    run_path<double>(GeomChain{sy.N}, sy, sys_idx, path, P, slice, tid, tp, bar);
    return;
  }
  switch (sy.L) {
#define MPK_CASE(LL)                                                             \
  case LL:                                                                       \
    run_path<double>(GeomSC<LL>{}, sy, sys_idx, path, P, slice, tid, tp, bar);    \
    break;
    MPK_FOR_EACH_L_FP64(MPK_CASE)
#undef MPK_CASE
    default:
      break;
  }
}

bool sweep_supports_L_fp64(int L) {
  switch (L) {
#define MPK_CASE(LL) case LL:
    MPK_FOR_EACH_L_FP64(MPK_CASE)
#undef MPK_CASE
    return true;
    default:
      return false;
  }
}

cudaError_t sweep_prepare_fp64() {
  return cudaFuncSetAttribute(sweep_kernel<double>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                              kSmemMax);
}

cudaError_t sweep_occupancy_fp64(int cta, int smem, int* blocks) {
  return cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks, sweep_kernel<double>, cta, smem);
}

cudaError_t launch_sweep_fp64(const SweepParams& p, int grid, int cta, int smem, cudaStream_t st) {
  sweep_kernel<double><<<grid, cta, smem, st>>>(p);
  return cudaGetLastError();
}

}  // namespace mpk
