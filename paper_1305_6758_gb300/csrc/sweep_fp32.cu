// FP32 form of the shared-memory sweep: FP32 spins, energy differences and
// Boltzmann factors; FP64 per-path accumulators.
#include "kernels.h"
#define REAL float
#define SUFFIX(f) f##_fp32
#define MPK_FOR_EACH_L MPK_FOR_EACH_L_FP32
#include "sweep.cuh"

namespace mpk {

template <typename Real, int kLattice>
__device__ __forceinline__ void dispatch_path(const DevSystem& sy, int sys_idx, int64_t path,
                                              const SweepParams& P, unsigned char* slice, int tid,
                                              int tp, int bar) {
  if constexpr (kLattice > 0) {
    run_path<Real>(GeomSC<kLattice>{}, sy, sys_idx, path, P, slice, tid, tp, bar);
  } else if constexpr (kLattice == kStreamKernel || stream_variant_L(kLattice) > 0) {
    // streamed paths are run by the kernel itself; nothing in shared memory only
  } else if constexpr (kLattice == kChainKernel) {
    run_path<Real>(GeomChain{sy.N}, sy, sys_idx, path, P, slice, tid, tp, bar);
  } else {
    if (sy.lattice == MP_LATTICE_CHAIN) {
      run_path<Real>(GeomChain{sy.N}, sy, sys_idx, path, P, slice, tid, tp, bar);
      return;
    }
    switch (sy.L) {
#define MPK_CASE(LL)                                                           \
  case LL:                                                                     \
    run_path<Real>(GeomSC<LL>{}, sy, sys_idx, path, P, slice, tid, tp, bar);   \
    break;
      MPK_FOR_EACH_L(MPK_CASE)
#undef MPK_CASE
      default:
        break;
    }
  }
}

// kernel of a variant (simple cubic L, chain, or mixed); nullptr if not built
static const void* kernel_of(int variant) {
  switch (variant) {
    case kMixedKernel: return reinterpret_cast<const void*>(sweep_kernel<REAL, kMixedKernel>);
    case kChainKernel: return reinterpret_cast<const void*>(sweep_kernel<REAL, kChainKernel>);
    case kStreamKernel: return reinterpret_cast<const void*>(sweep_kernel<REAL, kStreamKernel>);
    case stream_variant(64):
      return reinterpret_cast<const void*>(sweep_kernel<REAL, stream_variant(64)>);
#define MPK_CASE(LL) \
    case LL: return reinterpret_cast<const void*>(sweep_kernel<REAL, LL>);
      MPK_FOR_EACH_L(MPK_CASE)
#undef MPK_CASE
    default: return nullptr;
  }
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

cudaError_t SUFFIX(launch_sweep)(int variant, const SweepParams& p, int grid, int cta, int smem,
                                 cudaStream_t st) {
  const void* k = kernel_of(variant);
  if (!k) return cudaErrorInvalidValue;
  void* args[] = {const_cast<SweepParams*>(&p)};
  return cudaLaunchKernel(k, dim3(grid), dim3(cta), args, static_cast<size_t>(smem), st);
}

}  // namespace mpk
