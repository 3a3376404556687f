// Instantiation support for the sweep kernels of one precision.  The
// including translation unit defines REAL, SUFFIX and MPK_FOR_EACH_L (the
// compile-time lattice sizes of that precision); the kernels are spread over
// several translation units (sweep_<precision>*.cu) that compile in parallel,
// each exporting SUFFIX(sweep_part_<n>)(variant): the kernel of a variant it
// instantiates, or nullptr.
#pragma once
#include "kernels.h"
#include "sweep.cuh"

namespace mpk {

template <typename Real, int kLattice>
__device__ __forceinline__ void dispatch_path(const DevSystem& sy, int sys_idx, int64_t path,
                                              const SweepParams& P, unsigned char* slice, int tid,
                                              int tp, int bar) {
  if constexpr (kLattice > 0) {
    run_path<Real>(GeomSC<kLattice>{}, sy, sys_idx, path, P, slice, tid, tp, bar);
  } else if constexpr (kLattice == kStreamKernel || kLattice == kGlobalKernel ||
                       stream_variant_L(kLattice) > 0) {
    // streamed and in-place paths are run by the kernel itself; nothing in shared memory only
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
    run_path<Real>(GeomSC<LL, true>{}, sy, sys_idx, path, P, slice, tid, tp, bar); \
    break;
      MPK_FOR_EACH_L(MPK_CASE)
#undef MPK_CASE
      default:
        break;
    }
  }
}

}  // namespace mpk

#define MPK_PART_CASE(V) \
  case V:                \
    return reinterpret_cast<const void*>(sweep_kernel<REAL, V>);
