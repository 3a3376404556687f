// FP64 sweep kernels, part c: chains and the streamed kernels.
// (The host entry points and part a are in sweep_fp64.cu.)
#define REAL double
#define SUFFIX(f) f##_fp64
#define MPK_FOR_EACH_L MPK_FOR_EACH_L_FP64
#include "sweep_inst.cuh"

namespace mpk {

const void* SUFFIX(sweep_part_c)(int variant) {
  switch (variant) {
    MPK_PART_CASE(kChainKernel)
    MPK_PART_CASE(kStreamKernel)
    MPK_PART_CASE(kGlobalKernel)
    MPK_PART_CASE(stream_variant(32))
    MPK_PART_CASE(stream_variant(64))
    default: return nullptr;
  }
}

}  // namespace mpk
