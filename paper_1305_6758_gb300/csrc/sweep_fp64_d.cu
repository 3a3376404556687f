// FP64 sweep kernels, part d: the kernel for batches of uneven sizes.
// (The host entry points and part a are in sweep_fp64.cu.)
#define REAL double
#define SUFFIX(f) f##_fp64
#define MPK_FOR_EACH_L MPK_FOR_EACH_L_FP64
#include "sweep_inst.cuh"

namespace mpk {

const void* SUFFIX(sweep_part_d)(int variant) {
  switch (variant) {
    MPK_PART_CASE(kMixedKernel)
    default: return nullptr;
  }
}

}  // namespace mpk
