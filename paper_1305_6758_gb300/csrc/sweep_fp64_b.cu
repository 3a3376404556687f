// FP64 sweep kernels, part b: larger shared-memory lattice sizes.
// (The host entry points and part a are in sweep_fp64.cu.)
#define REAL double
#define SUFFIX(f) f##_fp64
#define MPK_FOR_EACH_L MPK_FOR_EACH_L_FP64
#include "sweep_inst.cuh"

namespace mpk {

const void* SUFFIX(sweep_part_b)(int variant) {
  switch (variant) {
    MPK_PART_CASE(12)
    MPK_PART_CASE(14)
    MPK_PART_CASE(16)
    MPK_PART_CASE(18)
    MPK_PART_CASE(20)
    default: return nullptr;
  }
}

}  // namespace mpk
