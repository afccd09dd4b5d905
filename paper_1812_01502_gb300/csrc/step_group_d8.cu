// step_group_d8.cu - register-resident group kernels for state dimension 8.
#include "bfpf_kernels.h"
#include "step_group.cuh"

namespace bfpf {

const void* group_kernel_d8(int kind, int a, int* G, bool staged, bool adapt, bool small) {

  if (kind != kLinearGaussian) return nullptr;
  return group_kernel_for<8, kLinearGaussian>(a, *G, staged, adapt, small);
}

}  // namespace bfpf
