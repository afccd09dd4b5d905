// step_group_d1.cu - register-resident group kernels for state dimension 1.
#include "bfpf_kernels.h"
#include "step_group.cuh"

namespace bfpf {

const void* group_kernel_d1(int kind, int a, int* G, bool staged, bool adapt, bool small) {
  if (kind == kStochVol) return group_kernel_for<1, kStochVol>(a, *G, staged, adapt, small);
  if (kind != kLinearGaussian) return nullptr;
  return group_kernel_for<1, kLinearGaussian>(a, *G, staged, adapt, small);
}

}  // namespace bfpf
