// step_pass_d1.cu - fused all-stages launches for state dimension 1.
#include "bfpf_kernels.h"
#include "step_pass.cuh"

namespace bfpf {

const void* pass_kernel_d1(int kind, int a) {
  if (kind == kStochVol) return pass_kernel_for<1, kStochVol>(a);
  if (kind == kLinearGaussian) return pass_kernel_for<1, kLinearGaussian>(a);
  return nullptr;
}

}  // namespace bfpf
