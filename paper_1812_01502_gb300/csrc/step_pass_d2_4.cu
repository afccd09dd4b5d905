// step_pass_d2_4.cu - fused all-stages launches for state dimensions 2 to 4.
#include "bfpf_kernels.h"
#include "step_pass.cuh"

namespace bfpf {

const void* pass_kernel_d2_4(int d, int kind, int a) {
  if (kind != kLinearGaussian) return nullptr;
  switch (d) {
    case 2: return pass_kernel_for<2, kLinearGaussian>(a);
    case 3: return pass_kernel_for<3, kLinearGaussian>(a);
    case 4: return pass_kernel_for<4, kLinearGaussian>(a);
    default: return nullptr;
  }
}

}  // namespace bfpf
