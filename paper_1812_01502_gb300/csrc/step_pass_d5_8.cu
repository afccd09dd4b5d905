// step_pass_d5_8.cu - fused all-stages launches for state dimensions 5 to 8.
#include "bfpf_kernels.h"
#include "step_pass.cuh"

namespace bfpf {

const void* pass_kernel_d5_8(int d, int kind, int a) {
  if (kind != kLinearGaussian) return nullptr;
  switch (d) {
    case 5: return pass_kernel_for<5, kLinearGaussian>(a);
    case 6: return pass_kernel_for<6, kLinearGaussian>(a);
    case 7: return pass_kernel_for<7, kLinearGaussian>(a);
    case 8: return pass_kernel_for<8, kLinearGaussian>(a);
    default: return nullptr;
  }
}

}  // namespace bfpf
