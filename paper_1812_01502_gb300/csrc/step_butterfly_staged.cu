// step_butterfly_staged.cu - the general tile kernel for the all-stages
// schedule (every stage of Algorithm 3 in each time step; Heine, Whiteley &
// Cemgil, arXiv 1812.01502, Section 3): the stage counter in the device state
// decides per launch whether to weight with g_n and whether to mutate.  A
// translation unit of its own so that it compiles in parallel with the
// default kernels of step_butterfly.cu.
#include "bfpf_kernels.h"
#include "step_tile.cuh"

namespace bfpf {

template <int D, int KIND>
static const void* staged_pick(bool wide) {
  return wide ? reinterpret_cast<const void*>(&step_butterfly_kernel<D, KIND, true, true>)
              : reinterpret_cast<const void*>(&step_butterfly_kernel<D, KIND, false, true>);
}

const void* select_staged_tile_kernel(int d, int kind, bool wide) {
  if (kind == kStochVol) return d == 1 ? staged_pick<1, kStochVol>(wide) : nullptr;
  if (kind != kLinearGaussian) return nullptr;
  switch (d) {
    case 1: return staged_pick<1, kLinearGaussian>(wide);
    case 2: return staged_pick<2, kLinearGaussian>(wide);
    case 3: return staged_pick<3, kLinearGaussian>(wide);
    case 4: return staged_pick<4, kLinearGaussian>(wide);
    case 5: return staged_pick<5, kLinearGaussian>(wide);
    case 6: return staged_pick<6, kLinearGaussian>(wide);
    case 7: return staged_pick<7, kLinearGaussian>(wide);
    case 8: return staged_pick<8, kLinearGaussian>(wide);
    default: return nullptr;
  }
}

}  // namespace bfpf
