// bfpf_kernels.h - host-side view of the kernels (internal to the library).
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

namespace bfpf {

// Kernel entry points for one (state dimension, model, wide-draw) variant.
struct KernelSet {
  const void* step;   // step_butterfly_kernel<D, KIND, WIDE>(StepParams)
  const void* init;   // init_particles_kernel<D, KIND>(StepParams)
};

// Picks the compiled variant; false if (d, kind) is not supported.
bool select_kernels(int d, int kind, bool wide, KernelSet& ks);

cudaError_t launch_philox_blocks(uint64_t seed, uint4 c, uint32_t count, uint32_t* out,
                                 cudaStream_t stream);

}  // namespace bfpf
