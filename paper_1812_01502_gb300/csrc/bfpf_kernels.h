// bfpf_kernels.h - host-side view of the kernels (internal to the library).
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

namespace bfpf {

// Kernel entry points for one (state dimension, model, wide-draw) variant.
struct KernelSet {
  const void* step;          // step_butterfly_kernel<D, KIND, WIDE, false>(StepParams)
  const void* step_staged;   // step_butterfly_kernel<D, KIND, WIDE, true>: all stages per step
  const void* init;          // init_particles_kernel<D, KIND>(StepParams)
};

// Picks the compiled variant of the general kernel; false if (d, kind) is not supported.
bool select_kernels(int d, int kind, bool wide, KernelSet& ks);
// The general kernel for the all-stages schedule (step_butterfly_staged.cu).
const void* select_staged_tile_kernel(int d, int kind, bool wide);
// The digit-set stage kernel step_sets_kernel<d, kind, wide>(StepParams) (step_sets.cu).
const void* select_sets_kernel(int d, int kind, bool wide);

// Register-resident group kernel step_group_kernel<d, kind, a, G, staged>(StepParams,
// GroupGeom) for a power-of-two radix a <= 32; sets *G (lanes per group).  nullptr if none.
const void* select_group_kernel(int d, int kind, int a, int* G, bool staged, bool adapt = false, bool small = false);
const void* group_kernel_d1(int kind, int a, int* G, bool staged, bool adapt, bool small);
const void* group_kernel_d2(int kind, int a, int* G, bool staged, bool adapt, bool small);
const void* group_kernel_d3(int kind, int a, int* G, bool staged, bool adapt, bool small);
const void* group_kernel_d4(int kind, int a, int* G, bool staged, bool adapt, bool small);
const void* group_kernel_d5(int kind, int a, int* G, bool staged, bool adapt, bool small);
const void* group_kernel_d6(int kind, int a, int* G, bool staged, bool adapt, bool small);
const void* group_kernel_d7(int kind, int a, int* G, bool staged, bool adapt, bool small);
const void* group_kernel_d8(int kind, int a, int* G, bool staged, bool adapt, bool small);

// Fused all-stages launch step_pass_kernel<d, kind, a>(StepParams, PassGeom):
// consecutive stages of one time step on digits of radix a (a power of two
// <= 32) over shared-memory tiles.  nullptr if none.
const void* select_pass_kernel(int d, int kind, int a);
const void* pass_kernel_d1(int kind, int a);
const void* pass_kernel_d2_4(int d, int kind, int a);
const void* pass_kernel_d5_8(int d, int kind, int a);

// Global-resampling comparator (radices = {N}, N > 1024): six kernels per step,
// launched in the order weight, refine, scan, bounds, resolve, advance, each
// taking (StepParams, GlobalParams).
struct GlobalKernels {
  const void* weight;
  const void* refine_reduce;
  const void* scan;
  const void* resolve;
  const void* advance;
};
bool select_global_kernels(int d, int kind, GlobalKernels& gk);

// Fully adapted schedule (step_adaptive.cu): adaptive_weight_kernel(StepParams) and
// adaptive_stage_kernel(StepParams, uint32_t j) for launch j of a step.
struct AdaptiveKernels {
  const void* weight;
  const void* stage;
};
bool select_adaptive_kernels(int d, int kind, bool wide, AdaptiveKernels& ak);

// AIRPF (step_islands.cu): island_stages_kernel(StepParams, IslandParams), one block of
// kIslandThreads threads with 8 * islands bytes of shared memory, and
// island_gather_kernel(StepParams, IslandParams).
struct IslandKernels {
  const void* stages;
  const void* gather;
};
bool select_island_kernels(int d, int kind, IslandKernels& ik);

// Batched filters (batch.cu): batch_class_kernel<D, KIND>(BatchParams, uint32_t u0) and
// batch_group_kernel<D, KIND>(same) run one time step of the work units u0 .. u0 + grid - 1
// (one class of model kind and dimension) whose digit is on the tile / the group path;
// batch_advance_kernel(BatchParams) advances the step; batch_init_kernel(BatchParams).
const void* batch_class_kernel_ptr(int kind, int d);
const void* batch_group_kernel_ptr(int kind, int d);
const void* batch_advance_kernel_ptr();
const void* batch_init_kernel_ptr();

cudaError_t launch_philox_blocks(uint64_t seed, uint4 c, uint32_t count, uint32_t* out,
                                 cudaStream_t stream);

}  // namespace bfpf
