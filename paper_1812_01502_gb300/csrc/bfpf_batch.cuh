// bfpf_batch.cuh - device-side description of a batch of independent filters.
#pragma once

#include "bfpf_device.cuh"

namespace bfpf {

// One filter of a batch (device memory, one per filter).
struct BatchFilter {
  float* x;                     // [d][N] states
  float* lV[2];                 // carried log weights, ping-pong by step parity
  uint32_t N, m, cap, pad;      // particles, digits, tile capacity
  uint32_t U;                   // work units (thread blocks) per step: unit j takes tiles j, j + U, ...
  uint32_t pbase;               // first slot of its units' partial sums (U > 1)
  RoundKeys rk;
  DevState st;                  // mu, mu_f, loglik, status of this filter
  ModelParams model;
  DigitGeom geom[kMaxDigits];
  // digits on the register-resident group path (bit k: digit k; power-of-two
  // radix <= 32 whose groups fill whole block iterations) and their geometry
  uint32_t gsel;
  GroupGeom gg[kMaxDigits];
};

struct BatchState {
  uint32_t n;                   // time step of the batch (all filters step together)
  uint32_t done;                // blocks finished with the current step
};

// Partial sums of one work unit: (max, sum e, sum e^2, sum e x_t), kBatchNP floats.
constexpr int kBatchNP = 3 + kMaxDim + 1;

struct BatchParams {
  BatchFilter* filters;
  const uint2* units;           // block b runs unit units[b] = {filter, j | U << 16} (largest work first)
  uint32_t nunits;
  float* partials;              // [sum of U over filters with U > 1][kBatchNP]
  BatchState* state;
  const float* y_ring;          // [F][ring][dy_max] observations
  double* inc_ring;             // [F][ring] likelihood increments
  float* mean_ring;             // [F][ring][d_max] filter means
  float* ess_ring;              // [F][ring]
  uint32_t F, ring, dy_max, d_max;
};

}  // namespace bfpf
