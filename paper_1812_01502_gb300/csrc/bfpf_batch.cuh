// bfpf_batch.cuh - device-side description of a batch of independent filters.
#pragma once

#include "bfpf_device.cuh"

namespace bfpf {

// One filter of a batch (device memory, one per filter).
struct BatchFilter {
  float* x;                     // [d][N] states
  float* lV[2];                 // carried log weights, ping-pong by step parity
  uint32_t N, m, cap, pad;      // particles, digits, tile capacity
  RoundKeys rk;
  DevState st;                  // mu, mu_f, loglik, status of this filter
  ModelParams model;
  DigitGeom geom[kMaxDigits];
};

struct BatchState {
  uint32_t n;                   // time step of the batch (all filters step together)
  uint32_t done;                // blocks finished with the current step
};

struct BatchParams {
  BatchFilter* filters;
  const uint32_t* order;        // block b runs filter order[b] (largest work first)
  BatchState* state;
  const float* y_ring;          // [F][ring][dy_max] observations
  double* inc_ring;             // [F][ring] likelihood increments
  float* mean_ring;             // [F][ring][d_max] filter means
  float* ess_ring;              // [F][ring]
  uint32_t F, ring, dy_max, d_max;
};

}  // namespace bfpf
