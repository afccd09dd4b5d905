// bfpf_model.cuh - the state-space models of the filter on the device.
//
// The HMM of Section 1.1 (eq. (HMM)): the potential g_n(x) = g(x, y_n) weights
// the particles, the kernel f(x, .) mutates them (Algorithm 1).
//   linear-Gaussian:  log g - c = -1/2 || Lr^{-1} (y - H x) ||^2,  f: x' = A x + Lq z
//   stochastic vol.:  log g - c = -x/2 - y^2 exp(-x) / (2 beta^2), f: x' = phi x + sigma z
// The constant c of log g is left to the likelihood (bfpf_epilogue.cuh).
#pragma once

#include "bfpf_device.cuh"

namespace bfpf {

template <int D, int KIND>
__device__ __forceinline__ float obs_log_term(const ModelParams& mp, const float* y, const float* x) {
  if constexpr (KIND == kStochVol) {
    return fmaf(-0.5f, x[0], -(y[0] * y[0] * mp.inv2b2) * ex2_ftz(x[0] * -1.4426950408889634f));
  } else {
    if (mp.flags & kHIdentity) {         // H = I implies dy = d: every bound is D
      float ss = 0.0f;
      if (mp.flags & kLrDiagonal) {
#pragma unroll
        for (int j = 0; j < D; ++j) {
          const float z = mp.Lri[j * kMaxDim + j] * (y[j] - x[j]);
          ss = fmaf(z, z, ss);
        }
      } else {
        float r[D];
#pragma unroll
        for (int j = 0; j < D; ++j) r[j] = y[j] - x[j];
#pragma unroll
        for (int j = 0; j < D; ++j) {
          float z = 0.0f;
#pragma unroll
          for (int u = 0; u <= j; ++u) z = fmaf(mp.Lri[j * kMaxDim + u], r[u], z);
          ss = fmaf(z, z, ss);
        }
      }
      return -0.5f * ss;
    }
    float r[kMaxDim];
#pragma unroll
    for (int j = 0; j < kMaxDim; ++j) {
      if (j < mp.dy) {
        float acc = y[j];
        if (mp.flags & kHIdentity) {
          acc -= (j < D) ? x[j] : 0.0f;
        } else {
#pragma unroll
          for (int t = 0; t < D; ++t) acc = fmaf(-mp.H[j * kMaxDim + t], x[t], acc);
        }
        r[j] = acc;
      }
    }
    float ss = 0.0f;
    if (mp.flags & kLrDiagonal) {
#pragma unroll
      for (int j = 0; j < kMaxDim; ++j)
        if (j < mp.dy) {
          const float z = mp.Lri[j * kMaxDim + j] * r[j];
          ss = fmaf(z, z, ss);
        }
    } else {
#pragma unroll
      for (int j = 0; j < kMaxDim; ++j)
        if (j < mp.dy) {
          float z = 0.0f;
#pragma unroll
          for (int u = 0; u <= j; ++u) z = fmaf(mp.Lri[j * kMaxDim + u], r[u], z);
          ss = fmaf(z, z, ss);
        }
    }
    return -0.5f * ss;
  }
}

template <int D, int KIND>
__device__ __forceinline__ void mutate(const ModelParams& mp, const float* xh, const float* z, float* out) {
  if constexpr (KIND == kStochVol) {
    out[0] = fmaf(mp.phi, xh[0], mp.sigma * z[0]);
  } else {
#pragma unroll
    for (int t = 0; t < D; ++t) {
      float acc = 0.0f;
      if (mp.flags & kADiagonal) {
        acc = mp.A[t * kMaxDim + t] * xh[t];
      } else {
#pragma unroll
        for (int u = 0; u < D; ++u) acc = fmaf(mp.A[t * kMaxDim + u], xh[u], acc);
      }
      if (mp.flags & kLqDiagonal) {
        acc = fmaf(mp.Lq[t * kMaxDim + t], z[t], acc);
      } else {
#pragma unroll
        for (int u = 0; u <= t; ++u) acc = fmaf(mp.Lq[t * kMaxDim + u], z[u], acc);
      }
      out[t] = acc;
    }
  }
}

// Non-finite log-weights are weight zero (and flagged).
__device__ __forceinline__ float sanitize_logweight(float lw, uint32_t& status) {
  if (lw != lw || lw == INFINITY) {
    status |= kStatusNonFinite;
    return -INFINITY;
  }
  return lw;
}

}  // namespace bfpf
