// step_adaptive.cuh - pieces of the fully adapted schedule (Section 1.2 of
// Heine, Whiteley & Cemgil, arXiv 1812.01502) shared by its tile kernel
// (step_adaptive.cu) and the register-resident group kernel (step_group.cuh):
// the mutation-only pass of a step whose remaining stages were skipped, and
// the end of a stage launch (ESS of the new stage weights -> skip decision).
#pragma once

#include "bfpf_device.cuh"
#include "bfpf_epilogue.cuh"
#include "bfpf_model.cuh"

namespace bfpf {

// End of a time step (thread 0 of the last block of launch m).
__device__ __forceinline__ void adaptive_end_step(const StepParams& p, DevState* st, uint32_t n) {
  if (p.rotate && st->last_k >= 0) st->start = ((uint32_t)st->last_k + 1u) % (uint32_t)p.m;
  st->skip = 0;
  st->done = 0;
  __threadfence();
  st->n = n + 1;
}

// Last launch of a step whose remaining stages were skipped: mutation only, the
// normals numbered group-major on digit g (as when this launch resamples).
template <int D, int KIND>
__device__ __forceinline__ void adaptive_mutate_only(const StepParams& p, const DigitGeom& g, uint32_t n) {
  DevState* st = p.st;
  const ModelParams& mp = p.model;
  if ((g.a & 3u) == 0) {
    // quads of members of one group: one Philox block per 4 normals
    for (uint32_t q = blockIdx.x * kBlock + threadIdx.x; q < p.N / 4; q += gridDim.x * kBlock) {
      const uint32_t pi0 = 4 * q;
      const uint32_t gid = fdiv(pi0, g.div_a), r0 = pi0 - gid * g.a;
      const uint32_t h = fdiv(gid, g.div_s), l = gid - h * g.s;
      const uint32_t ib = (h * g.a + r0) * g.s + l;       // particle of member r0
      float z[4 * D];
#pragma unroll
      for (int b = 0; b < D; ++b) {
        const uint4 w = philox4x32(make_uint4(q * D + b, n, kPurposePropagate, 0), p.rk);
        normals4_fast(w, z + 4 * b);
      }
#pragma unroll
      for (int e = 0; e < 4; ++e) {
        const uint32_t i = ib + e * g.s;
        float xh[D], xo[D];
#pragma unroll
        for (int t = 0; t < D; ++t) xh[t] = __ldcs(p.x + (size_t)t * p.N + i);
        mutate<D, KIND>(mp, xh, z + e * D, xo);
#pragma unroll
        for (int t = 0; t < D; ++t) __stcs(p.x + (size_t)t * p.N + i, xo[t]);
      }
    }
  } else {
    for (uint32_t i = blockIdx.x * kBlock + threadIdx.x; i < p.N; i += gridDim.x * kBlock) {
      const uint32_t r = (i / g.s) % g.a;
      const uint32_t gid = (i / (g.a * g.s)) * g.s + i % g.s;
      const uint32_t pi = gid * g.a + r;
      float xh[D], z[D], xo[D];
#pragma unroll
      for (int t = 0; t < D; ++t) {
        xh[t] = __ldcs(p.x + (size_t)t * p.N + i);
        const uint32_t nu = pi * D + t;
        const uint4 w = philox4x32(make_uint4(nu >> 2, n, kPurposePropagate, 0), p.rk);
        float zz[4];
        normals4_fast(w, zz);
        z[t] = zz[nu & 3u];
      }
      mutate<D, KIND>(mp, xh, z, xo);
#pragma unroll
      for (int t = 0; t < D; ++t) __stcs(p.x + (size_t)t * p.N + i, xo[t]);
    }
  }
  if (last_block_done(st)) adaptive_end_step(p, st, n);
}

// End of a stage launch that resampled on digit k: the partials hold
// (log V_G, 1, 1/a) per group, i.e. sum_i V_i and sum_i V_i^2 of the new stage
// weights; their ESS decides whether the next stage runs.
template <int D>
__device__ __forceinline__ void adaptive_stage_finish(const StepParams& p, Partial acc, float* accx, uint32_t status,
                                                      uint32_t lvp, uint32_t k, bool last, uint32_t n) {
  double S[2 + D];
  float Mx;
  if (!fold_partials<D>(p, acc, accx, status, S, Mx)) return;
  DevState* st = p.st;
  const double ess = (S[0] > 0.0 && S[1] > 0.0) ? S[0] * S[0] / ((double)p.N * S[1]) : 0.0;
  st->skip = (ess >= (double)p.theta) ? 1u : 0u;
  st->lvp = lvp ^ 1u;
  st->last_k = (int32_t)k;
  st->nstages += 1;
  if (last) {
    adaptive_end_step(p, st, n);
  } else {
    st->done = 0;
  }
}

}  // namespace bfpf
