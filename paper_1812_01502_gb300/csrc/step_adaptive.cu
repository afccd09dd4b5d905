// step_adaptive.cu - fully adapted augmented resampling (Heine, Whiteley &
// Cemgil, arXiv 1812.01502, Section 1.2): the ESS is evaluated before every
// stage of Algorithm 3, and once it reaches the threshold theta the step's
// remaining stages are skipped.  Weights that were not equalised carry over
// to the next step, so the carried log-weights are kept per particle.
//
// One time step = m + 1 launches:
//   launch 0      adaptive_weight_kernel: lw_i = lV_i + log g_n(zeta_i) - mu,
//                 the step's summaries (likelihood increment, mean, ESS) and
//                 the first decision (skip every stage if ESS >= theta);
//   launch 1 + j  adaptive_stage_kernel(j): stage on digit (start + j) mod m
//                 unless skipped; then the ESS of the new stage weights
//                 decides whether the next stage runs.  Launch m (j = m - 1)
//                 also mutates, resampled or not, and ends the step.
// A skipped launch that is not the last returns at once.  Every decision is
// written by the last block of one launch and read by the next launch.
// The draws of launch j use stage counter t = n m + j; with rotation the
// next step starts one digit after the last stage executed (Section 6.4).
#include <cfloat>

#include "bfpf_device.cuh"
#include "bfpf_epilogue.cuh"
#include "bfpf_kernels.h"
#include "bfpf_model.cuh"
#include "step_adaptive.cuh"
#include "step_tile.cuh"

namespace bfpf {

template <int D, int KIND>
__global__ void __launch_bounds__(kBlock) adaptive_weight_kernel(const __grid_constant__ StepParams p) {
  DevState* st = p.st;
  const ModelParams& mp = p.model;
  const uint32_t n = st->n;
  const uint32_t lvp = st->lvp;
  const float* __restrict__ lV_in = p.lV[lvp];
  float* __restrict__ lV_out = p.lV[lvp ^ 1u];
  const float muf = st->mu_f;
  float y[kMaxDim];
#pragma unroll
  for (int q = 0; q < kMaxDim; ++q) y[q] = (q < mp.dy) ? p.y_ring[(n % kRing) * mp.dy + q] : 0.0f;
  uint32_t status = 0;
  Partial acc{-INFINITY, 0.0f, 0.0f};
  float accx[D];
#pragma unroll
  for (int t = 0; t < D; ++t) accx[t] = 0.0f;
  for (uint32_t i = blockIdx.x * kBlock + threadIdx.x; i < p.N; i += gridDim.x * kBlock) {
    float xv[D];
#pragma unroll
    for (int t = 0; t < D; ++t) xv[t] = __ldcs(p.x + (size_t)t * p.N + i);
    const float lw = sanitize_logweight(__ldg(lV_in + i) + obs_log_term<D, KIND>(mp, y, xv) - muf, status);
    lV_out[i] = lw;
    merge_partial<D>(acc, accx, lw, 1.0f, 1.0f, xv);
  }
  double S[2 + D];
  float Mx;
  if (!fold_partials<D>(p, acc, accx, status, S, Mx)) return;
  const double ess = write_summaries<D>(p, S, Mx, n, muf);
  st->skip = (ess >= (double)p.theta) ? 1u : 0u;
  st->lvp = lvp ^ 1u;
  st->last_k = -1;
  st->done = 0;
}

template <int D, int KIND, bool WIDE>
__global__ void __launch_bounds__(kBlock) adaptive_stage_kernel(const __grid_constant__ StepParams p, uint32_t j) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  DevState* st = p.st;
  const uint32_t m = (uint32_t)p.m;
  const bool last = j + 1 == m;
  const uint32_t n = st->n;
  const uint32_t k = (st->start + j) % m;
  if (st->skip) {
    if (!last) return;                       // nothing to do, nothing to record
    adaptive_mutate_only<D, KIND>(p, p.geom[k], n);
    return;
  }
  const uint32_t lvp = st->lvp;
  TileCtx c;
  c.n = n;
  c.t = n * m + j;
  c.obs = false;
  c.mut = last;
  c.x = p.x;
  c.lV_in = p.lV[lvp];
  c.lV_out = p.lV[lvp ^ 1u];
  c.anc = nullptr;
  c.prec = nullptr;
  c.rk = &p.rk;
  c.mp = &p.model;
  c.g = &p.geom[k];
  c.N = p.N;
  c.cap = p.tile_cap;
  c.muf = 0.0f;
#pragma unroll
  for (int q = 0; q < kMaxDim; ++q) c.y[q] = 0.0f;
  uint32_t status = 0;
  Partial acc{-INFINITY, 0.0f, 0.0f};
  float accx[D];
#pragma unroll
  for (int t = 0; t < D; ++t) accx[t] = 0.0f;
  tile_steps<D, KIND, WIDE, true, true>(c, blockIdx.x, gridDim.x, smem_raw, acc, accx, status);
  adaptive_stage_finish<D>(p, acc, accx, status, lvp, k, last, n);
}

// ---------------------------------------------------------------------------
template <int D, int KIND>
static void adaptive_pick(bool wide, AdaptiveKernels& ak) {
  ak.weight = reinterpret_cast<const void*>(&adaptive_weight_kernel<D, KIND>);
  ak.stage = wide ? reinterpret_cast<const void*>(&adaptive_stage_kernel<D, KIND, true>)
                  : reinterpret_cast<const void*>(&adaptive_stage_kernel<D, KIND, false>);
}

bool select_adaptive_kernels(int d, int kind, bool wide, AdaptiveKernels& ak) {
  if (kind == kStochVol) {
    if (d != 1) return false;
    adaptive_pick<1, kStochVol>(wide, ak);
    return true;
  }
  if (kind != kLinearGaussian) return false;
  switch (d) {
    case 1: adaptive_pick<1, kLinearGaussian>(wide, ak); return true;
    case 2: adaptive_pick<2, kLinearGaussian>(wide, ak); return true;
    case 3: adaptive_pick<3, kLinearGaussian>(wide, ak); return true;
    case 4: adaptive_pick<4, kLinearGaussian>(wide, ak); return true;
    case 5: adaptive_pick<5, kLinearGaussian>(wide, ak); return true;
    case 6: adaptive_pick<6, kLinearGaussian>(wide, ak); return true;
    case 7: adaptive_pick<7, kLinearGaussian>(wide, ak); return true;
    case 8: adaptive_pick<8, kLinearGaussian>(wide, ak); return true;
    default: return false;
  }
}

}  // namespace bfpf
