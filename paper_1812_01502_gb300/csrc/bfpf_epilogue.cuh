// bfpf_epilogue.cuh - end of a time step, shared by the step kernels.
//
// Every thread carries a running partial (m, s1, s2, sx[d]) of the weighted
// particles it reduced:  s1 = sum e^{lw - m},  s2 = sum e^{2(lw - m)},
// sx = sum e^{lw - m} x.  finish_step() reduces them over the block, writes
// the block's partial, and the last block to arrive (last-block-done) folds
// all block partials in a fixed order with compensated FP32 sums, then
// computes in FP64:
//   likelihood increment  inc_n = log(N^-1 sum_i e^{lw_i}) + (mu_f - mu) + c_n
//   filter mean           sum_i e^{lw_i} x_i / sum_i e^{lw_i}
//   ESS (Section 1.2)     (sum e^{lw})^2 / (N sum e^{2 lw})
// and advances the device state (n, mu, cumulative FP64 log-likelihood).
// A stage that does not weight with an observation (all-stages schedule,
// stages after the first) writes no summaries and only moves the stage on.
#pragma once

#include "bfpf_device.cuh"

namespace bfpf {

struct Partial {
  float m, s1, s2;
};

// Merge a (max, sums) triple into the running partial, rescaling to the larger max.
template <int D>
__device__ __forceinline__ void merge_partial(Partial& acc, float* accx, float m, float s1, float s2,
                                              const float* sx) {
  if (m == -INFINITY) return;
  if (m > acc.m) {
    const float sc = expf(acc.m - m);
    acc.s1 = fmaf(acc.s1, sc, s1);
    acc.s2 = fmaf(acc.s2, sc * sc, s2);
#pragma unroll
    for (int t = 0; t < D; ++t) accx[t] = fmaf(accx[t], sc, sx[t]);
    acc.m = m;
  } else {
    const float sc = expf(m - acc.m);
    acc.s1 = fmaf(s1, sc, acc.s1);
    acc.s2 = fmaf(s2, sc * sc, acc.s2);
#pragma unroll
    for (int t = 0; t < D; ++t) accx[t] = fmaf(sx[t], sc, accx[t]);
  }
}

template <int D>
__device__ __forceinline__ void shfl_merge(Partial& acc, float* accx, int off) {
  Partial o;
  o.m = __shfl_down_sync(0xffffffffu, acc.m, off);
  o.s1 = __shfl_down_sync(0xffffffffu, acc.s1, off);
  o.s2 = __shfl_down_sync(0xffffffffu, acc.s2, off);
  float ox[D];
#pragma unroll
  for (int t = 0; t < D; ++t) ox[t] = __shfl_down_sync(0xffffffffu, accx[t], off);
  merge_partial<D>(acc, accx, o.m, o.s1, o.s2, ox);
}

// Grid-wide fold of the per-thread partials, called by every thread of every
// block exactly once.  Each block writes its partial; the last block to
// arrive (last-block-done) folds all block partials in a fixed order with
// compensated FP32 sums.  Returns true in thread 0 of the last block only,
// with S[0] = sum e^{lw - Mx}, S[1] = sum e^{2(lw - Mx)}, S[2 + t] = sum
// e^{lw - Mx} x_t (FP64) and Mx the global maximum.
template <int D>
__device__ __forceinline__ bool fold_partials(const StepParams& p, Partial acc, float* accx, uint32_t status,
                                              double* S, float& Mx_out) {
  constexpr int NP = 3 + D;
  constexpr int NW = kBlock / 32;
  __shared__ float s_red[NW][NP];
  __shared__ float s_redlo[NW][NP];
  __shared__ uint32_t s_last;
  DevState* st = p.st;
  const uint32_t tid = threadIdx.x;
  if (status) atomicOr(&st->status, status);
  const uint32_t lane = tid & 31u, warp = tid >> 5;
#pragma unroll
  for (int off = 16; off; off >>= 1) shfl_merge<D>(acc, accx, off);
  if (lane == 0) {
    s_red[warp][0] = acc.m;
    s_red[warp][1] = acc.s1;
    s_red[warp][2] = acc.s2;
#pragma unroll
    for (int t = 0; t < D; ++t) s_red[warp][3 + t] = accx[t];
  }
  __syncthreads();
  if (tid == 0) {
    Partial b{-INFINITY, 0.0f, 0.0f};
    float bx[D];
#pragma unroll
    for (int t = 0; t < D; ++t) bx[t] = 0.0f;
    for (int w = 0; w < NW; ++w) merge_partial<D>(b, bx, s_red[w][0], s_red[w][1], s_red[w][2], &s_red[w][3]);
    float* out = p.partials + (size_t)blockIdx.x * NP;
    out[0] = b.m;
    out[1] = b.s1;
    out[2] = b.s2;
#pragma unroll
    for (int t = 0; t < D; ++t) out[3 + t] = bx[t];
    __threadfence();
    const uint32_t prev = atomicAdd(&st->done, 1u);
    s_last = (prev == gridDim.x - 1) ? 1u : 0u;
  }
  __syncthreads();
  if (!s_last) return false;
  __threadfence();

  // Last block: fold all block partials (fixed order, compensated FP32), finish in FP64.
  const uint32_t G = gridDim.x;
  float Mx = -INFINITY;
  for (uint32_t b = tid; b < G; b += kBlock) Mx = fmaxf(Mx, __ldcg(p.partials + (size_t)b * NP));
#pragma unroll
  for (int off = 16; off; off >>= 1) Mx = fmaxf(Mx, __shfl_xor_sync(0xffffffffu, Mx, off));
  __syncthreads();
  if (lane == 0) s_red[warp][0] = Mx;
  __syncthreads();
  Mx = s_red[0][0];
  for (int w = 1; w < NW; ++w) Mx = fmaxf(Mx, s_red[w][0]);
  __syncthreads();

  float hi[NP - 1], lo[NP - 1];
#pragma unroll
  for (int v = 0; v < NP - 1; ++v) hi[v] = lo[v] = 0.0f;
  if (Mx != -INFINITY) {
    for (uint32_t b = tid; b < G; b += kBlock) {
      const float* pb = p.partials + (size_t)b * NP;
      const float mb = __ldcg(pb);
      if (mb == -INFINITY) continue;
      const float w = expf(mb - Mx);
      ff_add(hi[0], lo[0], __ldcg(pb + 1) * w);
      ff_add(hi[1], lo[1], __ldcg(pb + 2) * (w * w));
#pragma unroll
      for (int t = 0; t < D; ++t) ff_add(hi[2 + t], lo[2 + t], __ldcg(pb + 3 + t) * w);
    }
  }
#pragma unroll
  for (int off = 16; off; off >>= 1) {
#pragma unroll
    for (int v = 0; v < NP - 1; ++v) {
      const float oh = __shfl_down_sync(0xffffffffu, hi[v], off);
      const float ol = __shfl_down_sync(0xffffffffu, lo[v], off);
      ff_add(hi[v], lo[v], oh);
      lo[v] += ol;
    }
  }
  if (lane == 0) {
#pragma unroll
    for (int v = 0; v < NP - 1; ++v) {
      s_red[warp][v] = hi[v];
      s_redlo[warp][v] = lo[v];
    }
  }
  __syncthreads();
  if (tid != 0) return false;
  for (int v = 0; v < NP - 1; ++v) {
    float h = 0.0f, l = 0.0f;
    for (int w = 0; w < NW; ++w) {
      ff_add(h, l, s_red[w][v]);
      l += s_redlo[w][v];
    }
    S[v] = (double)h + (double)l;
  }
  Mx_out = Mx;
  return true;
}

// Writes the step's summaries from the folded sums (thread 0 of the last block):
// likelihood increment, filter mean and ESS into the output rings, the
// cumulative log-likelihood and the next normaliser.  Returns the ESS.
template <int D>
__device__ __forceinline__ double write_summaries(const StepParams& p, const double* S, float Mx, uint32_t n,
                                                  float muf, double* lme_out = nullptr) {
  DevState* st = p.st;
  const ModelParams& mp = p.model;
  const uint32_t slot = n % kRing;
  double lme, inc, ess;
  if (Mx == -INFINITY || !(S[0] > 0.0)) {
    lme = -INFINITY;
    inc = -INFINITY;
    ess = 0.0;
  } else {
    lme = (double)Mx + log(S[0] * (double)p.inv_N);
    inc = lme + ((double)muf - st->mu) + mp.c_obs;
    ess = S[0] * S[0] / ((double)p.N * S[1]);
  }
  p.inc_ring[slot] = inc;
  p.ess_ring[slot] = (float)ess;
  for (int t = 0; t < D; ++t) p.mean_ring[slot * mp.d + t] = (float)(S[2 + t] / S[0]);
  st->loglik += inc;
  st->mu = lme;
  st->mu_f = (float)lme;
  if (lme_out) *lme_out = lme;
  return ess;
}

// Last-block-done without partial sums: the last thread block of a launch to
// get here returns true in its thread 0 (the block counter is left for the
// caller to reset).
__device__ __forceinline__ bool last_block_done(DevState* st) {
  __shared__ uint32_t s_last_blk;
  __syncthreads();
  if (threadIdx.x == 0) {
    __threadfence();
    const uint32_t prev = atomicAdd(&st->done, 1u);
    s_last_blk = (prev == gridDim.x - 1) ? 1u : 0u;
  }
  __syncthreads();
  return s_last_blk && threadIdx.x == 0;
}

// End of one launch of the one-digit or all-stages schedule.
// ADVANCE = false (global resampling, which finishes the step in a later
// kernel): the last block leaves n alone and instead writes the global
// maximum log-weight and the single group's new log weight.
template <int D, bool ADVANCE = true>
__device__ __forceinline__ void finish_step(const StepParams& p, Partial acc, float* accx, const Sched& sc,
                                            uint32_t status, float muf, float* lv_single_out = nullptr) {
  double S[2 + D];
  float Mx;
  if (!fold_partials<D>(p, acc, accx, status, S, Mx)) return;
  DevState* st = p.st;
  const uint32_t n = sc.n;
  if (!sc.obs) {            // a later stage of the all-stages schedule: no summaries
    st->done = 0;
    __threadfence();
    if (sc.mut) {
      st->stage = 0;
      st->n = n + 1;
    } else {
      st->stage = st->stage + 1;
    }
    return;
  }
  double lme;
  write_summaries<D>(p, S, Mx, n, muf, &lme);
  st->done = 0;
  if constexpr (ADVANCE) {
    __threadfence();
    if (sc.mut) {
      st->stage = 0;
      st->n = n + 1;
    } else {
      st->stage = 1;
    }
  } else {
    st->gmax = Mx;
    if (lv_single_out) *lv_single_out = (float)lme;   // log of the one group's mean weight
  }
}

}  // namespace bfpf
