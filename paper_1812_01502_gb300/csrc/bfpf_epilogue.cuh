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

// Floats as order-preserving signed integers (for redux.sync max): a
// non-negative float keeps its bits, a negative one flips its magnitude bits.
__device__ __forceinline__ int float_order(float f) {
  const int i = __float_as_int(f);
  return i >= 0 ? i : (i ^ 0x7fffffff);
}
__device__ __forceinline__ float order_float(int i) { return __int_as_float(i >= 0 ? i : (i ^ 0x7fffffff)); }

// Natural log of a positive double x to about 1e-7 absolute: the exponent part
// exactly in FP64, log of the mantissa in [1, 2) by logf.
__device__ __forceinline__ double log_split(double x) {
  const long long b = __double_as_longlong(x);
  const int e = (int)((b >> 52) & 0x7ff) - 1023;
  const double m = __longlong_as_double((b & 0x000fffffffffffffLL) | 0x3ff0000000000000LL);
  return (double)e * 0.6931471805599453 + (double)logf((float)m);
}

// Grid-wide fold of the per-thread partials, called by every thread of every
// block exactly once.  Each block takes the largest of its threads' maxima
// (redux.sync), rescales every thread's sums to it (one exp per thread), sums
// them by shuffles and writes the block partial; the last block to arrive
// (last-block-done) folds all block partials in a fixed order with
// compensated FP32 sums.  Returns true in thread 0 of the last block only,
// with S[0] = sum e^{lw - Mx}, S[1] = sum e^{2(lw - Mx)}, S[2 + t] = sum
// e^{lw - Mx} x_t (FP64) and Mx the global maximum.
template <int D>
__device__ __forceinline__ bool fold_partials(const StepParams& p, Partial acc, float* accx, uint32_t status,
                                              double* S, float& Mx_out) {
  constexpr int NP = 3 + D;
  constexpr int NW = kBlock / 32;
  constexpr unsigned FULL = 0xffffffffu;
  __shared__ int s_max[NW];
  __shared__ float s_red[NW][NP];
  __shared__ float s_redlo[NW][NP];
  __shared__ uint32_t s_last;
  DevState* st = p.st;
  const uint32_t tid = threadIdx.x;
  if (status) atomicOr(&st->status, status);
  const uint32_t lane = tid & 31u, warp = tid >> 5;

  // ---- block partial: max, then rescaled sums ----
  int mi = __reduce_max_sync(FULL, float_order(acc.m));
  if (lane == 0) s_max[warp] = mi;
  __syncthreads();
  mi = s_max[0];
#pragma unroll
  for (int w = 1; w < NW; ++w) mi = max(mi, s_max[w]);
  const float bm = order_float(mi);
  const float sc = (acc.m == -INFINITY) ? 0.0f : expf(acc.m - bm);
  float v[NP - 1];
  v[0] = acc.s1 * sc;
  v[1] = acc.s2 * (sc * sc);
#pragma unroll
  for (int t = 0; t < D; ++t) v[2 + t] = accx[t] * sc;
#pragma unroll
  for (int off = 16; off; off >>= 1) {
#pragma unroll
    for (int k = 0; k < NP - 1; ++k) v[k] += __shfl_xor_sync(FULL, v[k], off);
  }
  if (lane == 0) {
#pragma unroll
    for (int k = 0; k < NP - 1; ++k) s_red[warp][k] = v[k];
  }
  __syncthreads();
  if (tid == 0) {
    float* out = p.partials + (size_t)blockIdx.x * NP;
    out[0] = bm;
#pragma unroll
    for (int k = 0; k < NP - 1; ++k) {
      float a = s_red[0][k];
      for (int w = 1; w < NW; ++w) a += s_red[w][k];
      out[1 + k] = a;
    }
    __threadfence();
    const uint32_t prev = atomicAdd(&st->done, 1u);
    s_last = (prev == gridDim.x - 1) ? 1u : 0u;
  }
  __syncthreads();
  if (!s_last) return false;
  __threadfence();

  // ---- last block: fold all block partials (fixed order, compensated FP32) ----
  // One pass: each thread folds its partials b = tid, tid + kBlock, ... against
  // its own running maximum (rescaling when a larger one arrives), then the
  // block's maximum rescales every thread's sums before the shuffle fold.
  const uint32_t G = gridDim.x;
  float mt = -INFINITY;
  float hi[NP - 1], lo[NP - 1];
#pragma unroll
  for (int k = 0; k < NP - 1; ++k) hi[k] = lo[k] = 0.0f;
  for (uint32_t b = tid; b < G; b += kBlock) {
    const float* pb = p.partials + (size_t)b * NP;
    const float mb = __ldcg(pb);
    float v[NP - 1];
#pragma unroll
    for (int k = 0; k < NP - 1; ++k) v[k] = __ldcg(pb + 1 + k);
    if (mb == -INFINITY) continue;
    float w = 1.0f;
    if (mb > mt) {
      const float r = (mt == -INFINITY) ? 0.0f : expf(mt - mb);
#pragma unroll
      for (int k = 0; k < NP - 1; ++k) {
        const float rk = (k == 1) ? r * r : r;
        hi[k] *= rk;
        lo[k] *= rk;
      }
      mt = mb;
    } else {
      w = expf(mb - mt);
    }
    ff_add(hi[0], lo[0], v[0] * w);
    ff_add(hi[1], lo[1], v[1] * (w * w));
#pragma unroll
    for (int t = 0; t < D; ++t) ff_add(hi[2 + t], lo[2 + t], v[2 + t] * w);
  }
  int gi = __reduce_max_sync(FULL, float_order(mt));
  __syncthreads();
  if (lane == 0) s_max[warp] = gi;
  __syncthreads();
  gi = s_max[0];
#pragma unroll
  for (int w = 1; w < NW; ++w) gi = max(gi, s_max[w]);
  const float Mx = order_float(gi);
  {
    const float r = (mt == -INFINITY) ? 0.0f : expf(mt - Mx);
#pragma unroll
    for (int k = 0; k < NP - 1; ++k) {
      const float rk = (k == 1) ? r * r : r;
      hi[k] *= rk;
      lo[k] *= rk;
    }
  }
#pragma unroll
  for (int off = 16; off; off >>= 1) {
#pragma unroll
    for (int k = 0; k < NP - 1; ++k) {
      const float oh = __shfl_down_sync(FULL, hi[k], off);
      const float ol = __shfl_down_sync(FULL, lo[k], off);
      ff_add(hi[k], lo[k], oh);
      lo[k] += ol;
    }
  }
  if (lane == 0) {
#pragma unroll
    for (int k = 0; k < NP - 1; ++k) {
      s_red[warp][k] = hi[k];
      s_redlo[warp][k] = lo[k];
    }
  }
  __syncthreads();
  if (tid != 0) return false;
#pragma unroll
  for (int k = 0; k < NP - 1; ++k) {
    float h = 0.0f, l = 0.0f;
    for (int w = 0; w < NW; ++w) {
      ff_add(h, l, s_red[w][k]);
      l += s_redlo[w][k];
    }
    S[k] = (double)h + (double)l;
  }
  Mx_out = Mx;
  return true;
}

// Writes the step's summaries from the folded sums (thread 0 of the last block):
// likelihood increment, filter mean and ESS into the output rings, the
// cumulative log-likelihood (FP64) and the next normaliser.  Returns the ESS.
// The log of the weight sum is taken as exponent (FP64) plus log of the
// mantissa (FP32), about 1e-7 absolute; mean and ESS are FP32 outputs.
template <int D>
__device__ __forceinline__ double write_summaries(const StepParams& p, const double* S, float Mx, uint32_t n,
                                                  float muf, double* lme_out = nullptr) {
  DevState* st = p.st;
  const ModelParams& mp = p.model;
  const uint32_t slot = n % kRing;
  const double mu_prev = st->mu;
  const double ll_prev = st->loglik;
  double lme, inc, ess;
  if (Mx == -INFINITY || !(S[0] > 0.0)) {
    lme = -INFINITY;
    inc = -INFINITY;
    ess = 0.0;
  } else {
    lme = (double)Mx + (log_split(S[0]) - log_split((double)p.N));
    inc = lme + ((double)muf - mu_prev) + mp.c_obs;
    const float s0 = (float)S[0];
    ess = (double)(s0 * s0 / ((float)p.N * (float)S[1]));
  }
  p.inc_ring[slot] = inc;
  p.ess_ring[slot] = (float)ess;
  const float inv_s0 = 1.0f / (float)S[0];
  for (int t = 0; t < D; ++t) p.mean_ring[slot * mp.d + t] = (float)S[2 + t] * inv_s0;
  st->loglik = ll_prev + inc;
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

// End of one launch of the one-digit or all-stages schedule; the launch ran
// adv stages (several when the all-stages schedule fuses consecutive digits).
// ADVANCE = false (global resampling, which finishes the step in a later
// kernel): the last block leaves n alone and instead writes the global
// maximum log-weight and the single group's new log weight.
template <int D, bool ADVANCE = true>
__device__ __forceinline__ void finish_step(const StepParams& p, Partial acc, float* accx, const Sched& sc,
                                            uint32_t status, float muf, float* lv_single_out = nullptr,
                                            uint32_t adv = 1u) {
  DevState* st = p.st;
  const uint32_t n = sc.n;
  if (!sc.obs) {            // a later stage of the all-stages schedule: no summaries,
    __shared__ uint32_t s_last_stage;   // only the last block to finish advances the stage
    if (status) atomicOr(&st->status, status);
    __syncthreads();
    if (threadIdx.x == 0) s_last_stage = (atomicAdd(&st->done, 1u) == gridDim.x - 1) ? 1u : 0u;
    __syncthreads();
    if (!s_last_stage || threadIdx.x != 0) return;
    st->done = 0;
    __threadfence();
    if (sc.mut) {
      st->stage = 0;
      st->n = n + 1;
    } else {
      st->stage = st->stage + adv;
    }
    return;
  }
  double S[2 + D];
  float Mx;
  if (!fold_partials<D>(p, acc, accx, status, S, Mx)) return;
  double lme;
  write_summaries<D>(p, S, Mx, n, muf, &lme);
  st->done = 0;
  if constexpr (ADVANCE) {
    __threadfence();
    if (sc.mut) {
      st->stage = 0;
      st->n = n + 1;
    } else {
      st->stage = adv;
    }
  } else {
    st->gmax = Mx;
    if (lv_single_out) *lv_single_out = (float)lme;   // log of the one group's mean weight
  }
}

}  // namespace bfpf
