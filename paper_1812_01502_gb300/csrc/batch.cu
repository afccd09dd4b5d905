// batch.cu - thousands of independent butterfly particle filters (uneven N,
// state dimension and radices) advanced one time step per kernel launch.
//
// Each filter is the filter of step_butterfly.cu (Algorithm 1 with one stage
// of Algorithm 3 per step, Heine, Whiteley & Cemgil, arXiv 1812.01502).  One
// launch covers a whole chunk of time steps of every filter of the batch:
// block b runs filter order[b] (filters sorted by decreasing work, so the
// largest start first) step after step with the shared tile code, finishing
// each step's likelihood increment, filter mean and ESS inside the block - a
// filter never needs another block, so nothing waits and blocks of small
// filters flow through the chunk without per-step launches.  The last block
// to finish advances the batch's step counter (last-block-done).
#include <cfloat>
#include <type_traits>

#include "bfpf_batch.cuh"
#include "bfpf_kernels.h"
#include "bfpf_model.cuh"
#include "step_tile.cuh"

namespace bfpf {

namespace {

// Block-level end of one filter's step (the single-block form of finish_step).
template <int D>
__device__ __forceinline__ void block_finish(const BatchParams& bp, BatchFilter& f, uint32_t fid, uint32_t n,
                                             Partial acc, float* accx, uint32_t status, float muf) {
  constexpr int NP = 3 + D;
  constexpr int NW = kBlock / 32;
  __shared__ float s_red[NW][NP];
  const uint32_t tid = threadIdx.x, lane = tid & 31u, warp = tid >> 5;
  if (status) atomicOr(&f.st.status, status);
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
    const uint32_t slot = n % bp.ring;
    double lme, inc, ess;
    if (b.m == -INFINITY || !(b.s1 > 0.0f)) {
      lme = -INFINITY;
      inc = -INFINITY;
      ess = 0.0;
    } else {
      lme = (double)b.m + log((double)b.s1 / (double)f.N);
      inc = lme + ((double)muf - f.st.mu) + f.model.c_obs;
      ess = (double)b.s1 * (double)b.s1 / ((double)f.N * (double)b.s2);
    }
    bp.inc_ring[(size_t)fid * bp.ring + slot] = inc;
    bp.ess_ring[(size_t)fid * bp.ring + slot] = (float)ess;
    for (int t = 0; t < D; ++t)
      bp.mean_ring[((size_t)fid * bp.ring + slot) * bp.d_max + t] = (float)((double)bx[t] / (double)b.s1);
    f.st.loglik += inc;
    f.st.mu = lme;
    f.st.mu_f = (float)lme;
  }
}

template <int D, int KIND>
__device__ __forceinline__ void batch_filter_step(const BatchParams& bp, BatchFilter& f, uint32_t fid, uint32_t n,
                                                  unsigned char* smem) {
  TileCtx ctx;
  const uint32_t k = n % f.m;
  ctx.n = n;
  ctx.t = n;          // one stage per time step
  ctx.obs = true;
  ctx.mut = true;
  ctx.x = f.x;
  ctx.lV_in = f.lV[n & 1u];
  ctx.lV_out = f.lV[(n & 1u) ^ 1u];
  ctx.anc = nullptr;
  ctx.prec = nullptr;
  ctx.rk = &f.rk;
  ctx.mp = &f.model;
  ctx.g = &f.geom[k];
  ctx.N = f.N;
  ctx.cap = f.cap;
  ctx.muf = f.st.mu_f;
  const float* yr = bp.y_ring + ((size_t)fid * bp.ring + n % bp.ring) * bp.dy_max;
#pragma unroll
  for (int j = 0; j < kMaxDim; ++j) ctx.y[j] = (j < (int)f.model.dy) ? yr[j] : 0.0f;
  uint32_t status = 0;
  Partial acc{-INFINITY, 0.0f, 0.0f};
  float accx[D];
#pragma unroll
  for (int t = 0; t < D; ++t) accx[t] = 0.0f;
  tile_steps<D, KIND, false>(ctx, 0, 1, smem, acc, accx, status);
  block_finish<D>(bp, f, fid, n, acc, accx, status, ctx.muf);
}

// Steps n0 .. n0 + steps - 1 of one filter: a filter never depends on another,
// so its block runs the whole chunk without any grid-wide synchronisation.
template <int D, int KIND>
__device__ __forceinline__ void batch_filter_steps(const BatchParams& bp, BatchFilter& f, uint32_t fid, uint32_t n0,
                                                   uint32_t steps, unsigned char* smem) {
  for (uint32_t j = 0; j < steps; ++j) {
    batch_filter_step<D, KIND>(bp, f, fid, n0 + j, smem);
    __syncthreads();   // this filter's normaliser and weights are in place for the next step
  }
}

}  // namespace

// One launch runs `steps` consecutive time steps of every filter (one block per filter).
__global__ void __launch_bounds__(kBlock) batch_step_kernel(const __grid_constant__ BatchParams bp, uint32_t steps) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ uint32_t s_last;
  const uint32_t n = bp.state->n;
  const uint32_t fid = bp.order[blockIdx.x];
  BatchFilter& f = bp.filters[fid];
  const int d = f.model.d;
  if (f.model.kind == kStochVol) {
    batch_filter_steps<1, kStochVol>(bp, f, fid, n, steps, smem_raw);
  } else {
    switch (d) {
      case 1: batch_filter_steps<1, kLinearGaussian>(bp, f, fid, n, steps, smem_raw); break;
      case 2: batch_filter_steps<2, kLinearGaussian>(bp, f, fid, n, steps, smem_raw); break;
      case 3: batch_filter_steps<3, kLinearGaussian>(bp, f, fid, n, steps, smem_raw); break;
      case 4: batch_filter_steps<4, kLinearGaussian>(bp, f, fid, n, steps, smem_raw); break;
      case 5: batch_filter_steps<5, kLinearGaussian>(bp, f, fid, n, steps, smem_raw); break;
      case 6: batch_filter_steps<6, kLinearGaussian>(bp, f, fid, n, steps, smem_raw); break;
      case 7: batch_filter_steps<7, kLinearGaussian>(bp, f, fid, n, steps, smem_raw); break;
      default: batch_filter_steps<8, kLinearGaussian>(bp, f, fid, n, steps, smem_raw); break;
    }
  }
  // the last block to finish advances the batch's step counter
  if (threadIdx.x == 0) {
    __threadfence();
    const uint32_t prev = atomicAdd(&bp.state->done, 1u);
    s_last = (prev == gridDim.x - 1) ? 1u : 0u;
  }
  __syncthreads();
  if (s_last && threadIdx.x == 0) {
    bp.state->done = 0;
    __threadfence();
    bp.state->n = n + steps;
  }
}

// Initial particles of every filter (one block per filter).
__global__ void __launch_bounds__(kBlock) batch_init_kernel(const __grid_constant__ BatchParams bp) {
  const BatchFilter& f = bp.filters[blockIdx.x];
  const ModelParams& mp = f.model;
  const uint32_t d = (uint32_t)mp.d;
  for (uint32_t i = threadIdx.x; i < f.N; i += kBlock) {
    float z[kMaxDim];
    for (uint32_t t = 0; t < d; ++t) {
      const uint32_t nu = i * d + t;
      const uint4 w = philox4x32(make_uint4(nu >> 2, 0, kPurposeInit, 0), f.rk);
      float zz[4];
      normals4(w, zz);
      z[t] = zz[nu & 3u];
    }
    for (uint32_t t = 0; t < d; ++t) {
      float v;
      if (mp.kind == kStochVol) {
        v = mp.sd0 * z[0];
      } else {
        v = mp.m0[t];
        for (uint32_t u = 0; u <= t; ++u) v = fmaf(mp.L0[t * kMaxDim + u], z[u], v);
      }
      f.x[(size_t)t * f.N + i] = v;
    }
  }
}

const void* batch_step_kernel_ptr() { return reinterpret_cast<const void*>(&batch_step_kernel); }
const void* batch_init_kernel_ptr() { return reinterpret_cast<const void*>(&batch_init_kernel); }

}  // namespace bfpf
