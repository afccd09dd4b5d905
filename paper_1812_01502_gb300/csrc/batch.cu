// batch.cu - thousands of independent butterfly particle filters (uneven N,
// state dimension and radices) advanced one time step per kernel launch.
//
// Each filter is the filter of step_butterfly.cu (Algorithm 1 with one stage
// of Algorithm 3 per step, Heine, Whiteley & Cemgil, arXiv 1812.01502).  One
// time step of every filter of the batch is one launch per class of filters
// (model kind and state dimension) and a launch that advances the step.  A filter's step is
// split into U work units (U from the filter's own size only, so a filter's
// results do not depend on the rest of the batch): unit j runs the tiles j,
// j + U, ... of the step's digit with the shared tile code.  A filter with one
// unit finishes its step (likelihood increment, filter mean, ESS) inside its
// block; with several, every unit writes its partial sums and the last unit to
// arrive folds them in unit order (last-block-done per filter, deterministic).
// A digit whose radix is a power of two <= 32 (groups filling whole block
// iterations) runs the register-resident group code of step_group.cuh
// instead of the tile code: unit j takes its block iterations j, j + U, ....
// Units are launched largest first, so that the big filters start at once and
// small ones fill the machine behind them.
#include <cfloat>
#include <type_traits>

#include "bfpf_batch.cuh"
#include "bfpf_kernels.h"
#include "bfpf_model.cuh"
#include "step_group.cuh"
#include "step_tile.cuh"

namespace bfpf {

namespace {

// Block reduction of the per-thread partials; the result is valid in thread 0.
template <int D>
__device__ __forceinline__ void block_partial(Partial& acc, float* accx, Partial& b, float* bx) {
  constexpr int NP = 3 + D;
  constexpr int NW = kBlock / 32;
  __shared__ float s_red[NW][NP];
  const uint32_t tid = threadIdx.x, lane = tid & 31u, warp = tid >> 5;
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
  b = Partial{-INFINITY, 0.0f, 0.0f};
#pragma unroll
  for (int t = 0; t < D; ++t) bx[t] = 0.0f;
  if (tid == 0)
    for (int w = 0; w < NW; ++w) merge_partial<D>(b, bx, s_red[w][0], s_red[w][1], s_red[w][2], &s_red[w][3]);
}

// The step's summaries of filter fid from its folded sums (one thread).
template <int D>
__device__ __forceinline__ void filter_summaries(const BatchParams& bp, BatchFilter& f, uint32_t fid, uint32_t n,
                                                 const Partial& b, const float* bx, float muf) {
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

// Unit j of U of filter fid at step n on the group path (radix A of digit k).
template <int D, int KIND, int A>
__device__ __forceinline__ void batch_group_pass(const BatchParams& bp, BatchFilter& f, uint32_t fid, uint32_t n,
                                                 uint32_t k, uint32_t j, uint32_t U, unsigned char* smem, Partial& acc,
                                                 float* accx, uint32_t& status) {
  constexpr int G = A / group_members_per_lane(A, D);
  using LY = GroupLayout<D, A, G>;
  static_assert(4 * (LY::kRowWords + LY::kTabWords) == (int)group_smem_bytes(D, A), "shared-memory size");
  uint32_t* const s_rows = reinterpret_cast<uint32_t*>(smem);
  uint32_t* const s_tab = s_rows + LY::kRowWords;
  GroupCtx c;
  c.x = f.x;
  c.lV_in = f.lV[n & 1u];
  c.lV_out = f.lV[(n & 1u) ^ 1u];
  c.anc = nullptr;
  c.prec = nullptr;
  c.N = f.N;
  c.n = n;
  c.t = n;            // one stage per time step
  c.obs = true;
  c.mut = true;
  c.muf = f.st.mu_f;
  const float* yr = bp.y_ring + ((size_t)fid * bp.ring + n % bp.ring) * bp.dy_max;
#pragma unroll
  for (int q = 0; q < kMaxDim; ++q) c.y[q] = (q < (int)f.model.dy) ? yr[q] : 0.0f;
  const RoundKeys rk = f.rk;    // in registers: the Philox rounds read every key
  group_iterations<D, KIND, A, G, false>(c, rk, f.model, f.gg[k], j, U, s_rows, s_tab, acc, accx, status);
}

// Unit j of U of filter fid at step n (GROUP: the digit is on the group path).
template <int D, int KIND, bool GROUP>
__device__ __forceinline__ void batch_unit_step(const BatchParams& bp, BatchFilter& f, uint32_t fid, uint32_t n,
                                                uint32_t j, uint32_t U, unsigned char* smem) {
  __shared__ uint32_t s_last;
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
  for (int q = 0; q < kMaxDim; ++q) ctx.y[q] = (q < (int)f.model.dy) ? yr[q] : 0.0f;
  uint32_t status = 0;
  Partial acc{-INFINITY, 0.0f, 0.0f};
  float accx[D];
#pragma unroll
  for (int t = 0; t < D; ++t) accx[t] = 0.0f;
  if constexpr (GROUP) {
    switch (f.geom[k].a) {
      case 2: batch_group_pass<D, KIND, 2>(bp, f, fid, n, k, j, U, smem, acc, accx, status); break;
      case 4: batch_group_pass<D, KIND, 4>(bp, f, fid, n, k, j, U, smem, acc, accx, status); break;
      case 8: batch_group_pass<D, KIND, 8>(bp, f, fid, n, k, j, U, smem, acc, accx, status); break;
      case 16: batch_group_pass<D, KIND, 16>(bp, f, fid, n, k, j, U, smem, acc, accx, status); break;
      default: batch_group_pass<D, KIND, 32>(bp, f, fid, n, k, j, U, smem, acc, accx, status); break;
    }
  } else {
    tile_steps<D, KIND, false>(ctx, j, U, smem, acc, accx, status);
  }
  if (status) atomicOr(&f.st.status, status);
  Partial b;
  float bx[D];
  block_partial<D>(acc, accx, b, bx);
  if (U == 1) {
    if (threadIdx.x == 0) filter_summaries<D>(bp, f, fid, n, b, bx, ctx.muf);
    return;
  }
  if (threadIdx.x == 0) {
    float* out = bp.partials + (size_t)(f.pbase + j) * kBatchNP;
    out[0] = b.m;
    out[1] = b.s1;
    out[2] = b.s2;
#pragma unroll
    for (int t = 0; t < D; ++t) out[3 + t] = bx[t];
    __threadfence();
    const uint32_t prev = atomicAdd(&f.st.done, 1u);
    s_last = (prev == U - 1) ? 1u : 0u;
  }
  __syncthreads();
  if (!s_last || threadIdx.x != 0) return;
  __threadfence();
  // last unit of the filter: fold the U partials in unit order
  Partial t{-INFINITY, 0.0f, 0.0f};
  float tx[D];
#pragma unroll
  for (int q = 0; q < D; ++q) tx[q] = 0.0f;
  for (uint32_t u = 0; u < U; ++u) {
    const float* pu = bp.partials + (size_t)(f.pbase + u) * kBatchNP;
    float ux[D];
#pragma unroll
    for (int q = 0; q < D; ++q) ux[q] = __ldcg(pu + 3 + q);
    merge_partial<D>(t, tx, __ldcg(pu), __ldcg(pu + 1), __ldcg(pu + 2), ux);
  }
  filter_summaries<D>(bp, f, fid, n, t, tx, ctx.muf);
  f.st.done = 0;
}

}  // namespace

// One time step of the work units u0 .. u0 + gridDim.x - 1, all of one model
// kind and state dimension (kernels per class, so that each keeps the
// registers its own dimension needs), split by the path of each unit's digit
// this step: the tile kernel returns at once for a unit on the group path and
// the group kernel for a unit on the tile path (all units of a filter take the
// same path in a step), so that the group code keeps the register budget of
// the single-filter group kernels.
template <int D, int KIND, bool GROUP>
__device__ __forceinline__ void batch_class_body(const BatchParams& bp, uint32_t u0, unsigned char* smem) {
  const uint32_t n = bp.state->n;
  const uint2 un = bp.units[u0 + blockIdx.x];
  const uint32_t fid = un.x, j = un.y & 0xffffu, U = un.y >> 16;
  BatchFilter& f = bp.filters[fid];
  const bool on_group = (f.gsel >> (n % f.m)) & 1u;
  if (on_group != GROUP) return;                  // block-uniform
  batch_unit_step<D, KIND, GROUP>(bp, f, fid, n, j, U, smem);
}

template <int D, int KIND>
__global__ void __launch_bounds__(kBlock, 2) batch_class_kernel(const __grid_constant__ BatchParams bp, uint32_t u0) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  batch_class_body<D, KIND, false>(bp, u0, smem_raw);
}

template <int D, int KIND>
__global__ void __launch_bounds__(kBlock, 2) batch_group_kernel(const __grid_constant__ BatchParams bp,
                                                                                uint32_t u0) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  batch_class_body<D, KIND, true>(bp, u0, smem_raw);
}

// After every class of a step: advance the batch's step counter.
__global__ void batch_advance_kernel(const __grid_constant__ BatchParams bp) {
  if (threadIdx.x == 0 && blockIdx.x == 0) bp.state->n = bp.state->n + 1;
}

const void* batch_class_kernel_ptr(int kind, int d) {
  if (kind == kStochVol) return d == 1 ? reinterpret_cast<const void*>(&batch_class_kernel<1, kStochVol>) : nullptr;
  switch (d) {
    case 1: return reinterpret_cast<const void*>(&batch_class_kernel<1, kLinearGaussian>);
    case 2: return reinterpret_cast<const void*>(&batch_class_kernel<2, kLinearGaussian>);
    case 3: return reinterpret_cast<const void*>(&batch_class_kernel<3, kLinearGaussian>);
    case 4: return reinterpret_cast<const void*>(&batch_class_kernel<4, kLinearGaussian>);
    case 5: return reinterpret_cast<const void*>(&batch_class_kernel<5, kLinearGaussian>);
    case 6: return reinterpret_cast<const void*>(&batch_class_kernel<6, kLinearGaussian>);
    case 7: return reinterpret_cast<const void*>(&batch_class_kernel<7, kLinearGaussian>);
    case 8: return reinterpret_cast<const void*>(&batch_class_kernel<8, kLinearGaussian>);
    default: return nullptr;
  }
}
const void* batch_group_kernel_ptr(int kind, int d) {
  if (kind == kStochVol) return d == 1 ? reinterpret_cast<const void*>(&batch_group_kernel<1, kStochVol>) : nullptr;
  switch (d) {
    case 1: return reinterpret_cast<const void*>(&batch_group_kernel<1, kLinearGaussian>);
    case 2: return reinterpret_cast<const void*>(&batch_group_kernel<2, kLinearGaussian>);
    case 3: return reinterpret_cast<const void*>(&batch_group_kernel<3, kLinearGaussian>);
    case 4: return reinterpret_cast<const void*>(&batch_group_kernel<4, kLinearGaussian>);
    case 5: return reinterpret_cast<const void*>(&batch_group_kernel<5, kLinearGaussian>);
    case 6: return reinterpret_cast<const void*>(&batch_group_kernel<6, kLinearGaussian>);
    case 7: return reinterpret_cast<const void*>(&batch_group_kernel<7, kLinearGaussian>);
    case 8: return reinterpret_cast<const void*>(&batch_group_kernel<8, kLinearGaussian>);
    default: return nullptr;
  }
}
const void* batch_advance_kernel_ptr() { return reinterpret_cast<const void*>(&batch_advance_kernel); }

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

const void* batch_init_kernel_ptr() { return reinterpret_cast<const void*>(&batch_init_kernel); }

}  // namespace bfpf
