// step_global.cu - one time step of the bootstrap particle filter with GLOBAL
// multinomial resampling (Algorithm 1 + Algorithm 2 of Heine, Whiteley &
// Cemgil, arXiv 1812.01502: every particle may copy any other), the
// comparator of the butterfly filter, for N above the size one thread block
// resamples (radices = {N}).
//
// The draw follows the same integer rule as the butterfly kernels with one
// group of N members: q_i = floor(fp32 exp(lw_i - max lw) 2^32), P = inclusive
// prefix (64-bit), u_i = floor(r_i Q / 2^64) with a 64-bit uniform r_i from
// counter (i/2, n, 3, 0), ancestor = #{j : P_j <= u_i}.  Three kernels:
//   1. weights: lw_i to memory, block partials -> last block: likelihood
//      increment, mean, ESS, the global maximum and the one group's weight;
//   2. scan: single-pass decoupled look-back prefix sum of q (tiles handed
//      out by an atomic ticket so a tile only waits on tiles already running;
//      waits are bounded and report kStatusTimeout); also records P at every
//      2^top_shift-th index (the top table of the search);
//   3. draws: top table in shared memory, binary search there, then inside
//      one segment of P in global memory; gather the ancestor's state (random
//      access), mutate, write the other state buffer; the last block advances n.
#include <cfloat>

#include "bfpf_device.cuh"
#include "bfpf_epilogue.cuh"
#include "bfpf_kernels.h"
#include "bfpf_model.cuh"

namespace bfpf {

namespace {

constexpr uint32_t kSpinLimit = 1u << 20;   // bounded wait on a predecessor tile (well under a second)

__device__ __forceinline__ unsigned long long ld_volatile_u64(const unsigned long long* p) {
  return *reinterpret_cast<const volatile unsigned long long*>(p);
}
__device__ __forceinline__ uint32_t ld_volatile_u32(const uint32_t* p) {
  return *reinterpret_cast<const volatile uint32_t*>(p);
}

}  // namespace

template <int D, int KIND>
__global__ void __launch_bounds__(kBlock) global_weight_kernel(const __grid_constant__ StepParams p,
                                                              const __grid_constant__ GlobalParams gp) {
  const ModelParams& mp = p.model;
  DevState* st = p.st;
  const uint32_t n = st->n;
  const float* __restrict__ X = gp.xbuf[n & 1u];
  const float lv = p.lV[n & 1u][0];            // one group: one carried weight
  const float muf = st->mu_f;
  const uint32_t N = p.N;
  float y[kMaxDim];
#pragma unroll
  for (int q = 0; q < kMaxDim; ++q) y[q] = (q < mp.dy) ? p.y_ring[(n % kRing) * mp.dy + q] : 0.0f;
  uint32_t status = 0;
  Partial acc{-INFINITY, 0.0f, 0.0f};
  float accx[D];
#pragma unroll
  for (int t = 0; t < D; ++t) accx[t] = 0.0f;
  for (uint32_t i = blockIdx.x * kBlock + threadIdx.x; i < N; i += gridDim.x * kBlock) {
    float xv[D];
#pragma unroll
    for (int t = 0; t < D; ++t) xv[t] = __ldcs(X + (size_t)t * N + i);
    const float lw = sanitize_logweight(lv + obs_log_term<D, KIND>(mp, y, xv) - muf, status);
    gp.lw[i] = lw;
    if (lw != -INFINITY) {
      float one[D];
#pragma unroll
      for (int t = 0; t < D; ++t) one[t] = xv[t];
      merge_partial<D>(acc, accx, lw, 1.0f, 1.0f, one);
    }
  }
  const Sched sc{n, n, 0u, true, true};   // one digit (m = 1): every step is one whole stage
  finish_step<D, false>(p, acc, accx, sc, status, muf, p.lV[(n & 1u) ^ 1u]);
}

__global__ void __launch_bounds__(kBlock) global_scan_kernel(const __grid_constant__ StepParams p,
                                                            const __grid_constant__ GlobalParams gp) {
  __shared__ unsigned long long s_warp[kBlock / 32];
  __shared__ unsigned long long s_prefix;
  __shared__ uint32_t s_tile;
  DevState* st = p.st;
  const uint32_t n = st->n;
  const uint32_t N = p.N;
  const float gmax = st->gmax;
  const uint32_t tid = threadIdx.x, lane = tid & 31u, warp = tid >> 5;
  if (tid == 0) s_tile = (uint32_t)(atomicAdd(&st->ticket, 1ull) - (unsigned long long)n * gp.nscan);
  __syncthreads();
  const uint32_t tile = s_tile;
  const uint32_t base = tile * kScanTile + tid * kScanItems;
  // integer weights of my 16 particles and their running sums
  unsigned long long run[kScanItems];
  unsigned long long tot = 0;
  float lwv[kScanItems];
  if (base + kScanItems <= N) {
#pragma unroll
    for (int q = 0; q < kScanItems / 4; ++q) {
      const float4 v = __ldcs(reinterpret_cast<const float4*>(gp.lw + base) + q);
      lwv[4 * q] = v.x; lwv[4 * q + 1] = v.y; lwv[4 * q + 2] = v.z; lwv[4 * q + 3] = v.w;
    }
  } else {
#pragma unroll
    for (int q = 0; q < kScanItems; ++q) lwv[q] = (base + q < N) ? gp.lw[base + q] : -INFINITY;
  }
  if (tid == 0 && tile == 0 && gmax == -INFINITY) atomicOr(&st->status, kStatusZeroGroup);
#pragma unroll
  for (int q = 0; q < kScanItems; ++q) {
    unsigned long long w = 0;
    if (gmax != -INFINITY) {
      const float e = exp_weight(lwv[q] - gmax);
      w = __float2ull_rz(e * 4294967296.0f);
    }
    tot += w;
    run[q] = tot;
  }
  // block-wide exclusive scan of the thread totals
  unsigned long long incl = tot;
#pragma unroll
  for (int off = 1; off < 32; off <<= 1) {
    const unsigned long long v = __shfl_up_sync(0xffffffffu, incl, off);
    if ((int)lane >= off) incl += v;
  }
  if (lane == 31) s_warp[warp] = incl;
  __syncthreads();
  if (warp == 0) {
    unsigned long long v = (lane < kBlock / 32) ? s_warp[lane] : 0ull;
#pragma unroll
    for (int off = 1; off < kBlock / 32; off <<= 1) {
      const unsigned long long o = __shfl_up_sync(0xffffffffu, v, off);
      if ((int)lane >= off) v += o;
    }
    if (lane < kBlock / 32) s_warp[lane] = v;   // inclusive over warps
  }
  __syncthreads();
  const unsigned long long warp_excl = (warp == 0) ? 0ull : s_warp[warp - 1];
  const unsigned long long thread_excl = warp_excl + incl - tot;
  const unsigned long long tile_total = s_warp[kBlock / 32 - 1];
  // decoupled look-back by warp 0, 32 predecessor tiles per round: every lane
  // waits (bounded) for its tile's aggregate or inclusive prefix; the nearest
  // tile with an inclusive prefix ends the walk
  if (warp == 0) {
    const uint32_t f_agg = 2u * n + 1u, f_pre = 2u * n + 2u;
    unsigned long long prefix = 0;
    if (tile == 0) {
      if (lane == 0) {
        gp.incl[0] = tile_total;
        __threadfence();
        atomicExch(gp.flag, f_pre);
      }
    } else {
      if (lane == 0) {
        gp.agg[tile] = tile_total;
        __threadfence();
        atomicExch(gp.flag + tile, f_agg);
      }
      // test hook: the stalled tile recognises no flag, so its wait runs out
      const bool stall = gp.stall_tile != 0 && tile == gp.stall_tile;
      bool timed_out = false;
      int32_t base = (int32_t)tile - 1;
      while (true) {
        const int32_t t = base - (int32_t)lane;
        uint32_t f = f_pre;                       // before tile 0: an inclusive prefix of 0
        unsigned long long v = 0;
        if (t >= 0) {
          uint32_t spins = 0;
          f = stall ? 0u : ld_volatile_u32(gp.flag + t);
          while (f != f_agg && f != f_pre) {
            if (++spins > kSpinLimit) {
              timed_out = true;                   // counted as an aggregate of 0
              break;
            }
            __nanosleep(32);
            f = stall ? 0u : ld_volatile_u32(gp.flag + t);
          }
          __threadfence();
          if (f == f_pre) v = ld_volatile_u64(gp.incl + t);
          else if (f == f_agg) v = ld_volatile_u64(gp.agg + t);
        }
        const unsigned ready = __ballot_sync(0xffffffffu, f == f_pre);
        const int first = ready ? __ffs(ready) - 1 : 32;   // nearest tile with a prefix
        unsigned long long c = ((int)lane <= first) ? v : 0ull;
#pragma unroll
        for (int off = 16; off; off >>= 1) c += __shfl_xor_sync(0xffffffffu, c, off);
        prefix += c;
        if (ready) break;
        base -= 32;
      }
      if (__any_sync(0xffffffffu, timed_out) && lane == 0) atomicOr(&st->status, kStatusTimeout);
      if (lane == 0) {
        gp.incl[tile] = prefix + tile_total;
        __threadfence();
        atomicExch(gp.flag + tile, f_pre);
      }
    }
    if (lane == 0) s_prefix = prefix;
  }
  __syncthreads();
  const unsigned long long off0 = s_prefix + thread_excl;
  const uint32_t seg_mask = (1u << gp.top_shift) - 1u;
#pragma unroll
  for (int q = 0; q < kScanItems; ++q) {
    const uint32_t i = base + q;
    if (i < N) {
      const unsigned long long P = off0 + run[q];
      gp.P[i] = P;
      if (((i + 1u) & seg_mask) == 0u || i == N - 1u) gp.top[i >> gp.top_shift] = P;
    }
  }
}

template <int D, int KIND>
__global__ void __launch_bounds__(kBlock) global_draw_kernel(const __grid_constant__ StepParams p,
                                                            const __grid_constant__ GlobalParams gp) {
  __shared__ unsigned long long s_top[kTopMax];
  __shared__ uint32_t s_last;
  const ModelParams& mp = p.model;
  DevState* st = p.st;
  const uint32_t n = st->n;
  const uint32_t N = p.N;
  const float* __restrict__ Xin = gp.xbuf[n & 1u];
  float* __restrict__ Xout = gp.xbuf[(n & 1u) ^ 1u];
  const uint32_t ntop = gp.ntop;
  for (uint32_t j = threadIdx.x; j < ntop; j += kBlock) s_top[j] = __ldcg(gp.top + j);
  __syncthreads();
  const unsigned long long Q = s_top[ntop - 1];
  uint32_t lsteps = 1;   // power of two > ntop / 2 for binary lifting over the table
  while (lsteps < ntop) lsteps <<= 1;
  const uint32_t seg = 1u << gp.top_shift;
  uint32_t fsteps = 1;
  while (fsteps < seg) fsteps <<= 1;
  // top table: number of its first ntop - 1 entries <= u (binary lifting in shared memory)
  auto top_count = [&](unsigned long long u) -> uint32_t {
    uint32_t c = 0;
    for (uint32_t stp = lsteps >> 1; stp; stp >>= 1)
      if (c + stp <= ntop - 1 && s_top[c + stp - 1] <= u) c += stp;
    return c;
  };
  auto search = [&](unsigned long long u) -> uint32_t {
    const uint32_t lo = top_count(u) << gp.top_shift;
    const uint32_t len = min(seg, N - lo);
    uint32_t f = 0;   // number of P_j <= u inside the segment (< len)
    for (uint32_t stp = fsteps >> 1; stp; stp >>= 1)
      if (f + stp <= len - 1 && __ldcg(gp.P + lo + f + stp - 1) <= u) f += stp;
    return lo + f;
  };
  // quads of consecutive particles share their Philox blocks
  const uint32_t nquad = (N % 4u == 0u) ? N / 4u : 0u;
  for (uint32_t q = blockIdx.x * kBlock + threadIdx.x; q < nquad; q += gridDim.x * kBlock) {
    const uint32_t i0 = 4u * q;
    const uint4 w0 = philox4x32_10(make_uint4(i0 >> 1, n, kPurposeResampleWide, 0), p.rk);
    const uint4 w1 = philox4x32_10(make_uint4((i0 >> 1) + 1, n, kPurposeResampleWide, 0), p.rk);
    const unsigned long long r64[4] = {((unsigned long long)w0.y << 32) | w0.x,
                                       ((unsigned long long)w0.w << 32) | w0.z,
                                       ((unsigned long long)w1.y << 32) | w1.x,
                                       ((unsigned long long)w1.w << 32) | w1.z};
    float z[4 * D];
#pragma unroll
    for (int b = 0; b < D; ++b) {
      const uint4 wz = philox4x32_10(make_uint4(q * D + b, n, kPurposePropagate, 0), p.rk);
      normals4(wz, z + 4 * b);
    }
    float xo[D][4];
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const uint32_t anc = (Q != 0) ? search(__umul64hi(r64[j], Q)) : i0 + j;
      float xh[D], o[D];
#pragma unroll
      for (int t = 0; t < D; ++t) xh[t] = __ldg(Xin + (size_t)t * N + anc);
      mutate<D, KIND>(mp, xh, z + j * D, o);
#pragma unroll
      for (int t = 0; t < D; ++t) xo[t][j] = o[t];
      if (p.anc) p.anc[i0 + j] = (int32_t)anc;
    }
#pragma unroll
    for (int t = 0; t < D; ++t)
      __stcs(reinterpret_cast<float4*>(Xout + (size_t)t * N + i0), make_float4(xo[t][0], xo[t][1], xo[t][2], xo[t][3]));
  }
  for (uint32_t i = 4u * nquad + blockIdx.x * kBlock + threadIdx.x; i < N; i += gridDim.x * kBlock) {
    const uint4 w = philox4x32_10(make_uint4(i >> 1, n, kPurposeResampleWide, 0), p.rk);
    const unsigned long long r64 = (i & 1u) ? (((unsigned long long)w.w << 32) | w.z)
                                             : (((unsigned long long)w.y << 32) | w.x);
    const uint32_t anc = (Q != 0) ? search(__umul64hi(r64, Q)) : i;
    float xh[D], xo[D], z[D];
#pragma unroll
    for (int t = 0; t < D; ++t) {
      xh[t] = __ldg(Xin + (size_t)t * N + anc);
      const uint32_t nu = i * D + t;
      const uint4 wz = philox4x32_10(make_uint4(nu >> 2, n, kPurposePropagate, 0), p.rk);
      float zz[4];
      normals4(wz, zz);
      z[t] = zz[nu & 3u];
    }
    mutate<D, KIND>(mp, xh, z, xo);
#pragma unroll
    for (int t = 0; t < D; ++t) __stcs(Xout + (size_t)t * N + i, xo[t]);
    if (p.anc) p.anc[i] = (int32_t)anc;
  }
  // the last block to finish advances the step counter
  __syncthreads();
  if (threadIdx.x == 0) {
    __threadfence();
    const uint32_t prev = atomicAdd(&st->done2, 1u);
    s_last = (prev == gridDim.x - 1) ? 1u : 0u;
  }
  __syncthreads();
  if (s_last && threadIdx.x == 0) {
    st->done2 = 0;
    __threadfence();
    st->n = n + 1;
  }
}

template <int D, int KIND>
static void fill_global(GlobalKernels& gk) {
  gk.weight = reinterpret_cast<const void*>(&global_weight_kernel<D, KIND>);
  gk.scan = reinterpret_cast<const void*>(&global_scan_kernel);
  gk.draw = reinterpret_cast<const void*>(&global_draw_kernel<D, KIND>);
}

bool select_global_kernels(int d, int kind, GlobalKernels& gk) {
  if (kind == kStochVol) {
    if (d != 1) return false;
    fill_global<1, kStochVol>(gk);
    return true;
  }
  switch (d) {
    case 1: fill_global<1, kLinearGaussian>(gk); return true;
    case 2: fill_global<2, kLinearGaussian>(gk); return true;
    case 3: fill_global<3, kLinearGaussian>(gk); return true;
    case 4: fill_global<4, kLinearGaussian>(gk); return true;
    case 5: fill_global<5, kLinearGaussian>(gk); return true;
    case 6: fill_global<6, kLinearGaussian>(gk); return true;
    case 7: fill_global<7, kLinearGaussian>(gk); return true;
    case 8: fill_global<8, kLinearGaussian>(gk); return true;
    default: return false;
  }
}

}  // namespace bfpf
