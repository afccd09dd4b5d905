// step_islands.cu - the augmented island resampling particle filter (AIRPF,
// Algorithm 4 of Heine, Whiteley & Cemgil, arXiv 1812.01502): N = M m
// particles in m = 2^S islands of M consecutive particles.  One time step =
// three launches:
//   1. within-island resampling (Algorithm 5): the stage kernel on digit 0 of
//      radices (M, m) with the observation weight and without mutation; the
//      carried weight it writes per group is the island weight of eq. (out weight);
//   2. island_stages_kernel: augmented island resampling (Algorithm 6, or the
//      modified Algorithm 7 that undoes pure swaps) on the m island weights,
//      S stages pairing island i with i xor 2^(s-1); one thread block, the
//      island weights and sample holders in shared memory;
//   3. island_gather_kernel: every particle of island i takes the particle at
//      the same place in the sample island i now holds, mutates, and writes the
//      other state buffer (an island may copy from any island).
#include <cfloat>

#include "bfpf_device.cuh"
#include "bfpf_epilogue.cuh"
#include "bfpf_kernels.h"
#include "bfpf_model.cuh"

namespace bfpf {

// Launched with one block of kIslandThreads threads and 8 * islands bytes of
// dynamic shared memory.
__global__ void __launch_bounds__(kIslandThreads) island_stages_kernel(const __grid_constant__ StepParams p,
                                                                        const __grid_constant__ IslandParams ip) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  float* V = reinterpret_cast<float*>(smem_raw);
  int32_t* H = reinterpret_cast<int32_t*>(V + ip.islands);
  const uint32_t n = p.st->n;
  const uint32_t tid = threadIdx.x;
  for (uint32_t i = tid; i < ip.islands; i += blockDim.x) {
    V[i] = ip.lW[i];
    H[i] = (int32_t)i;
  }
  __syncthreads();
  const float log2f_ = 0.69314718055994531f;
  __shared__ float s_red[3][kIslandThreads / 32];
  __shared__ uint32_t s_stop;
  uint32_t executed = 0;
  for (uint32_t s = 1; s <= ip.S; ++s) {
    if (ip.adaptive) {
      // AIRPF2: ESS of the island weights, (sum W)^2 / (m sum W^2); stop once >= theta
      const uint32_t lane = tid & 31u, warp = tid >> 5;
      float mx = -INFINITY;
      for (uint32_t i = tid; i < ip.islands; i += blockDim.x) mx = fmaxf(mx, V[i]);
#pragma unroll
      for (int off = 16; off; off >>= 1) mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, off));
      if (lane == 0) s_red[0][warp] = mx;
      __syncthreads();
      mx = -INFINITY;
      for (uint32_t w2 = 0; w2 < blockDim.x / 32; ++w2) mx = fmaxf(mx, s_red[0][w2]);
      float a1 = 0.0f, a2 = 0.0f;
      if (mx != -INFINITY) {
        for (uint32_t i = tid; i < ip.islands; i += blockDim.x) {
          const float e = expf(V[i] - mx);
          a1 += e;
          a2 = fmaf(e, e, a2);
        }
      }
#pragma unroll
      for (int off = 16; off; off >>= 1) {
        a1 += __shfl_xor_sync(0xffffffffu, a1, off);
        a2 += __shfl_xor_sync(0xffffffffu, a2, off);
      }
      if (lane == 0) {
        s_red[1][warp] = a1;
        s_red[2][warp] = a2;
      }
      __syncthreads();
      if (tid == 0) {
        double S1 = 0.0, S2 = 0.0;
        for (uint32_t w2 = 0; w2 < blockDim.x / 32; ++w2) {
          S1 += s_red[1][w2];
          S2 += s_red[2][w2];
        }
        const double ess = S1 * S1 / ((double)ip.islands * S2);   // NaN when every weight is zero
        s_stop = (ess >= (double)ip.theta) ? 1u : 0u;
      }
      __syncthreads();
      if (s_stop) break;
    }
    ++executed;
    const uint32_t lb = s - 1, b = 1u << lb;
    for (uint32_t q = tid; q < ip.islands / 2; q += blockDim.x) {
      const uint32_t i0 = ((q >> lb) << (lb + 1)) + (q & (b - 1));   // member 0: bit s-1 clear
      const uint32_t i1 = i0 + b;
      const float v0 = V[i0], v1 = V[i1];
      const float mx = fmaxf(v0, v1);
      float e0 = 0.0f, e1 = 0.0f;
      if (mx != -INFINITY) {
        e0 = exp_weight(v0 - mx);           // the larger weight is exactly 1
        e1 = exp_weight(v1 - mx);
      }
      const uint32_t q0 = __float2uint_rz(e0 * 16777216.0f);
      const uint32_t Q = q0 + __float2uint_rz(e1 * 16777216.0f);
      const uint4 w0 = philox4x32(make_uint4(i0 >> 2, n, kPurposeIsland, s), p.rk);
      const uint4 w1 = philox4x32(make_uint4(i1 >> 2, n, kPurposeIsland, s), p.rk);
      const uint32_t o0 = i0 & 3u, o1 = i1 & 3u;
      const uint32_t r0 = o0 == 0 ? w0.x : o0 == 1 ? w0.y : o0 == 2 ? w0.z : w0.w;
      const uint32_t r1 = o1 == 0 ? w1.x : o1 == 1 ? w1.y : o1 == 2 ? w1.z : w1.w;
      uint32_t c0 = 0, c1 = 1;              // an all-zero pair keeps its samples
      if (Q != 0) {
        c0 = (__umulhi(r0, Q) >= q0) ? 1u : 0u;   // #{j : P_j <= u}, P = (q0, Q)
        c1 = (__umulhi(r1, Q) >= q0) ? 1u : 0u;
      }
      if (!ip.plain && c0 == 1 && c1 == 0) {       // Algorithm 7: a pure swap is undone
        c0 = 0;
        c1 = 1;
      }
      const int32_t h0 = H[i0], h1 = H[i1];
      H[i0] = c0 ? h1 : h0;
      H[i1] = c1 ? h1 : h0;
      const float vn = (mx == -INFINITY) ? -INFINITY : mx + logf(e0 + e1) - log2f_;
      V[i0] = vn;
      V[i1] = vn;
    }
    __syncthreads();
  }
  for (uint32_t i = tid; i < ip.islands; i += blockDim.x) ip.src[i] = H[i];
  if (ip.adaptive) {        // carried weight of every particle = its island's weight
    for (uint32_t i = tid; i < ip.islands; i += blockDim.x) ip.lV_next[i] = V[i];
    if (tid == 0) p.st->nstages += executed;
  } else {
    for (uint32_t j = tid; j < ip.M; j += blockDim.x) ip.lV_next[j] = V[0];
  }
}

// Gather + mutation: particle (island i, place j) <- particle (src[i], j).
template <int D, int KIND>
__global__ void __launch_bounds__(kBlock) island_gather_kernel(const __grid_constant__ StepParams p,
                                                               const __grid_constant__ IslandParams ip) {
  DevState* st = p.st;
  const ModelParams& mp = p.model;
  const uint32_t n = st->n;
  const uint32_t N = p.N, M = ip.M;
  const float* __restrict__ X = p.x;
  float* __restrict__ Y = ip.x_out;
  if (M % 4 == 0) {                         // quads of particles inside one island
    for (uint32_t q = blockIdx.x * kBlock + threadIdx.x; q < N / 4; q += gridDim.x * kBlock) {
      const uint32_t i = 4 * q;
      const uint32_t isl = i / M;
      const uint32_t sp = (uint32_t)ip.src[isl] * M + (i - isl * M);
      float xh[4][D], z[4 * D], xo[D];
#pragma unroll
      for (int t = 0; t < D; ++t) {
        const float4 v = __ldg(reinterpret_cast<const float4*>(X + (size_t)t * N + sp));
        xh[0][t] = v.x; xh[1][t] = v.y; xh[2][t] = v.z; xh[3][t] = v.w;
      }
#pragma unroll
      for (int b = 0; b < D; ++b) {          // normals nu = i d + t, blocks of 4
        const uint4 w = philox4x32(make_uint4(q * D + b, n, kPurposePropagate, 0), p.rk);
        normals4_fast(w, z + 4 * b);
      }
      float out[D][4];
#pragma unroll
      for (int e = 0; e < 4; ++e) {
        mutate<D, KIND>(mp, xh[e], z + e * D, xo);
#pragma unroll
        for (int t = 0; t < D; ++t) out[t][e] = xo[t];
      }
#pragma unroll
      for (int t = 0; t < D; ++t)
        __stcs(reinterpret_cast<float4*>(Y + (size_t)t * N + i), make_float4(out[t][0], out[t][1], out[t][2], out[t][3]));
    }
  } else {
    for (uint32_t i = blockIdx.x * kBlock + threadIdx.x; i < N; i += gridDim.x * kBlock) {
      const uint32_t isl = i / M;
      const uint32_t sp = (uint32_t)ip.src[isl] * M + (i - isl * M);
      float xh[D], z[D], xo[D];
#pragma unroll
      for (int t = 0; t < D; ++t) {
        xh[t] = __ldg(X + (size_t)t * N + sp);
        const uint32_t nu = i * D + t;
        const uint4 w = philox4x32(make_uint4(nu >> 2, n, kPurposePropagate, 0), p.rk);
        float zz[4];
        normals4_fast(w, zz);
        z[t] = zz[nu & 3u];
      }
      mutate<D, KIND>(mp, xh, z, xo);
#pragma unroll
      for (int t = 0; t < D; ++t) __stcs(Y + (size_t)t * N + i, xo[t]);
    }
  }
  if (last_block_done(st)) {
    st->stage = 0;
    st->done = 0;
    __threadfence();
    st->n = n + 1;
  }
}

template <int D, int KIND>
static void island_pick(IslandKernels& ik) {
  ik.stages = reinterpret_cast<const void*>(&island_stages_kernel);
  ik.gather = reinterpret_cast<const void*>(&island_gather_kernel<D, KIND>);
}

bool select_island_kernels(int d, int kind, IslandKernels& ik) {
  if (kind == kStochVol) {
    if (d != 1) return false;
    island_pick<1, kStochVol>(ik);
    return true;
  }
  if (kind != kLinearGaussian) return false;
  switch (d) {
    case 1: island_pick<1, kLinearGaussian>(ik); return true;
    case 2: island_pick<2, kLinearGaussian>(ik); return true;
    case 3: island_pick<3, kLinearGaussian>(ik); return true;
    case 4: island_pick<4, kLinearGaussian>(ik); return true;
    case 5: island_pick<5, kLinearGaussian>(ik); return true;
    case 6: island_pick<6, kLinearGaussian>(ik); return true;
    case 7: island_pick<7, kLinearGaussian>(ik); return true;
    case 8: island_pick<8, kLinearGaussian>(ik); return true;
    default: return false;
  }
}

}  // namespace bfpf
