// step_butterfly.cu - one time step of the butterfly-interaction bootstrap
// particle filter as a single persistent kernel.
//
// Paper: Heine, Whiteley & Cemgil, arXiv 1812.01502.  Time step n runs the
// loop body of Algorithm 1 with Resample replaced by ONE stage of Algorithm 3
// on digit k = n mod m of the mixed-radix particle index:
//   weight     lw_i = log V_i + log g_n(zeta_i) - mu          (Algorithm 3, V_0 = g)
//   stage      V'_G = a_k^-1 sum_{j in G} V_j                 (eq. (V_defn_proofs))
//   resample   xi_i ~ sum_{j in G(i)} V_j delta_{zeta_j} / sum V_j   (integer rule)
//   mutate     zeta'_i ~ f(xi_i, .)                            (Algorithm 1)
// A group G = the a_k particles sharing every digit except k lies inside one
// tile, so the "exchange" of Section 1.2 is a gather from shared memory.
//
// Tile: nh blocks of the digits above k  x  a_k rows  x  nl columns of the
// digits below k.  Tile position p = row*nl + col, row = hh*a_k + r; global
// index i = base + row*s_k + col.  Each row is a contiguous run of nl states.
//
// This is the general kernel (any radix up to 1024, mixed radices that are
// not powers of two); step_group.cuh holds the faster register-resident
// kernel used for power-of-two radices up to 32.
//
// Integer resampling rule (shared specification with the oracle):
//   delta = fp32(lw - max_G lw), e = exp(delta) (FP32), q = floor(e 2^B)
//   (B = 24, or 32 for groups > 256), P = inclusive prefix over the group,
//   u = floor(r Q / 2^32) (or r Q / 2^64), ancestor = #{j : P_j <= u}.
// Random words are numbered group-major (pi = g a + r, see bfpf_device.cuh).
#include <cfloat>
#include <type_traits>

#include "bfpf_device.cuh"
#include "bfpf_epilogue.cuh"
#include "bfpf_kernels.h"
#include "bfpf_model.cuh"
#include "step_tile.cuh"

namespace bfpf {

// Initial particles zeta_0 ~ pi_0 (Algorithm 1, first loop).
template <int D, int KIND>
__global__ void __launch_bounds__(kBlock) init_particles_kernel(const __grid_constant__ StepParams p) {
  const ModelParams& mp = p.model;
  for (uint32_t i = blockIdx.x * kBlock + threadIdx.x; i < p.N; i += gridDim.x * kBlock) {
    float z[D];
#pragma unroll
    for (int t = 0; t < D; ++t) {
      const uint32_t nu = i * D + t;
      const uint4 w = philox4x32(make_uint4(nu >> 2, 0, kPurposeInit, 0), p.rk);
      float zz[4];
      normals4(w, zz);
      z[t] = zz[nu & 3u];
    }
#pragma unroll
    for (int t = 0; t < D; ++t) {
      float v;
      if constexpr (KIND == kStochVol) {
        v = mp.sd0 * z[0];
      } else {
        v = mp.m0[t];
#pragma unroll
        for (int u = 0; u <= t; ++u) v = fmaf(mp.L0[t * kMaxDim + u], z[u], v);
      }
      p.x[(size_t)t * p.N + i] = v;
    }
  }
}

__global__ void philox_blocks_kernel(uint32_t k0, uint32_t k1, uint4 c, uint32_t count, uint32_t* out) {
  for (uint32_t j = blockIdx.x * kBlock + threadIdx.x; j < count; j += gridDim.x * kBlock) {
    const uint4 w = philox4x32(make_uint4(c.x + j, c.y, c.z, c.w), k0, k1);
    reinterpret_cast<uint4*>(out)[j] = w;
  }
}

// ---------------------------------------------------------------------------
// Host-side dispatch
// ---------------------------------------------------------------------------
template <int D, int KIND, bool WIDE>
static void fill_step(KernelSet& ks) {
  ks.step = reinterpret_cast<const void*>(&step_butterfly_kernel<D, KIND, WIDE, false>);
  ks.step_staged = select_staged_tile_kernel(D, KIND, WIDE);
  ks.init = reinterpret_cast<const void*>(&init_particles_kernel<D, KIND>);
}

bool select_kernels(int d, int kind, bool wide, KernelSet& ks) {
#define BFPF_CASE(DD)                                         \
  case DD:                                                    \
    if (wide) fill_step<DD, kLinearGaussian, true>(ks);       \
    else fill_step<DD, kLinearGaussian, false>(ks);           \
    return true;
  if (kind == kStochVol) {
    if (d != 1) return false;
    if (wide) fill_step<1, kStochVol, true>(ks);
    else fill_step<1, kStochVol, false>(ks);
    return true;
  }
  switch (d) {
    BFPF_CASE(1)
    BFPF_CASE(2)
    BFPF_CASE(3)
    BFPF_CASE(4)
    BFPF_CASE(5)
    BFPF_CASE(6)
    BFPF_CASE(7)
    BFPF_CASE(8)
    default:
      return false;
  }
#undef BFPF_CASE
}

const void* select_group_kernel(int d, int kind, int a, int* G, bool staged, bool adapt, bool small) {
  switch (d) {
    case 1: return group_kernel_d1(kind, a, G, staged, adapt, small);
    case 2: return group_kernel_d2(kind, a, G, staged, adapt, small);
    case 3: return group_kernel_d3(kind, a, G, staged, adapt, small);
    case 4: return group_kernel_d4(kind, a, G, staged, adapt, small);
    case 5: return group_kernel_d5(kind, a, G, staged, adapt, small);
    case 6: return group_kernel_d6(kind, a, G, staged, adapt, small);
    case 7: return group_kernel_d7(kind, a, G, staged, adapt, small);
    case 8: return group_kernel_d8(kind, a, G, staged, adapt, small);
    default: return nullptr;
  }
}

const void* select_pass_kernel(int d, int kind, int a) {
  if (d == 1) return pass_kernel_d1(kind, a);
  if (d >= 2 && d <= 4) return pass_kernel_d2_4(d, kind, a);
  if (d >= 5 && d <= 8) return pass_kernel_d5_8(d, kind, a);
  return nullptr;
}

cudaError_t launch_philox_blocks(uint64_t seed, uint4 c, uint32_t count, uint32_t* out, cudaStream_t stream) {
  const uint32_t blocks = (count + kBlock - 1) / kBlock;
  philox_blocks_kernel<<<blocks ? (blocks > 4096 ? 4096 : blocks) : 1, kBlock, 0, stream>>>(
      (uint32_t)seed, (uint32_t)(seed >> 32), c, count, out);
  return cudaGetLastError();
}

}  // namespace bfpf
