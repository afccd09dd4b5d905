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

namespace bfpf {

namespace {

__device__ __forceinline__ unsigned long long mulhi64(unsigned long long a, unsigned long long b) {
  return __umul64hi(a, b);
}

}  // namespace

template <int D, int KIND, bool WIDE>
__global__ void __launch_bounds__(kBlock) step_butterfly_kernel(const __grid_constant__ StepParams p) {
  using PT = typename std::conditional<WIDE, unsigned long long, uint32_t>::type;
  extern __shared__ __align__(16) unsigned char smem_raw[];

  const uint32_t tid = threadIdx.x;
  const uint32_t cap = p.tile_cap;
  float* s_x = reinterpret_cast<float*>(smem_raw);
  float* s_lw = s_x + D * cap;
  PT* s_P = reinterpret_cast<PT*>(s_lw + cap);

  const ModelParams& mp = p.model;
  DevState* st = p.st;
  const uint32_t n = st->n;
  const uint32_t k = n % (uint32_t)p.m;
  const DigitGeom& g = p.geom[k];
  const uint32_t a = g.a, s = g.s, nl = g.nl, tn = g.tile_n;
  const bool wide_digit = g.wide != 0;
  const float* __restrict__ lV_in = p.lV[n & 1u];
  float* __restrict__ lV_out = p.lV[(n & 1u) ^ 1u];
  const float muf = st->mu_f;
  const uint32_t N = p.N;
  float y[kMaxDim];
#pragma unroll
  for (int j = 0; j < kMaxDim; ++j) y[j] = (j < mp.dy) ? p.y_ring[(n % kRing) * mp.dy + j] : 0.0f;
  uint32_t status = 0;
  const uint32_t ngroups = g.nh * nl;   // groups per tile

  // lifting steps of the ancestor search: largest power of two < a (0 if a == 1)
  uint32_t step0 = 1;
  while ((step0 << 1) < a) step0 <<= 1;
  if (a == 1) step0 = 0;

  Partial acc{-INFINITY, 0.0f, 0.0f};
  float accx[D];
#pragma unroll
  for (int t = 0; t < D; ++t) accx[t] = 0.0f;

  for (uint32_t tile = blockIdx.x; tile < g.ntiles; tile += gridDim.x) {
    const uint32_t th = fdiv(tile, g.div_tiles_l);
    const uint32_t tl = tile - th * g.tiles_l;
    const uint32_t h0 = th * g.nh, l0 = tl * nl;
    const uint32_t base = h0 * a * s + l0;

    __syncthreads();  // the previous tile's readers are done with shared memory

    // ---- load the tile's states (coalesced rows) ----
    if (g.quad) {
      for (uint32_t q = tid; q < (tn >> 2); q += kBlock) {
        const uint32_t pos = q << 2;
        const uint32_t row = fdiv(pos, g.div_nl);
        const uint32_t i = base + row * s + (pos - row * nl);
#pragma unroll
        for (int t = 0; t < D; ++t) {
          const float4 v = __ldcs(reinterpret_cast<const float4*>(p.x + (size_t)t * N + i));
          *reinterpret_cast<float4*>(s_x + t * cap + pos) = v;
        }
      }
    } else {
      for (uint32_t pos = tid; pos < tn; pos += kBlock) {
        const uint32_t row = fdiv(pos, g.div_nl);
        const uint32_t i = base + row * s + (pos - row * nl);
#pragma unroll
        for (int t = 0; t < D; ++t) s_x[t * cap + pos] = __ldcs(p.x + (size_t)t * N + i);
      }
    }
    __syncthreads();

    // ---- weights: lw = lV(group of the previous digit) + log g_n(x) - mu ----
    for (uint32_t pos = tid; pos < tn; pos += kBlock) {
      const uint32_t row = fdiv(pos, g.div_nl);
      const uint32_t i = base + row * s + (pos - row * nl);
      const uint32_t hp = fdiv(i, g.div_prev_as);
      const uint32_t lo = i - fdiv(i, g.div_prev_s) * g.prev_s;
      const float lv = __ldg(lV_in + hp * g.prev_s + lo);
      float xv[D];
#pragma unroll
      for (int t = 0; t < D; ++t) xv[t] = s_x[t * cap + pos];
      s_lw[pos] = sanitize_logweight(lv + obs_log_term<D, KIND>(mp, y, xv) - muf, status);
    }
    __syncthreads();

    // ---- per group: max, log-sum-exp, integer weights and prefix sums ----
    for (uint32_t gid = tid; gid < ngroups; gid += kBlock) {
      const uint32_t hh = fdiv(gid, g.div_nl);
      const uint32_t col = gid - hh * nl;
      const uint32_t p0 = hh * a * nl + col;
      float M = -INFINITY;
      for (uint32_t r = 0; r < a; ++r) M = fmaxf(M, s_lw[p0 + r * nl]);
      float s1 = 0.0f, s2 = 0.0f, sx[D];
#pragma unroll
      for (int t = 0; t < D; ++t) sx[t] = 0.0f;
      float L;
      if (M == -INFINITY) {
        for (uint32_t r = 0; r < a; ++r) s_P[p0 + r * nl] = 0;
        status |= kStatusZeroGroup;
        L = -INFINITY;
      } else {
        PT P = 0;
        for (uint32_t r = 0; r < a; ++r) {
          const uint32_t pos = p0 + r * nl;
          const float dl = s_lw[pos] - M;
          const float e = (dl == 0.0f) ? 1.0f : __expf(dl);
          s1 += e;
          s2 = fmaf(e, e, s2);
#pragma unroll
          for (int t = 0; t < D; ++t) sx[t] = fmaf(e, s_x[t * cap + pos], sx[t]);
          PT q;
          if (WIDE && wide_digit) q = (PT)__float2ull_rz(e * 4294967296.0f);
          else q = (PT)__float2uint_rz(e * 16777216.0f);
          P += q;
          s_P[pos] = P;
        }
        L = M + logf(s1);
      }
      lV_out[(h0 + hh) * s + l0 + col] = L - g.log_a;
      merge_partial<D>(acc, accx, M, s1, s2, sx);
    }
    __syncthreads();

    // ---- draw ancestors (group-major counters), gather, mutate, store ----
    // Work item = (member quad rq, group gid of the tile); consecutive threads
    // take consecutive groups, i.e. consecutive columns of a row.
    const uint32_t nq = (a + 3) >> 2;
    const bool a4 = (a & 3u) == 0;
    for (uint32_t it = tid; it < ngroups * nq; it += kBlock) {
      const uint32_t rq = fdiv(it, g.div_tgroups);
      const uint32_t gid = it - rq * ngroups;
      const uint32_t hh = fdiv(gid, g.div_nl);
      const uint32_t col = gid - hh * nl;
      const uint32_t gb = hh * a * nl + col;                 // tile position of member 0
      const uint32_t gc = (h0 + hh) * s + l0 + col;          // group index h*s + l
      const uint32_t ib = base + hh * a * s + col;           // global index of member 0
      const PT Q = s_P[gb + (a - 1) * nl];
      const uint32_t r0 = rq << 2;
      const uint32_t pi0 = gc * a + r0;
      uint32_t rw[4] = {0u, 0u, 0u, 0u};
      unsigned long long rw64[4] = {0ull, 0ull, 0ull, 0ull};
      float z[4 * D];
      if (a4) {   // pi0 % 4 == 0: whole counter blocks
        if (WIDE && wide_digit) {
          const uint4 w0 = philox4x32_10(make_uint4(pi0 >> 1, n, kPurposeResampleWide, 0), p.rk);
          const uint4 w1 = philox4x32_10(make_uint4((pi0 >> 1) + 1, n, kPurposeResampleWide, 0), p.rk);
          rw64[0] = ((unsigned long long)w0.y << 32) | w0.x;
          rw64[1] = ((unsigned long long)w0.w << 32) | w0.z;
          rw64[2] = ((unsigned long long)w1.y << 32) | w1.x;
          rw64[3] = ((unsigned long long)w1.w << 32) | w1.z;
        } else {
          const uint4 w = philox4x32_10(make_uint4(pi0 >> 2, n, kPurposeResample, 0), p.rk);
          rw[0] = w.x; rw[1] = w.y; rw[2] = w.z; rw[3] = w.w;
        }
#pragma unroll
        for (int b = 0; b < D; ++b) {
          const uint4 w = philox4x32_10(make_uint4((pi0 >> 2) * D + b, n, kPurposePropagate, 0), p.rk);
          normals4(w, z + 4 * b);
        }
      } else {    // members straddle counter blocks: one block per draw / normal
#pragma unroll
        for (int jj = 0; jj < 4; ++jj) {
          const uint32_t pi = pi0 + jj;
          if (r0 + jj >= a) break;
          if (WIDE && wide_digit) {
            const uint4 w = philox4x32_10(make_uint4(pi >> 1, n, kPurposeResampleWide, 0), p.rk);
            rw64[jj] = (pi & 1u) ? (((unsigned long long)w.w << 32) | w.z) : (((unsigned long long)w.y << 32) | w.x);
          } else {
            const uint4 w = philox4x32_10(make_uint4(pi >> 2, n, kPurposeResample, 0), p.rk);
            const uint32_t sel = pi & 3u;
            rw[jj] = sel == 0 ? w.x : sel == 1 ? w.y : sel == 2 ? w.z : w.w;
          }
#pragma unroll
          for (int t = 0; t < D; ++t) {
            const uint32_t nu = pi * D + t;
            const uint4 w = philox4x32_10(make_uint4(nu >> 2, n, kPurposePropagate, 0), p.rk);
            float zz[4];
            normals4(w, zz);
            z[jj * D + t] = zz[nu & 3u];
          }
        }
      }
#pragma unroll
      for (int jj = 0; jj < 4; ++jj) {
        const uint32_t r = r0 + jj;
        if (r >= a) break;
        PT u;
        if (WIDE && wide_digit) u = (PT)mulhi64(rw64[jj], (unsigned long long)Q);
        else u = (PT)(((unsigned long long)rw[jj] * Q) >> 32);
        uint32_t c = 0;
        for (uint32_t stp = step0; stp; stp >>= 1) {
          const uint32_t cand = c + stp;
          if (cand <= a - 1 && s_P[gb + (cand - 1) * nl] <= u) c = cand;
        }
        if (Q == 0) c = r;
        const uint32_t pa = gb + c * nl;
        float xh[D], xo[D];
#pragma unroll
        for (int t = 0; t < D; ++t) xh[t] = s_x[t * cap + pa];
        mutate<D, KIND>(mp, xh, z + jj * D, xo);
        const uint32_t i = ib + r * s;
#pragma unroll
        for (int t = 0; t < D; ++t) __stcs(p.x + (size_t)t * N + i, xo[t]);
        if (p.anc) p.anc[i] = (int32_t)(ib + c * s);
      }
    }
  }

  finish_step<D>(p, acc, accx, n, status, muf);
}

// Initial particles zeta_0 ~ pi_0 (Algorithm 1, first loop).
template <int D, int KIND>
__global__ void __launch_bounds__(kBlock) init_particles_kernel(const __grid_constant__ StepParams p) {
  const ModelParams& mp = p.model;
  for (uint32_t i = blockIdx.x * kBlock + threadIdx.x; i < p.N; i += gridDim.x * kBlock) {
    float z[D];
#pragma unroll
    for (int t = 0; t < D; ++t) {
      const uint32_t nu = i * D + t;
      const uint4 w = philox4x32_10(make_uint4(nu >> 2, 0, kPurposeInit, 0), p.rk);
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
    const uint4 w = philox4x32_10(make_uint4(c.x + j, c.y, c.z, c.w), k0, k1);
    reinterpret_cast<uint4*>(out)[j] = w;
  }
}

// ---------------------------------------------------------------------------
// Host-side dispatch
// ---------------------------------------------------------------------------
template <int D, int KIND, bool WIDE>
static void fill_step(KernelSet& ks) {
  ks.step = reinterpret_cast<const void*>(&step_butterfly_kernel<D, KIND, WIDE>);
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

const void* select_group_kernel(int d, int kind, int a, int* G) {
  switch (d) {
    case 1: return group_kernel_d1(kind, a, G);
    case 2: return group_kernel_d2(kind, a, G);
    case 3: return group_kernel_d3(kind, a, G);
    case 4: return group_kernel_d4(kind, a, G);
    case 5: return group_kernel_d5(kind, a, G);
    case 6: return group_kernel_d6(kind, a, G);
    case 7: return group_kernel_d7(kind, a, G);
    case 8: return group_kernel_d8(kind, a, G);
    default: return nullptr;
  }
}

cudaError_t launch_philox_blocks(uint64_t seed, uint4 c, uint32_t count, uint32_t* out, cudaStream_t stream) {
  const uint32_t blocks = (count + kBlock - 1) / kBlock;
  philox_blocks_kernel<<<blocks ? (blocks > 4096 ? 4096 : blocks) : 1, kBlock, 0, stream>>>(
      (uint32_t)seed, (uint32_t)(seed >> 32), c, count, out);
  return cudaGetLastError();
}

}  // namespace bfpf
