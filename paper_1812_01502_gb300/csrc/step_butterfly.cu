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
// Integer resampling rule (shared specification with the oracle):
//   delta = fp32(lw - max_G lw), e = exp(delta) (FP32), q = floor(e 2^B)
//   (B = 24, or 32 for groups > 256), P = inclusive prefix over the group,
//   u = floor(r Q / 2^32) (or r Q / 2^64), ancestor = #{j : P_j <= u}.
#include <cfloat>
#include <type_traits>

#include "bfpf_device.cuh"
#include "bfpf_kernels.h"

namespace bfpf {

namespace {

template <int D, int KIND>
__device__ __forceinline__ float obs_log_term(const ModelParams& mp, const float* y, const float* x) {
  if constexpr (KIND == kStochVol) {
    // log g - c = -x/2 - y^2 exp(-x) / (2 beta^2)
    return fmaf(-0.5f, x[0], -(y[0] * y[0]) * __expf(-x[0]) * mp.inv2b2);
  } else {
    // log g - c = -1/2 || Lr^{-1} (y - H x) ||^2
    float r[kMaxDim];
#pragma unroll
    for (int j = 0; j < kMaxDim; ++j) {
      if (j < mp.dy) {
        float acc = y[j];
        if (mp.flags & kHIdentity) {          // H is the identity
          acc -= (j < D) ? x[j] : 0.0f;
        } else {
#pragma unroll
          for (int t = 0; t < D; ++t) acc = fmaf(-mp.H[j * kMaxDim + t], x[t], acc);
        }
        r[j] = acc;
      }
    }
    float ss = 0.0f;
    if (mp.flags & kLrDiagonal) {              // Lr diagonal
#pragma unroll
      for (int j = 0; j < kMaxDim; ++j)
        if (j < mp.dy) {
          const float z = mp.Lri[j * kMaxDim + j] * r[j];
          ss = fmaf(z, z, ss);
        }
    } else {
#pragma unroll
      for (int j = 0; j < kMaxDim; ++j)
        if (j < mp.dy) {
          float z = 0.0f;
#pragma unroll
          for (int u = 0; u <= j; ++u) z = fmaf(mp.Lri[j * kMaxDim + u], r[u], z);
          ss = fmaf(z, z, ss);
        }
    }
    return -0.5f * ss;
  }
}

// zeta' = A xhat + Lq z  (linear-Gaussian)  or  phi xhat + sigma z  (SV)
template <int D, int KIND>
__device__ __forceinline__ void mutate(const ModelParams& mp, const float* xh, const float* z, float* out) {
  if constexpr (KIND == kStochVol) {
    out[0] = fmaf(mp.phi, xh[0], mp.sigma * z[0]);
  } else {
#pragma unroll
    for (int t = 0; t < D; ++t) {
      float acc = 0.0f;
      if (mp.flags & kADiagonal) {            // A diagonal
        acc = mp.A[t * kMaxDim + t] * xh[t];
      } else {
#pragma unroll
        for (int u = 0; u < D; ++u) acc = fmaf(mp.A[t * kMaxDim + u], xh[u], acc);
      }
      if (mp.flags & kLqDiagonal) {            // Lq diagonal
        acc = fmaf(mp.Lq[t * kMaxDim + t], z[t], acc);
      } else {
#pragma unroll
        for (int u = 0; u <= t; ++u) acc = fmaf(mp.Lq[t * kMaxDim + u], z[u], acc);
      }
      out[t] = acc;
    }
  }
}

struct Partial {
  float m, s1, s2;
};

// Merge a group's (max, sums) into the running block partial, rescaling to the larger max.
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

__device__ __forceinline__ unsigned long long mulhi64(unsigned long long a, unsigned long long b) {
  return __umul64hi(a, b);
}

}  // namespace

template <int D, int KIND, bool WIDE>
__global__ void __launch_bounds__(kBlock) step_butterfly_kernel(const __grid_constant__ StepParams p) {
  using PT = typename std::conditional<WIDE, unsigned long long, uint32_t>::type;
  constexpr int NP = 3 + D;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ float s_red[kBlock / 32][NP];
  __shared__ float s_redlo[kBlock / 32][NP];
  __shared__ uint32_t s_last;

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
      float lw = lv + obs_log_term<D, KIND>(mp, y, xv) - muf;
      if (lw != lw || lw == INFINITY) {
        lw = -INFINITY;
        status |= kStatusNonFinite;
      }
      s_lw[pos] = lw;
    }
    __syncthreads();

    // ---- per group: max, log-sum-exp, integer weights and prefix sums ----
    const uint32_t ngroups = g.nh * nl;
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

    // ---- draw ancestors, gather from shared memory, mutate, store ----
    const uint32_t key0 = p.seed_lo, key1 = p.seed_hi;
    if (g.quad) {
      for (uint32_t q = tid; q < (tn >> 2); q += kBlock) {
        const uint32_t pos0 = q << 2;
        const uint32_t row0 = fdiv(pos0, g.div_nl);
        const uint32_t i0 = base + row0 * s + (pos0 - row0 * nl);
        uint32_t rw[4] = {0u, 0u, 0u, 0u};
        unsigned long long rw64[4] = {0ull, 0ull, 0ull, 0ull};
        if (WIDE && wide_digit) {
          const uint4 w0 = philox4x32_10(make_uint4(i0 >> 1, n, kPurposeResampleWide, 0), key0, key1);
          const uint4 w1 = philox4x32_10(make_uint4((i0 >> 1) + 1, n, kPurposeResampleWide, 0), key0, key1);
          rw64[0] = ((unsigned long long)w0.y << 32) | w0.x;
          rw64[1] = ((unsigned long long)w0.w << 32) | w0.z;
          rw64[2] = ((unsigned long long)w1.y << 32) | w1.x;
          rw64[3] = ((unsigned long long)w1.w << 32) | w1.z;
        } else {
          const uint4 w = philox4x32_10(make_uint4(i0 >> 2, n, kPurposeResample, 0), key0, key1);
          rw[0] = w.x; rw[1] = w.y; rw[2] = w.z; rw[3] = w.w;
        }
        float z[4 * D];
#pragma unroll
        for (int b = 0; b < D; ++b) {
          const uint4 w = philox4x32_10(make_uint4((i0 >> 2) * D + b, n, kPurposePropagate, 0), key0, key1);
          normals4(w, z + 4 * b);
        }
        float outv[D][4];
#pragma unroll
        for (int j = 0; j < 4; ++j) {
          const uint32_t pos = pos0 + j;
          const uint32_t row = fdiv(pos, g.div_nl);
          const uint32_t col = pos - row * nl;
          const uint32_t hh = fdiv(row, g.div_a);
          const uint32_t r = row - hh * a;
          const uint32_t gb = hh * a * nl + col;
          const PT Q = s_P[gb + (a - 1) * nl];
          PT u;
          if (WIDE && wide_digit) u = (PT)mulhi64(rw64[j], (unsigned long long)Q);
          else u = (PT)(((unsigned long long)rw[j] * Q) >> 32);
          uint32_t c = 0;
          for (uint32_t stp = step0; stp; stp >>= 1) {
            const uint32_t cand = c + stp;
            if (cand <= a - 1 && s_P[gb + (cand - 1) * nl] <= u) c = cand;
          }
          if (Q == 0) c = r;
          const uint32_t pa = gb + c * nl;
          float xh[D];
#pragma unroll
          for (int t = 0; t < D; ++t) xh[t] = s_x[t * cap + pa];
          float xo[D];
          mutate<D, KIND>(mp, xh, z + j * D, xo);
#pragma unroll
          for (int t = 0; t < D; ++t) outv[t][j] = xo[t];
          if (p.anc) p.anc[i0 + j] = (int32_t)(i0 + j + (c - r) * s);
        }
#pragma unroll
        for (int t = 0; t < D; ++t)
          __stcs(reinterpret_cast<float4*>(p.x + (size_t)t * N + i0),
                 make_float4(outv[t][0], outv[t][1], outv[t][2], outv[t][3]));
      }
    } else {
      for (uint32_t pos = tid; pos < tn; pos += kBlock) {
        const uint32_t row = fdiv(pos, g.div_nl);
        const uint32_t col = pos - row * nl;
        const uint32_t i = base + row * s + col;
        const uint32_t hh = fdiv(row, g.div_a);
        const uint32_t r = row - hh * a;
        const uint32_t gb = hh * a * nl + col;
        const PT Q = s_P[gb + (a - 1) * nl];
        PT u;
        if (WIDE && wide_digit) {
          const uint4 w = philox4x32_10(make_uint4(i >> 1, n, kPurposeResampleWide, 0), key0, key1);
          const unsigned long long r64 = (i & 1u) ? (((unsigned long long)w.w << 32) | w.z)
                                                  : (((unsigned long long)w.y << 32) | w.x);
          u = (PT)mulhi64(r64, (unsigned long long)Q);
        } else {
          const uint4 w = philox4x32_10(make_uint4(i >> 2, n, kPurposeResample, 0), key0, key1);
          const uint32_t sel = i & 3u;
          const uint32_t rr = sel == 0 ? w.x : sel == 1 ? w.y : sel == 2 ? w.z : w.w;
          u = (PT)(((unsigned long long)rr * Q) >> 32);
        }
        uint32_t c = 0;
        for (uint32_t stp = step0; stp; stp >>= 1) {
          const uint32_t cand = c + stp;
          if (cand <= a - 1 && s_P[gb + (cand - 1) * nl] <= u) c = cand;
        }
        if (Q == 0) c = r;
        const uint32_t pa = gb + c * nl;
        float xh[D], z[D], xo[D];
#pragma unroll
        for (int t = 0; t < D; ++t) {
          xh[t] = s_x[t * cap + pa];
          const uint32_t nu = i * D + t;
          const uint4 w = philox4x32_10(make_uint4(nu >> 2, n, kPurposePropagate, 0), key0, key1);
          float zz[4];
          normals4(w, zz);
          z[t] = zz[nu & 3u];
        }
        mutate<D, KIND>(mp, xh, z, xo);
#pragma unroll
        for (int t = 0; t < D; ++t) __stcs(p.x + (size_t)t * N + i, xo[t]);
        if (p.anc) p.anc[i] = (int32_t)(i + (c - r) * s);
      }
    }
  }

  // ---- block partial -> global; the last block finishes the step ----
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
    for (int w = 0; w < kBlock / 32; ++w) merge_partial<D>(b, bx, s_red[w][0], s_red[w][1], s_red[w][2], &s_red[w][3]);
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
  if (!s_last) return;
  __threadfence();

  // Last block: combine all block partials in a fixed order with compensated
  // FP32 sums, then finish in FP64.
  const uint32_t G = gridDim.x;
  float Mx = -INFINITY;
  for (uint32_t b = tid; b < G; b += kBlock) Mx = fmaxf(Mx, __ldcg(p.partials + (size_t)b * NP));
#pragma unroll
  for (int off = 16; off; off >>= 1) Mx = fmaxf(Mx, __shfl_xor_sync(0xffffffffu, Mx, off));
  if (lane == 0) s_red[warp][0] = Mx;
  __syncthreads();
  Mx = s_red[0][0];
  for (int w = 1; w < kBlock / 32; ++w) Mx = fmaxf(Mx, s_red[w][0]);
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
  if (tid == 0) {
    double S[NP - 1];
    for (int v = 0; v < NP - 1; ++v) {
      float h = 0.0f, l = 0.0f;
      for (int w = 0; w < kBlock / 32; ++w) {
        ff_add(h, l, s_red[w][v]);
        l += s_redlo[w][v];
      }
      S[v] = (double)h + (double)l;
    }
    const uint32_t slot = n % kRing;
    double lme, inc, ess;
    if (Mx == -INFINITY || !(S[0] > 0.0)) {
      lme = -INFINITY;
      inc = -INFINITY;
      ess = 0.0;
    } else {
      lme = (double)Mx + log(S[0] * (double)p.inv_N);
      inc = lme + ((double)muf - st->mu) + mp.c_obs;
      ess = S[0] * S[0] / ((double)N * S[1]);
    }
    p.inc_ring[slot] = inc;
    p.ess_ring[slot] = (float)ess;
    for (int t = 0; t < D; ++t) p.mean_ring[slot * mp.d + t] = (float)(S[2 + t] / S[0]);
    st->loglik += inc;
    st->mu = lme;
    st->mu_f = (float)lme;
    st->done = 0;
    __threadfence();
    st->n = n + 1;
  }
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
      const uint4 w = philox4x32_10(make_uint4(nu >> 2, 0, kPurposeInit, 0), p.seed_lo, p.seed_hi);
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

cudaError_t launch_philox_blocks(uint64_t seed, uint4 c, uint32_t count, uint32_t* out, cudaStream_t stream) {
  const uint32_t blocks = (count + kBlock - 1) / kBlock;
  philox_blocks_kernel<<<blocks ? (blocks > 4096 ? 4096 : blocks) : 1, kBlock, 0, stream>>>(
      (uint32_t)seed, (uint32_t)(seed >> 32), c, count, out);
  return cudaGetLastError();
}

}  // namespace bfpf
