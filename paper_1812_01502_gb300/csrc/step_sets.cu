// step_sets.cu - Algorithm 3 with the paper's own stage matrices (eq. (A
// matrices) of Heine, Whiteley & Cemgil, arXiv 1812.01502): stage s = 1..S of
// a time step resamples within the groups of the digit SET {0, s} -- the
// a_0 a_s particles that share every digit except digits 0 and s (with radices
// (M, 2, ..., 2): the M particles of a PE and of its partner PE across bit
// s - 1).  Stage 1 weights with g_n, stage S mutates; the stage counter in the
// device state picks the stage.
//
// Tile: nh upper blocks x a_s rows x nl columns, nl a multiple of w = a_0;
// group (hh, cg) of a tile = rows 0..a_s-1 x columns cg w .. cg w + w - 1;
// member rho = r_s w + r_0 (digit s major, digit 0 minor) sits at tile
// position hh a_s nl + r_s nl + cg w + r_0.  Group index g = h (s_s / w) + l'
// (l' = digits 1..s-1), random words numbered pi = g a_0 a_s + rho.
#include <cfloat>
#include <type_traits>

#include "bfpf_device.cuh"
#include "bfpf_epilogue.cuh"
#include "bfpf_kernels.h"
#include "bfpf_model.cuh"
#include "step_tile.cuh"

namespace bfpf {

namespace {

template <int D, int KIND, bool WIDE>
__device__ __forceinline__ void set_tile_steps(const TileCtx& ctx, uint32_t first, uint32_t stride,
                                               unsigned char* smem_raw, Partial& acc, float* accx,
                                               uint32_t& status) {
  using PT = typename std::conditional<WIDE, unsigned long long, uint32_t>::type;
  const uint32_t tid = threadIdx.x;
  const uint32_t cap = ctx.cap;
  float* s_x = reinterpret_cast<float*>(smem_raw);
  float* s_lw = s_x + D * cap;
  PT* s_P = reinterpret_cast<PT*>(s_lw + cap);
  const ModelParams& mp = *ctx.mp;
  const RoundKeys& rk = *ctx.rk;
  const DigitGeom& g = *ctx.g;
  const uint32_t a = g.a, s = g.s, nl = g.nl, tn = g.tile_n, w = g.w;
  const uint32_t G = a * w;                 // members per group
  const uint32_t nlw = nl / w;              // groups per block of rows
  const uint32_t sw = s / w;
  const bool wide_digit = g.wide != 0;
  const float* __restrict__ lV_in = ctx.lV_in;
  float* __restrict__ lV_out = ctx.lV_out;
  float* __restrict__ X = ctx.x;
  const float muf = ctx.muf;
  const uint32_t N = ctx.N, n = ctx.n, t_st = ctx.t;
  const bool obs = ctx.obs, mut = ctx.mut;
  const float* y = ctx.y;
  const uint32_t ngroups = g.nh * nlw;
  uint32_t step0 = 1;                       // largest power of two < G
  while ((step0 << 1) < G) step0 <<= 1;
  // tile position of member rho of the group whose member 0 is at p0
  auto mpos = [&](uint32_t p0, uint32_t rho) -> uint32_t {
    const uint32_t rs = fdiv(rho, g.div_w);
    return p0 + rs * nl + (rho - rs * w);
  };

  for (uint32_t tile = first; tile < g.ntiles; tile += stride) {
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
          const float4 v = __ldcs(reinterpret_cast<const float4*>(X + (size_t)t * N + i));
          *reinterpret_cast<float4*>(s_x + t * cap + pos) = v;
        }
      }
    } else {
      for (uint32_t pos = tid; pos < tn; pos += kBlock) {
        const uint32_t row = fdiv(pos, g.div_nl);
        const uint32_t i = base + row * s + (pos - row * nl);
#pragma unroll
        for (int t = 0; t < D; ++t) s_x[t * cap + pos] = __ldcs(X + (size_t)t * N + i);
      }
    }
    __syncthreads();

    // ---- weights: lw = lV(group of the previous set) + log g_n(x) - mu ----
    for (uint32_t pos = tid; pos < tn; pos += kBlock) {
      const uint32_t row = fdiv(pos, g.div_nl);
      const uint32_t i = base + row * s + (pos - row * nl);
      const uint32_t hp = fdiv(i, g.div_prev_as);
      const uint32_t lo = i - fdiv(i, g.div_prev_s) * g.prev_s;
      const float lv = __ldg(lV_in + hp * g.prev_sw + fdiv(lo, g.div_w));
      float xv[D];
#pragma unroll
      for (int t = 0; t < D; ++t) xv[t] = s_x[t * cap + pos];
      s_lw[pos] = sanitize_logweight(obs ? lv + obs_log_term<D, KIND>(mp, y, xv) - muf : lv, status);
    }
    __syncthreads();

    // ---- per group: max, log-sum-exp, integer weights and prefix sums ----
    // (a team of T lanes per group, as in tile_steps; members rho in order)
    {
      const uint32_t T = g.team, lt = tid & (T - 1u);
      const uint32_t tpb = kBlock / T;
      const uint32_t C = (G + T - 1u) / T;
      const uint32_t rb = min(G, lt * C), re = min(G, rb + C);
      const uint32_t rounds = (ngroups + tpb - 1u) / tpb;
      for (uint32_t rd = 0; rd < rounds; ++rd) {
        const uint32_t gid = rd * tpb + tid / T;
        const bool active = gid < ngroups;
        uint32_t hh = 0, cg = 0;
        if (active) {
          hh = fdiv(gid, g.div_nlw);
          cg = gid - hh * nlw;
        }
        const uint32_t p0 = hh * a * nl + cg * w;
        float M = -INFINITY;
        if (active)
          for (uint32_t rho = rb; rho < re; ++rho) M = fmaxf(M, s_lw[mpos(p0, rho)]);
        for (uint32_t off = 1; off < T; off <<= 1) M = fmaxf(M, __shfl_xor_sync(0xffffffffu, M, off));
        float s1 = 0.0f, s2 = 0.0f, sx[D];
#pragma unroll
        for (int t = 0; t < D; ++t) sx[t] = 0.0f;
        PT run = 0;
        const bool live = active && M != -INFINITY;
        if (live) {
          for (uint32_t rho = rb; rho < re; ++rho) {
            const uint32_t pos = mpos(p0, rho);
            const float e = exp_weight(s_lw[pos] - M);
            s1 += e;
            s2 = fmaf(e, e, s2);
#pragma unroll
            for (int t = 0; t < D; ++t) sx[t] = fmaf(e, s_x[t * cap + pos], sx[t]);
            PT q;
            if (WIDE && wide_digit) q = (PT)__float2ull_rz(e * 4294967296.0f);
            else q = (PT)__float2uint_rz(e * 16777216.0f);
            run += q;
            s_P[pos] = run;
          }
        } else if (active) {
          for (uint32_t rho = rb; rho < re; ++rho) s_P[mpos(p0, rho)] = 0;
        }
        PT incl = run;
        for (uint32_t off = 1; off < T; off <<= 1) {
          const PT v = __shfl_up_sync(0xffffffffu, incl, off, T);
          if (lt >= off) incl += v;
        }
        const PT excl = incl - run;
        if (live && excl != 0)
          for (uint32_t rho = rb; rho < re; ++rho) s_P[mpos(p0, rho)] += excl;
        // each lane folds its own chunk into its running partial (same max M for the
        // whole team); only the group's sum of weights is needed here, for L
        float sg = s1;
        for (uint32_t off = 1; off < T; off <<= 1) sg += __shfl_xor_sync(0xffffffffu, sg, off);
        if (live) merge_partial<D>(acc, accx, M, s1, s2, sx);
        if (!active || lt != 0) continue;
        if (!live) status |= kStatusZeroGroup;
        const float L = live ? M + logf(sg) : -INFINITY;
        lV_out[(h0 + hh) * sw + l0 / w + cg] = L - g.log_a;
      }
    }
    __syncthreads();

    // ---- draw ancestors (group-major counters), gather, mutate, store ----
    const uint32_t nq = (G + 3) >> 2;
    const bool g4 = (G & 3u) == 0;
    for (uint32_t it = tid; it < ngroups * nq; it += kBlock) {
      const uint32_t rq = fdiv(it, g.div_tgroups);
      const uint32_t gid = it - rq * ngroups;
      const uint32_t hh = fdiv(gid, g.div_nlw);
      const uint32_t cg = gid - hh * nlw;
      const uint32_t p0 = hh * a * nl + cg * w;              // tile position of member 0
      const uint32_t gc = (h0 + hh) * sw + l0 / w + cg;      // group index
      const uint32_t ib = base + hh * a * s + cg * w;        // global index of member 0
      const PT Q = s_P[p0 + (a - 1) * nl + (w - 1)];
      const uint32_t r0q = rq << 2;
      const uint32_t pi0 = gc * G + r0q;
      uint32_t rw[4] = {0u, 0u, 0u, 0u};
      unsigned long long rw64[4] = {0ull, 0ull, 0ull, 0ull};
      float z[4 * D];
      if (g4) {   // pi0 % 4 == 0: whole counter blocks
        if (WIDE && wide_digit) {
          const uint4 w0 = philox4x32(make_uint4(pi0 >> 1, t_st, kPurposeResampleWide, 0), rk);
          const uint4 w1 = philox4x32(make_uint4((pi0 >> 1) + 1, t_st, kPurposeResampleWide, 0), rk);
          rw64[0] = ((unsigned long long)w0.y << 32) | w0.x;
          rw64[1] = ((unsigned long long)w0.w << 32) | w0.z;
          rw64[2] = ((unsigned long long)w1.y << 32) | w1.x;
          rw64[3] = ((unsigned long long)w1.w << 32) | w1.z;
        } else {
          const uint4 wv = philox4x32(make_uint4(pi0 >> 2, t_st, kPurposeResample, 0), rk);
          rw[0] = wv.x; rw[1] = wv.y; rw[2] = wv.z; rw[3] = wv.w;
        }
        if (mut) {
#pragma unroll
          for (int b = 0; b < D; ++b) {
            const uint4 wv = philox4x32(make_uint4((pi0 >> 2) * D + b, n, kPurposePropagate, 0), rk);
            normals4_fast(wv, z + 4 * b);
          }
        }
      } else {    // members straddle counter blocks: one block per draw / normal
#pragma unroll
        for (int jj = 0; jj < 4; ++jj) {
          const uint32_t pi = pi0 + jj;
          if (r0q + jj >= G) break;
          if (WIDE && wide_digit) {
            const uint4 wv = philox4x32(make_uint4(pi >> 1, t_st, kPurposeResampleWide, 0), rk);
            rw64[jj] = (pi & 1u) ? (((unsigned long long)wv.w << 32) | wv.z) : (((unsigned long long)wv.y << 32) | wv.x);
          } else {
            const uint4 wv = philox4x32(make_uint4(pi >> 2, t_st, kPurposeResample, 0), rk);
            const uint32_t sel = pi & 3u;
            rw[jj] = sel == 0 ? wv.x : sel == 1 ? wv.y : sel == 2 ? wv.z : wv.w;
          }
          if (!mut) continue;
#pragma unroll
          for (int t = 0; t < D; ++t) {
            const uint32_t nu = pi * D + t;
            const uint4 wv = philox4x32(make_uint4(nu >> 2, n, kPurposePropagate, 0), rk);
            float zz[4];
            normals4_fast(wv, zz);
            z[jj * D + t] = zz[nu & 3u];
          }
        }
      }
#pragma unroll
      for (int jj = 0; jj < 4; ++jj) {
        const uint32_t rho = r0q + jj;
        if (rho >= G) break;
        PT u;
        if (WIDE && wide_digit) u = (PT)mulhi64(rw64[jj], (unsigned long long)Q);
        else u = (PT)(((unsigned long long)rw[jj] * Q) >> 32);
        uint32_t c = 0;
        for (uint32_t stp = step0; stp; stp >>= 1) {
          const uint32_t cand = c + stp;
          if (cand <= G - 1 && s_P[mpos(p0, cand - 1)] <= u) c = cand;
        }
        if (Q == 0) c = rho;
        const uint32_t pa = mpos(p0, c);
        float xh[D], xo[D];
#pragma unroll
        for (int t = 0; t < D; ++t) xh[t] = s_x[t * cap + pa];
        if (mut) {
          mutate<D, KIND>(mp, xh, z + jj * D, xo);
        } else {
#pragma unroll
          for (int t = 0; t < D; ++t) xo[t] = xh[t];
        }
        const uint32_t rs = fdiv(rho, g.div_w);
        const uint32_t i = ib + rs * s + (rho - rs * w);
#pragma unroll
        for (int t = 0; t < D; ++t) __stcs(X + (size_t)t * N + i, xo[t]);
      }
    }
  }
}

}  // namespace

template <int D, int KIND, bool WIDE>
__global__ void __launch_bounds__(kBlock) step_sets_kernel(const __grid_constant__ StepParams p) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  DevState* st = p.st;
  const uint32_t S = (uint32_t)p.m - 1;     // stages per step
  const uint32_t n = st->n, stage = st->stage;
  Sched sc;
  sc.n = n;
  sc.t = n * S + stage;
  sc.k = 1 + stage;
  sc.obs = stage == 0;
  sc.mut = stage + 1 == S;
  TileCtx c;
  c.n = n;
  c.t = sc.t;
  c.obs = sc.obs;
  c.mut = sc.mut;
  c.x = p.x;
  c.lV_in = p.lV[sc.t & 1u];
  c.lV_out = p.lV[(sc.t & 1u) ^ 1u];
  c.anc = nullptr;
  c.prec = nullptr;
  c.rk = &p.rk;
  c.mp = &p.model;
  c.g = &p.geom[sc.k];
  c.N = p.N;
  c.cap = p.tile_cap;
  c.muf = st->mu_f;
#pragma unroll
  for (int j = 0; j < kMaxDim; ++j) c.y[j] = (j < p.model.dy) ? p.y_ring[(n % kRing) * p.model.dy + j] : 0.0f;
  uint32_t status = 0;
  Partial acc{-INFINITY, 0.0f, 0.0f};
  float accx[D];
#pragma unroll
  for (int t = 0; t < D; ++t) accx[t] = 0.0f;
  set_tile_steps<D, KIND, WIDE>(c, blockIdx.x, gridDim.x, smem_raw, acc, accx, status);
  finish_step<D>(p, acc, accx, sc, status, c.muf);
}

template <int D, int KIND>
static const void* sets_pick(bool wide) {
  return wide ? reinterpret_cast<const void*>(&step_sets_kernel<D, KIND, true>)
              : reinterpret_cast<const void*>(&step_sets_kernel<D, KIND, false>);
}

const void* select_sets_kernel(int d, int kind, bool wide) {
  if (kind == kStochVol) return d == 1 ? sets_pick<1, kStochVol>(wide) : nullptr;
  if (kind != kLinearGaussian) return nullptr;
  switch (d) {
    case 1: return sets_pick<1, kLinearGaussian>(wide);
    case 2: return sets_pick<2, kLinearGaussian>(wide);
    case 3: return sets_pick<3, kLinearGaussian>(wide);
    case 4: return sets_pick<4, kLinearGaussian>(wide);
    case 5: return sets_pick<5, kLinearGaussian>(wide);
    case 6: return sets_pick<6, kLinearGaussian>(wide);
    case 7: return sets_pick<7, kLinearGaussian>(wide);
    case 8: return sets_pick<8, kLinearGaussian>(wide);
    default: return nullptr;
  }
}

}  // namespace bfpf
