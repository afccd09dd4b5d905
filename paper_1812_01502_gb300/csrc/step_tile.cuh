// step_tile.cuh - the shared-memory tile form of one time step (general
// radices up to 1024), shared by the single-filter kernel (step_butterfly.cu)
// and the batched kernel (batch.cu).
//
// Tile: nh blocks of the digits above k x a_k rows x nl columns of the digits
// below k; tile position p = row*nl + col, row = hh*a_k + r; global index
// i = base + row*s_k + col.  Per tile: coalesced load of the states into
// shared memory, weights, per-group max / log-sum-exp / integer prefix sums
// (one thread per group), then per member quad: group-major Philox draws,
// ancestor search, gather from shared memory, mutation, store.
#pragma once

#include <cfloat>
#include <type_traits>

#include "bfpf_device.cuh"
#include "bfpf_epilogue.cuh"
#include "bfpf_model.cuh"

namespace bfpf {

__device__ __forceinline__ unsigned long long mulhi64(unsigned long long a, unsigned long long b) {
  return __umul64hi(a, b);
}

// Everything one time step does to the tiles first, first + stride, ... of one
// filter (the tile loop of the general kernel; also run by the batched kernel).
struct TileCtx {
  float* x;                  // [d][N] states (updated in place)
  const float* lV_in;        // carried log weights, groups of the previous digit
  float* lV_out;             // new carried log weights, groups of this digit
  int32_t* anc;              // ancestors (nullptr: not recorded)
  unsigned long long* prec;  // integer prefix sums of the draws (nullptr: not recorded)
  const RoundKeys* rk;
  const ModelParams* mp;
  const DigitGeom* g;        // geometry of this step's digit
  uint32_t N, n, cap;
  uint32_t t;                // stage counter (resampling counters)
  bool obs, mut;             // weight with g_n / mutate (see Sched)
  float muf;
  float y[kMaxDim];
};

// STAGED = false: every call weights with g_n and mutates (one stage per
// step); STAGED = true: ctx.obs / ctx.mut decide (all stages per step).
// ADAPT = true (fully adapted schedule): carried weights are per particle
// (lV_in[i], lV_out[i]), the observation weight was applied by a separate
// pass, and the partials accumulate the new stage weights V = exp(L_G - log a)
// of every member (for the ESS after the stage) instead of the weighted
// particles.
template <int D, int KIND, bool WIDE, bool STAGED = false, bool ADAPT = false>
__device__ __forceinline__ void tile_steps(const TileCtx& ctx, uint32_t first, uint32_t stride,
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
  const uint32_t a = g.a, s = g.s, nl = g.nl, tn = g.tile_n;
  const bool wide_digit = g.wide != 0;
  const float* __restrict__ lV_in = ctx.lV_in;
  float* __restrict__ lV_out = ctx.lV_out;
  float* __restrict__ X = ctx.x;
  const float muf = ctx.muf;
  const uint32_t N = ctx.N, n = ctx.n, t_st = STAGED ? ctx.t : ctx.n;
  const bool obs = STAGED ? ctx.obs : true;
  const bool mut = STAGED ? ctx.mut : true;
  const float* y = ctx.y;
  const uint32_t ngroups = g.nh * nl;   // groups per tile
  // lifting steps of the ancestor search: largest power of two < a (0 if a == 1)
  uint32_t step0 = 1;
  while ((step0 << 1) < a) step0 <<= 1;
  if (a == 1) step0 = 0;

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

    // ---- weights: lw = lV(group of the previous digit) + log g_n(x) - mu ----
    for (uint32_t pos = tid; pos < tn; pos += kBlock) {
      const uint32_t row = fdiv(pos, g.div_nl);
      const uint32_t i = base + row * s + (pos - row * nl);
      float lv;
      if constexpr (ADAPT) {
        lv = __ldg(lV_in + i);
      } else {
        const uint32_t hp = fdiv(i, g.div_prev_as);
        const uint32_t lo = i - fdiv(i, g.div_prev_s) * g.prev_s;
        lv = __ldg(lV_in + hp * g.prev_s + lo);
      }
      float xv[D];
#pragma unroll
      for (int t = 0; t < D; ++t) xv[t] = s_x[t * cap + pos];
      s_lw[pos] = sanitize_logweight(obs ? lv + obs_log_term<D, KIND>(mp, y, xv) - muf : lv, status);
    }
    __syncthreads();

    // ---- per group: max, log-sum-exp, integer weights and prefix sums ----
    // A team of T lanes (a power of two <= 32, T <= a) shares a group: lane lt
    // takes members [lt C, lt C + C), C = ceil(a / T); max and sums by xor-shuffle,
    // the prefix by an in-lane scan plus a shuffle scan over the team.  Every
    // lane runs the same number of rounds, so the shuffles see the whole warp.
    {
      const uint32_t T = g.team, lt = tid & (T - 1u);
      const uint32_t tpb = kBlock / T;
      const uint32_t C = (a + T - 1u) / T;
      const uint32_t rb = min(a, lt * C), re = min(a, rb + C);
      const uint32_t rounds = (ngroups + tpb - 1u) / tpb;
      for (uint32_t rd = 0; rd < rounds; ++rd) {
        const uint32_t gid = rd * tpb + tid / T;
        const bool active = gid < ngroups;
        uint32_t hh = 0, col = 0;
        if (active) {
          hh = fdiv(gid, g.div_nl);
          col = gid - hh * nl;
        }
        const uint32_t p0 = hh * a * nl + col;
        float M = -INFINITY;
        if (active)
          for (uint32_t r = rb; r < re; ++r) M = fmaxf(M, s_lw[p0 + r * nl]);
        for (uint32_t off = 1; off < T; off <<= 1) M = fmaxf(M, __shfl_xor_sync(0xffffffffu, M, off));
        float s1 = 0.0f, s2 = 0.0f, sx[D];
#pragma unroll
        for (int t = 0; t < D; ++t) sx[t] = 0.0f;
        PT run = 0;
        const bool live = active && M != -INFINITY;
        if (live) {
          for (uint32_t r = rb; r < re; ++r) {
            const uint32_t pos = p0 + r * nl;
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
          for (uint32_t r = rb; r < re; ++r) s_P[p0 + r * nl] = 0;
        }
        PT incl = run;
        for (uint32_t off = 1; off < T; off <<= 1) {
          const PT v = __shfl_up_sync(0xffffffffu, incl, off, T);
          if (lt >= off) incl += v;
        }
        const PT excl = incl - run;
        if (live && excl != 0)
          for (uint32_t r = rb; r < re; ++r) s_P[p0 + r * nl] += excl;
        if (ctx.prec && active) {    // test output: the integer prefix sums the draws use
          const uint32_t ib = base + hh * a * s + col;
          for (uint32_t r = rb; r < re; ++r) ctx.prec[ib + r * s] = (unsigned long long)s_P[p0 + r * nl];
        }
        // each lane folds its own chunk into its running partial (same max M for the
        // whole team); only the group's sum of weights is needed here, for L
        float sg = s1;
        for (uint32_t off = 1; off < T; off <<= 1) sg += __shfl_xor_sync(0xffffffffu, sg, off);
        if (!ADAPT && live) merge_partial<D>(acc, accx, M, s1, s2, sx);
        if (!active) continue;
        const float L = live ? M + logf(sg) : -INFINITY;
        if (!live && lt == 0) status |= kStatusZeroGroup;
        if constexpr (ADAPT) {
          const uint32_t ib = base + hh * a * s + col;       // global index of member 0
          for (uint32_t r = rb; r < re; ++r) lV_out[ib + r * s] = L - g.log_a;
          if (lt == 0) {
            float zx[D];
#pragma unroll
            for (int t = 0; t < D; ++t) zx[t] = 0.0f;
            merge_partial<D>(acc, accx, L, 1.0f, 1.0f / (float)a, zx);   // sum_i V_i, sum_i V_i^2 of the group
          }
        } else if (lt == 0) {
          lV_out[(h0 + hh) * s + l0 + col] = L - g.log_a;
        }
      }
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
          const uint4 w0 = philox4x32(make_uint4(pi0 >> 1, t_st, kPurposeResampleWide, 0), rk);
          const uint4 w1 = philox4x32(make_uint4((pi0 >> 1) + 1, t_st, kPurposeResampleWide, 0), rk);
          rw64[0] = ((unsigned long long)w0.y << 32) | w0.x;
          rw64[1] = ((unsigned long long)w0.w << 32) | w0.z;
          rw64[2] = ((unsigned long long)w1.y << 32) | w1.x;
          rw64[3] = ((unsigned long long)w1.w << 32) | w1.z;
        } else {
          const uint4 w = philox4x32(make_uint4(pi0 >> 2, t_st, kPurposeResample, 0), rk);
          rw[0] = w.x; rw[1] = w.y; rw[2] = w.z; rw[3] = w.w;
        }
        if (mut) {
#pragma unroll
          for (int b = 0; b < D; ++b) {
            const uint4 w = philox4x32(make_uint4((pi0 >> 2) * D + b, n, kPurposePropagate, 0), rk);
            normals4_fast(w, z + 4 * b);
          }
        }
      } else {    // members straddle counter blocks: one block per draw / normal
#pragma unroll
        for (int jj = 0; jj < 4; ++jj) {
          const uint32_t pi = pi0 + jj;
          if (r0 + jj >= a) break;
          if (WIDE && wide_digit) {
            const uint4 w = philox4x32(make_uint4(pi >> 1, t_st, kPurposeResampleWide, 0), rk);
            rw64[jj] = (pi & 1u) ? (((unsigned long long)w.w << 32) | w.z) : (((unsigned long long)w.y << 32) | w.x);
          } else {
            const uint4 w = philox4x32(make_uint4(pi >> 2, t_st, kPurposeResample, 0), rk);
            const uint32_t sel = pi & 3u;
            rw[jj] = sel == 0 ? w.x : sel == 1 ? w.y : sel == 2 ? w.z : w.w;
          }
          if (!mut) continue;
#pragma unroll
          for (int t = 0; t < D; ++t) {
            const uint32_t nu = pi * D + t;
            const uint4 w = philox4x32(make_uint4(nu >> 2, n, kPurposePropagate, 0), rk);
            float zz[4];
            normals4_fast(w, zz);
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
        if (mut) {
          mutate<D, KIND>(mp, xh, z + jj * D, xo);
        } else {
#pragma unroll
          for (int t = 0; t < D; ++t) xo[t] = xh[t];
        }
        const uint32_t i = ib + r * s;
#pragma unroll
        for (int t = 0; t < D; ++t) __stcs(X + (size_t)t * N + i, xo[t]);
        if (ctx.anc) ctx.anc[i] = (int32_t)(ib + c * s);
      }
    }
  }

}

// The general kernel: the tiles of one stage split over a persistent grid,
// then the end-of-step epilogue (step_butterfly.cu, step_butterfly_staged.cu
// instantiate it).
template <int D, int KIND, bool WIDE, bool STAGED>
__global__ void __launch_bounds__(kBlock) step_butterfly_kernel(const __grid_constant__ StepParams p) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  DevState* st = p.st;
  const Sched sc = STAGED ? sched_of(p, st) : Sched{st->n, st->n, st->n % (uint32_t)p.m, true, true};
  TileCtx c;
  c.n = sc.n;
  c.t = sc.t;
  c.obs = sc.obs;
  c.mut = sc.mut;
  c.x = p.x;
  c.lV_in = p.lV[sc.t & 1u];
  c.lV_out = p.lV[(sc.t & 1u) ^ 1u];
  c.anc = p.anc;
  c.prec = p.prec;
  c.rk = &p.rk;
  c.mp = &p.model;
  c.g = &p.geom[sc.k];
  c.N = p.N;
  c.cap = p.tile_cap;
  c.muf = st->mu_f;
#pragma unroll
  for (int j = 0; j < kMaxDim; ++j) c.y[j] = (j < p.model.dy) ? p.y_ring[(c.n % kRing) * p.model.dy + j] : 0.0f;
  uint32_t status = 0;
  Partial acc{-INFINITY, 0.0f, 0.0f};
  float accx[D];
#pragma unroll
  for (int t = 0; t < D; ++t) accx[t] = 0.0f;
  tile_steps<D, KIND, WIDE, STAGED>(c, blockIdx.x, gridDim.x, smem_raw, acc, accx, status);
  finish_step<D>(p, acc, accx, sc, status, c.muf);
}

}  // namespace bfpf
