// step_pass.cuh - several consecutive stages of the all-stages schedule in
// one launch.
//
// Paper: Heine, Whiteley & Cemgil, arXiv 1812.01502.  With every stage of
// Algorithm 3 inside each time step (Resample of Algorithm 1 = all of
// Algorithm 3), stage s of step n resamples within the groups of digit s with
// the stage weights V_s = A_s V_{s-1} (eq. (V_defn_proofs)), V_0 = g_n; the
// last stage is followed by the mutation.  A launch of this kernel runs the
// stages on digits k0 .. k0+J-1 (all of radix A) over tiles that contain
// every particle those stages can draw from (tile geometry: PassGeom).
//
// The loaded states do not move while the stages run: stage j only composes
// the ancestor map.  With c_j(p) the tile position that stage j draws for
// output position p, the state at p after stage j is the loaded state at
// A_{j+1}(p) = A_j(c_j(p)), A_0 = identity; the last stage of the launch
// gathers through its map, mutates when the launch ends the step, and stores.
//
// Weights.  Only the step's first stage (k0 = 0) weights with g_n, so its
// weights differ per particle.  After the stage on digit k a particle's
// carried weight is its group's mean, which depends only on its digits above
// k; by induction every later stage of the step gives identical weight
// vectors to all groups that share the digits above the stage's digit.  Such
// a stage computes one prefix-sum row per distinct value of those digits in
// the tile (the tile's "rows") and every group of the row draws against it;
// the draws themselves stay one per particle, with the group's own counter.
//
// The integer draw rule, the random-number counters and the float arithmetic
// of each weight are those of the one-stage kernels (step_group.cuh): with the
// same split of a group over lanes, and the same normaliser mu, the results
// are the same bit for bit.
#pragma once

#include "bfpf_device.cuh"
#include "bfpf_epilogue.cuh"
#include "bfpf_model.cuh"
#include "step_pass_layout.cuh"

namespace bfpf {

__host__ __device__ constexpr int pass_log2(int v) {
  int l = 0;
  while ((1 << l) < v) ++l;
  return l;
}

// z[q] = propagation normal nu0 + q of time step n, q < CNT.
template <int CNT>
__device__ __forceinline__ void pass_normals(uint32_t nu0, uint32_t n, const RoundKeys& rk, float* z) {
  if ((nu0 & 3u) == 0u && CNT % 4 == 0) {
#pragma unroll
    for (int b = 0; b < CNT / 4; ++b)
      normals4_fast(philox4x32(make_uint4((nu0 >> 2) + b, n, kPurposePropagate, 0), rk), z + 4 * b);
  } else {
    constexpr int NB = (CNT + 6) / 4;
    float zz[4 * NB];
#pragma unroll
    for (int b = 0; b < NB; ++b)
      normals4_fast(philox4x32(make_uint4((nu0 >> 2) + b, n, kPurposePropagate, 0), rk), zz + 4 * b);
    const uint32_t off = nu0 & 3u;
#pragma unroll
    for (int q = 0; q < CNT; ++q)
      z[q] = off == 0u ? zz[q] : off == 1u ? zz[q + 1] : off == 2u ? zz[q + 2] : zz[q + 3];
  }
}

// #{j : P_j <= u} in a prefix-sum row (layout: pass_row_stride).  The pivots
// (or the whole row for A <= 4) were loaded once for the draw unit.
template <int A>
__device__ __forceinline__ uint32_t pass_search(const uint32_t* row, const uint32_t* piv, uint32_t u) {
  // every P_j and u is below 2^29, so P_j + ~u has its top bit set exactly when P_j <= u
  const uint32_t nu = ~u;
  if constexpr (A == 2) {
    return (piv[0] + nu) >> 31;
  } else if constexpr (A == 4) {
    return ((piv[0] + nu) >> 31) + ((piv[1] + nu) >> 31) + ((piv[2] + nu) >> 31);
  } else {
    uint32_t b = 0;
#pragma unroll
    for (int q = 0; q < A / 4 - 1; ++q) b += (piv[q] + nu) >> 31;
    const uint4 v = *reinterpret_cast<const uint4*>(row + 4 * b);
    return 4 * b + ((v.x + nu) >> 31) + ((v.y + nu) >> 31) + ((v.z + nu) >> 31);
  }
}

// Three blocks per SM at d = 1 (80 registers), two above (128 registers: the
// weighting stage holds up to 16 state values of its members in registers).
template <int D, int KIND, int A>
__global__ void __launch_bounds__(kBlock, D == 1 ? 3 : 2) step_pass_kernel(const __grid_constant__ StepParams p,
                                                                          const __grid_constant__ PassGeom pg) {
  static_assert(A >= 2 && A <= 32 && (A & (A - 1)) == 0, "radix must be a power of two <= 32");
  constexpr int LA = pass_log2(A);
  constexpr int G = pass_lanes(D, A);          // lanes per group in the weighting stage
  constexpr int M = A / G;                     // members per lane there
  constexpr int MQ = A < 4 ? A : 4;            // members per draw unit (one Philox block)
  constexpr int RS = pass_row_stride(A);
  constexpr int NPV = A <= 4 ? A : A / 4;      // row words a thread loads for its searches (pivots incl. Q)
  // members per thread in the draw phase: up to 16, so that a full tile
  // still gives every thread of the block some (4096 / 16 = 256 at d = 1)
  constexpr int MBT = (int)(pass_tile_max(D) / (uint32_t)kBlock);
  constexpr int MB = A < MBT ? A : (MBT < MQ ? MQ : MBT);
  constexpr uint32_t NCH = A / MB;             // threads per group there
  constexpr unsigned FULL = 0xffffffffu;
  static_assert(M <= 16 && kBlock % G == 0, "bad weighting split");
  extern __shared__ __align__(16) unsigned char smem[];

  const uint32_t T = 1u << pg.log2T;
  const uint32_t TP = T + (T >> 5);
  const PassSmem lay = pass_smem_layout(D, A, T, pg.nrows);
  float* const s_x = reinterpret_cast<float*>(smem + lay.x);
  uint16_t* const s_anc = reinterpret_cast<uint16_t*>(smem + lay.anc);
  uint32_t* const s_rows = reinterpret_cast<uint32_t*>(smem + lay.rows);
  float* const s_lv = reinterpret_cast<float*>(smem + lay.lv);

  const ModelParams& mp = p.model;
  DevState* st = p.st;
  const uint32_t n = st->n;
  const uint32_t m = (uint32_t)p.m;
  const uint32_t J = pg.J;
  const bool obs = pg.k0 == 0;
  const bool mut = pg.k0 + J == m;
  const uint32_t t0 = n * m + pg.k0;
  // carried weights ping-pong by launch counter: launch (n, pass) reads buffer (n npass + pass) mod 2
  const uint32_t lvsel = (n * pg.npass + pg.pass) & 1u;
  const float* __restrict__ lV_in = p.lV[lvsel];
  float* __restrict__ lV_out = p.lV[lvsel ^ 1u];
  float* __restrict__ X = p.x;
  const uint32_t N = p.N;
  const float muf = st->mu_f;
  float y[kMaxDim];
#pragma unroll
  for (int q = 0; q < kMaxDim; ++q) y[q] = (q < mp.dy) ? p.y_ring[(n % kRing) * mp.dy + q] : 0.0f;
  const uint32_t log2L = pg.log2L, log2S = pg.log2S;
  const uint32_t Lmask = (1u << log2L) - 1u;
  const uint32_t log2NG = pg.log2T - LA;
  const uint32_t NG = 1u << log2NG;            // groups of a stage in one tile
  const uint32_t spmask = (1u << pg.log2sp) - 1u;
  const uint32_t tid = threadIdx.x, lane = tid & 31u, warp = tid >> 5;
  const bool whole = pg.log2tl == 0 && log2L == log2S;       // the tile is an index range
  const bool quad = whole || log2L >= 2;                      // runs of >= 4 consecutive indices
  uint32_t status = 0;
  Partial acc{-INFINITY, 0.0f, 0.0f};
  float accx[D];
#pragma unroll
  for (int t = 0; t < D; ++t) accx[t] = 0.0f;

  for (uint32_t tile = blockIdx.x; tile < pg.ntiles; tile += gridDim.x) {
    uint32_t base_i;
    if (whole) {
      base_i = tile << pg.log2T;
    } else {
      const uint32_t hi = tile >> pg.log2tl;
      const uint32_t lo0 = (tile & ((1u << pg.log2tl) - 1u)) << log2L;
      base_i = lo0 + (hi << (pg.log2B + log2S));
    }
    // particle index of tile position pos
    auto i_of = [&](uint32_t pos) -> uint32_t { return base_i + (pos & Lmask) + ((pos >> log2L) << log2S); };

    __syncthreads();   // the previous tile is done with shared memory

    // ---- load the tile's states ----
    if (quad) {
      for (uint32_t q = tid; q < (T >> 2); q += kBlock) {
        const uint32_t pos = q << 2;
        const uint32_t i = i_of(pos);
#pragma unroll
        for (int t = 0; t < D; ++t) {
          const float4 v = *reinterpret_cast<const float4*>(X + (size_t)t * N + i);
          float* dst = s_x + t * TP + pass_xpad(pos);    // the 4 positions share one 32-block
          dst[0] = v.x;
          dst[1] = v.y;
          dst[2] = v.z;
          dst[3] = v.w;
        }
      }
    } else {
      for (uint32_t pos = tid; pos < T; pos += kBlock) {
        const uint32_t i = i_of(pos);
#pragma unroll
        for (int t = 0; t < D; ++t) s_x[t * TP + pass_xpad(pos)] = X[(size_t)t * N + i];
      }
    }
    __syncthreads();

    for (uint32_t j = 0; j < J; ++j) {
      const uint32_t log2sig = log2L + j * LA;       // in-tile stride of this stage's digit
      const uint32_t sigmask = (1u << log2sig) - 1u;
      const uint32_t log2sk = log2S + j * LA;        // its stride s_k among all N particles
      const uint32_t skmask = (1u << log2sk) - 1u;
      const uint32_t t = t0 + j;                     // stage counter: resampling words
      const bool wstage = obs && j == 0;             // weights with g_n, per particle
      const bool last = j + 1 == J;
      float* const lv_cur = s_lv + (j & 1u) * pg.nrows;
      const float* const lv_prev = s_lv + ((j & 1u) ^ 1u) * pg.nrows;
      const uint16_t* const anc_old = s_anc + ((j & 1u) ^ 1u) * T;
      uint16_t* const anc_new = s_anc + (j & 1u) * T;

      // ---- A: prefix-sum rows ----
      if (wstage) {
        // One row per group (the step's weighting stage; here s_k0 = 1, so L = 1
        // and group gi is the positions gi A .. gi A + A - 1).  G lanes per
        // group, M consecutive members per lane, as in the group kernel.
        constexpr uint32_t GPI = kBlock / G;
        const uint32_t tg = tid / G, jl = tid % G;
        for (uint32_t g0 = 0; g0 < NG; g0 += GPI) {
          const uint32_t gi = g0 + tg;
          const bool valid = gi < NG;                // the same for the G lanes of a group
          // lanes past the last group read group 0's states (and write nothing)
          const uint32_t pos0 = ((valid ? gi : 0u) << LA) + jl * M;
          // the tile is the index range from base_i, and a group's carried
          // weights (digit m - 1's groups: index i mod s_{m-1}) are consecutive
          const uint32_t i0 = base_i + pos0;
          const uint32_t lv0 = i0 & spmask;
          float lw[M], xv[M][D];
          if constexpr (M % 4 == 0) {
#pragma unroll
            for (int q = 0; q < M / 4; ++q) {
#pragma unroll
              for (int c = 0; c < D; ++c) {
                const float4 v = *reinterpret_cast<const float4*>(X + (size_t)c * N + i0 + 4 * q);
                xv[4 * q][c] = v.x;
                xv[4 * q + 1][c] = v.y;
                xv[4 * q + 2][c] = v.z;
                xv[4 * q + 3][c] = v.w;
              }
              const float4 v = __ldg(reinterpret_cast<const float4*>(lV_in + lv0) + q);
              lw[4 * q] = v.x;
              lw[4 * q + 1] = v.y;
              lw[4 * q + 2] = v.z;
              lw[4 * q + 3] = v.w;
            }
          } else {
#pragma unroll
            for (int mm = 0; mm < M; ++mm) {
#pragma unroll
              for (int c = 0; c < D; ++c) xv[mm][c] = s_x[c * TP + pass_xpad(pos0 + mm)];
              lw[mm] = __ldg(lV_in + lv0 + mm);
            }
          }
#pragma unroll
          for (int mm = 0; mm < M; ++mm)
            lw[mm] = valid ? lw[mm] + (obs_log_term<D, KIND>(mp, y, xv[mm]) - muf)
                           : 0.0f;                   // a finite dummy: no side effects below
          float mx = lw[0];
#pragma unroll
          for (int mm = 1; mm < M; ++mm) mx = fmaxf(mx, lw[mm]);
#pragma unroll
          for (int off = 1; off < G; off <<= 1) mx = fmaxf(mx, __shfl_xor_sync(FULL, mx, off));
          float s1 = 0.0f, s2 = 0.0f, sx[D];
          uint32_t P[M];
          uint32_t run = 0;
#pragma unroll
          for (int c = 0; c < D; ++c) sx[c] = 0.0f;
#pragma unroll
          for (int mm = 0; mm < M; ++mm) {
            const float e = exp_weight(lw[mm] - mx);
            s1 += e;
            s2 = fmaf(e, e, s2);
#pragma unroll
            for (int c = 0; c < D; ++c) sx[c] = fmaf(e, xv[mm][c], sx[c]);
            run += __float2uint_rz(e * 16777216.0f);
            P[mm] = run;
          }
          float s1_lane = s1;
#pragma unroll
          for (int off = 1; off < G; off <<= 1) s1 += __shfl_xor_sync(FULL, s1, off);
          // Rare path (a non-finite log-weight, or a group whose weights are all
          // zero): recompute with sanitised weights.  Entered by the whole warp
          // when any of its groups needs it, so that the shuffles stay converged;
          // for the other groups it recomputes the same values.
          if (__any_sync(FULL, !(s1 >= 1.0f && s1 <= (float)A))) {
#pragma unroll
            for (int mm = 0; mm < M; ++mm) lw[mm] = sanitize_logweight(lw[mm], status);
            mx = -INFINITY;
#pragma unroll
            for (int mm = 0; mm < M; ++mm) mx = fmaxf(mx, lw[mm]);
#pragma unroll
            for (int off = 1; off < G; off <<= 1) mx = fmaxf(mx, __shfl_xor_sync(FULL, mx, off));
            const bool live = mx != -INFINITY;
            s1 = 0.0f;
            s2 = 0.0f;
            run = 0;
#pragma unroll
            for (int c = 0; c < D; ++c) sx[c] = 0.0f;
#pragma unroll
            for (int mm = 0; mm < M; ++mm) {
              const float e = live ? exp_weight(lw[mm] - mx) : 0.0f;
              s1 += e;
              s2 = fmaf(e, e, s2);
#pragma unroll
              for (int c = 0; c < D; ++c) sx[c] = fmaf(e, xv[mm][c], sx[c]);
              run += __float2uint_rz(e * 16777216.0f);
              P[mm] = run;
            }
            s1_lane = s1;
#pragma unroll
            for (int off = 1; off < G; off <<= 1) s1 += __shfl_xor_sync(FULL, s1, off);
            if (!live && jl == 0 && valid) status |= kStatusZeroGroup;
          }
          uint32_t incl = run;
#pragma unroll
          for (int off = 1; off < G; off <<= 1) {
            const uint32_t v = __shfl_up_sync(FULL, incl, off, G);
            if ((int)jl >= off) incl += v;
          }
          const uint32_t Q = (G > 1) ? __shfl_sync(FULL, incl, G - 1, G) : incl;
          const uint32_t excl = incl - run;
          if (valid) {
            uint32_t* const row = s_rows + gi * RS;
#pragma unroll
            for (int mm = 0; mm < M; ++mm) {
              const uint32_t r = jl * M + mm;
              const uint32_t v = P[mm] + excl;
              row[r] = v;
              if (A >= 8 && (r & 3u) == 3u) row[A + (r >> 2)] = v;
            }
            if (jl == 0) lv_cur[gi] = (Q != 0) ? (mx + logf(s1) - pg.log_a) : -INFINITY;
            merge_partial<D>(acc, accx, mx, s1_lane, s2, sx);
          }
        }
      } else {
        // One row per distinct value of the digits above this stage's digit in
        // the tile: member r of row rho sits at position
        // (r << log2sig) + (rho << (log2sig + LA)).  One lane per member, 32 / A
        // rows per warp at a time.  The weight sum follows the group kernel's
        // order (M0 consecutive members per lane, then an xor tree).
        constexpr int M0 = group_members_per_lane(A, D);
        constexpr int G0 = A / M0;
        constexpr uint32_t RPW = 32 / A;
        const uint32_t nrj = T >> (log2sig + LA);
        const uint32_t seg = lane / A, r = lane % A;
        for (uint32_t rb = warp * RPW; rb < nrj; rb += (kBlock / 32) * RPW) {
          const uint32_t rho = rb + seg;
          const bool valid = rho < nrj;              // the same for the A lanes of a row
          float w = -INFINITY;
          if (valid) {
            if (j == 0) {   // the carried weight of the group of digit k0 - 1 holding member r
              const uint32_t i = i_of((r << log2sig) + (rho << (log2sig + LA)));
              w = __ldg(lV_in + (((i >> log2S) << pg.log2sp) | (i & spmask)));
            } else {        // ... of the previous stage's row (r, rho)
              w = lv_prev[r + (rho << LA)];
            }
            w = sanitize_logweight(w, status);
          }
          float mx = w;
#pragma unroll
          for (int off = 1; off < A; off <<= 1) mx = fmaxf(mx, __shfl_xor_sync(FULL, mx, off));
          const bool live = mx != -INFINITY;
          const float e = live ? exp_weight(w - mx) : 0.0f;
          uint32_t P = __float2uint_rz(e * 16777216.0f);
#pragma unroll
          for (int off = 1; off < A; off <<= 1) {
            const uint32_t v = __shfl_up_sync(FULL, P, off, A);
            if ((int)r >= off) P += v;
          }
          const uint32_t Q = __shfl_sync(FULL, P, A - 1, A);
          float s1 = 0.0f;
#pragma unroll
          for (int mm = 0; mm < M0; ++mm) s1 += __shfl_sync(FULL, e, (int)((r / M0) * M0) + mm, A);
#pragma unroll
          for (int off = 1; off < G0; off <<= 1) s1 += __shfl_xor_sync(FULL, s1, off * M0);
          if (valid) {
            uint32_t* const row = s_rows + rho * RS;
            row[r] = P;
            if (A >= 8 && (r & 3u) == 3u) row[A + (r >> 2)] = P;
            if (r == 0) {
              lv_cur[rho] = (Q != 0) ? (mx + logf(s1) - pg.log_a) : -INFINITY;
              if (!live) status |= kStatusZeroGroup;
            }
          }
        }
      }
      __syncthreads();

      // the new carried weights of the launch's last digit, one per group
      if (last) {
        for (uint32_t gi = tid; gi < NG; gi += kBlock) {
          const uint32_t base = (gi & sigmask) | ((gi >> log2sig) << (log2sig + LA));
          const uint32_t i0 = i_of(base);
          lV_out[((i0 >> (log2sk + LA)) << log2sk) | (i0 & skmask)] = lv_cur[gi >> log2sig];
        }
      }

      // ---- B: one draw per particle.  A thread takes MB consecutive members of
      // one group (MB a power of two dividing A): group gi of the stage has its
      // member 0 at position base and its row at gi >> log2sig; the words of
      // MQ members come from one Philox block ----
      for (uint32_t u = tid; u < NG * NCH; u += kBlock) {
        const uint32_t gi = u & (NG - 1u);
        const uint32_t rb0 = (u >> log2NG) * MB;
        const uint32_t base = (gi & sigmask) | ((gi >> log2sig) << (log2sig + LA));
        const uint32_t* const row = s_rows + (gi >> log2sig) * RS;
        const uint32_t i0 = i_of(base);
        const uint32_t g = ((i0 >> (log2sk + LA)) << log2sk) | (i0 & skmask);   // the group's number
        uint32_t piv[NPV];
        if constexpr (A == 2) {
          const uint2 v = *reinterpret_cast<const uint2*>(row);
          piv[0] = v.x;
          piv[1] = v.y;
        } else if constexpr (A == 4) {
          const uint4 v = *reinterpret_cast<const uint4*>(row);
          piv[0] = v.x;
          piv[1] = v.y;
          piv[2] = v.z;
          piv[3] = v.w;
        } else if constexpr (A == 8) {
          const uint2 v = *reinterpret_cast<const uint2*>(row + A);
          piv[0] = v.x;
          piv[1] = v.y;
        } else {
#pragma unroll
          for (int q = 0; q < NPV / 4; ++q) {
            const uint4 v = *reinterpret_cast<const uint4*>(row + A + 4 * q);
            piv[4 * q] = v.x;
            piv[4 * q + 1] = v.y;
            piv[4 * q + 2] = v.z;
            piv[4 * q + 3] = v.w;
          }
        }
        const uint32_t Q = piv[NPV - 1];
        // new map entries of a stage on the lowest in-tile digit (members
        // adjacent): gathered in registers and stored 16 bytes at a time
        constexpr int NPK = (MB >= 8) ? MB / 2 : 1;
        uint32_t pk[NPK];
#pragma unroll
        for (int q = 0; q < NPK; ++q) pk[q] = 0u;
        const bool packed = (MB >= 8) && log2sig == 0 && !last;
#pragma unroll
        for (int q4 = 0; q4 < MB / MQ; ++q4) {
          const uint32_t pi0 = g * A + rb0 + q4 * MQ;       // group-major index of the unit's first member
          uint32_t rw[MQ];
          {
            const uint4 w = philox4x32(make_uint4(pi0 >> 2, t, kPurposeResample, 0), p.rk);
            if constexpr (MQ == 4) {
              rw[0] = w.x;
              rw[1] = w.y;
              rw[2] = w.z;
              rw[3] = w.w;
            } else {
              const bool hi2 = (pi0 & 2u) != 0u;
              rw[0] = hi2 ? w.z : w.x;
              rw[1] = hi2 ? w.w : w.y;
            }
          }
          // propagation normals NQ members at a time (fewer registers at d = 6, 8,
          // where a pair's normals still start on a Philox block)
          constexpr int NQ = (D == 6 || D == 8) && MQ == 4 ? 2 : MQ;
#pragma unroll
          for (int h = 0; h < MQ / NQ; ++h) {
            float z[NQ * D];
            if (last && mut) pass_normals<NQ * D>((pi0 + h * NQ) * D, n, p.rk, z);
#pragma unroll
            for (int mq2 = 0; mq2 < NQ; ++mq2) {
              const int mb = q4 * MQ + h * NQ + mq2;           // member of the thread's run
              const uint32_t r = rb0 + mb;
              uint32_t c = pass_search<A>(row, piv, __umulhi(rw[h * NQ + mq2], Q));   // floor(r Q / 2^32) against P
              if (Q == 0) c = r;                                                  // an all-zero group keeps its particles
              const uint32_t pc = base + (c << log2sig);
              const uint32_t src = (j == 0) ? pc : (uint32_t)anc_old[pc];
              if (!last) {
                if (packed) {
                  if constexpr (MB >= 8) pk[mb >> 1] |= src << (16 * (mb & 1));
                } else {
                  anc_new[base + (r << log2sig)] = (uint16_t)src;
                }
              } else {
                float xh[D], xo[D];
#pragma unroll
                for (int cc = 0; cc < D; ++cc) xh[cc] = s_x[cc * TP + pass_xpad(src)];
                if (mut) {
                  mutate<D, KIND>(mp, xh, z + mq2 * D, xo);
                } else {
#pragma unroll
                  for (int cc = 0; cc < D; ++cc) xo[cc] = xh[cc];
                }
                const uint32_t i = i0 + (r << log2sk);
#pragma unroll
                for (int cc = 0; cc < D; ++cc) X[(size_t)cc * N + i] = xo[cc];
              }
            }
          }
        }
        if constexpr (MB >= 8) {
          if (packed) {
            uint4* dst = reinterpret_cast<uint4*>(anc_new + base + rb0);   // 16-byte aligned: base + rb0 is a multiple of 8
#pragma unroll
            for (int q = 0; q < NPK / 4; ++q) dst[q] = make_uint4(pk[4 * q], pk[4 * q + 1], pk[4 * q + 2], pk[4 * q + 3]);
          }
        }
      }
      __syncthreads();   // this stage's rows and map are read; the next stage overwrites them
    }
  }
  const Sched sc{n, t0, pg.k0, obs, mut};
  finish_step<D>(p, acc, accx, sc, status, muf, nullptr, J);
}

// Kernel for (D, KIND, A); nullptr for an unsupported combination.
template <int D, int KIND>
inline const void* pass_kernel_for(int a) {
  switch (a) {
    case 2: return reinterpret_cast<const void*>(&step_pass_kernel<D, KIND, 2>);
    case 4: return reinterpret_cast<const void*>(&step_pass_kernel<D, KIND, 4>);
    case 8: return reinterpret_cast<const void*>(&step_pass_kernel<D, KIND, 8>);
    case 16: return reinterpret_cast<const void*>(&step_pass_kernel<D, KIND, 16>);
    case 32: return reinterpret_cast<const void*>(&step_pass_kernel<D, KIND, 32>);
    default: return nullptr;
  }
}

}  // namespace bfpf
