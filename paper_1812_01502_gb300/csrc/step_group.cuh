// step_group.cuh - one time step of the butterfly particle filter with the
// interaction groups held in registers (power-of-two radix A <= 32).
//
// Paper: Heine, Whiteley & Cemgil, arXiv 1812.01502.  Time step n is the loop
// body of Algorithm 1 with ONE stage of Algorithm 3 on digit k = n mod m:
//   weight     lw_i = log V_i + log g_n(zeta_i) - mu           (V_0 = g)
//   stage      V'_G = A^-1 sum_{j in G} V_j                     (eq. (V_defn_proofs))
//   resample   xi_i ~ sum_{j in G(i)} V_j delta_{zeta_j} / sum V_j   (integer rule)
//   mutate     zeta'_i ~ f(xi_i, .)                             (Algorithm 1)
//
// Work mapping: a group of A members (the A particles sharing every digit
// but k) is owned by G consecutive lanes of one warp, each holding M = A/G
// members in registers: group max / sums by xor-shuffles, the integer prefix
// sum by an in-thread scan plus a shuffle scan over the G lanes.  Prefix sums
// and states are staged in shared memory in a [member][group] layout so that
// the ancestor search and the gather read different banks across a warp.
// With one lane per group (G = 1) only warp-level synchronisation is needed
// inside the loop, and loads and stores go straight to global memory: for a
// fixed member, consecutive lanes own consecutive groups, i.e. consecutive
// addresses when s_k >= 32.  With a group spread over G >= 8 lanes, a warp's
// direct accesses would use at most half of every sector they touch (members
// s_k apart); there the block loads and stores its whole tile of
// D x A x (groups per iteration) states through the state table in address
// order (coalesced for every digit), at the price of block-wide barriers.
//
// Integer resampling rule (shared with the oracle): delta = fp32(lw - max),
// e = exp(delta), q = floor(e 2^24), P = inclusive prefix, Q = P_{A-1},
// u = floor(r Q / 2^32), ancestor = #{j : P_j <= u}, found in two 4-ary
// levels: the bucket from the pivots P_3, P_7, ... (registers when one lane
// holds the whole group, else one 16-byte shared-memory load), then the
// bucket's 4 sums from one 16-byte shared-memory load.
#pragma once

#include "bfpf_device.cuh"
#include "bfpf_epilogue.cuh"
#include "bfpf_model.cuh"
#include "step_adaptive.cuh"
#include "step_group_layout.cuh"

namespace bfpf {

// STAGED = false: one stage per time step (every launch weights and mutates).
// STAGED = true: the stage schedule of the device state decides both (all
// stages per step, Sched); a separate instantiation keeps the default path's
// registers unchanged.
// ADAPT = true: stage launch gg.j of the fully adapted schedule without
// rotation (digit gg.k = gg.j): skipped when the ESS already reached the
// threshold (the last launch then only mutates), per-particle carried weights
// in and out, and the ESS of the new stage weights decides the next stage.
// Cooperative tile of one block iteration (groups g0 .. g0 + GPB - 1 of the
// digit with stride s = 2^log2s): element (t, member r, group gi) lives at
// X[t N + off] and in the state table at (t A + r) LD + gi; a thread takes the
// same PH elements of every component, located once.  When s >= GPB the
// tile's groups share h and form GPB consecutive columns of every member row
// (off = base + r s + gi); when s < GPB (then s divides GPB and g0) its particles
// are the consecutive range of length A GPB from base = h0 A s.  Either way
// consecutive threads take consecutive addresses.
// Largest divisor of n that is at most 8.
constexpr int load_chunk(int n) {
  int c = n < 8 ? n : 8;
  while (n % c) --c;
  return c;
}

template <int D, int A, int GPB, int LD>
struct GroupTile {
  static constexpr uint32_t kRow = (uint32_t)A * GPB;   // elements per state component
  static constexpr int PH = (int)(kRow / kBlock);        // elements of a component per thread
  static constexpr int PER = D * PH;
  static_assert(kRow % kBlock == 0, "tile rows must split evenly over the block");
  uint32_t off[PH], tix[PH];   // my elements of component 0: row offset, table index
  __device__ __forceinline__ GroupTile(uint32_t batch, uint32_t log2s, uint32_t log2as) {
    const uint32_t g0 = batch * GPB;
    const uint32_t h0 = g0 >> log2s, l0 = g0 & ((1u << log2s) - 1u);
    const bool wide_s = (1u << log2s) >= (uint32_t)GPB;
    const uint32_t base = (h0 << log2as) + l0;
#pragma unroll
    for (int ph = 0; ph < PH; ++ph) {
      const uint32_t e = threadIdx.x + (uint32_t)ph * kBlock;
      uint32_t r, gi;
      if (wide_s) {
        r = e / GPB;
        gi = e % GPB;
        off[ph] = base + (r << log2s) + gi;
      } else {
        r = (e >> log2s) & (A - 1u);
        gi = ((e >> log2as) << log2s) | (e & ((1u << log2s) - 1u));
        off[ph] = base + e;
      }
      tix[ph] = r * LD + gi;
    }
  }
  __device__ __forceinline__ void load(const float* __restrict__ X, uint32_t N, uint32_t* tab) const {
    constexpr int CH = load_chunk(PER);             // loads in flight per thread
#pragma unroll
    for (int c = 0; c < PER; c += CH) {
      float v[CH];
#pragma unroll
      for (int q = 0; q < CH; ++q) {
        const int t = (c + q) / PH, ph = (c + q) % PH;
        v[q] = __ldcs(X + (size_t)t * N + off[ph]);
      }
#pragma unroll
      for (int q = 0; q < CH; ++q) {
        const int t = (c + q) / PH, ph = (c + q) % PH;
        tab[tix[ph] + (uint32_t)(t * A * LD)] = __float_as_uint(v[q]);
      }
    }
  }
  __device__ __forceinline__ void store(float* __restrict__ X, uint32_t N, const uint32_t* tab) const {
#pragma unroll 4
    for (int el = 0; el < PER; ++el) {
      const int t = el / PH, ph = el % PH;
      __stcs(X + (size_t)t * N + off[ph], __uint_as_float(tab[tix[ph] + (uint32_t)(t * A * LD)]));
    }
  }
};

// What one stage reads and writes of its filter, besides the model and the
// round keys (passed separately so that they stay in parameter space).
struct GroupCtx {
  float* x;                 // [d][N] states
  const float* lV_in;       // carried log weights of the previous stage
  float* lV_out;            // ... of this stage
  int32_t* anc;             // optional ancestors
  unsigned long long* prec; // optional prefix sums of the draws (test output)
  uint32_t N;
  uint32_t n;               // time step: observation and propagation normals
  uint32_t t;               // stage counter: resampling words
  bool obs, mut;            // weight with g_n / mutate in this stage
  float muf;                // FP32 normaliser subtracted from the log weights
  float y[kMaxDim];         // observation y_n
};

// Block iterations first, first + stride, ... < gg.nbatch of one stage on a
// radix-A digit: every group's weights, draws, gather and mutation; the
// block's partial sums accumulate into (acc, accx) and status bits into status.
template <int D, int KIND, int A, int G, bool ADAPT>
__device__ __forceinline__ void group_iterations(const GroupCtx& c, const RoundKeys& rk, const ModelParams& mp,
                                                 const GroupGeom& gg, uint32_t first, uint32_t stride,
                                                 uint32_t* s_rows, uint32_t* s_tab, Partial& acc, float* accx,
                                                 uint32_t& status) {
  static_assert(A >= 2 && A <= 32 && (A & (A - 1)) == 0, "radix must be a power of two <= 32");
  static_assert(G >= 1 && G <= A && A % G == 0, "bad lanes per group");
  using LY = GroupLayout<D, A, G>;
  constexpr int M = A / G;                 // members per lane
  constexpr int GPB = LY::GPB;
  constexpr int LD = LY::LD;
  constexpr int PIV = LY::PIV;
  constexpr int RS = LY::RS;
  constexpr unsigned FULL = 0xffffffffu;
  // tile through the state table (block barriers) for groups over 8 or more
  // lanes: their direct accesses would use at most half of every sector
  // (with G lanes per group a warp's access spans G runs of 32/G floats)
  constexpr bool COAL = (G >= 8) && !ADAPT;

  const uint32_t tid = threadIdx.x;
  const uint32_t tg = tid / G, j = tid % G;
  const bool obs = c.obs, mut = c.mut;
  const uint32_t n = c.n;
  const float* __restrict__ lV_in = c.lV_in;
  float* __restrict__ lV_out = c.lV_out;
  float* __restrict__ X = c.x;
  const float muf = c.muf;
  const uint32_t N = c.N;
  const float* y = c.y;
  const uint32_t log2s = gg.log2s, log2as = gg.log2as;
  const uint32_t smask = (1u << log2s) - 1u;
  const bool contiguous = (log2s == 0) && (M % 4 == 0);   // digit 0: members are adjacent
  uint32_t* const col = s_tab + tg;                        // my group's column of the state table
  uint32_t* const row = s_rows + tg * RS;                  // my group's prefix-sum row

  for (uint32_t batch = first; batch < gg.nbatch; batch += stride) {
    const uint32_t g = batch * GPB + tg;              // group index h*s + l
    const uint32_t h = g >> log2s;
    const uint32_t l = g & smask;
    const uint32_t ig = (h << log2as) + l;            // global index of member 0
    const uint32_t i0 = ig + ((j * M) << log2s);      // my first member
    const float* lvp = lV_in + ((((h * A + j * M) * gg.lv_mul) + (l & gg.lv_lmask)) & gg.lv_mask);

    // ---- load my members, weight them (lw = log V + log g_n - mu) ----
    float xv[M][D];
    float lw[M];
    if constexpr (COAL) {
      __syncthreads();                               // the previous iteration's store has read the table
      GroupTile<D, A, GPB, LD>(batch, log2s, log2as).load(X, N, s_tab);
      __syncthreads();
#pragma unroll
      for (int mm = 0; mm < M; ++mm) {
#pragma unroll
        for (int t = 0; t < D; ++t) xv[mm][t] = __uint_as_float(col[(t * A + j * M + mm) * LD]);
        lw[mm] = __ldg(lvp + mm * gg.lv_mul);
      }
    } else if (contiguous) {
#pragma unroll
      for (int q = 0; q < M / 4; ++q) {
#pragma unroll
        for (int t = 0; t < D; ++t) {
          const float4 v = __ldcs(reinterpret_cast<const float4*>(X + (size_t)t * N + i0) + q);
          xv[4 * q][t] = v.x; xv[4 * q + 1][t] = v.y; xv[4 * q + 2][t] = v.z; xv[4 * q + 3][t] = v.w;
        }
        const float4 v = __ldg(reinterpret_cast<const float4*>(lvp) + q);
        lw[4 * q] = v.x; lw[4 * q + 1] = v.y; lw[4 * q + 2] = v.z; lw[4 * q + 3] = v.w;
      }
    } else {
#pragma unroll
      for (int mm = 0; mm < M; ++mm) {
        const uint32_t i = i0 + (mm << log2s);
#pragma unroll
        for (int t = 0; t < D; ++t) xv[mm][t] = __ldcs(X + (size_t)t * N + i);
        lw[mm] = __ldg(lvp + mm * gg.lv_mul);
      }
    }
    if (obs) {
#pragma unroll
      for (int mm = 0; mm < M; ++mm) lw[mm] += obs_log_term<D, KIND>(mp, y, xv[mm]) - muf;
    }

    // ---- group max, weights, integer prefix sums ----
    float mx = lw[0];
#pragma unroll
    for (int mm = 1; mm < M; ++mm) mx = fmaxf(mx, lw[mm]);
#pragma unroll
    for (int off = 1; off < G; off <<= 1) mx = fmaxf(mx, __shfl_xor_sync(FULL, mx, off));
    float s1 = 0.0f, s2 = 0.0f, sx[D];
    uint32_t P[M];
    uint32_t run = 0;
#pragma unroll
    for (int t = 0; t < D; ++t) sx[t] = 0.0f;
#pragma unroll
    for (int mm = 0; mm < M; ++mm) {
      const float e = exp_weight(lw[mm] - mx);         // the group maximum weighs exactly 1
      s1 += e;
      if (obs) {                                       // the step's summaries: this stage weights with g_n
        s2 = fmaf(e, e, s2);
#pragma unroll
        for (int t = 0; t < D; ++t) sx[t] = fmaf(e, xv[mm][t], sx[t]);
      }
      run += __float2uint_rz(e * 16777216.0f);
      P[mm] = run;
    }
    float s1_lane = s1;                              // my members' share (the group's, with G = 1)
#pragma unroll
    for (int off = 1; off < G; off <<= 1) s1 += __shfl_xor_sync(FULL, s1, off);
    bool redo = !(s1 >= 1.0f && s1 <= (float)A);
    // with several lanes per group the whole warp takes the rare path when any
    // group of it needs it, so that its shuffles stay converged (the other
    // groups recompute the same values)
    if constexpr (G > 1) redo = __any_sync(FULL, redo);
    if (redo) {
      // Rare path: a non-finite log-weight (NaN / +inf -> weight zero) or a group
      // whose weights are all zero.  Recompute the group with sanitised weights.
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
      for (int t = 0; t < D; ++t) sx[t] = 0.0f;
#pragma unroll
      for (int mm = 0; mm < M; ++mm) {
        const float e = live ? exp_weight(lw[mm] - mx) : 0.0f;
        s1 += e;
        s2 = fmaf(e, e, s2);
#pragma unroll
        for (int t = 0; t < D; ++t) sx[t] = fmaf(e, xv[mm][t], sx[t]);
        run += __float2uint_rz(e * 16777216.0f);
        P[mm] = run;
      }
      s1_lane = s1;
#pragma unroll
      for (int off = 1; off < G; off <<= 1) s1 += __shfl_xor_sync(FULL, s1, off);
      if (!live && j == 0) status |= kStatusZeroGroup;
    }
    uint32_t incl = run;
#pragma unroll
    for (int off = 1; off < G; off <<= 1) {
      const uint32_t v = __shfl_up_sync(FULL, incl, off, G);
      if ((int)j >= off) incl += v;
    }
    const uint32_t Q = (G > 1) ? __shfl_sync(FULL, incl, G - 1, G) : incl;
    const uint32_t excl = incl - run;
#pragma unroll
    for (int mm = 0; mm < M; ++mm) P[mm] += excl;
    if (c.prec) {                  // test output: the integer prefix sums the draws use
#pragma unroll
      for (int mm = 0; mm < M; ++mm) c.prec[i0 + (mm << log2s)] = P[mm];
    }
    if constexpr (M % 4 == 0) {
#pragma unroll
      for (int q = 0; q < M / 4; ++q)
        *reinterpret_cast<uint4*>(row + j * M + 4 * q) = make_uint4(P[4 * q], P[4 * q + 1], P[4 * q + 2], P[4 * q + 3]);
    } else {
#pragma unroll
      for (int mm = 0; mm < M; ++mm) row[j * M + mm] = P[mm];
    }
    if constexpr (PIV > 0 && G > 1) {   // one lane per group keeps its pivots in registers
#pragma unroll
      for (int mm = 0; mm < M; ++mm)
        if (((j * M + mm) & 3u) == 3u) row[A + ((j * M + mm) >> 2)] = P[mm];
    }
    if constexpr (!COAL) {                           // (the cooperative load filled the table)
#pragma unroll
      for (int mm = 0; mm < M; ++mm) {
        const uint32_t r = j * M + mm;
#pragma unroll
        for (int t = 0; t < D; ++t) col[(t * A + r) * LD] = __float_as_uint(xv[mm][t]);
      }
    }
    if constexpr (ADAPT) {           // per-particle carried weights; partial of the new stage weights
      const float lv_new = (Q != 0) ? (mx + logf(s1) - gg.log_a) : -INFINITY;
      if (contiguous) {
#pragma unroll
        for (int q = 0; q < M / 4; ++q)
          reinterpret_cast<float4*>(lV_out + i0)[q] = make_float4(lv_new, lv_new, lv_new, lv_new);
      } else {
#pragma unroll
        for (int mm = 0; mm < M; ++mm) lV_out[i0 + (mm << log2s)] = lv_new;
      }
      if (j == 0 && Q != 0) {
        float zx[D];
#pragma unroll
        for (int t = 0; t < D; ++t) zx[t] = 0.0f;
        merge_partial<D>(acc, accx, lv_new + gg.log_a, 1.0f, 1.0f / (float)A, zx);
      }
    } else {
      if (j == 0) lV_out[g] = (Q != 0) ? (mx + logf(s1) - gg.log_a) : -INFINITY;
      // every lane folds its own members' sums into its partial (the block's
      // fold adds the lanes up), so the group needs no cross-lane sums of them
      if (obs) merge_partial<D>(acc, accx, mx, s1_lane, s2, sx);
    }
    __syncwarp();

    // ---- per 4 members: random words (group-major counters), draws, gather, mutate, store ----
    const uint32_t pi0 = g * A + j * M;
    // Bucket pivots P_3, P_7, ... of a group held whole by one lane.
    uint32_t piv[PIV > 1 ? PIV - 1 : 1];
    if constexpr (G == 1 && PIV > 1) {
#pragma unroll
      for (int q = 0; q < PIV - 1; ++q) piv[q] = P[4 * q + 3];
    }
    float xo[M][D];
    uint32_t coff[M];          // ancestor's digit k
#pragma unroll
    for (int q4 = 0; q4 < (M + 3) / 4; ++q4) {
      constexpr int MQ = (M < 4) ? M : 4;             // members handled in this round
      uint32_t rw[MQ];
      {
        const uint4 w = philox4x32(make_uint4((pi0 >> 2) + q4, c.t, kPurposeResample, 0), rk);
        if constexpr (M >= 4) {
          rw[0] = w.x; rw[1] = w.y; rw[2] = w.z; rw[3] = w.w;
        } else {
#pragma unroll
          for (int mm = 0; mm < MQ; ++mm) {
            const uint32_t o = ((pi0 & 3u) + mm) & 3u;
            rw[mm] = o == 0 ? w.x : o == 1 ? w.y : o == 2 ? w.z : w.w;
          }
        }
      }
      float z[MQ * D];
      if (!mut) {
        // not the last stage of the step: no mutation, no propagation normals
      } else if constexpr ((MQ * D) % 4 == 0) {              // then the first normal number is a multiple of 4
        const uint32_t c0 = ((pi0 + 4 * q4) * D) >> 2;
#pragma unroll
        for (int b = 0; b < MQ * D / 4; ++b) {
          const uint4 w = philox4x32(make_uint4(c0 + b, n, kPurposePropagate, 0), rk);
          normals4_fast(w, z + 4 * b);
        }
      } else if constexpr (4 % (MQ * D) == 0) {       // 1 or 2 normals inside one block
        const uint32_t nu0 = pi0 * D;
        const uint4 w = philox4x32(make_uint4(nu0 >> 2, n, kPurposePropagate, 0), rk);
        float zz[4];
        normals4_fast(w, zz);
        const uint32_t off = nu0 & 3u;
#pragma unroll
        for (int q = 0; q < MQ * D; ++q) {
          const uint32_t o = off + q;
          z[q] = o == 0 ? zz[0] : o == 1 ? zz[1] : o == 2 ? zz[2] : zz[3];
        }
      } else {
        constexpr int NB = (MQ * D + 6) / 4;
        const uint32_t nu0 = (pi0 + 4 * q4) * D;
        float zz[4 * NB];
#pragma unroll
        for (int b = 0; b < NB; ++b) {
          const uint4 w = philox4x32(make_uint4((nu0 >> 2) + b, n, kPurposePropagate, 0), rk);
          normals4_fast(w, zz + 4 * b);
        }
        const uint32_t off = nu0 & 3u;
#pragma unroll
        for (int q = 0; q < MQ * D; ++q) z[q] = zz[off + q];
      }
#pragma unroll
      for (int mq = 0; mq < MQ; ++mq) {
        const int mm = 4 * q4 + mq;
        const uint32_t u = __umulhi(rw[mq], Q);       // floor(r Q / 2^32)
        // #{j : P_j <= u}: 4-ary, two levels.  Every P_j and u is below 2^29
        // (at most 32 members of at most 2^24 each), so P_j + ~u = P_j - u - 1
        // has its top bit set exactly when P_j <= u.
        const uint32_t nu = ~u;
        uint32_t c;
        if constexpr (A == 2) {
          c = (row[0] + nu) >> 31;
        } else {
          uint32_t b = 0;                              // bucket: pivots P_{4b+3} <= u
          if constexpr (G == 1 && PIV > 1) {
#pragma unroll
            for (int q = 0; q < PIV - 1; ++q) b += (piv[q] + nu) >> 31;
          } else if constexpr (PIV > 0) {
#pragma unroll
            for (int q = 0; q < PIV / 4 + (PIV % 4 ? 1 : 0); ++q) {
              const uint4 pv = *reinterpret_cast<const uint4*>(row + A + 4 * q);
              const uint32_t pvs[4] = {pv.x, pv.y, pv.z, pv.w};
#pragma unroll
              for (int e = 0; e < 4; ++e)
                if (4 * q + e < PIV - 1) b += (pvs[e] + nu) >> 31;
            }
          }
          const uint4 v = *reinterpret_cast<const uint4*>(row + 4 * b);
          c = 4 * b + ((v.x + nu) >> 31) + ((v.y + nu) >> 31) + ((v.z + nu) >> 31);
        }
        if (Q == 0) c = j * M + mm;                    // an all-zero group keeps its particles
        float xh[D];
#pragma unroll
        for (int t = 0; t < D; ++t) xh[t] = __uint_as_float(col[(t * A + c) * LD]);
        if (mut) {
          mutate<D, KIND>(mp, xh, z + mq * D, xo[mm]);
        } else {
#pragma unroll
          for (int t = 0; t < D; ++t) xo[mm][t] = xh[t];
        }
        coff[mm] = c;
      }
    }
    if constexpr (COAL) {
      __syncthreads();                               // every gather of the iteration is done
#pragma unroll
      for (int mm = 0; mm < M; ++mm)
#pragma unroll
        for (int t = 0; t < D; ++t) col[(t * A + j * M + mm) * LD] = __float_as_uint(xo[mm][t]);
      __syncthreads();
      GroupTile<D, A, GPB, LD>(batch, log2s, log2as).store(X, N, s_tab);
    } else if (contiguous) {
#pragma unroll
      for (int q = 0; q < M / 4; ++q)
#pragma unroll
        for (int t = 0; t < D; ++t)
          __stcs(reinterpret_cast<float4*>(X + (size_t)t * N + i0) + q,
                 make_float4(xo[4 * q][t], xo[4 * q + 1][t], xo[4 * q + 2][t], xo[4 * q + 3][t]));
    } else {
#pragma unroll
      for (int mm = 0; mm < M; ++mm)
#pragma unroll
        for (int t = 0; t < D; ++t) __stcs(X + (size_t)t * N + i0 + (mm << log2s), xo[mm][t]);
    }
    if (c.anc) {
#pragma unroll
      for (int mm = 0; mm < M; ++mm) c.anc[i0 + (mm << log2s)] = (int32_t)(ig + (coff[mm] << log2s));
    }
    __syncwarp();
  }
}

template <int D, int KIND, int A, int G, bool STAGED, bool ADAPT = false>
__device__ __forceinline__ void step_group_body(const StepParams& p, const GroupGeom& gg) {
  using LY = GroupLayout<D, A, G>;
  __shared__ __align__(16) uint32_t s_rows[LY::kRowWords];
  __shared__ uint32_t s_tab[LY::kTabWords];
  const ModelParams& mp = p.model;
  DevState* st = p.st;
  if constexpr (ADAPT) {
    if (st->skip) {
      if (!gg.last) return;                     // nothing to do, nothing to record
      adaptive_mutate_only<D, KIND>(p, p.geom[gg.k], st->n);
      return;
    }
  }
  const Sched sc = ADAPT ? Sched{st->n, st->n * (uint32_t)p.m + gg.j, gg.k, false, gg.last != 0}
                         : STAGED ? sched_of(p, st) : Sched{st->n, st->n, 0u, true, true};
  const uint32_t lvsel = ADAPT ? st->lvp : (sc.t & 1u);
  GroupCtx c;
  c.x = p.x;
  c.lV_in = p.lV[lvsel];
  c.lV_out = p.lV[lvsel ^ 1u];
  c.anc = p.anc;
  c.prec = p.prec;
  c.N = p.N;
  c.n = sc.n;
  c.t = sc.t;
  c.obs = (STAGED || ADAPT) ? sc.obs : true;
  c.mut = (STAGED || ADAPT) ? sc.mut : true;
  c.muf = st->mu_f;
#pragma unroll
  for (int q = 0; q < kMaxDim; ++q) c.y[q] = (q < mp.dy) ? p.y_ring[(sc.n % kRing) * mp.dy + q] : 0.0f;
  uint32_t status = 0;
  Partial acc{-INFINITY, 0.0f, 0.0f};
  float accx[D];
#pragma unroll
  for (int t = 0; t < D; ++t) accx[t] = 0.0f;
  group_iterations<D, KIND, A, G, ADAPT>(c, p.rk, mp, gg, blockIdx.x, gridDim.x, s_rows, s_tab, acc, accx, status);
  if constexpr (ADAPT) {
    adaptive_stage_finish<D>(p, acc, accx, status, lvsel, gg.k, gg.last != 0, sc.n);
  } else {
    finish_step<D>(p, acc, accx, sc, status, c.muf);
  }
}

template <int D, int KIND, int A, int G, bool STAGED, bool ADAPT = false>
__global__ void __launch_bounds__(kBlock) step_group_kernel(const __grid_constant__ StepParams p,
                                                           const __grid_constant__ GroupGeom gg) {
  step_group_body<D, KIND, A, G, STAGED, ADAPT>(p, gg);
}

// The same for d >= 5, with at most 80 registers so that three blocks share
// an SM (a few bytes of spills; with two blocks per SM the 8-D step was short
// of warps to hide its latencies).  The staged instantiations of radices below
// 16 keep the unbounded build: bounded, they spill about 160 bytes at d = 8.
template <int D, int KIND, int A, int G, bool STAGED, bool ADAPT = false>
__global__ void __launch_bounds__(kBlock, 3) step_group_kernel_d5(const __grid_constant__ StepParams p,
                                                                  const __grid_constant__ GroupGeom gg) {
  step_group_body<D, KIND, A, G, STAGED, ADAPT>(p, gg);
}

// SMALL: at most two members per lane, for populations too small to fill the
// GPU with the default split (shorter per-thread chains, more thread blocks).
template <int D, int KIND, int A, bool STAGED, bool ADAPT, bool SMALL>
inline const void* group_kernel_pick(int& G) {
  constexpr int MD = group_members_per_lane(A, D);
  constexpr int M = (SMALL && MD > 2) ? 2 : MD;
  constexpr int GG = A / M;
  G = GG;
  if constexpr (D >= 5 && (!STAGED || A >= 16))
    return reinterpret_cast<const void*>(&step_group_kernel_d5<D, KIND, A, GG, STAGED, ADAPT>);
  return reinterpret_cast<const void*>(&step_group_kernel<D, KIND, A, GG, STAGED, ADAPT>);
}

template <int D, int KIND, bool STAGED, bool ADAPT, bool SMALL>
inline const void* group_kernel_for_s(int a, int& G) {
  switch (a) {
    case 2: return group_kernel_pick<D, KIND, 2, STAGED, ADAPT, SMALL>(G);
    case 4: return group_kernel_pick<D, KIND, 4, STAGED, ADAPT, SMALL>(G);
    case 8: return group_kernel_pick<D, KIND, 8, STAGED, ADAPT, SMALL>(G);
    case 16: return group_kernel_pick<D, KIND, 16, STAGED, ADAPT, SMALL>(G);
    case 32: return group_kernel_pick<D, KIND, 32, STAGED, ADAPT, SMALL>(G);
    default: return nullptr;
  }
}

// staged: all stages per step; adapt: the fully adapted schedule (no rotation);
// small: the two-members-per-lane split (not for the adapted schedule)
template <int D, int KIND>
inline const void* group_kernel_for(int a, int& G, bool staged, bool adapt, bool small) {
  if (adapt) return group_kernel_for_s<D, KIND, false, true, false>(a, G);
  if (small)
    return staged ? group_kernel_for_s<D, KIND, true, false, true>(a, G)
                  : group_kernel_for_s<D, KIND, false, false, true>(a, G);
  return staged ? group_kernel_for_s<D, KIND, true, false, false>(a, G)
                : group_kernel_for_s<D, KIND, false, false, false>(a, G);
}

}  // namespace bfpf
