// step_global.cu - one time step of the bootstrap particle filter with GLOBAL
// multinomial resampling (Algorithm 1 + Algorithm 2 of Heine, Whiteley &
// Cemgil, arXiv 1812.01502: every particle may copy any other), the
// comparator of the butterfly filter, for N above the size one thread block
// resamples (radices = {N}).
//
// The draw follows the same integer rule as the butterfly kernels with one
// group of N members: q_i = floor(fp32 exp(lw_i - max lw) 2^32), P = inclusive
// prefix (64-bit), u_i = floor(r_i Q / 2^64) with a 64-bit uniform r_i from
// counter (i/2, n, 3, 0), ancestor = #{j : P_j <= u_i}.  Six phases in
// five launches (2 and 3 share one):
//   1. weights: lw_i to memory, block partials -> last block: likelihood
//      increment, mean, ESS, the global maximum and the one group's weight;
//      every draw (its index i) is also filed under its coarse bin (the top
//      cbits bits of r_i), counted per chunk of particles in shared memory so
//      that one global atomic reserves a run of slots per bin and chunk;
//   2. refine: the same per coarse bin, filing every draw under its bucket
//      b = top log2b bits of r_i (fixed capacity per bucket, an overflow list
//      behind it); r_i is recomputed from its counter, so a filed draw is
//      only its 4-byte index;
//   3. reduce: the integer weights q_i = floor(exp(lw_i - max lw) 2^32) summed
//      per tile of 4096 particles; the last block turns the tile sums into
//      tile offsets and the total Q;
//   4. scan: every tile's prefix sums P from its offset (loads and stores
//      staged through shared memory so that both are coalesced), and the
//      bucket edges: u is monotone in r, so bucket b covers the u interval
//      from u_b = floor(b 2^(64-log2b) Q / 2^64) to the next bucket's start,
//      and jb[b] = #{j : P_j <= u_b} is the particle j with
//      P_{j-1} <= u_b < P_j, found by the thread that holds it;
//   5. resolve: one block per bucket stages P[jb[b] .. jb[b+1]) and the
//      states x[jb[b] .. jb[b+1]] in shared memory, files the staged P_j into
//      equal bins of the bucket's u interval (a shared-memory histogram and
//      its scan: a guide table), counts P_j <= u_i there for every particle of
//      the bucket from its bin's first index (its index was filed by phases
//      1 and 2), gathers and mutates, and writes the particle's new state; a
//      bucket whose index range is longer than the staging buffer, and the
//      overflow list, search P in global memory (r_i again from its counter);
//   6. advance: one thread clears the overflow counts and advances n.
// No kernel waits on another block.
// Every particle's ancestor is #{j : P_j <= u_i} whatever the bucket layout:
// bucketing only decides where the count is taken.
#include <cfloat>

#include "bfpf_device.cuh"
#include "bfpf_epilogue.cuh"
#include "bfpf_global.cuh"
#include "bfpf_kernels.h"
#include "bfpf_model.cuh"

namespace bfpf {

namespace {

}  // namespace

// Bucket of a uniform: its top log2b bits.
__device__ __forceinline__ uint32_t bucket_of(unsigned long long r, uint32_t log2b) {
  return log2b ? (uint32_t)(r >> (64u - log2b)) : 0u;
}

// The 64-bit uniform of particle i's draw at step n: words (2(i%2), 2(i%2)+1)
// of the Philox block with counter (i/2, n, 3, 0).
__device__ __forceinline__ unsigned long long draw_uniform(const StepParams& p, uint32_t i, uint32_t n) {
  const uint4 w = philox4x32(make_uint4(i >> 1, n, kPurposeResampleWide, 0), p.rk);
  return (i & 1u) ? (((unsigned long long)w.w << 32) | w.z) : (((unsigned long long)w.y << 32) | w.x);
}

// File draw i straight into its bucket (or the overflow list): the path of the
// rare draws whose coarse bin was full.
__device__ __forceinline__ void file_direct(const StepParams& p, const GlobalParams& gp, uint32_t i, uint32_t n) {
  const uint32_t b = bucket_of(draw_uniform(p, i, n), gp.log2b);
  const uint32_t pos = atomicAdd(gp.cnt + b, 1u);
  if (pos < gp.cap) gp.slot[(size_t)b * gp.cap + pos] = i;
  else gp.ovf[atomicAdd(gp.cnt + gp.buckets, 1u)] = i;
}

// File one block's chunk of draws (thread t holds V of them: index i, bin,
// valid) into nbins bins of capacity cap: dst[bin * cap + pos] = i, pos
// reserved from gcnt[bin]; a draw whose bin is full goes to ovf[*ovf_cnt++].
// The chunk is counted per bin in shared memory, each non-empty bin reserves
// its run with one global atomic, and the draws are ordered by bin in shared
// memory first so that consecutive threads write consecutive slots.
// Shared memory: s_cnt[nbins], s_off[nbins], s_buf[kBlock * V] of {i, bin}.
template <int V>
__device__ __forceinline__ void file_chunk(const uint32_t (&i)[V], const uint32_t (&bin)[V], const bool (&valid)[V],
                                           uint32_t nbins, uint32_t* gcnt, uint32_t* dst, uint32_t cap,
                                           uint32_t* ovf_cnt, uint32_t* ovf, uint32_t* s_cnt, uint32_t* s_off,
                                           uint2* s_buf) {
  constexpr int NW = kBlock / 32;
  __shared__ uint32_t s_wsum[NW];
  __shared__ uint32_t s_total;
  const uint32_t tid = threadIdx.x, lane = tid & 31u, warp = tid >> 5;
  for (uint32_t k = tid; k < nbins; k += kBlock) s_cnt[k] = 0;
  __syncthreads();
  uint32_t rank[V];
#pragma unroll
  for (int j = 0; j < V; ++j) rank[j] = valid[j] ? atomicAdd(s_cnt + bin[j], 1u) : 0u;
  __syncthreads();
  // exclusive scan of the counts (E consecutive bins per thread) and one
  // global reservation per non-empty bin
  const uint32_t E = (nbins + kBlock - 1u) / kBlock;
  const uint32_t k0 = min(tid * E, nbins), k1 = min(k0 + E, nbins);
  uint32_t sum = 0;
  for (uint32_t k = k0; k < k1; ++k) sum += s_cnt[k];
  uint32_t incl = sum;
#pragma unroll
  for (int off = 1; off < 32; off <<= 1) {
    const uint32_t v = __shfl_up_sync(0xffffffffu, incl, off);
    if ((int)lane >= off) incl += v;
  }
  if (lane == 31) s_wsum[warp] = incl;
  __syncthreads();
  if (warp == 0) {
    uint32_t v = (lane < NW) ? s_wsum[lane] : 0u;
#pragma unroll
    for (int off = 1; off < NW; off <<= 1) {
      const uint32_t o = __shfl_up_sync(0xffffffffu, v, off);
      if ((int)lane >= off) v += o;
    }
    if (lane < NW) s_wsum[lane] = v;
    if (lane == NW - 1) s_total = v;
  }
  __syncthreads();
  uint32_t run = (warp ? s_wsum[warp - 1] : 0u) + incl - sum;
  for (uint32_t k = k0; k < k1; ++k) {
    const uint32_t c = s_cnt[k];
    s_off[k] = run;
    run += c;
    s_cnt[k] = c ? atomicAdd(gcnt + k, c) : 0u;   // the run's first slot in the bin
  }
  __syncthreads();
#pragma unroll
  for (int j = 0; j < V; ++j)
    if (valid[j]) s_buf[s_off[bin[j]] + rank[j]] = make_uint2(i[j], bin[j]);
  __syncthreads();
  const uint32_t total = s_total;
  for (uint32_t k = tid; k < total; k += kBlock) {
    const uint2 e = s_buf[k];
    const uint32_t b = e.y;
    const uint32_t pos = s_cnt[b] + (k - s_off[b]);
    if (pos < cap) dst[(size_t)b * cap + pos] = e.x;
    else ovf[atomicAdd(ovf_cnt, 1u)] = e.x;
  }
  __syncthreads();                                 // the caller reuses the shared buffers
}

// Weights and the coarse filing.  The particles are taken in chunks of
// kBlock * V consecutive indices (V per thread); every draw of a chunk is
// filed under its coarse bin, the top cbits bits of r_i.
template <int D, int KIND>
__global__ void __launch_bounds__(kBlock) global_weight_kernel(const __grid_constant__ StepParams p,
                                                              const __grid_constant__ GlobalParams gp) {
  constexpr int V = global_weight_vec(D);
  constexpr uint32_t CH = kBlock * V;
  extern __shared__ __align__(16) unsigned char s_dyn[];
  uint2* const s_buf = reinterpret_cast<uint2*>(s_dyn);                 // [CH]
  uint32_t* const s_cnt = reinterpret_cast<uint32_t*>(s_buf + CH);      // [2^cbits]
  const ModelParams& mp = p.model;
  DevState* st = p.st;
  const uint32_t n = st->n;
  const float* __restrict__ X = gp.xbuf[n & 1u];
  const float lv = p.lV[n & 1u][0];            // one group: one carried weight
  const float muf = st->mu_f;
  const uint32_t N = p.N;
  const uint32_t tid = threadIdx.x;
  float y[kMaxDim];
#pragma unroll
  for (int q = 0; q < kMaxDim; ++q) y[q] = (q < mp.dy) ? p.y_ring[(n % kRing) * mp.dy + q] : 0.0f;
  uint32_t status = 0;
  Partial acc{-INFINITY, 0.0f, 0.0f};
  float accx[D];
#pragma unroll
  for (int t = 0; t < D; ++t) accx[t] = 0.0f;
  const uint32_t cbits = gp.cbits, nbins = 1u << cbits;
  uint32_t* const s_off = s_cnt + nbins;                                 // [2^cbits]
  const bool vec = (N % 4u) == 0u;
  const uint32_t nchunk = (N + CH - 1u) / CH;
  for (uint32_t ch = blockIdx.x; ch < nchunk; ch += gridDim.x) {   // block-uniform loop
    const uint32_t i0 = ch * CH + tid * V;
    const bool full = vec && i0 + V <= N;
    float xv[V][D];
    float lw[V];
    if (full) {
#pragma unroll
      for (int t = 0; t < D; ++t) {
#pragma unroll
        for (int h = 0; h < V / 4; ++h) {
          const float4 v = __ldcs(reinterpret_cast<const float4*>(X + (size_t)t * N + i0) + h);
          xv[4 * h][t] = v.x; xv[4 * h + 1][t] = v.y; xv[4 * h + 2][t] = v.z; xv[4 * h + 3][t] = v.w;
        }
      }
    } else {
#pragma unroll
      for (int j = 0; j < V; ++j)
#pragma unroll
        for (int t = 0; t < D; ++t) xv[j][t] = (i0 + j < N) ? __ldcs(X + (size_t)t * N + i0 + j) : 0.0f;
    }
#pragma unroll
    for (int j = 0; j < V; ++j)
      lw[j] = (i0 + j < N) ? sanitize_logweight(lv + obs_log_term<D, KIND>(mp, y, xv[j]) - muf, status) : -INFINITY;
    if (full) {
#pragma unroll
      for (int h = 0; h < V / 4; ++h)
        reinterpret_cast<float4*>(gp.lw + i0)[h] = make_float4(lw[4 * h], lw[4 * h + 1], lw[4 * h + 2], lw[4 * h + 3]);
    } else {
#pragma unroll
      for (int j = 0; j < V; ++j)
        if (i0 + j < N) gp.lw[i0 + j] = lw[j];
    }
#pragma unroll
    for (int h = 0; h < V / 4; ++h) {            // one partial merge per four particles
      const float m4 = fmaxf(fmaxf(lw[4 * h], lw[4 * h + 1]), fmaxf(lw[4 * h + 2], lw[4 * h + 3]));
      if (m4 != -INFINITY) {
        float s1 = 0.0f, s2 = 0.0f, sx[D];
#pragma unroll
        for (int t = 0; t < D; ++t) sx[t] = 0.0f;
#pragma unroll
        for (int j = 4 * h; j < 4 * h + 4; ++j) {
          const float e = exp_weight(lw[j] - m4);   // 0 for a log-weight of -inf
          s1 += e;
          s2 = fmaf(e, e, s2);
#pragma unroll
          for (int t = 0; t < D; ++t) sx[t] = fmaf(e, xv[j][t], sx[t]);
        }
        merge_partial<D>(acc, accx, m4, s1, s2, sx);
      }
    }
    // uniforms (pairs of particles share a Philox block) and their coarse bins
    uint32_t ii[V], cb[V];
    bool valid[V];
#pragma unroll
    for (int h = 0; h < V / 2; ++h) {
      const uint4 w = philox4x32(make_uint4(i0 / 2u + h, n, kPurposeResampleWide, 0), p.rk);
      cb[2 * h] = bucket_of(((unsigned long long)w.y << 32) | w.x, cbits);
      cb[2 * h + 1] = bucket_of(((unsigned long long)w.w << 32) | w.z, cbits);
    }
#pragma unroll
    for (int j = 0; j < V; ++j) {
      ii[j] = i0 + j;
      valid[j] = i0 + j < N;
    }
    file_chunk<V>(ii, cb, valid, nbins, gp.ccnt, gp.cslot, gp.ccap, gp.ccnt + nbins, gp.covf, s_cnt, s_off, s_buf);
  }
  const Sched sc{n, n, 0u, true, true};   // one digit (m = 1): every step is one whole stage
  finish_step<D, false>(p, acc, accx, sc, status, muf, p.lV[(n & 1u) ^ 1u]);
}

// Fine filing: block (coarse bin cb, segment sg) takes kRefineSeg entries of
// the bin and files each under its bucket (the next log2b - cbits bits of r),
// the same way.  Draws of the coarse overflow list are filed one by one.
__device__ __forceinline__ void refine_body(const StepParams& p, const GlobalParams& gp, uint32_t blk, uint32_t nblk) {
  extern __shared__ __align__(16) unsigned char s_dyn[];
  uint2* const s_buf = reinterpret_cast<uint2*>(s_dyn);                 // [kRefineSeg]
  uint32_t* const s_cnt = reinterpret_cast<uint32_t*>(s_buf + kRefineSeg);
  const uint32_t tid = threadIdx.x;
  const uint32_t n = p.st->n;
  const uint32_t cbits = gp.cbits, fbits = gp.log2b - cbits, nfine = 1u << fbits;
  uint32_t* const s_off = s_cnt + nfine;
  const uint32_t cb = blk / gp.nseg, sg = blk % gp.nseg;
  const uint32_t cfill = min(__ldcg(gp.ccnt + cb), gp.ccap);
  const uint32_t e0 = sg * kRefineSeg;
  if (e0 < cfill) {                                // block-uniform
    const size_t cbase = (size_t)cb * gp.ccap;
    uint32_t ii[kRefineItems], fb[kRefineItems];
    bool valid[kRefineItems];
#pragma unroll
    for (int q = 0; q < kRefineItems; ++q) {
      const uint32_t e = e0 + q * kBlock + tid;
      valid[q] = e < cfill;
      ii[q] = valid[q] ? __ldcs(gp.cslot + cbase + e) : 0u;
    }
#pragma unroll
    for (int q = 0; q < kRefineItems; ++q)
      fb[q] = valid[q] ? (bucket_of(draw_uniform(p, ii[q], n), gp.log2b) & (nfine - 1u)) : 0u;
    const size_t b0 = (size_t)cb << fbits;         // this coarse bin's first bucket
    file_chunk<kRefineItems>(ii, fb, valid, nfine, gp.cnt + b0, gp.slot + b0 * gp.cap, gp.cap, gp.cnt + gp.buckets,
                             gp.ovf, s_cnt, s_off, s_buf);
  }
  const uint32_t nco = __ldcg(gp.ccnt + (1u << cbits));
  for (uint32_t e = blk * kBlock + tid; e < nco; e += nblk * kBlock)
    file_direct(p, gp, __ldcg(gp.covf + e), n);
}

// floor(e 2^32) for e in [0, 1]: below 1, e 2^32 < 2^32 (the largest float
// below 1 is 1 - 2^-24) and the 32-bit round-toward-zero conversion is exact;
// e = 1 (the population's maximum) weighs 2^32.
__device__ __forceinline__ unsigned long long floor_scaled_2p32(float e) {
  return e >= 1.0f ? (1ull << 32) : (unsigned long long)__float2uint_rz(e * 4294967296.0f);
}

// Integer weight of log-weight lw, with the population's maximum log-weight
// gmax weighing exactly 2^32 (the same on both scan passes).
__device__ __forceinline__ unsigned long long global_qweight(float lw, float gmax) {
  return floor_scaled_2p32(exp_weight(lw - gmax));
}

// 3a. reduce: the sum of the integer weights of every scan tile; the last
// block to finish turns the tile sums into tile offsets (their exclusive
// prefix sums) and the total Q, toff[nscan].
__device__ __forceinline__ void reduce_body(const StepParams& p, const GlobalParams& gp, uint32_t blk) {
  __shared__ unsigned long long s_warp[kBlock / 32];
  __shared__ bool s_last;
  const uint32_t N = p.N;
  const uint32_t tid = threadIdx.x, lane = tid & 31u, warp = tid >> 5;
  const float gmax = p.st->gmax;
  const uint32_t tbase = blk * kScanTile;
  unsigned long long sum = 0;
  if (gmax != -INFINITY) {
    const bool vec = (N % 4u) == 0u;
#pragma unroll
    for (int k = 0; k < kScanItems / 4; ++k) {     // the scan pass reads the tile again, from L2
      const uint32_t i4 = tbase + 4u * (k * kBlock + tid);
      if (vec && i4 + 4u <= N) {
        const float4 v = __ldcg(reinterpret_cast<const float4*>(gp.lw + i4));
        sum += global_qweight(v.x, gmax) + global_qweight(v.y, gmax) + global_qweight(v.z, gmax) +
               global_qweight(v.w, gmax);
      } else {
#pragma unroll
        for (int e = 0; e < 4; ++e)
          if (i4 + e < N) sum += global_qweight(__ldcg(gp.lw + i4 + e), gmax);
      }
    }
  }
#pragma unroll
  for (int off = 16; off; off >>= 1) sum += __shfl_xor_sync(0xffffffffu, sum, off);
  if (lane == 0) s_warp[warp] = sum;
  __syncthreads();
  if (tid == 0) {
    unsigned long long tsum = 0;
#pragma unroll
    for (int w = 0; w < kBlock / 32; ++w) tsum += s_warp[w];
    gp.tsum[blk] = tsum;
    __threadfence();
    s_last = atomicAdd(gp.done, 1u) == gp.nscan - 1u;
  }
  __syncthreads();
  if (!s_last) return;
  // last block: exclusive prefix of the tile sums, E consecutive tiles per thread
  __threadfence();
  const uint32_t nt = gp.nscan;
  const uint32_t E = (nt + kBlock - 1u) / kBlock;
  const uint32_t k0 = min(tid * E, nt), k1 = min(k0 + E, nt);
  unsigned long long tot = 0;
  for (uint32_t k = k0; k < k1; ++k) tot += __ldcg(gp.tsum + k);   // E consecutive sums: one line per thread
  unsigned long long incl = tot;
#pragma unroll
  for (int off = 1; off < 32; off <<= 1) {
    const unsigned long long v = __shfl_up_sync(0xffffffffu, incl, off);
    if ((int)lane >= off) incl += v;
  }
  __syncthreads();                                 // s_warp is reused
  if (lane == 31) s_warp[warp] = incl;
  __syncthreads();
  unsigned long long run = incl - tot;
  for (int w = 0; w < (int)warp; ++w) run += s_warp[w];
  for (uint32_t k = k0; k < k1; ++k) {
    gp.toff[k] = run;
    run += __ldcg(gp.tsum + k);
  }
  if (tid == kBlock - 1) {
    gp.toff[nt] = run;                             // Q: the last thread's running sum ends at the total
    *gp.done = 0;                                  // ready for the next step
  }
}

// Kernels 2 and 3 in one launch: the refine blocks are bound by instruction
// issue, the reduce blocks by memory, so the two share the SMs.  The first
// nred blocks reduce (none when one tile holds every particle: the scan then
// takes its own total), the rest refine.
__global__ void __launch_bounds__(kBlock) global_refine_reduce_kernel(const __grid_constant__ StepParams p,
                                                                     const __grid_constant__ GlobalParams gp) {
  const uint32_t nred = gp.nscan > 1u ? gp.nscan : 0u;
  if (blockIdx.x < nred) reduce_body(p, gp, blockIdx.x);
  else refine_body(p, gp, blockIdx.x - nred, gridDim.x - nred);
}

// Bucket edge b: the smallest u of bucket b, floor(b 2^(64-log2b) Q / 2^64);
// Q itself for b = buckets (a bound above every u).
__device__ __forceinline__ unsigned long long edge_u(uint32_t b, unsigned long long Q, uint32_t log2b,
                                                     uint32_t buckets) {
  if (b >= buckets) return Q;
  return log2b ? __umul64hi((unsigned long long)b << (64u - log2b), Q) : 0ull;
}

// #{b in [0, buckets) : edge_u(b) < v} for 0 <= v <= Q: a float estimate of
// ceil(v buckets / Q), corrected to the exact count (the edges are
// non-decreasing in b, so each loop only moves toward the answer).
__device__ __forceinline__ uint32_t edges_below(unsigned long long v, unsigned long long Q, uint32_t log2b,
                                                uint32_t buckets) {
  if (v == 0) return 0;
  const float est = ceilf(__ull2float_rn(v) / __ull2float_rn(Q) * (float)buckets);
  uint32_t b = (uint32_t)fminf(fmaxf(est, 0.0f), (float)buckets);
  while (b > 0 && edge_u(b - 1u, Q, log2b, buckets) >= v) --b;
  while (b < buckets && edge_u(b, Q, log2b, buckets) < v) ++b;
  return b;
}

// 3b. scan: the prefix sums of one tile from its offset (no waiting on other
// tiles: the offsets come from the reduce pass), and the bucket edges that
// fall in the tile.  Edge b belongs to the particle j with P_{j-1} <= u_b < P_j
// (P_{-1} = 0), and then jb[b] = #{P <= u_b} = j; the last edge, u = Q - 1,
// likewise.  Loads and stores of the tile are staged through shared memory so
// that both are coalesced.
__global__ void __launch_bounds__(kBlock, 4) global_scan_kernel(const __grid_constant__ StepParams p,
                                                            const __grid_constant__ GlobalParams gp) {
  // the tile's log-weights, then its prefix sums, one padding word every 32
  // floats / 16 doubles so that thread-contiguous accesses hit distinct banks
  __shared__ unsigned long long s_buf[kScanTile + kScanTile / 16];
  __shared__ unsigned long long s_warp[kBlock / 32];
  DevState* st = p.st;
  const uint32_t N = p.N;
  const float gmax = st->gmax;
  const uint32_t tid = threadIdx.x, lane = tid & 31u, warp = tid >> 5;
  const uint32_t tile = blockIdx.x;
  const uint32_t tbase = tile * kScanTile;
  float* const s_f = reinterpret_cast<float*>(s_buf);
  const bool vec = (N % 4u) == 0u;
#pragma unroll
  for (int k = 0; k < kScanItems / 4; ++k) {      // coalesced load of the tile
    const uint32_t idx = 4u * (k * kBlock + tid);
    float v[4];
    if (vec && tbase + idx + 4u <= N) {
      const float4 w = __ldcs(reinterpret_cast<const float4*>(gp.lw + tbase + idx));
      v[0] = w.x; v[1] = w.y; v[2] = w.z; v[3] = w.w;
    } else {
#pragma unroll
      for (int e = 0; e < 4; ++e) v[e] = (tbase + idx + e < N) ? __ldcs(gp.lw + tbase + idx + e) : -INFINITY;
    }
#pragma unroll
    for (int e = 0; e < 4; ++e) s_f[idx + e + ((idx + e) >> 5)] = v[e];
  }
  __syncthreads();
  // integer weights of my 16 consecutive particles and their running sums
  unsigned long long run[kScanItems];
  unsigned long long tot = 0;
  if (tid == 0 && tile == 0 && gmax == -INFINITY) atomicOr(&st->status, kStatusZeroGroup);
#pragma unroll
  for (int q = 0; q < kScanItems; ++q) {
    const uint32_t idx = tid * kScanItems + q;
    const float lw = s_f[idx + (idx >> 5)];
    tot += (gmax != -INFINITY) ? global_qweight(lw, gmax) : 0ull;
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
  __syncthreads();                                 // (also: every thread has read its log-weights)
  // one tile: its own offset (0) and total; else both from the reduce pass
  const bool single = gp.nscan == 1u;
  unsigned long long lo = (single ? 0ull : __ldcg(gp.toff + tile)) + incl - tot;   // P before my first particle
  unsigned long long btot = 0;
#pragma unroll
  for (int w = 0; w < kBlock / 32; ++w) {
    if (w < (int)warp) lo += s_warp[w];
    btot += s_warp[w];
  }
#pragma unroll
  for (int q = 0; q < kScanItems; ++q) {
    const uint32_t idx = tid * kScanItems + q;
    s_buf[idx + (idx >> 4)] = lo + run[q];
  }
  __syncthreads();
#pragma unroll
  for (int k = 0; k < kScanItems; ++k) {          // coalesced store of the tile
    const uint32_t idx = k * kBlock + tid;
    if (tbase + idx < N) gp.P[tbase + idx] = s_buf[idx + (idx >> 4)];
  }
  // bucket edges u_b in [lo, hi): usually none in one thread's 16 particles
  const unsigned long long Q = single ? btot : __ldcg(gp.toff + gp.nscan);
  const uint32_t j0 = tbase + tid * kScanItems;
  if (Q != 0) {
    const unsigned long long hi = lo + tot;
    if (hi > lo) {
      const uint32_t L = gp.log2b, B = gp.buckets;
      const uint32_t be = edges_below(hi, Q, L, B);
      for (uint32_t b = edges_below(lo, Q, L, B); b < be; ++b) {
        const unsigned long long u = edge_u(b, Q, L, B);
        uint32_t c = 0;
        for (int q = 0; q < kScanItems; ++q) {
          const uint32_t idx = tid * kScanItems + q;
          c += (s_buf[idx + (idx >> 4)] <= u) ? 1u : 0u;
        }
        gp.jb[b] = j0 + c;
      }
      if (lo <= Q - 1u && Q - 1u < hi) {           // the last edge
        uint32_t c = 0;
        for (int q = 0; q < kScanItems; ++q) {
          const uint32_t idx = tid * kScanItems + q;
          c += (s_buf[idx + (idx >> 4)] <= Q - 1u) ? 1u : 0u;
        }
        gp.jb[B] = j0 + c;
      }
    }
  } else {                                         // no weight anywhere: every edge is 0
    for (uint32_t b = tile * kBlock + tid; b <= gp.buckets; b += gridDim.x * kBlock) gp.jb[b] = 0;
  }
}

static_assert(kGuideBins % kBlock == 0, "guide bins are scanned kGuideBins / kBlock per thread");

// Bin of a value v of the bucket's u interval [ulo, ulo + W] among the
// kGuideBins bins of the guide table: (v - ulo) >> shift, with the shift that
// makes W >> shift < kGuideBins.  A monotone function of v, which is all the
// exact count below relies on.
__device__ __forceinline__ uint32_t guide_bin(unsigned long long v, unsigned long long ulo, uint32_t shift) {
  return (uint32_t)((v - ulo) >> shift);
}
constexpr uint32_t kGuideLog2 = 10;
static_assert((1u << kGuideLog2) == kGuideBins, "guide bins: a power of two");

// Ancestor, gather and mutation of particle i with uniform r.  Its ancestor
// lies in [lo, lo + len]: ancestor = lo + #{j in [lo, lo + len) : P_j <= u},
// counted in the staged copy (sP, with the guide table sG[t] = #{staged P_j
// of a bin before t}; states sX with row stride SC + 1) or in global memory.
// In the staged copy every P_j of a bin before u's is <= u and every P_j of a
// later bin is > u, so the count starts at sG[bin(u)] and scans u's own bin.
template <int D, int KIND>
__device__ __forceinline__ void resolve_draw(const StepParams& p, const GlobalParams& gp, const float* __restrict__ Xin,
                                             float* __restrict__ Xout, unsigned long long Q, uint32_t n, uint32_t i,
                                             bool staged, uint32_t lo, uint32_t len,
                                             const unsigned long long* sP, const float* sX, const uint32_t* sG,
                                             unsigned long long ulo, uint32_t gshift) {
  constexpr uint32_t SC = global_stage_alloc(D);
  const uint32_t N = p.N;
  const unsigned long long r = draw_uniform(p, i, n);
  uint32_t anc = i;                                // an all-zero population keeps its particles
  float xh[D];
  if (Q != 0) {
    const unsigned long long u = __umul64hi(r, Q);
    uint32_t c = 0;
    if (staged) {
      c = sG[guide_bin(u, ulo, gshift)];
      while (c < len && sP[c] <= u) ++c;
#pragma unroll
      for (int t = 0; t < D; ++t) xh[t] = sX[t * (SC + 1u) + c];
    } else {
      const unsigned long long* Pg = gp.P + lo;
      for (uint32_t stp = len ? (1u << (31 - __clz(len))) : 0u; stp; stp >>= 1)
        if (c + stp <= len && __ldcg(Pg + c + stp - 1u) <= u) c += stp;
#pragma unroll
      for (int t = 0; t < D; ++t) xh[t] = __ldg(Xin + (size_t)t * N + lo + c);
    }
    anc = lo + c;
  } else {
#pragma unroll
    for (int t = 0; t < D; ++t) xh[t] = __ldg(Xin + (size_t)t * N + i);
  }
  // propagation normals nu = i d + t: Philox block nu / 4, Box-Muller pairs of its words
  float z[D];
  {
    uint4 w = make_uint4(0, 0, 0, 0);
    float z0 = 0.0f, z1 = 0.0f;
    const uint32_t nu0 = i * D;
#pragma unroll
    for (int t = 0; t < D; ++t) {
      const uint32_t nu = nu0 + t;
      if (t == 0 || (nu & 3u) == 0u) w = philox4x32(make_uint4(nu >> 2, n, kPurposePropagate, 0), p.rk);
      if (t == 0 || (nu & 1u) == 0u) box_muller_fast((nu & 2u) ? w.z : w.x, (nu & 2u) ? w.w : w.y, z0, z1);
      z[t] = (nu & 1u) ? z1 : z0;
    }
  }
  float xo[D];
  mutate<D, KIND>(p.model, xh, z, xo);
#pragma unroll
  for (int t = 0; t < D; ++t) Xout[(size_t)t * N + i] = xo[t];
  if (p.anc) p.anc[i] = (int32_t)anc;
}

// One block per bucket (grid = buckets), then the overflow list grid-stride.
template <int D, int KIND>
__global__ void __launch_bounds__(kBlock) global_resolve_kernel(const __grid_constant__ StepParams p,
                                                               const __grid_constant__ GlobalParams gp) {
  constexpr uint32_t SC = global_stage_alloc(D);
  extern __shared__ __align__(16) unsigned char s_dyn[];
  unsigned long long* const sP = reinterpret_cast<unsigned long long*>(s_dyn);   // [SC]
  float* const sX = reinterpret_cast<float*>(sP + SC);                            // [D][SC + 1]
  uint32_t* const sG = reinterpret_cast<uint32_t*>(sX + D * (SC + 1u));           // [kGuideBins]
  __shared__ uint32_t s_wsum[kBlock / 32];
  DevState* st = p.st;
  const uint32_t n = st->n;
  const uint32_t N = p.N;
  const uint32_t tid = threadIdx.x, b = blockIdx.x;
  const float* __restrict__ Xin = gp.xbuf[n & 1u];
  float* __restrict__ Xout = gp.xbuf[(n & 1u) ^ 1u];
  const unsigned long long Q = __ldcg(gp.P + (N - 1u));
  const uint32_t filled = min(__ldcg(gp.cnt + b), gp.cap);
  const uint32_t lo = __ldcg(gp.jb + b);
  const uint32_t len = __ldcg(gp.jb + b + 1u) - lo;
  const bool staged = Q != 0 && len < gp.stage_cap;
  const size_t s0 = (size_t)b * gp.cap;
  // the first kPre draws of every thread are loaded with the fill count and
  // the bucket edges (slots past the fill count hold stale indices, never
  // used), so that the slot, edge and staging latencies overlap
  constexpr int kPre = 4;
  uint32_t pre[kPre];
#pragma unroll
  for (int k = 0; k < kPre; ++k) {
    const uint32_t e = tid + k * kBlock;
    pre[k] = e < gp.cap ? __ldcs(gp.slot + s0 + e) : 0u;
  }
  // the bucket's u interval [ulo, uhi] and the shift of its guide bins
  const unsigned long long ulo = (gp.log2b && b) ? __umul64hi((unsigned long long)b << (64u - gp.log2b), Q) : 0ull;
  const unsigned long long uhi = (b + 1u < gp.buckets) ? __umul64hi((unsigned long long)(b + 1u) << (64u - gp.log2b), Q) : Q;
  const uint32_t wbits = 64u - (uint32_t)__clzll(uhi - ulo);    // bit length of the interval's width
  const uint32_t gshift = wbits > kGuideLog2 ? wbits - kGuideLog2 : 0u;
  if (staged) {
    for (uint32_t j = tid; j < len; j += kBlock) sP[j] = __ldcg(gp.P + lo + j);
#pragma unroll
    for (int t = 0; t < D; ++t)
      for (uint32_t j = tid; j <= len; j += kBlock) sX[t * (SC + 1u) + j] = __ldg(Xin + (size_t)t * N + lo + j);
    for (uint32_t k = tid; k < kGuideBins; k += kBlock) sG[k] = 0u;
  }
  __syncthreads();
  if (staged) {                                    // guide table: histogram of the bins, then its scan
    for (uint32_t j = tid; j < len; j += kBlock) atomicAdd(sG + guide_bin(sP[j], ulo, gshift), 1u);
    __syncthreads();
    constexpr uint32_t E = kGuideBins / kBlock;    // consecutive bins per thread
    uint32_t cnt[E], sum = 0;
#pragma unroll
    for (uint32_t e = 0; e < E; ++e) {
      cnt[e] = sG[tid * E + e];
      sum += cnt[e];
    }
    const uint32_t lane = tid & 31u, warp = tid >> 5;
    uint32_t incl = sum;
#pragma unroll
    for (int off = 1; off < 32; off <<= 1) {
      const uint32_t v = __shfl_up_sync(0xffffffffu, incl, off);
      if ((int)lane >= off) incl += v;
    }
    if (lane == 31) s_wsum[warp] = incl;
    __syncthreads();
    uint32_t base = incl - sum;
    for (uint32_t w = 0; w < warp; ++w) base += s_wsum[w];
#pragma unroll
    for (uint32_t e = 0; e < E; ++e) {
      sG[tid * E + e] = base;
      base += cnt[e];
    }
  }
  __syncthreads();
  if (tid == 0) {                                  // zero the counters for the next step
    gp.cnt[b] = 0;                                 // (read above by every thread)
    if (b < (1u << gp.cbits)) gp.ccnt[b] = 0;
  }
#pragma unroll
  for (int k = 0; k < kPre; ++k)
    if (tid + k * kBlock < filled) resolve_draw<D, KIND>(p, gp, Xin, Xout, Q, n, pre[k], staged, lo, len, sP, sX, sG, ulo, gshift);
  for (uint32_t e = tid + kPre * kBlock; e < filled; e += kBlock) {
    const uint32_t i = __ldcs(gp.slot + s0 + e);
    resolve_draw<D, KIND>(p, gp, Xin, Xout, Q, n, i, staged, lo, len, sP, sX, sG, ulo, gshift);
  }
  const uint32_t nov = __ldcg(gp.cnt + gp.buckets);
  for (uint32_t e = b * kBlock + tid; e < nov; e += gridDim.x * kBlock) {
    const uint32_t i = __ldcg(gp.ovf + e);
    resolve_draw<D, KIND>(p, gp, Xin, Xout, Q, n, i, false, 0u, N, sP, sX, sG, 0ull, 0u);
  }
}

// End of the step (one thread, after the resolve kernel): clear the overflow
// counts and advance the step counter.  A separate launch, so that no resolve
// block waits for its scattered stores before it retires.
__global__ void global_advance_kernel(const __grid_constant__ StepParams p, const __grid_constant__ GlobalParams gp) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  gp.cnt[gp.buckets] = 0;
  gp.ccnt[1u << gp.cbits] = 0;
  p.st->n = p.st->n + 1;
}

template <int D, int KIND>
static void fill_global(GlobalKernels& gk) {
  gk.weight = reinterpret_cast<const void*>(&global_weight_kernel<D, KIND>);
  gk.scan = reinterpret_cast<const void*>(&global_scan_kernel);
  gk.refine_reduce = reinterpret_cast<const void*>(&global_refine_reduce_kernel);
  gk.resolve = reinterpret_cast<const void*>(&global_resolve_kernel<D, KIND>);
  gk.advance = reinterpret_cast<const void*>(&global_advance_kernel);
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
