// bfpf_global.cuh - buffers and sizes of the global-resampling path
// (radices = {N}, N above one thread block): Algorithm 2 of Heine, Whiteley &
// Cemgil, arXiv 1812.01502, over all N particles.
#pragma once

#include <cstdint>

#include "bfpf_device.cuh"

namespace bfpf {

// Buffers of the global-resampling path (m = 1, N > kMaxCtaRadix).
// The draws are resolved by bucket: particle i goes to bucket b = the top
// log2b bits of its 64-bit uniform r_i, so every bucket covers one interval of
// u = floor(r Q / 2^64) and hence one index range [jb[b], jb[b+1]] of
// ancestors, which is staged in shared memory.
struct GlobalParams {
  float* xbuf[2];                 // states, ping-pong by time-step parity (gather is random)
  float* lw;                      // [N] log-weights of the step
  unsigned long long* P;          // [N] inclusive prefix sums of the integer weights
  unsigned long long* tsum;       // [nscan] integer-weight sum of every scan tile
  unsigned long long* toff;       // [nscan + 1] tile offsets (exclusive prefix of tsum); toff[nscan] = Q
  uint32_t* done;                 // blocks of the reduce pass finished (zero between steps)
  // A filed draw is its particle index i: the uniform r_i is a function of the
  // counter (i/2, n, 3, 0), recomputed wherever it is needed.
  uint32_t* slot;                 // [buckets][cap] draws filed by bucket
  uint32_t* cnt;                  // [buckets + 1] fill counts (zero between steps); last: overflow count
  uint32_t* cslot;                // [2^cbits][ccap] draws filed by coarse bin (top cbits bits of r)
  uint32_t* ccnt;                 // [2^cbits + 1] coarse fill counts (zero between steps); last: overflow count
  uint32_t* covf;                 // [N] draws whose coarse bin was full
  uint32_t* ovf;                  // [N] draws whose bucket was full
  uint32_t* jb;                   // [buckets + 1] jb[b] = #{j : P_j <= lowest u of bucket b}
  uint32_t nscan;                 // scan tiles of kScanTile particles
  uint32_t log2b, buckets;        // buckets = 2^log2b
  uint32_t cbits, ccap, nseg;     // coarse bins 2^cbits (cbits <= 12, log2b - cbits <= 12), their
                                  // capacity, refine blocks per coarse bin
  uint32_t cap;                   // slots per bucket
  uint32_t stage_cap;             // longest index range staged in shared memory (<= global_stage_alloc(d))
};

// Consecutive particles per thread of the global weight kernel.
__host__ __device__ constexpr int global_weight_vec(int d) { return d <= 2 ? 8 : 4; }
// Indices of P (and states) the resolve kernel's shared-memory buffer holds.
__host__ __device__ constexpr uint32_t global_stage_alloc(int d) { return d <= 2 ? 2048u : 1024u; }

// Bins of the resolve kernel's guide table over a bucket's u interval.
constexpr uint32_t kGuideBins = 1024;

constexpr int kScanItems = 16;
constexpr uint32_t kMaxCoarse = 4096;                          // coarse bins and buckets per coarse bin
constexpr int kRefineItems = 8;                                // draws per thread of a refine block
constexpr uint32_t kRefineSeg = kBlock * kRefineItems;        // draws per refine block
constexpr uint32_t kScanTile = kBlock * kScanItems;   // 4096 particles

}  // namespace bfpf
