// step_pass_layout.cuh - tile and shared-memory layout of the fused
// all-stages launches (step_pass.cuh), shared with the host code that plans
// them.
#pragma once

#include <cstdint>

#include "bfpf_device.cuh"
#include "step_group_layout.cuh"

namespace bfpf {

// One launch of the all-stages schedule that runs the stages on the J
// consecutive digits k0 .. k0+J-1 of a time step, all of radix A (a power of
// two <= 32).  Its tiles hold L consecutive values of the digits below k0
// (every value when L = s_k0), every value of the J digits (B = A^J of them),
// and, when L = s_k0, several consecutive values of the digits above: tile
// position pos = (hh B + mi) L + l is particle
//   i = base + (pos mod L) + (pos div L) s_k0,
// base = tile T when L = s_k0 (the tile is the index range [tile T, tile T + T)),
// else lo0 + hi B s_k0 with hi = tile div (s_k0 / L), lo0 = (tile mod (s_k0 / L)) L.
struct PassGeom {
  uint32_t k0, J;          // first digit, digits in the launch
  uint32_t pass, npass;    // launch position in the step, launches per step
  uint32_t log2L, log2S;   // log2 L, log2 s_k0
  uint32_t log2B, log2T;   // log2 A^J, log2 of the tile size T
  uint32_t log2tl;         // log2 (s_k0 / L): tiles per block of higher digits (0 when L = s_k0)
  uint32_t ntiles;
  uint32_t log2sp;         // log2 of the stride of digit k0 - 1 (digit m - 1 when k0 = 0)
  uint32_t nrows;          // prefix-sum rows held at once (see pass_smem_layout)
  float log_a;             // log A
};

// Largest tile (particles) of a fused launch at state dimension D: states,
// ancestor maps and prefix-sum rows stay within about 70 KB, three blocks
// per SM.
__host__ __device__ constexpr uint32_t pass_tile_max(int D) { return D == 1 ? 4096u : D <= 4 ? 2048u : 1024u; }

// Words per prefix-sum row: P_0 .. P_{A-1}, then for A >= 8 the bucket
// pivots P_3, P_7, ..., padded to 4 mod 8 words so that the 16-byte loads of
// eight lanes (different rows) fall on distinct banks; A <= 4 is dense.
__host__ __device__ constexpr int pass_row_stride(int A) {
  return A <= 4 ? A : (A + A / 4) + ((12 - (A + A / 4) % 8) % 8);
}

// Lanes per group in the weighting stage: the register-resident group
// kernel's split of a radix-A group at dimension D, or more lanes when a full
// tile would leave threads of the block without a group.
__host__ __device__ constexpr int pass_lanes(int D, int A) {
  int G = A / group_members_per_lane(A, D);
  while (G < A && (int)(pass_tile_max(D) / (uint32_t)A) * G < kBlock) G *= 2;
  return G;
}

// Padded index of tile position pos in a state row of the shared tile: one
// spare word per 32 keeps reads of lanes A positions apart (the weighting
// stage, when a lane's members are fewer than four) on distinct banks.
__host__ __device__ constexpr uint32_t pass_xpad(uint32_t pos) { return pos + (pos >> 5); }

struct PassSmem {
  uint32_t x, anc, rows, lv, total;   // byte offsets of each part, total bytes
};

// States [D][T + T/32] (FP32), two ancestor maps [2][T] (16-bit tile
// positions), nrows prefix-sum rows, and two arrays of nrows row
// log-weights (this stage's and the previous one's).
__host__ __device__ constexpr PassSmem pass_smem_layout(int D, int A, uint32_t T, uint32_t nrows) {
  PassSmem s{0u, 0u, 0u, 0u, 0u};
  const uint32_t TP = T + (T >> 5);
  s.x = 0u;
  s.anc = ((4u * (uint32_t)D * TP) + 15u) & ~15u;
  s.rows = s.anc + ((4u * T + 15u) & ~15u);
  s.lv = s.rows + ((4u * nrows * (uint32_t)pass_row_stride(A) + 15u) & ~15u);
  s.total = s.lv + 8u * nrows;
  return s;
}

}  // namespace bfpf
