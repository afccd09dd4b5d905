// step_group_layout.cuh - work split and shared-memory layout of the
// register-resident group kernels (step_group.cuh), shared with the host code
// that plans launches and sizes shared memory.
#pragma once

#include <cstdint>

#include "bfpf_device.cuh"

namespace bfpf {

// Members per lane of a radix-A group at state dimension D: the largest power
// of two m <= A with m D <= 16 state values in registers; G = A / m lanes.
__host__ __device__ constexpr int group_members_per_lane(int A, int D) {
  int m = 1;
  while (m * 2 <= A && m * 2 * D <= 16) m *= 2;
  return m;
}

// Shared-memory layout of a stage on a radix-A digit with G lanes per group.
// Prefix-sum rows, one per group: P_0 .. P_{A-1}, then the bucket pivots
// P_3, P_7, ... (A >= 8); the row stride RS = 4 mod 8 words puts the 16-byte
// loads of 8 lanes (different groups) on distinct banks.  States: a
// [t][member][group] table (leading dimension LD), so that the gather of a
// warp reads distinct banks.
template <int D, int A, int G>
struct GroupLayout {
  static constexpr int GPB = kBlock / G;                  // groups per block iteration
  static constexpr int LD = GPB + (G > 1 ? 1 : 0);
  static constexpr int PIV = (A >= 8) ? A / 4 : 0;
  static constexpr int RS = (A + PIV) + ((12 - (A + PIV) % 8) % 8);
  static constexpr int kRowWords = GPB * RS;
  static constexpr int kTabWords = D * A * LD;
  static_assert(RS % 8 == 4 && RS >= A + PIV, "row stride");
};

// Shared-memory bytes of a one-stage group pass on radix A at dimension D
// (members per lane as group_members_per_lane), and the largest over the
// radices 2 .. 32.
__host__ __device__ constexpr uint32_t group_smem_bytes(int D, int A) {
  const int G = A / group_members_per_lane(A, D);
  const int GPB = kBlock / G;
  const int LD = GPB + (G > 1 ? 1 : 0);
  const int PIV = (A >= 8) ? A / 4 : 0;
  const int RS = (A + PIV) + ((12 - (A + PIV) % 8) % 8);
  return 4u * (uint32_t)(GPB * RS + D * A * LD);
}
__host__ __device__ constexpr uint32_t group_smem_bytes_max(int D) {
  uint32_t b = 0;
  for (int A = 2; A <= 32; A *= 2) b = b > group_smem_bytes(D, A) ? b : group_smem_bytes(D, A);
  return b;
}

}  // namespace bfpf
