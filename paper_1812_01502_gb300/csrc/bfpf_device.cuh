// bfpf_device.cuh - device-side building blocks of the butterfly particle filter.
//
// Philox4x32-7 (Salmon, Moraes, Dror & Shaw, SC'11), Box-Muller normals,
// division by run-time invariant integers (Granlund & Montgomery, PLDI'94),
// float-float compensated sums (Knuth's TwoSum), and the parameter blocks the
// kernels receive.  The random-stream layout (which counter feeds which
// draw) is a fixed convention of this library:
//
//   key = (seed mod 2^32, seed div 2^32)
//   initial normals      counter (nu/4, 0, 0, 0),  nu = i*d + t
//   propagation normals  counter (nu/4, n, 1, 0),  nu = pi*d + t   at time step n
//   resampling uniforms  counter (pi/4, n, 2, 0)   word pi%4            (groups of <= 256)
//   wide uniforms        counter (pi/2, n, 3, 0)   words 2(pi%2)+{0,1}  (groups of > 256)
//
// pi = g*a_k + r numbers the particles group by group at step n (digit k =
// n mod m): g = (i / (a_k s_k)) s_k + i % s_k is i's group, r its digit k.
//
// Box-Muller pair (w0, w1) -> normals 4c, 4c+1 and (w2, w3) -> 4c+2, 4c+3 of
// block c; u = (2*(w0>>9)+1) 2^-24 and v = (w1>>8) 2^-24 are exact FP32 values.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

namespace bfpf {

constexpr int kMaxDigits = 32;
constexpr int kMaxDim = 8;
constexpr int kBlock = 256;
constexpr uint32_t kNarrowMaxRadix = 256;   // groups up to this size use 24-bit weights, 32-bit draws
constexpr uint32_t kMaxCtaRadix = 1024;     // largest group resampled inside one thread block
constexpr uint32_t kRing = 1024;            // observation / per-step output ring length

constexpr uint32_t kPurposeInit = 0;
constexpr uint32_t kPurposePropagate = 1;
constexpr uint32_t kPurposeResample = 2;
constexpr uint32_t kPurposeResampleWide = 3;
constexpr uint32_t kPurposeIsland = 4;       // island-level draws of augmented island resampling

constexpr uint32_t kStatusNonFinite = 1u;
constexpr uint32_t kStatusZeroGroup = 2u;

enum ModelKind : int { kLinearGaussian = 1, kStochVol = 2 };

// ---------------------------------------------------------------------------
// Philox4x32 with seven rounds.  Salmon et al. report Philox4x32 free of
// TestU01 BigCrush failures from seven rounds on and use ten as a safety
// margin; this library takes seven (the oracle implements the same count).
// The round keys (k0 + r W0, k1 + r W1) depend only on the seed; kernels take
// them precomputed from their parameter block so that the xor with the round
// key reads a constant operand.
constexpr int kPhiloxRounds = 7;

struct RoundKeys {
  uint32_t k[2 * kPhiloxRounds];   // k[2r], k[2r+1]: round r
};

inline RoundKeys make_round_keys(uint64_t seed) {
  RoundKeys rk;
  uint32_t k0 = (uint32_t)seed, k1 = (uint32_t)(seed >> 32);
  for (int r = 0; r < kPhiloxRounds; ++r) {
    rk.k[2 * r] = k0;
    rk.k[2 * r + 1] = k1;
    k0 += 0x9E3779B9u;
    k1 += 0xBB67AE85u;
  }
  return rk;
}

__device__ __forceinline__ uint4 philox_round(uint4 c, uint32_t k0, uint32_t k1) {
  const uint64_t p0 = (uint64_t)c.x * 0xD2511F53u;
  const uint64_t p1 = (uint64_t)c.z * 0xCD9E8D57u;
  return make_uint4((uint32_t)(p1 >> 32) ^ c.y ^ k0, (uint32_t)p1, (uint32_t)(p0 >> 32) ^ c.w ^ k1, (uint32_t)p0);
}

__device__ __forceinline__ uint4 philox4x32(uint4 c, const RoundKeys& rk) {
#pragma unroll
  for (int r = 0; r < kPhiloxRounds; ++r) c = philox_round(c, rk.k[2 * r], rk.k[2 * r + 1]);
  return c;
}

__device__ __forceinline__ uint4 philox4x32(uint4 c, uint32_t k0, uint32_t k1) {
#pragma unroll
  for (int r = 0; r < kPhiloxRounds; ++r) {
    c = philox_round(c, k0, k1);
    k0 += 0x9E3779B9u;
    k1 += 0xBB67AE85u;
  }
  return c;
}

// Two standard normals from two 32-bit words (see the layout above), with
// CUDA's full-precision logf / sqrtf / sincospif.
__device__ __forceinline__ void box_muller(uint32_t wa, uint32_t wb, float& z0, float& z1) {
  const float u = __uint2float_rn(((wa >> 9) << 1) | 1u) * 0x1p-24f;   // exact, in (0, 1)
  const float v = __uint2float_rn(wb >> 8) * 0x1p-24f;                 // exact, in [0, 1)
  const float rad = sqrtf(-2.0f * logf(u));
  float s, c;
  sincospif(2.0f * v, &s, &c);
  z0 = rad * c;
  z1 = rad * s;
}

__device__ __forceinline__ void normals4(uint4 w, float z[4]) {
  box_muller(w.x, w.y, z[0], z[1]);
  box_muller(w.z, w.w, z[2], z[3]);
}

// Special-function-unit approximations with flush-to-zero.  The arguments
// the kernels pass are never subnormal (uniforms >= 2^-24, radii^2 >= 2^-23,
// angles and weight exponents of normal size or zero), and there the .ftz
// forms return the same values as the plain forms without their subnormal
// scaling steps.
__device__ __forceinline__ float lg2_ftz(float x) {
  float r;
  asm("lg2.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
  return r;
}
__device__ __forceinline__ float ex2_ftz(float x) {
  float r;
  asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
  return r;
}
__device__ __forceinline__ float sqrt_ftz(float x) {
  float r;
  asm("sqrt.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
  return r;
}
__device__ __forceinline__ float sin_ftz(float x) {
  float r;
  asm("sin.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
  return r;
}
__device__ __forceinline__ float cos_ftz(float x) {
  float r;
  asm("cos.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
  return r;
}

// The same transform on the special-function units: -2 ln u from lg2.approx
// (absolute error about 2^-22 in log2 u), except for u > 63/64 where
// -ln u = t + t^2/2 + t^3/3 + t^4/4 with t = 1 - u (exact in FP32; truncation
// below 2e-8 relative) keeps the small radii accurate; the angle is taken in
// [-pi, pi) where sin/cos.approx have absolute error about 2^-21:
// cos(2 pi v) = -cos(2 pi (v - 1/2)).  Normals differ from the full-precision
// transform by < 4e-6 absolute.  u = (2 floor(w0 / 2^9) + 1) 2^-24 is built
// from its bits: 1 + floor(w0 / 2^9) 2^-23 minus (1 - 2^-24), exact in FP32.
__device__ __forceinline__ void box_muller_fast(uint32_t wa, uint32_t wb, float& z0, float& z1) {
  const float u = __uint_as_float((wa >> 9) | 0x3f800000u) - 0.99999994039535522f;
  const float v = __uint2float_rn(wb >> 8) * 0x1p-24f;
  float r2;
  if (u > 0.984375f) {
    const float t = 1.0f - u;
    const float poly = fmaf(fmaf(fmaf(t, 0.25f, 1.0f / 3.0f), t, 0.5f), t, 1.0f);
    r2 = (t + t) * poly;
  } else {
    r2 = -1.3862943611198906f * lg2_ftz(u);   // -2 ln 2 log2 u
  }
  const float rad = sqrt_ftz(r2);
  const float ang = 6.283185307179586f * (v - 0.5f);
  z0 = -rad * cos_ftz(ang);
  z1 = -rad * sin_ftz(ang);
}

__device__ __forceinline__ void normals4_fast(uint4 w, float z[4]) {
  box_muller_fast(w.x, w.y, z[0], z[1]);
  box_muller_fast(w.z, w.w, z[2], z[3]);
}

// exp(x) for the integer weights, x = lw - max <= 0: ex2.approx.ftz.f32 of
// x log2(e).  The PTX ISA specifies ex2.approx(+-0) = +1, and 0 * log2(e) is
// exactly 0, so the group maximum always weighs exactly 1 (q = 2^B).
__device__ __forceinline__ float exp_weight(float x) {
  return ex2_ftz(x * 1.4426950408889634f);
}

// ---------------------------------------------------------------------------
// Division by an invariant divisor: q = floor(x / d) for 0 <= x < 2^32.
// With l = ceil(log2 d) and mul = floor(2^32 (2^l - d) / d) + 1,
// q = (mulhi(x, mul) + x) >> l   (33-bit intermediate).
// ---------------------------------------------------------------------------
struct FastDiv {
  uint32_t d;
  uint32_t mul;
  uint32_t shift;
};

inline FastDiv make_fastdiv(uint32_t d) {
  FastDiv f{d, 1u, 0u};
  uint32_t l = 0;
  while ((1ull << l) < d) ++l;
  f.shift = l;
  f.mul = (uint32_t)((((1ull << l) - d) << 32) / d + 1ull);
  return f;
}

__device__ __forceinline__ uint32_t fdiv(uint32_t x, const FastDiv& f) {
  return (uint32_t)(((uint64_t)__umulhi(x, f.mul) + x) >> f.shift);
}

// ---------------------------------------------------------------------------
// TwoSum-compensated float accumulation (hi + lo represents the sum).
// ---------------------------------------------------------------------------
__device__ __forceinline__ void ff_add(float& hi, float& lo, float v) {
  const float s = __fadd_rn(hi, v);
  const float bb = __fsub_rn(s, hi);
  const float err = __fadd_rn(__fsub_rn(hi, __fsub_rn(s, bb)), __fsub_rn(v, bb));
  hi = s;
  lo = __fadd_rn(lo, err);
}

// ---------------------------------------------------------------------------
// Parameter blocks
// ---------------------------------------------------------------------------
struct DigitGeom {
  uint32_t a;         // radix a_k
  uint32_t s;         // stride s_k = a_0 ... a_{k-1}
  uint32_t H;         // N / (a_k s_k): number of blocks of the digits above k
  uint32_t nh, nl;    // a tile is nh upper-digit blocks x a_k rows x nl lower-digit columns
  uint32_t tiles_l;   // s_k / nl
  uint32_t ntiles;    // (H / nh) * tiles_l
  uint32_t tile_n;    // nh * a_k * nl particles
  uint32_t quad;      // 1 if every tile splits into aligned runs of 4 consecutive indices
  uint32_t prev_s;    // stride of digit k-1 (mod m), whose groups carry the weights
  float log_a;        // log(a_k)
  uint32_t wide;      // a_k > kNarrowMaxRadix: 32-bit weights, 64-bit draws, 64-bit prefix sums
  FastDiv div_nl, div_a, div_tiles_l, div_prev_as, div_prev_s, div_tgroups;
  // digit-set stages {0, k} (step_sets.cu): w = a_0 columns per group, prev_sw =
  // prev_s / w; 1 and prev_s for a plain digit stage
  uint32_t w, prev_sw;
  FastDiv div_w, div_nlw;
  uint32_t team;      // lanes per group in the tile kernels' group phase (power of two <= 32)
  FastDiv div_s;      // division by s_k
};

// Geometry of one digit for the register-resident group kernel (power-of-two
// radices): group g = h*s + l has members i = h*a*s + r*s + l; the carried
// weight of member r is lV[((h*a + r)*lv_mul + (l & lv_lmask)) & lv_mask].
struct GroupGeom {
  uint32_t log2s;     // log2 s_k
  uint32_t log2as;    // log2 (a_k s_k)
  uint32_t nbatch;    // (N / a_k) / groups per thread block
  uint32_t lv_mul, lv_lmask, lv_mask;
  float log_a;
  uint32_t j, k, last;   // fully adapted schedule: launch position, digit, last launch of the step
};

// ModelParams::flags: structure of the linear-Gaussian matrices (lets the
// kernels skip multiplications by known zeros)
constexpr int kHIdentity = 1, kLrDiagonal = 2, kLqDiagonal = 4, kADiagonal = 8;

struct ModelParams {
  int kind;
  int d, dy;
  int flags;
  float A[kMaxDim * kMaxDim];     // transition matrix (row-major)
  float Lq[kMaxDim * kMaxDim];    // transition-noise factor (lower triangular)
  float H[kMaxDim * kMaxDim];     // observation matrix (dy x d)
  float Lri[kMaxDim * kMaxDim];   // inverse of the observation-noise factor (lower triangular)
  float m0[kMaxDim];
  float L0[kMaxDim * kMaxDim];
  float phi, sigma, inv2b2, sd0;  // stochastic volatility
  double c_obs;                   // state-independent part of log g (enters the likelihood only)
};

struct DevState {
  uint32_t n;          // time index of the next observation
  uint32_t done;       // thread blocks finished with the current step
  uint32_t status;     // sticky kStatus* bits
  float mu_f;          // FP32 copy of mu, subtracted by the kernels
  double mu;           // carried normaliser (log-mean carried weight)
  double loglik;       // cumulative log-likelihood (FP64)
  float gmax;          // global resampling: maximum log-weight of the step
  uint32_t done2;      // reserved (zero)
  uint32_t stage;      // next stage of time step n (0 unless every stage runs in each step)
  // fully adapted schedule (per-particle carried weights)
  uint32_t lvp;        // which lV buffer holds the current weights
  uint32_t skip;       // the ESS reached the threshold: the step's remaining stages are skipped
  int32_t last_k;      // digit of the last stage executed in this step (-1: none yet)
  uint32_t start;      // digit the step's stages start at (rotated start)
  unsigned long long nstages;   // resampling stages executed so far
};

struct StepParams {
  RoundKeys rk;        // Philox round keys of the seed
  float* x;            // [d][N] particle states (updated in place)
  float* lV[2];        // carried log stage weights, ping-pong by stage-counter parity
  int32_t* anc;        // [N] ancestors of the last step (nullptr = not recorded)
  unsigned long long* prec;   // [N] inclusive prefix sums of the integer weights within each
                              // particle's group at the last step (nullptr = not recorded)
  DevState* st;
  float* partials;     // [grid][3 + d] per-block partial sums
  const float* y_ring; // [kRing][dy]
  double* inc_ring;    // [kRing]
  float* mean_ring;    // [kRing][d]
  float* ess_ring;     // [kRing]
  uint32_t N;
  int m;
  uint32_t seed_lo, seed_hi;
  uint32_t tile_cap;   // shared-memory tile capacity (particles)
  float inv_N;
  uint32_t sps;        // resampling stages per time step: 1 (one digit per step) or m (all of them)
  float theta;         // fully adapted schedule: ESS threshold in (0, 1] (above 1: every stage)
  uint32_t rotate;     // fully adapted schedule: start each step one digit after the last stage run
  ModelParams model;
  DigitGeom geom[kMaxDigits];
};

// Where one launch sits in the stage schedule.  The stage counter t counts
// every resampling stage run so far; stage t works on digit k = t mod m.
// With one stage per step (sps = 1) t = n and each launch is a whole step.
// With all m stages per step (Algorithm 1 whose Resample is all of Algorithm
// 3, sps = m) step n runs stages t = n m .. n m + m - 1: only the first
// multiplies the observation weight g_n in (V_0 = g), only the last mutates.
struct Sched {
  uint32_t n;     // time index (observation, mutation counters, output slot)
  uint32_t t;     // stage counter (resampling counters, carried-weight parity)
  uint32_t k;     // digit of this stage
  bool obs;       // weight with g_n and produce the step's summaries
  bool mut;       // mutate after resampling (last stage of the step)
};

__device__ __forceinline__ Sched sched_of(const StepParams& p, const DevState* st) {
  Sched sc;
  sc.n = st->n;
  const uint32_t stage = st->stage;
  sc.t = sc.n * p.sps + stage;
  sc.k = sc.t % (uint32_t)p.m;
  sc.obs = stage == 0;
  sc.mut = stage + 1 == p.sps;
  return sc;
}

// Augmented island resampling (AIRPF): islands of M consecutive particles.
constexpr int kIslandThreads = 1024;
constexpr uint32_t kMaxIslands = 16384;   // island weights and holders fit in shared memory
struct IslandParams {
  float* x_out;         // [d][N] states after the island gather and the mutation
  int32_t* src;         // [islands] island whose sample island i holds after the island stages
  const float* lW;      // [islands] log island weights from the within-island stage
  float* lV_next;       // [M] carried log weights of the next step (all equal)
  uint32_t M, islands, S;
  uint32_t plain;       // 1: Algorithm 6 as printed (no undoing of swaps)
  uint32_t adaptive;    // 1: ESS test before every island stage (AIRPF2); lV_next then per island
  float theta;          // its threshold
};

}  // namespace bfpf
