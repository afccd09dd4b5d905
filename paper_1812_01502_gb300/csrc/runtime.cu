// runtime.cu - host runtime and C ABI (include/bfpf.h) of the butterfly
// particle filter: argument checking, tile planning, workspace layout,
// kernel launches, CUDA-graph replay of chunks of time steps.
//
// The problem a handle solves is the HMM of Section 1.1 of Heine, Whiteley &
// Cemgil (arXiv 1812.01502) filtered by Algorithm 1 with one stage of
// Algorithm 3 per time step; see step_butterfly.cu for the step itself.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <map>
#include <mutex>
#include <new>
#include <string>
#include <vector>

#include "bfpf.h"
#include "bfpf_batch.cuh"
#include "bfpf_device.cuh"
#include "bfpf_global.cuh"
#include "bfpf_kernels.h"
#include "step_group_layout.cuh"
#include "step_pass_layout.cuh"

#include <nvtx3/nvToolsExt.h>

using namespace bfpf;

namespace {

// NVTX range for profilers and tracers (a no-op unless a tool is attached).
struct Trace {
  explicit Trace(const char* name) { nvtxRangePushA(name); }
  ~Trace() { nvtxRangePop(); }
  Trace(const Trace&) = delete;
  Trace& operator=(const Trace&) = delete;
};

thread_local std::string t_error;

constexpr size_t kAlign = 256;

size_t align_up(size_t v) { return (v + kAlign - 1) / kAlign * kAlign; }

struct Layout {
  size_t st, x, lv0, lv1, anc, prec, partials, y_ring, inc_ring, mean_ring, ess_ring, total;
  size_t x2, lw, P, tsum, toff, done;       // global resampling only (x2: also AIRPF)
  size_t slot, cnt, ovf, jb, cslot, ccnt, covf;   // global resampling: draws filed by coarse bin, then bucket
  size_t src;                               // AIRPF: island sources
};

// The kernel that runs the steps on one digit.
struct DigitPlan {
  const void* kernel = nullptr;
  bool group = false;         // register-resident group kernel (else the general tile kernel)
  int lanes = 0;              // lanes per group (group kernel)
  GroupGeom gg{};
  int grid = 0;
  size_t smem = 0;            // dynamic shared memory (general kernel)
};

struct Plan {
  int d = 0, dy = 0, kind = 0, m = 0;
  uint32_t N = 0;
  bool wide = false;          // some radix > kNarrowMaxRadix
  uint32_t min_a = 0;
  uint32_t cap = 0;           // tile capacity (particles)
  uint32_t max_tiles = 0;
  int grid = 0;
  size_t smem = 0;
  bool record = false;
  bool record_draws = false;  // PF_RECORD_DRAWS: integer prefix sums of the step's draws (test output)
  uint32_t sps = 1;           // resampling stages per time step (1, or m with PF_ALL_STAGES)
  bool adaptive = false;      // PF_ADAPTIVE: m + 1 launches per step, per-particle carried weights
  bool rotate = false;
  float theta = 0.5f;
  AdaptiveKernels ak{};
  bool sets = false;          // PF_DIGIT_SETS: stage s on digits {0, s}, m - 1 launches per step
  bool islands = false;       // PF_ISLANDS: radices (M, m), 3 launches per step
  bool island_plain = false;
  bool island_adaptive = false;   // PF_ISLANDS | PF_ADAPTIVE (AIRPF2): ESS test before every island stage
  float island_theta = 0.5f;
  IslandKernels ik{};
  int chunk_len = 64;
  KernelSet ks{};
  ModelParams mp{};
  DigitGeom geom[kMaxDigits]{};
  DigitPlan dp[kMaxDigits]{};
  int max_grid = 0;
  bool global = false;        // radices = {N} with N > kMaxCtaRadix: global resampling kernels
  GlobalKernels gk{};
  int grid_weight = 0;
  uint32_t nscan = 0;
  uint32_t log2b = 0, buckets = 1, bucket_cap = 0, stage_cap = 0;   // bucketed draws
  uint32_t cbits = 0, ccap = 0, nseg = 1;                            // coarse bins
  size_t smem_resolve = 0, smem_weight = 0, smem_refine = 0;
  // All-stages schedule on power-of-two radices <= 32: npass fused launches per
  // step (step_pass.cuh), each running consecutive digits of one radix; 0 = one
  // launch per stage.
  int npass = 0;
  PassGeom pg[kMaxDigits]{};
  const void* pass_kernel[kMaxDigits]{};
  size_t pass_smem[kMaxDigits]{};
  int pass_grid[kMaxDigits]{};
  Layout lay{};
};

}  // namespace

struct pf_handle {
  int device = 0;
  cudaStream_t stream = nullptr;
  cudaStream_t cap_stream = nullptr;
  bool own_ws = false;
  unsigned char* ws = nullptr;
  size_t ws_bytes = 0;
  Plan plan;
  StepParams P{};
  GlobalParams GP{};
  uint64_t n_host = 0;     // time steps enqueued
  uint64_t n_pushed = 0;   // observations copied into the ring
  std::vector<cudaGraphExec_t> graphs;   // chunk graphs, one per radix phase (n mod m)
  uint32_t launch_j[kMaxDigits] = {};    // stage-launch arguments of the fully adapted schedule
  StepParams Pisl[2]{};                  // AIRPF: step parameters by step parity (states ping-pong)
  IslandParams ipar[2]{};
  uint32_t flags = 0;                    // pf_options.flags at creation
  uint64_t seed = 0;
  int32_t radices[kMaxDigits] = {};
  std::string err;
};

namespace {

pf_status fail(const pf_handle* h, pf_status s, const std::string& msg) {
  if (h) const_cast<pf_handle*>(h)->err = msg;
  else t_error = msg;
  return s;
}

#define PF_CUDA(h, call)                                                              \
  do {                                                                                \
    cudaError_t e_ = (call);                                                          \
    if (e_ != cudaSuccess)                                                            \
      return fail((h), PF_ECUDA, std::string(#call) + ": " + cudaGetErrorString(e_)); \
  } while (0)

// True if p is host memory (outputs written there need the stream synchronised).
bool is_host_ptr(const void* p) {
  if (!p) return false;
  cudaPointerAttributes attr;
  if (cudaPointerGetAttributes(&attr, p) != cudaSuccess) {
    cudaGetLastError();
    return true;
  }
  return attr.type == cudaMemoryTypeHost || attr.type == cudaMemoryTypeUnregistered;
}

bool is_lower_triangular(const double* M, int n) {
  for (int i = 0; i < n; ++i)
    for (int j = i + 1; j < n; ++j)
      if (M[i * n + j] != 0.0) return false;
  return true;
}

// Fill the device model block from the caller's model (doubles -> floats).
pf_status build_model(const pf_model* model, ModelParams& mp, std::string& msg) {
  if (!model) { msg = "model is NULL"; return PF_EINVAL; }
  std::memset(&mp, 0, sizeof(mp));
  mp.kind = model->kind;
  if (model->kind == PF_MODEL_STOCH_VOL) {
    if (model->d != 1 || model->dy != 1) { msg = "stochastic volatility needs d = dy = 1"; return PF_EINVAL; }
    if (!(std::fabs(model->phi) < 1.0) || !(model->sigma > 0.0) || !(model->beta > 0.0)) {
      msg = "stochastic volatility needs |phi| < 1, sigma > 0, beta > 0";
      return PF_EINVAL;
    }
    mp.d = mp.dy = 1;
    mp.phi = (float)model->phi;
    mp.sigma = (float)model->sigma;
    mp.inv2b2 = (float)(1.0 / (2.0 * model->beta * model->beta));
    mp.sd0 = (float)(model->sigma / std::sqrt(1.0 - model->phi * model->phi));
    mp.c_obs = -0.5 * std::log(2.0 * M_PI * model->beta * model->beta);
    return PF_OK;
  }
  if (model->kind != PF_MODEL_LINEAR_GAUSSIAN) { msg = "unknown model kind"; return PF_EINVAL; }
  const int d = model->d, dy = model->dy;
  if (d < 1 || d > kMaxDim || dy < 1 || dy > kMaxDim) {
    msg = "linear-Gaussian model needs 1 <= d, dy <= 8";
    return PF_EINVAL;
  }
  if (!model->H && dy != d) { msg = "H = NULL (identity) needs dy == d"; return PF_EINVAL; }
  mp.d = d;
  mp.dy = dy;
  auto get = [](const double* M, int r, int c, int cols, bool ident) -> double {
    if (M) return M[r * cols + c];
    return (ident && r == c) ? 1.0 : 0.0;
  };
  int flags = kHIdentity | kLrDiagonal | kLqDiagonal | kADiagonal;
  for (int i = 0; i < d; ++i)
    for (int j = 0; j < d; ++j) {
      const double a = get(model->A, i, j, d, true), q = get(model->Lq, i, j, d, true),
                   l0 = get(model->L0, i, j, d, true);
      if (!std::isfinite(a) || !std::isfinite(q) || !std::isfinite(l0)) { msg = "non-finite matrix entry"; return PF_EINVAL; }
      if (j > i && (q != 0.0 || l0 != 0.0)) { msg = "Lq and L0 must be lower triangular"; return PF_EINVAL; }
      mp.A[i * kMaxDim + j] = (float)a;
      mp.Lq[i * kMaxDim + j] = (float)q;
      mp.L0[i * kMaxDim + j] = (float)l0;
      if (i != j && a != 0.0) flags &= ~kADiagonal;
      if (i != j && q != 0.0) flags &= ~kLqDiagonal;
    }
  for (int i = 0; i < dy; ++i)
    for (int j = 0; j < d; ++j) {
      const double hv = get(model->H, i, j, d, true);
      if (!std::isfinite(hv)) { msg = "non-finite H entry"; return PF_EINVAL; }
      mp.H[i * kMaxDim + j] = (float)hv;
      if (hv != ((i == j) ? 1.0 : 0.0)) flags &= ~kHIdentity;
    }
  if (dy != d) flags &= ~kHIdentity;
  // Lr^{-1} by forward substitution (double), and the likelihood constant.
  std::vector<double> Lr(dy * dy), Li(dy * dy, 0.0);
  for (int i = 0; i < dy; ++i)
    for (int j = 0; j < dy; ++j) Lr[i * dy + j] = get(model->Lr, i, j, dy, true);
  if (!is_lower_triangular(Lr.data(), dy)) { msg = "Lr must be lower triangular"; return PF_EINVAL; }
  double logdet = 0.0;
  for (int i = 0; i < dy; ++i) {
    if (!(Lr[i * dy + i] != 0.0) || !std::isfinite(Lr[i * dy + i])) { msg = "Lr needs a nonzero finite diagonal"; return PF_EINVAL; }
    logdet += std::log(std::fabs(Lr[i * dy + i]));
    for (int j = 0; j < i; ++j)
      if (Lr[i * dy + j] != 0.0) flags &= ~kLrDiagonal;
  }
  for (int c = 0; c < dy; ++c) {        // solve Lr * col = e_c
    for (int i = 0; i < dy; ++i) {
      double v = (i == c) ? 1.0 : 0.0;
      for (int j = 0; j < i; ++j) v -= Lr[i * dy + j] * Li[j * dy + c];
      Li[i * dy + c] = v / Lr[i * dy + i];
    }
  }
  for (int i = 0; i < dy; ++i)
    for (int j = 0; j < dy; ++j) mp.Lri[i * kMaxDim + j] = (float)Li[i * dy + j];
  for (int i = 0; i < d; ++i) mp.m0[i] = model->m0 ? (float)model->m0[i] : 0.0f;
  mp.c_obs = -logdet - 0.5 * dy * std::log(2.0 * M_PI);
  mp.flags = flags;
  return PF_OK;
}

uint32_t largest_divisor_at_most(uint32_t n, uint32_t limit) {
  if (limit >= n) return n;
  for (uint32_t v = std::max<uint32_t>(limit, 1); v > 1; --v)
    if (n % v == 0) return v;
  return 1;
}

bool plan_passes(Plan& pl, const int32_t* radices, int m);

pf_status make_plan(const pf_model* model, int64_t N64, const int32_t* radices, int32_t m,
                    const pf_options* opts, Plan& pl, std::string& msg) {
  pf_options opts_rec;
  if (opts && (opts->flags & PF_RECORD_DRAWS)) {   // records the ancestors too, with the same limits
    opts_rec = *opts;
    opts_rec.flags |= PF_RECORD_ANCESTORS;
    opts = &opts_rec;
    pl.record_draws = true;
  }
  const pf_status bs = build_model(model, pl.mp, msg);
  if (bs != PF_OK) return bs;
  pl.d = pl.mp.d;
  pl.dy = pl.mp.dy;
  pl.kind = pl.mp.kind;
  if (!radices || m < 1 || m > kMaxDigits) { msg = "need 1 <= m <= 32 radices"; return PF_EINVAL; }
  if (N64 < 2 || N64 >= (int64_t(1) << 31)) { msg = "need 2 <= N < 2^31"; return PF_EINVAL; }
  int64_t prod = 1;
  pl.min_a = 0xffffffffu;
  // AIRPF: digit 1 counts the islands and is never run by the stage kernels
  pl.islands = opts && (opts->flags & PF_ISLANDS);
  pl.island_plain = pl.islands && (opts->flags & PF_ISLANDS_PLAIN);
  if (pl.islands) {
    if (opts->flags & (PF_ALL_STAGES | PF_ROTATE | PF_DIGIT_SETS | PF_RECORD_ANCESTORS)) {
      msg = "PF_ISLANDS cannot be combined with PF_ALL_STAGES, PF_ROTATE, PF_DIGIT_SETS or PF_RECORD_ANCESTORS";
      return PF_EINVAL;
    }
    if (opts->flags & PF_ADAPTIVE) {     // AIRPF2
      if (!(opts->ess_threshold >= 0.0f)) { msg = "ess_threshold must be >= 0"; return PF_EINVAL; }
      pl.island_adaptive = true;
      pl.island_theta = opts->ess_threshold > 0.0f ? opts->ess_threshold : 0.5f;
    }
    if (m != 2 || radices[1] < 2 || radices[1] > (int64_t)kMaxIslands || (radices[1] & (radices[1] - 1))) {
      msg = "PF_ISLANDS needs radices (M, m) with m a power of two, 2 <= m <= 16384";
      return PF_EINVAL;
    }
  }
  for (int k = 0; k < m; ++k) {
    const int64_t a = radices[k];
    const bool run = !(pl.islands && k == 1);
    if (a < 2) { msg = "every radix must be >= 2"; return PF_EINVAL; }
    if (run && m > 1 && a > (int64_t)kMaxCtaRadix) { msg = "radices must be <= 1024 when m > 1"; return PF_EINVAL; }
    prod *= a;
    if (prod > N64) break;
    pl.min_a = std::min<uint32_t>(pl.min_a, (uint32_t)a);
    if (run && a > (int64_t)kNarrowMaxRadix) pl.wide = true;
  }
  if (prod != N64) { msg = "the product of the radices must equal N"; return PF_EINVAL; }
  pl.N = (uint32_t)N64;
  pl.m = m;
  const int d = pl.d;
  if (m == 1 && N64 > (int64_t)kMaxCtaRadix) {
    // Global multinomial resampling (Algorithm 2) across thread blocks.
    if (opts && (opts->flags & PF_ADAPTIVE)) {
      msg = "PF_ADAPTIVE needs every group within one thread block (N <= 1024 when m = 1)";
      return PF_EINVAL;
    }
    pl.global = true;
    pl.wide = true;
    if (!select_global_kernels(d, pl.kind, pl.gk)) { msg = "unsupported (d, model) combination"; return PF_EINVAL; }
    if (!select_kernels(d, pl.kind, true, pl.ks)) { msg = "unsupported (d, model) combination"; return PF_EINVAL; }
    pl.nscan = (pl.N + kScanTile - 1) / kScanTile;
    // Draws are resolved per bucket of their uniform: about stage_cap / 2 to
    // stage_cap draws per bucket (a population in random index order puts
    // about as many prefix sums as draws in a bucket's u interval), so that a
    // bucket's index range normally fits the shared-memory staging buffer
    // (8 + 4 d bytes per index).
    const bool small_buckets = opts && (opts->flags & PF_TEST_SMALL_BUCKETS);
    pl.stage_cap = global_stage_alloc(d);
    uint32_t lgN = 0, lgc = 0;
    while ((2ull << lgN) <= pl.N) ++lgN;            // floor(log2 N)
    while ((2u << lgc) <= pl.stage_cap) ++lgc;      // log2 stage_cap
    pl.log2b = lgN > lgc - 1 ? std::min<uint32_t>(lgN - (lgc - 1), 24u) : 0u;
    // small populations: at least 2^8 buckets (but at least 256 draws each) so
    // that the resolve launch has blocks for every SM
    if (lgN >= 8u) pl.log2b = std::max<uint32_t>(pl.log2b, std::min<uint32_t>(lgN - 8u, 8u));
    pl.buckets = 1u << pl.log2b;
    const uint32_t mu = (uint32_t)((pl.N + pl.buckets - 1) / pl.buckets);
    const uint32_t sd = (uint32_t)std::ceil(std::sqrt((double)mu));
    // 8 standard deviations of the binomial fill above its mean; the rare
    // excess goes to the overflow list.  The test hook forces overflow.
    pl.bucket_cap = small_buckets ? 16u : std::min<uint32_t>(pl.N, mu + 8u * sd + 64u);
    if (small_buckets) pl.stage_cap = 64u;          // most buckets then search in global memory
    // Coarse bins: the top half of the bucket bits, filed first
    pl.cbits = (pl.log2b + 1u) / 2u;
    const uint32_t muc = (uint32_t)((pl.N + (1u << pl.cbits) - 1) >> pl.cbits);
    const uint32_t sdc = (uint32_t)std::ceil(std::sqrt((double)muc));
    pl.ccap = small_buckets ? 64u : std::min<uint32_t>(pl.N, muc + 8u * sdc + 64u);
    pl.nseg = (pl.ccap + kRefineSeg - 1) / kRefineSeg;
    pl.smem_weight = (size_t)8 * kBlock * global_weight_vec(d) + (size_t)8 * (1u << pl.cbits);
    pl.smem_refine = (size_t)8 * kRefineSeg + (size_t)8 * (1u << (pl.log2b - pl.cbits));
    pl.smem_resolve = (size_t)8 * global_stage_alloc(d) + (size_t)4 * d * (global_stage_alloc(d) + 1u) +
                      (size_t)4 * kGuideBins;
    DigitGeom& g = pl.geom[0];
    g.a = pl.N;
    g.s = 1;
    g.H = 1;
    g.log_a = (float)std::log((double)pl.N);
    g.wide = 1;
    pl.record = opts && (opts->flags & PF_RECORD_ANCESTORS);
    pl.chunk_len = (opts && opts->chunk_len > 0) ? std::min<int>(opts->chunk_len, (int)kRing) : 64;
    pl.sps = 1;               // one digit: the single stage is the whole of Algorithm 3
    return PF_OK;
  }
  uint32_t target = (opts && opts->tile > 0) ? (uint32_t)opts->tile : (d == 1 ? 4096u : d <= 4 ? 2048u : 1024u);
  target = std::max<uint32_t>(target, 4);
  uint32_t s = 1;
  pl.cap = 0;
  pl.max_tiles = 0;
  for (int k = 0; k < m; ++k) {
    DigitGeom& g = pl.geom[k];
    const uint32_t a = (uint32_t)radices[k];
    g.a = a;
    g.s = s;
    g.H = pl.N / (a * s);
    if ((uint64_t)a * s <= target) {
      g.nl = s;
      g.nh = largest_divisor_at_most(g.H, target / (a * s));
    } else {
      g.nh = 1;
      g.nl = largest_divisor_at_most(s, std::max<uint32_t>(1, target / a));
    }
    g.tiles_l = s / g.nl;
    g.ntiles = (g.H / g.nh) * g.tiles_l;
    g.tile_n = g.nh * a * g.nl;
    g.quad = (g.nl == s) ? ((g.tile_n % 4 == 0) && (pl.N % 4 == 0)) : ((g.nl % 4 == 0) && (s % 4 == 0));
    g.log_a = (float)std::log((double)a);
    g.wide = a > kNarrowMaxRadix ? 1u : 0u;
    g.div_nl = make_fastdiv(g.nl);
    g.div_a = make_fastdiv(a);
    g.div_s = make_fastdiv(s);
    g.div_tiles_l = make_fastdiv(g.tiles_l);
    if (!(pl.islands && k == 1)) {
      pl.cap = std::max(pl.cap, g.tile_n);
      pl.max_tiles = std::max(pl.max_tiles, g.ntiles);
    }
    s *= a;
  }
  for (int k = 0; k < m; ++k) {
    const int kp = (k + m - 1) % m;
    DigitGeom& g = pl.geom[k];
    g.prev_s = pl.geom[kp].s;
    g.div_prev_as = make_fastdiv(pl.geom[kp].a * pl.geom[kp].s);
    g.div_prev_s = make_fastdiv(pl.geom[kp].s);
  }
  // Lanes per group in the tile kernels' group phase: one lane for groups of up
  // to 32 members (a serial pass is cheapest there), else a power of two <= 32
  // that leaves each lane at least 8 members.
  auto team_for = [](uint32_t members) {
    uint32_t t = 1;
    if (members <= 32) return t;
    while (t * 2 <= 32 && t * 2 * 8 <= members) t *= 2;
    return t;
  };
  for (int k = 0; k < m; ++k) {
    DigitGeom& g = pl.geom[k];
    g.team = team_for(g.a);
    g.div_tgroups = make_fastdiv(g.nh * g.nl);
    g.w = 1;
    g.prev_sw = g.prev_s;
    g.div_w = make_fastdiv(1);
    g.div_nlw = g.div_nl;
  }
  pl.sets = opts && (opts->flags & PF_DIGIT_SETS);
  if (pl.sets) {
    // Digit sets {0, k}, k = 1..m-1 (eq. (A matrices)): groups of a_0 a_k members.
    if (opts->flags & (PF_ALL_STAGES | PF_ADAPTIVE | PF_ISLANDS | PF_RECORD_ANCESTORS)) {
      msg = "PF_DIGIT_SETS cannot be combined with the other schedule flags or PF_RECORD_ANCESTORS";
      return PF_EINVAL;
    }
    if (m < 2) { msg = "PF_DIGIT_SETS needs at least two radices"; return PF_EINVAL; }
    const uint32_t w = (uint32_t)radices[0];
    pl.cap = 0;
    pl.max_tiles = 0;
    pl.wide = false;
    for (int k = 1; k < m; ++k) {
      if ((uint64_t)w * (uint64_t)radices[k] > kMaxCtaRadix) {
        msg = "PF_DIGIT_SETS needs a_0 * a_k <= 1024 for every k";
        return PF_EINVAL;
      }
    }
    for (int k = 1; k < m; ++k) {
      DigitGeom& g = pl.geom[k];
      const uint32_t a = g.a, sk = g.s;
      const uint32_t G = a * w;
      if ((uint64_t)a * sk <= target) {
        g.nl = sk;
        g.nh = largest_divisor_at_most(g.H, std::max<uint32_t>(1, target / (a * sk)));
      } else {
        g.nh = 1;
        g.nl = w * largest_divisor_at_most(sk / w, std::max<uint32_t>(1, target / G));
      }
      g.tiles_l = sk / g.nl;
      g.ntiles = (g.H / g.nh) * g.tiles_l;
      g.tile_n = g.nh * a * g.nl;
      g.quad = (g.nl == sk) ? ((g.tile_n % 4 == 0) && (pl.N % 4 == 0)) : ((g.nl % 4 == 0) && (sk % 4 == 0));
      g.log_a = (float)std::log((double)G);
      g.wide = G > kNarrowMaxRadix ? 1u : 0u;
      g.div_nl = make_fastdiv(g.nl);
      g.div_tiles_l = make_fastdiv(g.tiles_l);
      const int kp = (k == 1) ? m - 1 : k - 1;          // the previous stage's set {0, kp}
      g.prev_s = pl.geom[kp].s;
      g.div_prev_as = make_fastdiv(pl.geom[kp].a * pl.geom[kp].s);
      g.div_prev_s = make_fastdiv(pl.geom[kp].s);
      g.w = w;
      g.prev_sw = pl.geom[kp].s / w;
      g.div_w = make_fastdiv(w);
      g.div_nlw = make_fastdiv(g.nl / w);
      g.div_tgroups = make_fastdiv(g.nh * (g.nl / w));
      g.team = team_for(G);
      pl.cap = std::max(pl.cap, g.tile_n);
      pl.max_tiles = std::max(pl.max_tiles, g.ntiles);
      if (g.wide) pl.wide = true;
    }
  }
  pl.sps = (opts && (opts->flags & PF_ALL_STAGES)) ? (uint32_t)m : pl.sets ? (uint32_t)m - 1 : 1u;
  if (pl.islands) {           // the within-island stage is stage 0 of a two-stage step
    pl.sps = 2;
    if (pl.island_adaptive) {   // carried weights per island: the within-island stage reads lV[i / M]
      DigitGeom& g0 = pl.geom[0];
      g0.prev_s = 1;
      g0.prev_sw = 1;
      g0.div_prev_as = make_fastdiv(g0.a);
      g0.div_prev_s = make_fastdiv(1);
    }
    if (!select_island_kernels(d, pl.kind, pl.ik)) { msg = "unsupported (d, model) combination"; return PF_EINVAL; }
  }
  if (pl.sps > 1 && opts && (opts->flags & PF_RECORD_ANCESTORS)) {
    msg = "PF_RECORD_ANCESTORS records one stage; it cannot be combined with PF_ALL_STAGES";
    return PF_EINVAL;
  }
  if (opts && (opts->flags & PF_ADAPTIVE) && !pl.islands) {
    if (opts->flags & (PF_ALL_STAGES | PF_RECORD_ANCESTORS)) {
      msg = "PF_ADAPTIVE cannot be combined with PF_ALL_STAGES or PF_RECORD_ANCESTORS";
      return PF_EINVAL;
    }
    if (!(opts->ess_threshold >= 0.0f)) { msg = "ess_threshold must be >= 0"; return PF_EINVAL; }
    pl.adaptive = true;
    pl.rotate = (opts->flags & PF_ROTATE) != 0;
    pl.theta = opts->ess_threshold > 0.0f ? opts->ess_threshold : 0.5f;
    if (!select_adaptive_kernels(d, pl.kind, pl.wide, pl.ak)) { msg = "unsupported (d, model) combination"; return PF_EINVAL; }
  }
  const bool staged = pl.sps > 1;
  constexpr uint32_t kSmallBatches = 128;
  // Register-resident group kernel: every radix a power of two, a_k <= 32, and the
  // groups of digit k fill whole thread-block iterations.
  bool pow2 = true;
  for (int k = 0; k < m; ++k) pow2 = pow2 && ((radices[k] & (radices[k] - 1)) == 0);
  for (int k = 0; k < m; ++k) {
    DigitPlan& dp = pl.dp[k];
    const DigitGeom& g = pl.geom[k];
    int G = 0;
    // the fully adapted schedule uses group kernels unless rotation makes a launch's digit data-dependent
    const bool adapt_group = pl.adaptive && !pl.rotate;
    const void* gk = (pow2 && g.a <= 32 && !(pl.adaptive && pl.rotate) && !pl.sets && !pl.island_adaptive)
                         ? select_group_kernel(pl.d, pl.kind, (int)g.a, &G, staged, adapt_group)
                         : nullptr;
    if (gk && G > 0) {
      uint32_t gpb = kBlock / G;
      const uint32_t ngroups = pl.N / g.a;
      // A population whose groups fill fewer than kSmallBatches thread-block
      // iterations takes the two-members-per-lane split: more blocks, shorter chains.
      if (!adapt_group && ngroups % gpb == 0 && ngroups / gpb < kSmallBatches) {
        int Gs = 0;
        const void* gks = select_group_kernel(pl.d, pl.kind, (int)g.a, &Gs, staged, false, true);
        if (gks && Gs > 0 && ngroups % (kBlock / Gs) == 0) {
          gk = gks;
          G = Gs;
          gpb = kBlock / G;
        }
      }
      if (ngroups % gpb == 0) {
        dp.kernel = gk;
        dp.group = true;
        dp.lanes = G;
        uint32_t l2s = 0, l2as = 0;
        while ((1u << l2s) < g.s) ++l2s;
        while ((1u << l2as) < g.a * g.s) ++l2as;
        dp.gg.log2s = l2s;
        dp.gg.log2as = l2as;
        dp.gg.nbatch = ngroups / gpb;
        const int kp = (k + m - 1) % m;
        const uint32_t sp = pl.geom[kp].s;
        if (k == 0) {
          dp.gg.lv_mul = 1;
          dp.gg.lv_lmask = 0;
          dp.gg.lv_mask = sp - 1;       // s_{m-1} = N / a_{m-1}
        } else {
          dp.gg.lv_mul = sp;
          dp.gg.lv_lmask = sp - 1;
          dp.gg.lv_mask = 0xffffffffu;
        }
        dp.gg.log_a = g.log_a;
        if (adapt_group) {            // per-particle carried weights: index = member's particle index
          dp.gg.lv_mul = g.s;
          dp.gg.lv_lmask = g.s - 1;
          dp.gg.lv_mask = 0xffffffffu;
          dp.gg.j = (uint32_t)k;
          dp.gg.k = (uint32_t)k;
          dp.gg.last = (k == m - 1) ? 1u : 0u;
        }
      }
    }
  }
  pl.cap = (pl.cap + 3) / 4 * 4;
  pl.smem = (size_t)(d + 1) * pl.cap * 4 + (size_t)pl.cap * (pl.wide ? 8 : 4);
  pl.record = opts && (opts->flags & PF_RECORD_ANCESTORS);
  if (staged && !pl.sets && !pl.islands && pow2 && !(opts && (opts->flags & PF_TEST_STAGE_PER_LAUNCH))) {
    bool small_radix = true;
    for (int k = 0; k < m; ++k) small_radix = small_radix && radices[k] <= 32;
    if (small_radix && !plan_passes(pl, radices, m)) pl.npass = 0;
    // A population below 2^16 whose digits fuse into more than half as many
    // launches keeps one launch per stage: there the group kernels' split (two
    // members per lane for small populations) keeps more threads busy than the
    // fused tiles, and few launches are saved (measured on the 7-D workload).
    if (pl.npass && pl.N < 65536u && 2 * pl.npass > m) pl.npass = 0;
  }
  pl.chunk_len = (opts && opts->chunk_len > 0) ? std::min<int>(opts->chunk_len, (int)kRing) : 64;
  if (!select_kernels(d, pl.kind, pl.wide, pl.ks)) { msg = "unsupported (d, model) combination"; return PF_EINVAL; }
  return PF_OK;
}

// Splits the m digits of the all-stages schedule into fused launches: a launch
// takes consecutive digits of one radix while a tile holding every particle
// its stages can draw from fits pass_tile_max(d) and keeps runs of at least 16
// consecutive indices per state row (or the tile is a whole index range).
// False when a radix has no fused kernel (the schedule then keeps one launch
// per stage).
bool plan_passes(Plan& pl, const int32_t* radices, int m) {
  auto lg2 = [](uint32_t v) { uint32_t l = 0; while ((1u << l) < v) ++l; return l; };
  const uint32_t Tmax = pass_tile_max(pl.d);
  int np = 0;
  for (int k0 = 0; k0 < m;) {
    const uint32_t A = (uint32_t)radices[k0];
    const uint32_t S = pl.geom[k0].s;
    auto fits = [&](uint64_t B) { return B <= Tmax && ((uint64_t)S * B <= Tmax || Tmax / B >= 16u); };
    // A launch takes another digit only while its tiles stay within cap
    // particles, so that populations above 1024 keep at least 16 tiles (thread
    // blocks): one block running a dozen stages on 4096 particles took 48 us a
    // step where two launches of 16 blocks took 25 us (1-D, radix 2).
    uint32_t cap = 1024;
    while (cap * 2u <= pl.N / 16u) cap *= 2u;
    cap = std::min(cap, Tmax);
    auto grows = [&](uint64_t B) { return fits(B) && ((uint64_t)S * B <= cap || 16u * B <= cap); };
    uint32_t J = 1, B = A;
    while (k0 + (int)J < m && (uint32_t)radices[k0 + J] == A && grows((uint64_t)B * A)) {
      B *= A;
      ++J;
    }
    const void* kern = select_pass_kernel(pl.d, pl.kind, (int)A);
    if (!kern || !fits(B)) return false;
    PassGeom& g = pl.pg[np];
    // Tiles of up to Tmax particles, smaller where that leaves fewer than
    // about 512 tiles (small populations: more thread blocks).
    uint32_t fill = 1;
    while (fill * 2u <= pl.N / 512u) fill *= 2u;
    // L = s_k0 (the tile is an index range) unless that tile would pass the cap
    // and L < s_k0 keeps within it
    const bool whole = (uint64_t)S * B <= cap || ((uint64_t)S * B <= Tmax && 16u * B > cap);
    const uint32_t L = whole ? S : std::max(16u, std::min(Tmax / B, fill / B));
    // (at least 4: the tile is loaded in runs of 4 consecutive particles)
    const uint32_t T = whole ? std::max({4u, S * B, std::min(Tmax, fill)}) : L * B;
    g.k0 = (uint32_t)k0;
    g.J = J;
    g.pass = (uint32_t)np;
    g.log2L = lg2(L);
    g.log2S = lg2(S);
    g.log2B = lg2(B);
    g.log2T = lg2(T);
    g.log2tl = whole ? 0u : lg2(S / L);
    g.ntiles = pl.N / T;
    g.log2sp = lg2(pl.geom[k0 == 0 ? m - 1 : k0 - 1].s);
    g.nrows = (k0 == 0) ? T / A : T >> (g.log2L + lg2(A));
    g.log_a = pl.geom[k0].log_a;
    pl.pass_kernel[np] = kern;
    pl.pass_smem[np] = pass_smem_layout(pl.d, (int)A, T, g.nrows).total;
    ++np;
    k0 += (int)J;
  }
  pl.npass = np;
  for (int q = 0; q < np; ++q) pl.pg[q].npass = (uint32_t)np;
  return true;
}

// The dynamic shared-memory limit is an attribute of the kernel, shared by every
// handle in the process: raise it when a handle needs more, never lower it
// (another handle may be running the same kernel with a larger tile).
cudaError_t raise_smem_limit(const void* kernel, size_t bytes) {
  static std::mutex mu;
  static std::map<std::pair<int, const void*>, size_t> limit;
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  std::lock_guard<std::mutex> lock(mu);
  size_t& cur = limit[{dev, kernel}];
  if (bytes <= cur) return cudaSuccess;
  e = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
  if (e == cudaSuccess) cur = bytes;
  return e;
}

// Needs a CUDA device: occupancy decides the persistent grid size.
pf_status finish_plan_global(Plan& pl, const pf_options* opts, int sms, std::string& msg) {
  int nw = 0;
  cudaError_t e = raise_smem_limit(pl.gk.resolve, pl.smem_resolve);
  if (e == cudaSuccess)
    e = raise_smem_limit(pl.gk.weight, pl.smem_weight);
  if (e == cudaSuccess)
    e = raise_smem_limit(pl.gk.refine_reduce, pl.smem_refine);
  if (e == cudaSuccess) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nw, pl.gk.weight, kBlock, pl.smem_weight);
  if (e != cudaSuccess) { msg = std::string("CUDA: ") + cudaGetErrorString(e); return PF_ECUDA; }
  const int units = (int)((pl.N + kBlock - 1) / kBlock);
  int gw = (opts && opts->grid > 0) ? opts->grid : std::max(1, nw) * sms;
  pl.grid_weight = std::max(1, std::min(gw, units));
  pl.max_grid = pl.grid_weight;
  pl.grid = pl.grid_weight;
  Layout& L = pl.lay;
  size_t off = 0;
  auto take = [&](size_t bytes) { size_t o = off; off = align_up(off + bytes); return o; };
  L.st = take(sizeof(DevState));
  L.x = take((size_t)4 * pl.d * pl.N);
  L.x2 = take((size_t)4 * pl.d * pl.N);
  L.lv0 = take(4);
  L.lv1 = take(4);
  L.anc = pl.record ? take((size_t)4 * pl.N) : 0;
  L.partials = take((size_t)4 * (3 + pl.d) * pl.grid_weight);
  L.y_ring = take((size_t)4 * kRing * pl.dy);
  L.inc_ring = take((size_t)8 * kRing);
  L.mean_ring = take((size_t)4 * kRing * pl.d);
  L.ess_ring = take((size_t)4 * kRing);
  L.lw = take((size_t)4 * pl.N);
  L.P = take((size_t)8 * pl.N);
  L.slot = take((size_t)4 * pl.buckets * pl.bucket_cap);
  L.cnt = take((size_t)4 * (pl.buckets + 1u));
  L.cslot = take((size_t)4 * (1u << pl.cbits) * pl.ccap);
  L.ccnt = take((size_t)4 * ((1u << pl.cbits) + 1u));
  L.covf = take((size_t)4 * pl.N);
  L.ovf = take((size_t)4 * pl.N);
  L.jb = take((size_t)4 * (pl.buckets + 1u));
  L.tsum = take((size_t)8 * pl.nscan);
  L.toff = take((size_t)8 * (pl.nscan + 1u));
  L.done = take(4);
  L.total = off;
  return PF_OK;
}

pf_status finish_plan(Plan& pl, const pf_options* opts, std::string& msg) {
  int dev = 0, sms = 0, nb = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (e == cudaSuccess && pl.global) return finish_plan_global(pl, opts, sms, msg);
  const void* tile_kernel = pl.adaptive ? pl.ak.stage
                            : pl.sets ? select_sets_kernel(pl.d, pl.kind, pl.wide)
                            : pl.sps > 1 ? pl.ks.step_staged : pl.ks.step;
  if (!tile_kernel) { msg = "unsupported (d, model) combination"; return PF_EINVAL; }
  if (e == cudaSuccess)   // opt in beyond the 48 KB default whatever the size
    e = raise_smem_limit(tile_kernel, pl.smem);
  if (e == cudaSuccess) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, tile_kernel, kBlock, pl.smem);
  if (e != cudaSuccess) { msg = std::string("CUDA: ") + cudaGetErrorString(e); return PF_ECUDA; }
  if (nb < 1) { msg = "tile does not fit in shared memory; choose a smaller tile"; return PF_EINVAL; }
  pl.max_grid = 0;
  for (int k = 0; k < pl.m; ++k) {
    DigitPlan& dp = pl.dp[k];
    int units = 0, per_sm = 0;
    if (dp.group) {
      e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, dp.kernel, kBlock, 0);
      if (e != cudaSuccess) { msg = std::string("CUDA: ") + cudaGetErrorString(e); return PF_ECUDA; }
      units = (int)dp.gg.nbatch;
    } else {
      dp.kernel = tile_kernel;
      dp.smem = pl.smem;
      per_sm = nb;
      units = (int)pl.geom[k].ntiles;
    }
    int grid = (opts && opts->grid > 0) ? opts->grid : std::max(1, per_sm) * sms;
    dp.grid = std::max(1, std::min(grid, units));
    pl.max_grid = std::max(pl.max_grid, dp.grid);
  }
  for (int q = 0; q < pl.npass; ++q) {
    int per_sm = 0;
    e = raise_smem_limit(pl.pass_kernel[q], pl.pass_smem[q]);
    if (e == cudaSuccess)
      e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, pl.pass_kernel[q], kBlock, pl.pass_smem[q]);
    if (e != cudaSuccess) { msg = std::string("CUDA: ") + cudaGetErrorString(e); return PF_ECUDA; }
    if (per_sm < 1) { msg = "fused stage tile does not fit in shared memory"; return PF_EINVAL; }
    const int grid = (opts && opts->grid > 0) ? opts->grid : per_sm * sms;
    pl.pass_grid[q] = std::max(1, std::min(grid, (int)pl.pg[q].ntiles));
    pl.max_grid = std::max(pl.max_grid, pl.pass_grid[q]);
  }
  const int grid = pl.max_grid;
  pl.grid = grid;
  Layout& L = pl.lay;
  size_t off = 0;
  auto take = [&](size_t bytes) { size_t o = off; off = align_up(off + bytes); return o; };
  L.st = take(sizeof(DevState));
  L.x = take((size_t)4 * pl.d * pl.N);
  const size_t nlv = pl.adaptive ? pl.N : pl.N / pl.min_a;   // per particle, or per smallest group
  L.lv0 = take((size_t)4 * nlv);
  L.lv1 = take((size_t)4 * nlv);
  L.anc = pl.record ? take((size_t)4 * pl.N) : 0;
  L.prec = pl.record_draws ? take((size_t)8 * pl.N) : 0;
  L.partials = take((size_t)4 * (3 + pl.d) * grid);
  L.y_ring = take((size_t)4 * kRing * pl.dy);
  L.inc_ring = take((size_t)8 * kRing);
  L.mean_ring = take((size_t)4 * kRing * pl.d);
  L.ess_ring = take((size_t)4 * kRing);
  if (pl.islands) {
    L.x2 = take((size_t)4 * pl.d * pl.N);
    L.src = take((size_t)4 * pl.geom[1].a);
    const int smem_isl = (int)(8 * pl.geom[1].a);
    e = raise_smem_limit(pl.ik.stages, (size_t)smem_isl);
    if (e != cudaSuccess) { msg = std::string("CUDA: ") + cudaGetErrorString(e); return PF_ECUDA; }
  }
  L.total = off;
  return PF_OK;
}

// Launch the kernel(s) of stage t of the schedule (digit t mod m).
cudaError_t launch_step(pf_handle* h, cudaStream_t stream, uint64_t t) {
  if (h->plan.global) {
    void* args[] = {&h->P, &h->GP};
    cudaError_t e = cudaLaunchKernel(h->plan.gk.weight, dim3(h->plan.grid_weight), dim3(kBlock), args,
                                     h->plan.smem_weight, stream);
    if (e == cudaSuccess)
      e = cudaLaunchKernel(h->plan.gk.refine_reduce,
                           dim3((h->plan.nscan > 1 ? h->plan.nscan : 0u) + (1u << h->plan.cbits) * h->plan.nseg),
                           dim3(kBlock), args, h->plan.smem_refine, stream);
    if (e == cudaSuccess) e = cudaLaunchKernel(h->plan.gk.scan, dim3(h->plan.nscan), dim3(kBlock), args, 0, stream);
    if (e == cudaSuccess)
      e = cudaLaunchKernel(h->plan.gk.resolve, dim3(h->plan.buckets), dim3(kBlock), args, h->plan.smem_resolve, stream);
    if (e == cudaSuccess) e = cudaLaunchKernel(h->plan.gk.advance, dim3(1), dim3(32), args, 0, stream);
    return e;
  }
  if (h->plan.islands) {    // within-island stage, island stages, gather + mutation
    const Plan& pl = h->plan;
    const uint64_t n = t / 3;
    const uint32_t j = (uint32_t)(t % 3), par = (uint32_t)(n & 1u);
    if (j == 0) {
      const DigitPlan& dp = pl.dp[0];
      if (dp.group) {
        void* args[] = {&h->Pisl[par], const_cast<GroupGeom*>(&dp.gg)};
        return cudaLaunchKernel(dp.kernel, dim3(dp.grid), dim3(kBlock), args, 0, stream);
      }
      void* args[] = {&h->Pisl[par]};
      return cudaLaunchKernel(dp.kernel, dim3(dp.grid), dim3(kBlock), args, dp.smem, stream);
    }
    void* args[] = {&h->Pisl[par], &h->ipar[par]};
    if (j == 1)
      return cudaLaunchKernel(pl.ik.stages, dim3(1), dim3(kIslandThreads), args, (size_t)8 * pl.geom[1].a, stream);
    return cudaLaunchKernel(pl.ik.gather, dim3(pl.max_grid), dim3(kBlock), args, 0, stream);
  }
  if (h->plan.adaptive) {   // launch 0 of a step weights, launch 1 + j runs stage j
    const Plan& pl = h->plan;
    const uint32_t j = (uint32_t)(t % (uint64_t)(pl.m + 1));
    if (j == 0) {
      void* args[] = {&h->P};
      return cudaLaunchKernel(pl.ak.weight, dim3(pl.max_grid), dim3(kBlock), args, 0, stream);
    }
    const DigitPlan& dp = pl.dp[j - 1];
    if (dp.group) {                 // no rotation: launch j - 1 works on digit j - 1
      void* args[] = {&h->P, const_cast<GroupGeom*>(&dp.gg)};
      return cudaLaunchKernel(dp.kernel, dim3(dp.grid), dim3(kBlock), args, 0, stream);
    }
    h->launch_j[j - 1] = j - 1;
    void* args[] = {&h->P, &h->launch_j[j - 1]};
    return cudaLaunchKernel(pl.ak.stage, dim3(pl.max_grid), dim3(kBlock), args, pl.smem, stream);
  }
  if (h->plan.npass) {      // fused all-stages launch t mod npass of its step
    Plan& pl = h->plan;
    const int q = (int)(t % (uint64_t)pl.npass);
    void* args[] = {&h->P, &pl.pg[q]};
    return cudaLaunchKernel(pl.pass_kernel[q], dim3(pl.pass_grid[q]), dim3(kBlock), args, pl.pass_smem[q], stream);
  }
  const uint64_t kd = h->plan.sets ? 1 + t % (uint64_t)(h->plan.m - 1) : t % (uint64_t)h->plan.m;
  DigitPlan& dp = h->plan.dp[kd];
  if (dp.group) {
    void* args[] = {&h->P, &dp.gg};
    return cudaLaunchKernel(dp.kernel, dim3(dp.grid), dim3(kBlock), args, 0, stream);
  }
  void* args[] = {&h->P};
  return cudaLaunchKernel(dp.kernel, dim3(dp.grid), dim3(kBlock), args, dp.smem, stream);
}

}  // namespace

extern "C" {

pf_status pf_workspace_size(const pf_model* model, int64_t N, const int32_t* radices, int32_t m,
                            const pf_options* opts, size_t* bytes) {
  if (!bytes) return fail(nullptr, PF_EINVAL, "bytes is NULL");
  Plan pl;
  std::string msg;
  pf_status s = make_plan(model, N, radices, m, opts, pl, msg);
  if (s == PF_OK) s = finish_plan(pl, opts, msg);
  if (s != PF_OK) return fail(nullptr, s, msg);
  *bytes = pl.lay.total;
  return PF_OK;
}

pf_status pf_create(const pf_model* model, int64_t N, const int32_t* radices, int32_t m, uint64_t seed,
                    const pf_options* opts, void* workspace, size_t workspace_bytes, pf_handle** out) {
  if (!out) return fail(nullptr, PF_EINVAL, "out is NULL");
  *out = nullptr;
  pf_handle* h = new (std::nothrow) pf_handle();
  if (!h) return fail(nullptr, PF_ENOMEM, "host allocation failed");
  std::string msg;
  pf_status s = make_plan(model, N, radices, m, opts, h->plan, msg);
  if (s == PF_OK) s = finish_plan(h->plan, opts, msg);
  if (s != PF_OK) {
    delete h;
    return fail(nullptr, s, msg);
  }
  Plan& pl = h->plan;
  cudaGetDevice(&h->device);
  h->stream = opts ? static_cast<cudaStream_t>(opts->stream) : nullptr;
  h->flags = opts ? opts->flags : 0u;
  h->seed = seed;
  for (int32_t k = 0; k < m; ++k) h->radices[k] = radices[k];
  if (workspace) {
    if (workspace_bytes < pl.lay.total) {
      delete h;
      return fail(nullptr, PF_ENOMEM, "workspace smaller than pf_workspace_size()");
    }
    if (reinterpret_cast<uintptr_t>(workspace) % kAlign) {
      delete h;
      return fail(nullptr, PF_EINVAL, "workspace must be 256-byte aligned");
    }
    h->ws = static_cast<unsigned char*>(workspace);
    h->ws_bytes = workspace_bytes;
  } else {
    cudaError_t e = cudaMalloc(&h->ws, pl.lay.total);
    if (e != cudaSuccess) {
      delete h;
      return fail(nullptr, PF_ENOMEM, std::string("cudaMalloc: ") + cudaGetErrorString(e));
    }
    h->own_ws = true;
    h->ws_bytes = pl.lay.total;
  }
  cudaError_t e = cudaStreamCreateWithFlags(&h->cap_stream, cudaStreamNonBlocking);
  if (e != cudaSuccess) {
    if (h->own_ws) cudaFree(h->ws);
    delete h;
    return fail(nullptr, PF_ECUDA, std::string("cudaStreamCreate: ") + cudaGetErrorString(e));
  }
  StepParams& P = h->P;
  const Layout& L = pl.lay;
  P.x = reinterpret_cast<float*>(h->ws + L.x);
  P.lV[0] = reinterpret_cast<float*>(h->ws + L.lv0);
  P.lV[1] = reinterpret_cast<float*>(h->ws + L.lv1);
  P.anc = pl.record ? reinterpret_cast<int32_t*>(h->ws + L.anc) : nullptr;
  // the global path keeps its prefix sums in L.P; the others record them on request
  P.prec = (pl.record_draws && !pl.global) ? reinterpret_cast<unsigned long long*>(h->ws + L.prec) : nullptr;
  P.st = reinterpret_cast<DevState*>(h->ws + L.st);
  P.partials = reinterpret_cast<float*>(h->ws + L.partials);
  P.y_ring = reinterpret_cast<const float*>(h->ws + L.y_ring);
  P.inc_ring = reinterpret_cast<double*>(h->ws + L.inc_ring);
  P.mean_ring = reinterpret_cast<float*>(h->ws + L.mean_ring);
  P.ess_ring = reinterpret_cast<float*>(h->ws + L.ess_ring);
  P.N = pl.N;
  P.m = pl.m;
  P.seed_lo = (uint32_t)seed;
  P.seed_hi = (uint32_t)(seed >> 32);
  P.rk = make_round_keys(seed);
  P.tile_cap = pl.cap;
  P.inv_N = (float)(1.0 / pl.N);
  P.sps = pl.sps;
  P.theta = pl.theta;
  P.rotate = pl.rotate ? 1u : 0u;
  P.model = pl.mp;
  std::memcpy(P.geom, pl.geom, sizeof(P.geom));
  if (pl.islands) {
    float* xb[2] = {P.x, reinterpret_cast<float*>(h->ws + L.x2)};
    for (int par = 0; par < 2; ++par) {
      h->Pisl[par] = P;
      h->Pisl[par].x = xb[par];
      IslandParams& ip = h->ipar[par];
      ip.x_out = xb[par ^ 1];
      ip.src = reinterpret_cast<int32_t*>(h->ws + L.src);
      ip.lW = P.lV[1];          // the within-island stage (stage counter 2n) writes lV[1]
      ip.lV_next = P.lV[0];     // and reads lV[0]
      ip.M = pl.geom[0].a;
      ip.islands = pl.geom[1].a;
      uint32_t S = 0;
      while ((1u << S) < ip.islands) ++S;
      ip.S = S;
      ip.plain = pl.island_plain ? 1u : 0u;
      ip.adaptive = pl.island_adaptive ? 1u : 0u;
      ip.theta = pl.island_theta;
    }
  }
  if (pl.global) {
    GlobalParams& G = h->GP;
    G.xbuf[0] = P.x;
    G.xbuf[1] = reinterpret_cast<float*>(h->ws + L.x2);
    G.lw = reinterpret_cast<float*>(h->ws + L.lw);
    G.P = reinterpret_cast<unsigned long long*>(h->ws + L.P);
    G.tsum = reinterpret_cast<unsigned long long*>(h->ws + L.tsum);
    G.toff = reinterpret_cast<unsigned long long*>(h->ws + L.toff);
    G.done = reinterpret_cast<uint32_t*>(h->ws + L.done);
    G.slot = reinterpret_cast<uint32_t*>(h->ws + L.slot);
    G.cnt = reinterpret_cast<uint32_t*>(h->ws + L.cnt);
    G.ovf = reinterpret_cast<uint32_t*>(h->ws + L.ovf);
    G.cslot = reinterpret_cast<uint32_t*>(h->ws + L.cslot);
    G.ccnt = reinterpret_cast<uint32_t*>(h->ws + L.ccnt);
    G.covf = reinterpret_cast<uint32_t*>(h->ws + L.covf);
    G.jb = reinterpret_cast<uint32_t*>(h->ws + L.jb);
    G.cbits = pl.cbits;
    G.ccap = pl.ccap;
    G.nseg = pl.nseg;
    G.nscan = pl.nscan;
    G.log2b = pl.log2b;
    G.buckets = pl.buckets;
    G.cap = pl.bucket_cap;
    G.stage_cap = pl.stage_cap;
  }

  // Algorithm 1, first loop: zeta_0 ~ pi_0; carried weights start at zero.
  auto bail = [&](cudaError_t err, const char* what) {
    std::string m2 = std::string(what) + ": " + cudaGetErrorString(err);
    cudaStreamDestroy(h->cap_stream);
    if (h->own_ws) cudaFree(h->ws);
    delete h;
    return fail(nullptr, PF_ECUDA, m2);
  };
  e = cudaMemsetAsync(h->ws + L.st, 0, sizeof(DevState), h->stream);
  if (e != cudaSuccess) return bail(e, "cudaMemsetAsync");
  e = cudaMemsetAsync(h->ws + L.lv0, 0, pl.global ? 4 : (size_t)4 * (pl.adaptive ? pl.N : pl.N / pl.min_a),
                      h->stream);
  if (e != cudaSuccess) return bail(e, "cudaMemsetAsync");
  if (pl.global) {
    e = cudaMemsetAsync(h->ws + L.done, 0, 4, h->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(h->ws + L.cnt, 0, (size_t)4 * (pl.buckets + 1u), h->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(h->ws + L.ccnt, 0, (size_t)4 * ((1u << pl.cbits) + 1u), h->stream);
    if (e != cudaSuccess) return bail(e, "cudaMemsetAsync");
  }
  int sms = 0;
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, h->device);
  const uint32_t blocks = std::min<uint32_t>((pl.N + kBlock - 1) / kBlock, (uint32_t)std::max(1, sms) * 8);
  void* args[] = {&h->P};
  e = cudaLaunchKernel(pl.ks.init, dim3(blocks), dim3(kBlock), args, 0, h->stream);
  if (e != cudaSuccess) return bail(e, "init kernel");
  *out = h;
  return PF_OK;
}

pf_status pf_step(pf_handle* h, const float* y_n, float* mean_out, double* loglik_inc, float* ess_out) {
  if (!h) return fail(nullptr, PF_EINVAL, "handle is NULL");
  if (!y_n) return fail(h, PF_EINVAL, "y_n is NULL");
  if (h->n_pushed != h->n_host) return fail(h, PF_ESTATE, "observations pushed but not consumed");
  pf_status s = pf_push_observations(h, y_n, 1);
  if (s == PF_OK) s = pf_advance(h, 1, mean_out, loglik_inc, ess_out);
  return s;
}

pf_status pf_push_observations(pf_handle* h, const float* y, int32_t T) {
  if (!h) return fail(nullptr, PF_EINVAL, "handle is NULL");
  if (T < 0 || (T > 0 && !y)) return fail(h, PF_EINVAL, "need T >= 0 and y != NULL");
  if (h->n_pushed + (uint64_t)T - h->n_host > kRing)
    return fail(h, PF_ESTATE, "more than 1024 observations pushed ahead of the steps taken");
  const Plan& pl = h->plan;
  int32_t done = 0;
  while (done < T) {   // at most two contiguous pieces of the ring
    const uint32_t slot = (uint32_t)(h->n_pushed % kRing);
    const int32_t L = std::min<int32_t>(T - done, (int32_t)(kRing - slot));
    PF_CUDA(h, cudaMemcpyAsync(const_cast<float*>(h->P.y_ring) + (size_t)slot * pl.dy, y + (size_t)done * pl.dy,
                               (size_t)4 * pl.dy * L, cudaMemcpyDefault, h->stream));
    h->n_pushed += L;
    done += L;
  }
  return PF_OK;
}

namespace {

// L steps on pushed observations, starting at step h->n_host (L * sps stage
// launches, from stage counter t0 = n_host * sps): a captured graph (one per
// radix phase t0 mod m, since the kernel depends on the digit) when L is the
// chunk length, else individual launches.
pf_status enqueue_steps(pf_handle* h, int32_t L) {
  Trace tr("bfpf steps");
  const Plan& pl = h->plan;
  const uint64_t lps = pl.islands ? 3 : pl.adaptive ? (uint64_t)pl.m + 1
                                       : pl.npass ? (uint64_t)pl.npass : pl.sps;   // launches per step
  const uint64_t t0 = h->n_host * lps;
  const int64_t launches = (int64_t)L * (int64_t)lps;
  if (L == pl.chunk_len && L > 1) {
    if (h->graphs.empty()) h->graphs.assign(pl.m, nullptr);
    cudaGraphExec_t& exec =
        h->graphs[pl.islands ? h->n_host & 1u : (pl.adaptive || pl.sets || pl.npass) ? 0 : t0 % (uint64_t)pl.m];
    if (!exec) {
      cudaGraph_t graph = nullptr;
      PF_CUDA(h, cudaStreamBeginCapture(h->cap_stream, cudaStreamCaptureModeThreadLocal));
      cudaError_t le = cudaSuccess;
      for (int64_t j = 0; j < launches && le == cudaSuccess; ++j) le = launch_step(h, h->cap_stream, t0 + j);
      cudaError_t ce = cudaStreamEndCapture(h->cap_stream, &graph);
      if (le != cudaSuccess) return fail(h, PF_ECUDA, std::string("capture launch: ") + cudaGetErrorString(le));
      if (ce != cudaSuccess) return fail(h, PF_ECUDA, std::string("cudaStreamEndCapture: ") + cudaGetErrorString(ce));
      cudaError_t ie = cudaGraphInstantiate(&exec, graph, 0);
      cudaGraphDestroy(graph);
      if (ie != cudaSuccess) {
        exec = nullptr;
        return fail(h, PF_ECUDA, std::string("cudaGraphInstantiate: ") + cudaGetErrorString(ie));
      }
    }
    PF_CUDA(h, cudaGraphLaunch(exec, h->stream));
  } else {
    for (int64_t j = 0; j < launches; ++j) PF_CUDA(h, launch_step(h, h->stream, t0 + j));
  }
  return PF_OK;
}

}  // namespace

pf_status pf_advance(pf_handle* h, int32_t T, float* means, double* loglik_incs, float* ess) {
  if (!h) return fail(nullptr, PF_EINVAL, "handle is NULL");
  if (T < 0) return fail(h, PF_EINVAL, "need T >= 0");
  if (h->n_host + (uint64_t)T > h->n_pushed) return fail(h, PF_ESTATE, "fewer observations pushed than steps asked");
  const Plan& pl = h->plan;
  int32_t done = 0;
  while (done < T) {
    const uint32_t slot0 = (uint32_t)(h->n_host % kRing);
    const int32_t L = std::min<int32_t>({pl.chunk_len, T - done, (int32_t)(kRing - slot0)});
    pf_status s = enqueue_steps(h, L);
    if (s != PF_OK) return s;
    if (means)
      PF_CUDA(h, cudaMemcpyAsync(means + (size_t)done * pl.d, h->P.mean_ring + (size_t)slot0 * pl.d,
                                 (size_t)4 * pl.d * L, cudaMemcpyDefault, h->stream));
    if (loglik_incs)
      PF_CUDA(h, cudaMemcpyAsync(loglik_incs + done, h->P.inc_ring + slot0, (size_t)8 * L, cudaMemcpyDefault,
                                 h->stream));
    if (ess)
      PF_CUDA(h, cudaMemcpyAsync(ess + done, h->P.ess_ring + slot0, (size_t)4 * L, cudaMemcpyDefault, h->stream));
    h->n_host += L;
    done += L;
  }
  PF_CUDA(h, cudaGetLastError());
  if (is_host_ptr(means) || is_host_ptr(loglik_incs) || is_host_ptr(ess)) PF_CUDA(h, cudaStreamSynchronize(h->stream));
  return PF_OK;
}

pf_status pf_run(pf_handle* h, const float* y, int32_t T, float* means, double* loglik_incs, float* ess) {
  if (!h) return fail(nullptr, PF_EINVAL, "handle is NULL");
  if (T < 0 || (T > 0 && !y)) return fail(h, PF_EINVAL, "need T >= 0 and y != NULL");
  if (h->n_pushed != h->n_host) return fail(h, PF_ESTATE, "observations pushed but not consumed");
  const Plan& pl = h->plan;
  int32_t done = 0;
  while (done < T) {
    const uint32_t slot0 = (uint32_t)(h->n_host % kRing);
    const int32_t L = std::min<int32_t>({pl.chunk_len, T - done, (int32_t)(kRing - slot0)});
    pf_status s = pf_push_observations(h, y + (size_t)done * pl.dy, L);
    if (s == PF_OK) s = pf_advance(h, L, means ? means + (size_t)done * pl.d : nullptr,
                                  loglik_incs ? loglik_incs + done : nullptr, ess ? ess + done : nullptr);
    if (s != PF_OK) return s;
    done += L;
  }
  return PF_OK;
}

pf_status pf_loglik(const pf_handle* h, double* out) {
  if (!h || !out) return fail(h, PF_EINVAL, "NULL argument");
  DevState st;
  PF_CUDA(h, cudaMemcpyAsync(&st, h->P.st, sizeof(st), cudaMemcpyDeviceToHost, h->stream));
  PF_CUDA(h, cudaStreamSynchronize(h->stream));
  *out = st.loglik;
  return PF_OK;
}

pf_status pf_get_state(const pf_handle* h, float* x, float* lV, double* scalars) {
  if (!h) return fail(nullptr, PF_EINVAL, "handle is NULL");
  const Plan& pl = h->plan;
  DevState st;
  PF_CUDA(h, cudaMemcpyAsync(&st, h->P.st, sizeof(st), cudaMemcpyDeviceToHost, h->stream));
  PF_CUDA(h, cudaStreamSynchronize(h->stream));
  const float* xcur = pl.global ? h->GP.xbuf[st.n & 1u] : pl.islands ? h->Pisl[st.n & 1u].x : h->P.x;
  if (x) PF_CUDA(h, cudaMemcpyAsync(x, xcur, (size_t)4 * pl.d * pl.N, cudaMemcpyDeviceToHost, h->stream));
  PF_CUDA(h, cudaStreamSynchronize(h->stream));
  if (lV && pl.adaptive) {
    PF_CUDA(h, cudaMemcpyAsync(lV, h->P.lV[st.lvp & 1u], (size_t)4 * pl.N, cudaMemcpyDeviceToHost, h->stream));
    PF_CUDA(h, cudaStreamSynchronize(h->stream));
  } else if (lV) {
    const uint64_t t = (uint64_t)st.n * pl.sps + st.stage;   // stage counter
    const int kp = pl.sets ? (int)(1 + (t + pl.m - 2) % (pl.m - 1)) : (int)((t + pl.m - 1) % pl.m);
    const size_t cnt = pl.global ? 1 : pl.island_adaptive ? pl.N / pl.geom[0].a
                                     : pl.N / (pl.geom[kp].a * pl.geom[kp].w);
    // (fused all-stages launches alternate the buffers per launch: step n starts on (n npass) mod 2)
    const uint64_t sel = pl.npass ? (uint64_t)st.n * (uint64_t)pl.npass : t;
    PF_CUDA(h, cudaMemcpyAsync(lV, h->P.lV[sel & 1u], 4 * cnt, cudaMemcpyDeviceToHost, h->stream));
    PF_CUDA(h, cudaStreamSynchronize(h->stream));
  }
  if (scalars) {
    scalars[0] = (double)st.n;
    scalars[1] = st.loglik;
    scalars[2] = st.mu;
    scalars[3] = (double)st.mu_f;
  }
  return PF_OK;
}

pf_status pf_get_ancestors(const pf_handle* h, int32_t* anc) {
  if (!h || !anc) return fail(h, PF_EINVAL, "NULL argument");
  if (!h->P.anc) return fail(h, PF_ESTATE, "ancestors are not recorded (create with PF_RECORD_ANCESTORS)");
  PF_CUDA(h, cudaMemcpyAsync(anc, h->P.anc, (size_t)4 * h->plan.N, cudaMemcpyDeviceToHost, h->stream));
  PF_CUDA(h, cudaStreamSynchronize(h->stream));
  return PF_OK;
}

pf_status pf_get_draw_prefix(const pf_handle* h, uint64_t* prefix) {
  if (!h || !prefix) return fail(h, PF_EINVAL, "NULL argument");
  const void* src = nullptr;
  if (h->plan.global) src = h->ws + h->plan.lay.P;
  else if (h->P.prec) src = h->P.prec;
  else return fail(h, PF_ESTATE, "draws are not recorded (create with PF_RECORD_DRAWS)");
  PF_CUDA(h, cudaMemcpyAsync(prefix, src, (size_t)8 * h->plan.N, cudaMemcpyDeviceToHost, h->stream));
  PF_CUDA(h, cudaStreamSynchronize(h->stream));
  return PF_OK;
}

pf_status pf_get_status(const pf_handle* h, uint32_t* bits) {
  if (!h || !bits) return fail(h, PF_EINVAL, "NULL argument");
  DevState st;
  PF_CUDA(h, cudaMemcpyAsync(&st, h->P.st, sizeof(st), cudaMemcpyDeviceToHost, h->stream));
  PF_CUDA(h, cudaStreamSynchronize(h->stream));
  *bits = st.status;
  return PF_OK;
}

// ---------------------------------------------------------------------------
// Checkpoint / resume: the whole device workspace plus the host counters.
// ---------------------------------------------------------------------------
namespace {

struct CheckpointHeader {
  char magic[8];            // "BFPFCKP1"
  uint32_t version;
  uint32_t N;
  int32_t m, d, dy, kind;
  int32_t radices[kMaxDigits];
  uint32_t flags, pad;
  uint64_t seed;
  uint64_t model_hash;      // FNV-1a of the device model parameters
  uint64_t ws_bytes;
  uint64_t n_host, n_pushed;
};

uint64_t fnv1a(const void* data, size_t n) {
  const unsigned char* b = static_cast<const unsigned char*>(data);
  uint64_t hsh = 1469598103934665603ull;
  for (size_t i = 0; i < n; ++i) {
    hsh ^= b[i];
    hsh *= 1099511628211ull;
  }
  return hsh;
}

void fill_header(const pf_handle* h, CheckpointHeader& hd) {
  std::memset(&hd, 0, sizeof(hd));
  std::memcpy(hd.magic, "BFPFCKP1", 8);
  hd.version = 1;
  hd.N = h->plan.N;
  hd.m = h->plan.m;
  hd.d = h->plan.d;
  hd.dy = h->plan.dy;
  hd.kind = h->plan.kind;
  for (int k = 0; k < h->plan.m; ++k) hd.radices[k] = h->radices[k];
  hd.flags = h->flags;
  hd.seed = h->seed;
  hd.model_hash = fnv1a(&h->plan.mp, sizeof(h->plan.mp));
  hd.ws_bytes = h->plan.lay.total;
  hd.n_host = h->n_host;
  hd.n_pushed = h->n_pushed;
}

}  // namespace

pf_status pf_checkpoint_size(const pf_handle* h, size_t* bytes) {
  if (!h || !bytes) return fail(h, PF_EINVAL, "NULL argument");
  *bytes = sizeof(CheckpointHeader) + h->plan.lay.total;
  return PF_OK;
}

pf_status pf_save(const pf_handle* h, void* buf, size_t len) {
  Trace tr("bfpf save");
  if (!h || !buf) return fail(h, PF_EINVAL, "NULL argument");
  if (len < sizeof(CheckpointHeader) + h->plan.lay.total) return fail(h, PF_EINVAL, "buffer smaller than pf_checkpoint_size()");
  CheckpointHeader hd;
  fill_header(h, hd);
  std::memcpy(buf, &hd, sizeof(hd));
  PF_CUDA(h, cudaMemcpyAsync(static_cast<unsigned char*>(buf) + sizeof(hd), h->ws, h->plan.lay.total,
                             cudaMemcpyDeviceToHost, h->stream));
  PF_CUDA(h, cudaStreamSynchronize(h->stream));
  return PF_OK;
}

pf_status pf_load(pf_handle* h, const void* buf, size_t len) {
  Trace tr("bfpf load");
  if (!h || !buf) return fail(h, PF_EINVAL, "NULL argument");
  if (len < sizeof(CheckpointHeader)) return fail(h, PF_EINVAL, "buffer too small for a checkpoint");
  CheckpointHeader hd, mine;
  std::memcpy(&hd, buf, sizeof(hd));
  fill_header(h, mine);
  if (std::memcmp(hd.magic, mine.magic, 8) != 0 || hd.version != mine.version)
    return fail(h, PF_EINVAL, "not a checkpoint of this library");
  if (hd.N != mine.N || hd.m != mine.m || hd.d != mine.d || hd.dy != mine.dy || hd.kind != mine.kind ||
      std::memcmp(hd.radices, mine.radices, sizeof(hd.radices)) != 0 || hd.flags != mine.flags ||
      hd.seed != mine.seed || hd.model_hash != mine.model_hash || hd.ws_bytes != mine.ws_bytes)
    return fail(h, PF_EINVAL, "the checkpoint was taken from a filter with another model, N, radices, seed or options");
  if (len < sizeof(hd) + hd.ws_bytes) return fail(h, PF_EINVAL, "checkpoint truncated");
  PF_CUDA(h, cudaMemcpyAsync(h->ws, static_cast<const unsigned char*>(buf) + sizeof(hd), hd.ws_bytes,
                             cudaMemcpyHostToDevice, h->stream));
  PF_CUDA(h, cudaStreamSynchronize(h->stream));
  h->n_host = hd.n_host;
  h->n_pushed = hd.n_pushed;
  return PF_OK;
}

pf_status pf_stage_count(const pf_handle* h, uint64_t* out) {
  if (!h || !out) return fail(h, PF_EINVAL, "NULL argument");
  DevState st;
  PF_CUDA(h, cudaMemcpyAsync(&st, h->P.st, sizeof(st), cudaMemcpyDeviceToHost, h->stream));
  PF_CUDA(h, cudaStreamSynchronize(h->stream));
  *out = (h->plan.adaptive || h->plan.island_adaptive) ? st.nstages : (uint64_t)st.n * h->plan.sps + st.stage;
  return PF_OK;
}

pf_status pf_describe(const pf_handle* h, char* buf, size_t len) {
  if (!h || !buf || len == 0) return fail(h, PF_EINVAL, "NULL argument");
  const Plan& pl = h->plan;
  std::string o = "{\"N\": " + std::to_string(pl.N) + ", \"d\": " + std::to_string(pl.d) +
                  ", \"stages_per_step\": " + std::to_string(pl.sps) +
                  ", \"launches_per_step\": " +
                  std::to_string(pl.global ? 5 : pl.islands ? 3 : pl.adaptive ? pl.m + 1 : pl.npass ? pl.npass : (int)pl.sps) +
                  ", \"adaptive\": " + (pl.adaptive ? "true" : "false") +
                  ", \"rotate\": " + (pl.rotate ? "true" : "false") +
                  ", \"ess_threshold\": " + std::to_string(pl.adaptive ? pl.theta : 0.0f) +
                  ", \"islands\": " + std::to_string(pl.islands ? pl.geom[1].a : 0) +
                  ", \"digit_sets\": " + (pl.sets ? "true" : "false") +
                  ", \"island_resampling\": \"" + (pl.islands ? (pl.island_plain ? "algorithm6" : "algorithm7") : "") +
                  (pl.island_adaptive ? "+adapted" : "") +
                  "\", \"digits\": [";
  if (pl.global)
    o += "{\"a\": " + std::to_string(pl.N) + ", \"s\": 1, \"kernel\": \"global\", \"scan_tiles\": " +
         std::to_string(pl.nscan) + ", \"grid\": " + std::to_string(pl.grid_weight) + ", \"buckets\": " +
         std::to_string(pl.buckets) + ", \"bucket_cap\": " + std::to_string(pl.bucket_cap) +
         ", \"stage_cap\": " + std::to_string(pl.stage_cap) + ", \"coarse_bins\": " +
         std::to_string(1u << pl.cbits) + ", \"coarse_cap\": " + std::to_string(pl.ccap) + "}";
  else
  for (int k = 0; k < pl.m; ++k) {
    const DigitPlan& dp = pl.dp[k];
    const DigitGeom& g = pl.geom[k];
    if (k) o += ", ";
    o += "{\"a\": " + std::to_string(g.a) + ", \"s\": " + std::to_string(g.s) + ", \"kernel\": \"" +
         (dp.group ? "group" : "tile") + "\", " +
         (dp.group ? "\"lanes\": " + std::to_string(dp.lanes) : "\"tile\": " + std::to_string(g.tile_n)) +
         ", \"grid\": " + std::to_string(dp.grid) + "}";
  }
  o += "]";
  if (pl.npass) {
    o += ", \"fused\": [";
    for (int q = 0; q < pl.npass; ++q) {
      const PassGeom& g = pl.pg[q];
      if (q) o += ", ";
      o += "{\"k0\": " + std::to_string(g.k0) + ", \"digits\": " + std::to_string(g.J) + ", \"tile\": " +
           std::to_string(1u << g.log2T) + ", \"lows\": " + std::to_string(1u << g.log2L) + ", \"grid\": " +
           std::to_string(pl.pass_grid[q]) + ", \"smem\": " + std::to_string(pl.pass_smem[q]) + "}";
    }
    o += "]";
  }
  o += "}";
  const size_t nb = std::min(len - 1, o.size());
  std::memcpy(buf, o.data(), nb);
  buf[nb] = 0;
  return PF_OK;
}

pf_status pf_destroy(pf_handle* h) {
  if (!h) return PF_OK;
  cudaError_t e = cudaStreamSynchronize(h->stream);
  for (cudaGraphExec_t g : h->graphs)
    if (g) cudaGraphExecDestroy(g);
  if (h->cap_stream) cudaStreamDestroy(h->cap_stream);
  if (h->own_ws && h->ws) cudaFree(h->ws);
  delete h;
  if (e != cudaSuccess) return fail(nullptr, PF_ECUDA, std::string("cudaStreamSynchronize: ") + cudaGetErrorString(e));
  return PF_OK;
}

const char* pf_last_error(const pf_handle* h) {
  if (h) return h->err.c_str();
  return t_error.c_str();
}

pf_status pf_philox_blocks(uint64_t seed, uint32_t c0, uint32_t c1, uint32_t c2, uint32_t c3, int64_t count,
                           uint32_t* out, void* stream) {
  if (!out || count < 0 || count > 0x7fffffff) return fail(nullptr, PF_EINVAL, "bad arguments");
  if (count == 0) return PF_OK;
  cudaError_t e = launch_philox_blocks(seed, make_uint4(c0, c1, c2, c3), (uint32_t)count, out,
                                       static_cast<cudaStream_t>(stream));
  if (e != cudaSuccess) return fail(nullptr, PF_ECUDA, std::string("philox kernel: ") + cudaGetErrorString(e));
  return PF_OK;
}

}  // extern "C"

// ---------------------------------------------------------------------------
// pf_step_noalloc: one step with the temporaries in a fixed, library-owned
// scratch area instead of an allocated workspace.
// ---------------------------------------------------------------------------
namespace {

constexpr int kNoAllocMaxBlocks = 2048;
constexpr size_t kNoAllocStateOff = 0;
constexpr size_t kNoAllocPartialsOff = 256;
constexpr size_t kNoAllocPartialsBytes = (size_t)4 * (3 + kMaxDim) * kNoAllocMaxBlocks;   // 90,112
constexpr size_t kNoAllocYOff = kNoAllocPartialsOff + kNoAllocPartialsBytes;
constexpr size_t kNoAllocIncOff = kNoAllocYOff + (size_t)4 * kRing * kMaxDim;
constexpr size_t kNoAllocMeanOff = kNoAllocIncOff + (size_t)8 * kRing;
constexpr size_t kNoAllocEssOff = kNoAllocMeanOff + (size_t)4 * kRing * kMaxDim;
constexpr size_t kNoAllocBytes = 192 * 1024;
static_assert(kNoAllocEssOff + 4 * kRing <= kNoAllocBytes, "scratch layout exceeds its size");
constexpr int kNoAllocMaxDevices = 64;

// The scratch area.  In host code this name is only a stand-in for the
// symbol; its device address comes from cudaGetSymbolAddress below.
static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocBytes];

std::mutex g_noalloc_mutex;
unsigned char* g_noalloc_addr[kNoAllocMaxDevices] = {};

// Device address of the scratch area on the current device, resolved once per device.
cudaError_t noalloc_scratch(unsigned char** out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= kNoAllocMaxDevices) return cudaErrorInvalidDevice;
  std::lock_guard<std::mutex> lock(g_noalloc_mutex);
  if (!g_noalloc_addr[dev]) {
    void* ptr = nullptr;
    e = cudaGetSymbolAddress(&ptr, g_noalloc_scratch);
    if (e != cudaSuccess) return e;
    g_noalloc_addr[dev] = static_cast<unsigned char*>(ptr);
  }
  *out = g_noalloc_addr[dev];
  return cudaSuccess;
}

struct NoAllocStart {
  double mu;
  uint32_t n;
  uint32_t dy;
  float y[kMaxDim];
};

// Clears the device state block (block counter, status, likelihood) and puts
// this step's observation and normaliser in place.
__global__ void noalloc_start_kernel(DevState* st, float* y_ring, NoAllocStart s) {
  if (threadIdx.x == 0) {
    st->n = s.n;
    st->stage = 0;
    st->done = 0;
    st->status = 0;
    st->mu = s.mu;
    st->mu_f = (float)s.mu;
    st->loglik = 0.0;
    for (uint32_t j = 0; j < s.dy; ++j) y_ring[(s.n % kRing) * s.dy + j] = s.y[j];
  }
}

}  // namespace

extern "C" pf_status pf_step_noalloc(const pf_model* model, int64_t N, const int32_t* radices, int32_t m,
                                     uint64_t seed, uint32_t n, double mu, float* x, const float* lV_in,
                                     float* lV_out, const float* y_n, double* out, float* mean_out,
                                     uint32_t* status_out, void* stream) {
  if (!x || !lV_in || !lV_out || !y_n || !out) return fail(nullptr, PF_EINVAL, "NULL argument");
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  if (st) {   // the scratch address and the launch plan belong to the current device
    int cur = 0, sdev = 0;
    cudaError_t e0 = cudaGetDevice(&cur);
    if (e0 == cudaSuccess) e0 = cudaStreamGetDevice(st, &sdev);
    if (e0 != cudaSuccess) return fail(nullptr, PF_ECUDA, std::string("stream device: ") + cudaGetErrorString(e0));
    if (sdev != cur) return fail(nullptr, PF_EINVAL, "the stream belongs to another device than the current one");
  }
  Plan pl;
  std::string msg;
  pf_status s = make_plan(model, N, radices, m, nullptr, pl, msg);
  if (s == PF_OK && pl.global) {
    s = PF_EINVAL;
    msg = "global resampling (radices = {N}, N > 1024) needs a handle from pf_create";
  }
  if (s == PF_OK) s = finish_plan(pl, nullptr, msg);
  if (s != PF_OK) return fail(nullptr, s, msg);
  unsigned char* scratch = nullptr;
  cudaError_t e = noalloc_scratch(&scratch);
  if (e != cudaSuccess) return fail(nullptr, PF_ECUDA, std::string("cudaGetSymbolAddress: ") + cudaGetErrorString(e));

  StepParams P{};
  P.rk = make_round_keys(seed);
  P.x = x;
  P.lV[n & 1u] = const_cast<float*>(lV_in);
  P.lV[(n & 1u) ^ 1u] = lV_out;
  P.anc = nullptr;
  P.st = reinterpret_cast<DevState*>(scratch + kNoAllocStateOff);
  P.partials = reinterpret_cast<float*>(scratch + kNoAllocPartialsOff);
  P.y_ring = reinterpret_cast<const float*>(scratch + kNoAllocYOff);
  P.inc_ring = reinterpret_cast<double*>(scratch + kNoAllocIncOff);
  P.mean_ring = reinterpret_cast<float*>(scratch + kNoAllocMeanOff);
  P.ess_ring = reinterpret_cast<float*>(scratch + kNoAllocEssOff);
  P.N = pl.N;
  P.m = pl.m;
  P.seed_lo = (uint32_t)seed;
  P.seed_hi = (uint32_t)(seed >> 32);
  P.tile_cap = pl.cap;
  P.inv_N = (float)(1.0 / pl.N);
  P.sps = 1;
  P.model = pl.mp;
  std::memcpy(P.geom, pl.geom, sizeof(P.geom));

  NoAllocStart start{};
  start.mu = mu;
  start.n = n;
  start.dy = (uint32_t)pl.dy;
  for (int j = 0; j < pl.dy; ++j) start.y[j] = y_n[j];
  noalloc_start_kernel<<<1, 32, 0, st>>>(P.st, const_cast<float*>(P.y_ring), start);
  e = cudaGetLastError();
  if (e != cudaSuccess) return fail(nullptr, PF_ECUDA, std::string("start kernel: ") + cudaGetErrorString(e));
  DigitPlan& dp = pl.dp[n % (uint32_t)pl.m];
  // The scratch area holds the partial sums of at most kNoAllocMaxBlocks blocks.
  // The step kernels stride over their units by gridDim and the fold of the
  // partials runs over gridDim, so a smaller grid only takes more iterations.
  const int grid = std::min(dp.grid, kNoAllocMaxBlocks);
  if (dp.group) {
    void* args[] = {&P, &dp.gg};
    e = cudaLaunchKernel(dp.kernel, dim3(grid), dim3(kBlock), args, 0, st);
  } else {
    void* args[] = {&P};
    e = cudaLaunchKernel(dp.kernel, dim3(grid), dim3(kBlock), args, dp.smem, st);
  }
  if (e != cudaSuccess) return fail(nullptr, PF_ECUDA, std::string("step kernel: ") + cudaGetErrorString(e));
  const uint32_t slot = n % kRing;
  DevState dst;
  float ess = 0.0f;
  e = cudaMemcpyAsync(&dst, P.st, sizeof(dst), cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaMemcpyAsync(&out[0], P.inc_ring + slot, 8, cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaMemcpyAsync(&ess, P.ess_ring + slot, 4, cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess && mean_out)
    e = cudaMemcpyAsync(mean_out, P.mean_ring + (size_t)slot * pl.d, (size_t)4 * pl.d, cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) return fail(nullptr, PF_ECUDA, std::string("copy back: ") + cudaGetErrorString(e));
  out[1] = dst.mu;
  out[2] = (double)ess;
  if (status_out) *status_out = dst.status;
  return PF_OK;
}

// ---------------------------------------------------------------------------
// Batches of independent filters
// ---------------------------------------------------------------------------
struct pf_batch {
  int device = 0;
  cudaStream_t stream = nullptr;
  cudaStream_t cap_stream = nullptr;
  cudaStream_t side = nullptr;              // the tile-path kernels of a step run beside the group path
  cudaEvent_t fork_ev = nullptr, join_ev = nullptr;
  bool own_ws = false;
  unsigned char* ws = nullptr;
  size_t ws_bytes = 0;
  int F = 0, ring = 64, dy_max = 1, d_max = 1;
  size_t smem = 0;
  BatchParams BP{};
  std::vector<BatchFilter> host_filters;    // host copy (pointers, sizes, geometry)
  std::vector<uint2> units;                 // {filter, j | U << 16}, by class, largest work first
  struct Class {
    const void* kernel;                     // tile path
    const void* gkernel;                    // group path
    uint32_t u0, count;                     // the class's units
    uint32_t g0, gcount;                    // units that may be on the group path (a prefix of the class)
    uint32_t t0, tcount;                    // units that may be on the tile path (a suffix)
  };
  std::vector<Class> classes;               // one or two kernel launches per class and step
  uint64_t n_host = 0;
  cudaGraphExec_t graph = nullptr;
  std::string err;
  ~pf_batch() {                             // the workspace is freed by its owner's paths
    if (graph) cudaGraphExecDestroy(graph);
    if (cap_stream) cudaStreamDestroy(cap_stream);
    if (side) cudaStreamDestroy(side);
    if (fork_ev) cudaEventDestroy(fork_ev);
    if (join_ev) cudaEventDestroy(join_ev);
  }
};

namespace {

struct BatchLayout {
  size_t state, filters, units, partials, y_ring, inc_ring, mean_ring, ess_ring, total;
  std::vector<size_t> x, lv0, lv1;
  std::vector<uint32_t> U, pbase;   // work units of every filter, first partial slot
  uint32_t nunits = 0, nslots = 0;
};

// Work of one filter's step in particle-dimensions, and the default work of one
// thread block (a 2^14-particle filter of dimension 1, or 2^11 particles of dimension 8).
inline double batch_work(const Plan& pl) { return (double)pl.N * (pl.d + 1); }
constexpr double kBatchUnitWork = 32768.0;
constexpr double kBatchUnitParticles = 16384.0;

// Plan every filter and lay the batch out in one workspace.
// Group-path geometry of digit k of a batch filter: a power-of-two radix <= 32
// whose groups fill whole block iterations (members per lane as for a single
// filter's default split), with its carried weights indexed from digit k - 1.
bool batch_group_geom(const Plan& pl, int k, GroupGeom& gg) {
  const DigitGeom& g = pl.geom[k];
  const uint32_t a = g.a;
  if (a < 2 || a > 32 || (a & (a - 1)) != 0) return false;
  const uint32_t G = a / (uint32_t)group_members_per_lane((int)a, pl.d);
  const uint32_t gpb = kBlock / G;
  const uint32_t ngroups = pl.N / a;
  if (ngroups % gpb != 0) return false;
  std::memset(&gg, 0, sizeof(gg));
  while ((1u << gg.log2s) < g.s) ++gg.log2s;
  while ((1u << gg.log2as) < a * g.s) ++gg.log2as;
  gg.nbatch = ngroups / gpb;
  const int kp = (k + pl.m - 1) % pl.m;
  const uint32_t sp = pl.geom[kp].s;
  if (k == 0) {
    gg.lv_mul = 1;
    gg.lv_lmask = 0;
    gg.lv_mask = sp - 1;          // s_{m-1} = N / a_{m-1}
  } else {
    gg.lv_mul = sp;
    gg.lv_lmask = sp - 1;
    gg.lv_mask = 0xffffffffu;
  }
  gg.log_a = g.log_a;
  return true;
}

pf_status plan_batch(int32_t F, const pf_model* models, const int64_t* N, const int32_t* radices, const int32_t* m,
                     const pf_options* opts, std::vector<Plan>& plans, BatchLayout& L, int& ring, int& dy_max,
                     int& d_max, size_t& smem, std::string& msg) {
  if (F < 1 || !models || !N || !radices || !m) { msg = "need F >= 1 and non-NULL arrays"; return PF_EINVAL; }
  plans.resize(F);
  ring = (opts && opts->chunk_len > 0) ? std::min<int>(opts->chunk_len, (int)kRing) : 64;
  dy_max = d_max = 1;
  smem = 0;
  size_t roff = 0;
  for (int32_t f = 0; f < F; ++f) {
    if (m[f] < 1 || m[f] > kMaxDigits) { msg = "filter " + std::to_string(f) + ": need 1 <= m <= 32"; return PF_EINVAL; }
    pf_options o{};
    const int d = models[f].d;
    o.tile = (opts && opts->tile > 0) ? opts->tile : (d <= 1 ? 4096 : d <= 4 ? 2048 : 1024);
    pf_status s = make_plan(&models[f], N[f], radices + roff, m[f], &o, plans[f], msg);
    if (s != PF_OK) { msg = "filter " + std::to_string(f) + ": " + msg; return s; }
    roff += (size_t)m[f];
    if (plans[f].global || plans[f].wide) {
      msg = "filter " + std::to_string(f) + ": batches need radices <= 256 (and N <= 1024 when m = 1)";
      return PF_EINVAL;
    }
    dy_max = std::max(dy_max, plans[f].dy);
    d_max = std::max(d_max, plans[f].d);
    smem = std::max(smem, plans[f].smem);
    GroupGeom gg;
    for (int k = 0; k < plans[f].m; ++k)
      if (batch_group_geom(plans[f], k, gg)) smem = std::max<size_t>(smem, group_smem_bytes_max(d));
  }
  // Work units: a filter's step is split into U = ceil(work / unit work) blocks
  // (at most the fewest tiles of any of its digits), from the filter's own size
  // only; opts->grid > 0 sets the unit work (particle-dimensions per block).
  const double unit_work = (opts && opts->grid > 0) ? (double)opts->grid : kBatchUnitWork;
  L.U.resize(F);
  L.pbase.resize(F);
  L.nunits = L.nslots = 0;
  for (int32_t f = 0; f < F; ++f) {
    uint32_t tiles = 0xffffffffu;
    for (int k = 0; k < plans[f].m; ++k) tiles = std::min(tiles, plans[f].geom[k].ntiles);
    // at most kBatchUnitParticles particles per unit, so that no unit of a
    // cheap (small d) filter outweighs an SM's fair share of its class
    const double want = std::max(std::ceil(batch_work(plans[f]) / unit_work),
                                 std::ceil((double)plans[f].N / kBatchUnitParticles));
    const uint32_t U = (uint32_t)std::max(1.0, std::min({want, (double)tiles, 65535.0}));
    L.U[f] = U;
    L.pbase[f] = (U > 1) ? L.nslots : 0u;
    if (U > 1) L.nslots += U;
    L.nunits += U;
  }
  size_t off = 0;
  auto take = [&](size_t bytes) { size_t o = off; off = align_up(off + bytes); return o; };
  L.state = take(sizeof(BatchState));
  L.filters = take(sizeof(BatchFilter) * (size_t)F);
  L.units = take(8 * (size_t)L.nunits);
  L.partials = take((size_t)4 * kBatchNP * std::max(1u, L.nslots));
  L.y_ring = take((size_t)4 * F * ring * dy_max);
  L.inc_ring = take((size_t)8 * F * ring);
  L.mean_ring = take((size_t)4 * F * ring * d_max);
  L.ess_ring = take((size_t)4 * F * ring);
  L.x.resize(F);
  L.lv0.resize(F);
  L.lv1.resize(F);
  for (int32_t f = 0; f < F; ++f) {
    L.x[f] = take((size_t)4 * plans[f].d * plans[f].N);
    L.lv0[f] = take((size_t)4 * (plans[f].N / plans[f].min_a));
    L.lv1[f] = take((size_t)4 * (plans[f].N / plans[f].min_a));
  }
  L.total = off;
  return PF_OK;
}

pf_status bfail(const pf_batch* b, pf_status s, const std::string& msg) {
  if (b) const_cast<pf_batch*>(b)->err = msg;
  else t_error = msg;
  return s;
}

#define PF_BCUDA(b, call)                                                              \
  do {                                                                                 \
    cudaError_t e_ = (call);                                                           \
    if (e_ != cudaSuccess)                                                             \
      return bfail((b), PF_ECUDA, std::string(#call) + ": " + cudaGetErrorString(e_)); \
  } while (0)

}  // namespace

extern "C" {

pf_status pf_batch_workspace_size(int32_t F, const pf_model* models, const int64_t* N, const int32_t* radices,
                                  const int32_t* m, const pf_options* opts, size_t* bytes) {
  if (!bytes) return bfail(nullptr, PF_EINVAL, "bytes is NULL");
  std::vector<Plan> plans;
  BatchLayout L;
  int ring, dy_max, d_max;
  size_t smem;
  std::string msg;
  pf_status s = plan_batch(F, models, N, radices, m, opts, plans, L, ring, dy_max, d_max, smem, msg);
  if (s != PF_OK) return bfail(nullptr, s, msg);
  *bytes = L.total;
  return PF_OK;
}

pf_status pf_batch_create(int32_t F, const pf_model* models, const int64_t* N, const int32_t* radices,
                          const int32_t* m, const uint64_t* seeds, const pf_options* opts, void* workspace,
                          size_t workspace_bytes, pf_batch** out) {
  if (!out || !seeds) return bfail(nullptr, PF_EINVAL, "NULL argument");
  *out = nullptr;
  pf_batch* b = new (std::nothrow) pf_batch();
  if (!b) return bfail(nullptr, PF_ENOMEM, "host allocation failed");
  std::vector<Plan> plans;
  BatchLayout L;
  std::string msg;
  pf_status s = plan_batch(F, models, N, radices, m, opts, plans, L, b->ring, b->dy_max, b->d_max, b->smem, msg);
  if (s != PF_OK) {
    delete b;
    return bfail(nullptr, s, msg);
  }
  cudaError_t e = cudaGetDevice(&b->device);
  if (e != cudaSuccess) {
    delete b;
    return bfail(nullptr, PF_ECUDA, std::string("CUDA: ") + cudaGetErrorString(e));
  }
  b->F = F;
  b->stream = opts ? static_cast<cudaStream_t>(opts->stream) : nullptr;
  if (workspace) {
    if (workspace_bytes < L.total || reinterpret_cast<uintptr_t>(workspace) % kAlign) {
      delete b;
      return bfail(nullptr, PF_EINVAL, "workspace too small or not 256-byte aligned");
    }
    b->ws = static_cast<unsigned char*>(workspace);
    b->ws_bytes = workspace_bytes;
  } else {
    e = cudaMalloc(&b->ws, L.total);
    if (e != cudaSuccess) {
      delete b;
      return bfail(nullptr, PF_ENOMEM, std::string("cudaMalloc: ") + cudaGetErrorString(e));
    }
    b->own_ws = true;
    b->ws_bytes = L.total;
  }
  e = cudaStreamCreateWithFlags(&b->cap_stream, cudaStreamNonBlocking);
  if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&b->side, cudaStreamNonBlocking);
  if (e == cudaSuccess) e = cudaEventCreateWithFlags(&b->fork_ev, cudaEventDisableTiming);
  if (e == cudaSuccess) e = cudaEventCreateWithFlags(&b->join_ev, cudaEventDisableTiming);
  if (e != cudaSuccess) {
    if (b->own_ws) cudaFree(b->ws);
    delete b;
    return bfail(nullptr, PF_ECUDA, std::string("cudaStreamCreate: ") + cudaGetErrorString(e));
  }
  b->host_filters.resize(F);
  std::vector<std::pair<double, uint2>> work;
  work.reserve(L.nunits);
  for (int32_t f = 0; f < F; ++f) {
    BatchFilter& bf = b->host_filters[f];
    std::memset(&bf, 0, sizeof(bf));
    const Plan& pl = plans[f];
    bf.x = reinterpret_cast<float*>(b->ws + L.x[f]);
    bf.lV[0] = reinterpret_cast<float*>(b->ws + L.lv0[f]);
    bf.lV[1] = reinterpret_cast<float*>(b->ws + L.lv1[f]);
    bf.N = pl.N;
    bf.m = (uint32_t)pl.m;
    bf.cap = pl.cap;
    bf.rk = make_round_keys(seeds[f]);
    bf.model = pl.mp;
    std::memcpy(bf.geom, pl.geom, sizeof(bf.geom));
    bf.gsel = 0;
    for (int k = 0; k < pl.m; ++k)
      if (batch_group_geom(pl, k, bf.gg[k])) bf.gsel |= 1u << k;
    bf.U = L.U[f];
    bf.pbase = L.pbase[f];
    const double uw = batch_work(pl) / L.U[f];
    for (uint32_t j = 0; j < L.U[f]; ++j) work.push_back({-uw, make_uint2((uint32_t)f, j | (L.U[f] << 16))});
  }
  // classes of (model kind, dimension); inside a class the units of filters
  // whose every digit is on the group path first, then those with digits on
  // both paths, then those on the tile path only (so that each path's kernel
  // covers one contiguous range of units), each part largest first
  auto cls = [&](const uint2& u) { return plans[u.x].kind * 16 + plans[u.x].d; };
  auto paths = [&](const uint2& u) {          // 0: group only, 1: both, 2: tile only
    const BatchFilter& hf = b->host_filters[u.x];
    const uint32_t all = (hf.m >= 32) ? 0xffffffffu : ((1u << hf.m) - 1u);
    const uint32_t g = hf.gsel & all;
    return g == all ? 0 : (g != 0 ? 1 : 2);
  };
  std::stable_sort(work.begin(), work.end(), [&](const std::pair<double, uint2>& x, const std::pair<double, uint2>& y) {
    const int cx = cls(x.second), cy = cls(y.second);
    if (cx != cy) return cx < cy;
    const int px = paths(x.second), py = paths(y.second);
    return px != py ? px < py : x.first < y.first;
  });
  b->units.resize(work.size());
  for (size_t u = 0; u < work.size(); ++u) b->units[u] = work[u].second;
  for (size_t u = 0; u < work.size(); ++u) {
    if (u == 0 || cls(work[u].second) != cls(work[u - 1].second)) {
      const Plan& pl = plans[work[u].second.x];
      b->classes.push_back({batch_class_kernel_ptr(pl.kind, pl.d), batch_group_kernel_ptr(pl.kind, pl.d), (uint32_t)u,
                            0u, (uint32_t)u, 0u, (uint32_t)u, 0u});
    }
    auto& c = b->classes.back();
    c.count += 1;
    const int pk = paths(work[u].second);
    if (pk <= 1) c.gcount = (uint32_t)u + 1u - c.g0;          // group range: [g0, g0 + gcount)
    if (pk >= 1 && c.tcount == 0) c.t0 = (uint32_t)u;         // tile range: [t0, t0 + tcount)
    if (pk >= 1) c.tcount = (uint32_t)u + 1u - c.t0;
  }
  for (const auto& c : b->classes) {
    if (!c.kernel || !c.gkernel) {
      delete b;
      return bfail(nullptr, PF_EINVAL, "unsupported (d, model) combination in the batch");
    }
    e = raise_smem_limit(c.kernel, b->smem);
    if (e == cudaSuccess) e = raise_smem_limit(c.gkernel, b->smem);
    if (e != cudaSuccess) {
      delete b;
      return bfail(nullptr, PF_ECUDA, std::string("CUDA: ") + cudaGetErrorString(e));
    }
  }
  BatchParams& P = b->BP;
  P.filters = reinterpret_cast<BatchFilter*>(b->ws + L.filters);
  P.units = reinterpret_cast<const uint2*>(b->ws + L.units);
  P.nunits = L.nunits;
  P.partials = reinterpret_cast<float*>(b->ws + L.partials);
  P.state = reinterpret_cast<BatchState*>(b->ws + L.state);
  P.y_ring = reinterpret_cast<const float*>(b->ws + L.y_ring);
  P.inc_ring = reinterpret_cast<double*>(b->ws + L.inc_ring);
  P.mean_ring = reinterpret_cast<float*>(b->ws + L.mean_ring);
  P.ess_ring = reinterpret_cast<float*>(b->ws + L.ess_ring);
  P.F = (uint32_t)F;
  P.ring = (uint32_t)b->ring;
  P.dy_max = (uint32_t)b->dy_max;
  P.d_max = (uint32_t)b->d_max;
  auto bail = [&](cudaError_t err, const char* what) {
    std::string m2 = std::string(what) + ": " + cudaGetErrorString(err);
    cudaStreamSynchronize(b->stream);
    if (b->own_ws) cudaFree(b->ws);
    delete b;
    return bfail(nullptr, PF_ECUDA, m2);
  };
  e = cudaMemcpyAsync(P.filters, b->host_filters.data(), sizeof(BatchFilter) * (size_t)F, cudaMemcpyHostToDevice,
                      b->stream);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(const_cast<uint2*>(P.units), b->units.data(), 8 * b->units.size(), cudaMemcpyHostToDevice,
                        b->stream);
  if (e == cudaSuccess) e = cudaMemsetAsync(P.state, 0, sizeof(BatchState), b->stream);
  for (int32_t f = 0; f < F && e == cudaSuccess; ++f)
    e = cudaMemsetAsync(b->ws + L.lv0[f], 0, (size_t)4 * (plans[f].N / plans[f].min_a), b->stream);
  if (e != cudaSuccess) return bail(e, "batch set-up copy");
  void* args[] = {&b->BP};
  e = cudaLaunchKernel(batch_init_kernel_ptr(), dim3(F), dim3(kBlock), args, 0, b->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(b->stream);   // host copies above must complete
  if (e != cudaSuccess) return bail(e, "batch init");
  *out = b;
  return PF_OK;
}

pf_status pf_batch_run(pf_batch* b, const float* y, int32_t T, double* loglik_incs, float* means, float* ess) {
  Trace tr("bfpf batch run");
  if (!b) return bfail(nullptr, PF_EINVAL, "batch is NULL");
  if (T < 0 || (T > 0 && !y)) return bfail(b, PF_EINVAL, "need T >= 0 and y != NULL");
  const int R = b->ring, F = b->F;
  // one time step: a launch per class of filters, then the step counter
  // One time step: the tile-path kernels (small filters, short) on the side
  // stream beside the group-path kernels (they touch disjoint filters), both
  // joined before the kernel that advances the step counter.
  bool any_tile = false;
  for (const auto& c : b->classes) any_tile = any_tile || c.tcount != 0;
  auto launch_step = [&](cudaStream_t s) -> cudaError_t {
    cudaError_t le = cudaSuccess;
    if (any_tile) {
      le = cudaEventRecord(b->fork_ev, s);
      if (le == cudaSuccess) le = cudaStreamWaitEvent(b->side, b->fork_ev, 0);
      for (auto& c : b->classes) {
        if (le != cudaSuccess || !c.tcount) continue;
        uint32_t u0 = c.t0;
        void* cargs[] = {&b->BP, &u0};
        le = cudaLaunchKernel(c.kernel, dim3(c.tcount), dim3(kBlock), cargs, b->smem, b->side);
      }
      if (le == cudaSuccess) le = cudaEventRecord(b->join_ev, b->side);
    }
    for (auto& c : b->classes) {
      if (le != cudaSuccess || !c.gcount) continue;
      uint32_t u0 = c.g0;
      void* cargs[] = {&b->BP, &u0};
      le = cudaLaunchKernel(c.gkernel, dim3(c.gcount), dim3(kBlock), cargs, b->smem, s);
    }
    if (le == cudaSuccess && any_tile) le = cudaStreamWaitEvent(s, b->join_ev, 0);
    if (le != cudaSuccess) return le;
    void* aargs[] = {&b->BP};
    return cudaLaunchKernel(batch_advance_kernel_ptr(), dim3(1), dim3(32), aargs, 0, s);
  };
  int32_t done = 0;
  while (done < T) {
    const uint32_t slot0 = (uint32_t)(b->n_host % (uint64_t)R);
    const int32_t L = std::min<int32_t>(R - (int32_t)slot0, T - done);
    const size_t yw = (size_t)4 * b->dy_max;
    PF_BCUDA(b, cudaMemcpy2DAsync(const_cast<float*>(b->BP.y_ring) + (size_t)slot0 * b->dy_max, yw * R,
                                  y + (size_t)done * b->dy_max, yw * T, yw * L, F, cudaMemcpyDefault, b->stream));
    if (L == R && R > 1) {
      if (!b->graph) {
        cudaGraph_t graph = nullptr;
        PF_BCUDA(b, cudaStreamBeginCapture(b->cap_stream, cudaStreamCaptureModeThreadLocal));
        cudaError_t le = cudaSuccess;        // the launches of every time step of the chunk
        for (int32_t j = 0; j < L && le == cudaSuccess; ++j) le = launch_step(b->cap_stream);
        cudaError_t ce = cudaStreamEndCapture(b->cap_stream, &graph);
        if (le != cudaSuccess) return bfail(b, PF_ECUDA, std::string("capture launch: ") + cudaGetErrorString(le));
        if (ce != cudaSuccess) return bfail(b, PF_ECUDA, std::string("cudaStreamEndCapture: ") + cudaGetErrorString(ce));
        cudaError_t ie = cudaGraphInstantiate(&b->graph, graph, 0);
        cudaGraphDestroy(graph);
        if (ie != cudaSuccess) {
          b->graph = nullptr;
          return bfail(b, PF_ECUDA, std::string("cudaGraphInstantiate: ") + cudaGetErrorString(ie));
        }
      }
      PF_BCUDA(b, cudaGraphLaunch(b->graph, b->stream));
    } else {
      for (int32_t j = 0; j < L; ++j) PF_BCUDA(b, launch_step(b->stream));
    }
    if (loglik_incs)
      PF_BCUDA(b, cudaMemcpy2DAsync(loglik_incs + done, (size_t)8 * T, b->BP.inc_ring + slot0, (size_t)8 * R,
                                    (size_t)8 * L, F, cudaMemcpyDefault, b->stream));
    if (ess)
      PF_BCUDA(b, cudaMemcpy2DAsync(ess + done, (size_t)4 * T, b->BP.ess_ring + slot0, (size_t)4 * R, (size_t)4 * L,
                                    F, cudaMemcpyDefault, b->stream));
    if (means) {
      const size_t mw = (size_t)4 * b->d_max;
      PF_BCUDA(b, cudaMemcpy2DAsync(means + (size_t)done * b->d_max, mw * T, b->BP.mean_ring + (size_t)slot0 * b->d_max,
                                    mw * R, mw * L, F, cudaMemcpyDefault, b->stream));
    }
    b->n_host += L;
    done += L;
  }
  PF_BCUDA(b, cudaGetLastError());
  if (loglik_incs || means || ess) PF_BCUDA(b, cudaStreamSynchronize(b->stream));
  return PF_OK;
}

pf_status pf_batch_loglik(const pf_batch* b, double* out) {
  if (!b || !out) return bfail(b, PF_EINVAL, "NULL argument");
  std::vector<BatchFilter> tmp(b->F);
  PF_BCUDA(b, cudaMemcpyAsync(tmp.data(), b->BP.filters, sizeof(BatchFilter) * (size_t)b->F, cudaMemcpyDeviceToHost,
                              b->stream));
  PF_BCUDA(b, cudaStreamSynchronize(b->stream));
  for (int f = 0; f < b->F; ++f) out[f] = tmp[f].st.loglik;
  return PF_OK;
}

pf_status pf_batch_get_state(const pf_batch* b, int32_t f, float* x, float* lV, double* scalars) {
  if (!b || f < 0 || f >= b->F) return bfail(b, PF_EINVAL, "bad batch or filter index");
  BatchFilter bf;
  BatchState bs;
  PF_BCUDA(b, cudaMemcpyAsync(&bf, b->BP.filters + f, sizeof(bf), cudaMemcpyDeviceToHost, b->stream));
  PF_BCUDA(b, cudaMemcpyAsync(&bs, b->BP.state, sizeof(bs), cudaMemcpyDeviceToHost, b->stream));
  PF_BCUDA(b, cudaStreamSynchronize(b->stream));
  if (x) PF_BCUDA(b, cudaMemcpyAsync(x, bf.x, (size_t)4 * bf.model.d * bf.N, cudaMemcpyDeviceToHost, b->stream));
  if (lV) {
    const uint32_t kp = (bs.n + bf.m - 1) % bf.m;
    PF_BCUDA(b, cudaMemcpyAsync(lV, bf.lV[bs.n & 1u], (size_t)4 * (bf.N / bf.geom[kp].a), cudaMemcpyDeviceToHost,
                                b->stream));
  }
  PF_BCUDA(b, cudaStreamSynchronize(b->stream));
  if (scalars) {
    scalars[0] = (double)bs.n;
    scalars[1] = bf.st.loglik;
    scalars[2] = bf.st.mu;
    scalars[3] = (double)bf.st.mu_f;
  }
  return PF_OK;
}

const char* pf_batch_last_error(const pf_batch* b) {
  if (b) return b->err.c_str();
  return t_error.c_str();
}

pf_status pf_batch_destroy(pf_batch* b) {
  if (!b) return PF_OK;
  cudaError_t e = cudaStreamSynchronize(b->stream);
  if (b->own_ws && b->ws) cudaFree(b->ws);
  delete b;
  if (e != cudaSuccess) return bfail(nullptr, PF_ECUDA, std::string("cudaStreamSynchronize: ") + cudaGetErrorString(e));
  return PF_OK;
}

}  // extern "C"
