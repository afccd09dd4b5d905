/*
 * bfpf.h - C ABI of the butterfly-interaction bootstrap particle filter.
 *
 * The filter is the one of Heine, Whiteley & Cemgil, "Parallelising particle
 * filters with butterfly interactions" (arXiv 1812.01502): Algorithm 1
 * (bootstrap particle filter) whose resampling step is one stage of
 * Algorithm 3 (augmented resampling) per time step.  Particle indices
 * 0..N-1 are read in mixed radix N = a_0 a_1 ... a_{m-1} (digit 0 least
 * significant); at time step n the particles resample only inside groups
 * that share every digit except digit k = n mod m, i.e. the stage matrix is
 * A_k = I (x) 1_{1/a_k} (x) I (eq. (A matrices) of Section 1.2 generalised to
 * mixed radix, as the Remark after Lemma 3 allows), and the stage weights
 * V_k = A_k V_{k-1} carry into the next time step.
 *
 * Conventions (all entry points):
 *  - Every function returns a pf_status; PF_OK is 0.  On failure the handle
 *    (or, for calls without a handle, the calling thread) records a message
 *    that pf_last_error() returns.  No entry point aborts the process.
 *  - All device work is enqueued on the handle's CUDA stream and is
 *    asynchronous, except where an output goes to host memory or the
 *    description says "synchronises".
 *  - A handle is not thread-safe; use one handle per host thread or lock.
 *  - There is no CPU fallback: without a usable CUDA device every call that
 *    needs one returns PF_ECUDA.
 *  - Pointers documented "host or device" are copied with cudaMemcpyDefault
 *    (unified virtual addressing); device pointers must belong to the
 *    handle's device.
 */
#ifndef BFPF_H
#define BFPF_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    PF_OK = 0,
    PF_EINVAL = 1,    /* invalid argument: sizes, radices, model, null pointers   */
    PF_ENOMEM = 2,    /* workspace too small or device allocation failed          */
    PF_ECUDA = 3,     /* a CUDA runtime call failed (message has the CUDA error)   */
    PF_ETIMEOUT = 4,  /* reserved (no kernel of the library waits on another)       */
    PF_ESTATE = 5     /* call not valid in the handle's current state              */
} pf_status;

typedef enum {
    PF_MODEL_LINEAR_GAUSSIAN = 1,
    PF_MODEL_STOCH_VOL = 2
} pf_model_kind;

/*
 * The hidden Markov model of Section 1.1 (eq. (HMM)):
 *   X_0 ~ pi_0,  X_n | X_{n-1} ~ f(X_{n-1}, .),  Y_n | X_n ~ g(X_n, .),  n >= 0.
 *
 * PF_MODEL_LINEAR_GAUSSIAN:
 *   pi_0 = N(m0, L0 L0^T);  X_n = A X_{n-1} + Lq eps_n;  Y_n = H X_n + Lr w_n,
 *   eps, w standard normal.  d = state dimension (1..8), dy = observation
 *   dimension (1..8).  Matrices are row-major double arrays that the library
 *   copies at pf_create (the caller keeps ownership): A d*d, Lq d*d lower
 *   triangular, H dy*d, Lr dy*dy lower triangular with nonzero diagonal,
 *   m0 d, L0 d*d lower triangular.  NULL means identity (zero for m0; H = NULL
 *   needs dy == d).  (Section 6.1's experiment: A = Lq = H = L0 = I,
 *   Lr = I/2, m0 = 0.)
 * PF_MODEL_STOCH_VOL (d = dy = 1):
 *   pi_0 = N(0, sigma^2/(1-phi^2));  X_n = phi X_{n-1} + sigma v_n;
 *   Y_n = beta exp(X_n/2) w_n;  requires |phi| < 1, sigma > 0, beta > 0.
 */
typedef struct {
    int32_t kind;         /* pf_model_kind */
    int32_t d;
    int32_t dy;
    const double* A;
    const double* Lq;
    const double* H;
    const double* Lr;
    const double* m0;
    const double* L0;
    double phi, sigma, beta;
} pf_model;

/* pf_options.flags */
#define PF_RECORD_ANCESTORS 1u   /* keep the ancestor index of every particle of the last step */
/* Run every stage of Algorithm 3 in each time step (Algorithm 1 whose
 * Resample is the whole of Algorithm 3, Section 3): step n weights with
 * g_n, then resamples on digits 0, 1, ..., m-1 in turn with stage weights
 * V_s = A_s V_{s-1} (Section 3, eq. (V_defn_proofs)), then mutates.  After the
 * last stage every carried weight is equal (Lemma 3(c)).  Without the flag
 * each step runs the one stage on digit n mod m (the default, cheapest
 * schedule).  Consecutive digits of one radix (a power of two <= 32) share a
 * kernel launch while the particles their stages can exchange fit one
 * shared-memory tile (4096 particles at d = 1, 2048 at d <= 4, 1024 above),
 * unless N < 2^16 and that saves fewer than half of the launches; otherwise
 * one launch per stage, m per time step (pf_describe lists the launches).  Cannot be combined with PF_RECORD_ANCESTORS (EINVAL).  Ignored
 * when m = 1. */
#define PF_ALL_STAGES 2u
/* Fully adapted augmented resampling (Section 1.2): each time step weights
 * with g_n, then runs the stages of Algorithm 3 on digits 0, 1, ..., m-1 in
 * turn while the effective sample size (Section 1.2) of the current weights
 * is below pf_options.ess_threshold, skipping the rest once it is reached;
 * then mutates.  Weights that were not equalised carry over to the next
 * step, so carried log-weights are kept per particle (N floats; pf_get_state
 * returns N of them).  m + 1 kernel launches per time step.  Radices must
 * keep every group within one thread block (each a_k <= 1024; m = 1 needs
 * N <= 1024).  Cannot be combined with PF_ALL_STAGES or PF_RECORD_ANCESTORS. */
#define PF_ADAPTIVE 4u
/* With PF_ADAPTIVE: start each step's stages one digit after the last stage
 * executed (the rotation proposed in Section 6.4) instead of at digit 0. */
#define PF_ROTATE 8u
/* Augmented island resampling particle filter (AIRPF, Algorithm 4) with the
 * modified island resampling of Algorithm 7: radices must be (M, m) -- m =
 * 2^S islands of M consecutive particles (2 <= M <= 1024, 2 <= m <= 16384,
 * m a power of two).  Each step weights with g_n, resamples multinomially
 * within every island (Algorithm 5; island weight = mean g of the island),
 * runs the S stages of augmented island resampling on the island weights
 * (whole islands are copied; a draw in which two paired islands would only
 * swap their samples is undone), then mutates.  3 kernel launches per step.
 * Cannot be combined with the other schedule flags or PF_RECORD_ANCESTORS. */
#define PF_ISLANDS 16u
/* With PF_ISLANDS: island resampling as in Algorithm 6 (swaps are kept). */
#define PF_ISLANDS_PLAIN 32u
/* Algorithm 3 with the paper's own stage matrices (eq. (A matrices)): each
 * time step runs stages s = 1..m-1, stage s resampling within the groups of
 * the digit SET {0, s} -- the a_0 a_s particles that share every digit except
 * digits 0 and s (radices (M, 2, ..., 2): a PE's M particles together with
 * its partner PE's across bit s-1).  Stage 1 weights with g_n, stage m-1
 * mutates; afterwards every carried weight is equal (Lemma 3(c)).  Needs
 * m >= 2 and a_0 a_s <= 1024; m - 1 launches per step.  Cannot be combined
 * with the other schedule flags or PF_RECORD_ANCESTORS. */
#define PF_DIGIT_SETS 64u
/* Parity output: also keep, for every particle, the inclusive prefix sum P of
 * the integer weights within its group at the last step (the numbers the
 * integer draw of Algorithm 2 / Algorithm 3's sampling line compares its
 * uniform with; read by pf_get_draw_prefix).  Implies PF_RECORD_ANCESTORS and
 * its limits.  Adds 8N bytes of workspace. */
#define PF_RECORD_DRAWS 128u
/* Test hook for the global-resampling draws (radices = {N}, N > 1024): every
 * bucket of draws holds 16 particles and stages at most 64 indices, so most
 * draws go through the overflow list and most buckets search P in global
 * memory.  Results are those of the normal path; only slower. */
#define PF_TEST_SMALL_BUCKETS 0x40000000u
/* Test hook for PF_ALL_STAGES: one launch per stage even where consecutive
 * digits of one radix (a power of two <= 32) would share a fused launch.  The
 * same filter; with the fused kernels' lane split the same numbers. */
#define PF_TEST_STAGE_PER_LAUNCH 0x20000000u

typedef struct {
    int32_t tile;        /* target particles per thread-block tile; 0 = automatic            */
    int32_t chunk_len;   /* time steps per CUDA-graph replay in pf_run; 0 = 64 (max 1024)    */
    uint32_t flags;      /* PF_RECORD_ANCESTORS | PF_ALL_STAGES | PF_ADAPTIVE | PF_ROTATE |  */
                         /* PF_ISLANDS | PF_ISLANDS_PLAIN | PF_DIGIT_SETS                    */
    int32_t grid;        /* persistent thread blocks; 0 = automatic (SMs x occupancy)        */
    void* stream;        /* cudaStream_t to run on; NULL = the legacy default stream          */
    float ess_threshold; /* PF_ADAPTIVE: a stage runs while ESS < ess_threshold; 0 = 0.5.     */
                         /* Values above 1 run every stage; values <= 1/N run none.          */
} pf_options;

typedef struct pf_handle pf_handle;

/*
 * Device workspace needed by pf_create for this problem: particle states
 * (4*d*N bytes), carried log-weights (2 * 4N/min(a) bytes), optional
 * ancestors (4N), per-block partial sums and small rings for observations
 * and per-step outputs; global resampling (radices = {N}, N > 1024) adds a
 * second state buffer (4dN), log-weights (4N), prefix sums (8N), the draws
 * filed by bucket as 4-byte indices (about 4N, twice) and two overflow lists
 * (4N each).  opts may be NULL.
 * Errors: PF_EINVAL (bad model / N / radices, see pf_create).
 */
pf_status pf_workspace_size(const pf_model* model, int64_t N, const int32_t* radices,
                            int32_t m, const pf_options* opts, size_t* bytes);

/*
 * Create a filter for `model` with N = radices[0] * ... * radices[m-1]
 * particles (Assumption A1 of the paper with paper-m = N / M generalised to
 * mixed radix).  Every radix must be >= 2 and <= 1024, except that m == 1
 * (radices = {N}: the global-resampling bootstrap filter of Algorithm 2) allows
 * any N.  N < 2^31.  `seed` keys the counter-based random stream (Philox4x32 with seven rounds),
 * so a run is reproducible given (model, N, radices, seed, observations).
 *
 * workspace: device memory of at least pf_workspace_size() bytes, 256-byte
 *   aligned, owned by the caller, who must keep it alive until pf_destroy; or
 *   NULL, in which case the library allocates (cudaMalloc) and frees its own.
 * Draws pi_0 (Algorithm 1, first loop) on the stream before returning.
 * Errors: PF_EINVAL, PF_ENOMEM (workspace_bytes too small / allocation
 *   failed), PF_ECUDA.  On error *out is set to NULL.
 */
pf_status pf_create(const pf_model* model, int64_t N, const int32_t* radices, int32_t m,
                    uint64_t seed, const pf_options* opts, void* workspace,
                    size_t workspace_bytes, pf_handle** out);

/*
 * One time step n (n = number of steps taken so far): weight the particles
 * with g(., y_n), run one augmented-resampling stage on digit n mod m, and
 * mutate (Algorithm 1 loop body).  y_n: dy floats, host or device.
 * Optional outputs (NULL to skip; host or device): mean_out (d floats) = the
 * weighted filtering mean estimate of E[X_n | y_0..y_n]; loglik_inc (1
 * double) = log p^(y_n | y_0..y_{n-1}); ess_out (1 float) = the effective
 * sample size fraction of Section 1.2 computed from the carried weights.
 * Host outputs synchronise the stream.
 */
pf_status pf_step(pf_handle* h, const float* y_n, float* mean_out, double* loglik_inc,
                  float* ess_out);

/*
 * T time steps over y (T x dy floats, row-major, host or device), in chunks
 * of opts.chunk_len steps replayed from a captured CUDA graph.  Optional
 * per-step outputs (NULL to skip; host or device): means (T x d floats),
 * loglik_incs (T doubles), ess (T floats).  Host outputs synchronise.
 */
pf_status pf_run(pf_handle* h, const float* y, int32_t T, float* means, double* loglik_incs,
                 float* ess);

/*
 * Streaming form of pf_run, for callers that feed observations as they arrive:
 * pf_push_observations copies T observations (T x dy floats, host or device)
 * into the handle's device ring for the next T time steps not yet pushed; at
 * most 1024 observations may be pushed ahead of the steps taken (else
 * PF_ESTATE).  pf_advance then takes T time steps on pushed observations
 * (fewer pushed than T: PF_ESTATE) and writes the optional per-step outputs
 * exactly as pf_run does.  pf_advance with T = 1 is one kernel launch.
 */
pf_status pf_push_observations(pf_handle* h, const float* y, int32_t T);
pf_status pf_advance(pf_handle* h, int32_t T, float* means, double* loglik_incs, float* ess);

/* Cumulative log-likelihood estimate log p^(y_0..y_{n-1}) accumulated in
 * FP64 across time.  Synchronises the stream. */
pf_status pf_loglik(const pf_handle* h, double* out);

/*
 * Copy the filter state to host memory (synchronises; any pointer may be NULL):
 *   x        N*d floats, state-major: x[t*N + i] = component t of particle i
 *            (the prediction particles of the next step);
 *   lV       N / a_{k'} floats: carried log stage weights, one per group of the
 *            digit k' of the last stage run (k' = (n-1) mod m; m-1 with
 *            PF_ALL_STAGES; all zero before the first step), group index
 *            (i / (a_{k'} s_{k'})) * s_{k'} + i % s_{k'}, s_{k'} = a_0 ... a_{k'-1};
 *            with PF_ADAPTIVE: N floats, one per particle;
 *            with PF_DIGIT_SETS: N / (a_0 a_{m-1}) floats, one per group of the
 *            last set {0, m-1} (index (i / (a_{m-1} s_{m-1})) (s_{m-1} / a_0)
 *            + (i % s_{m-1}) / a_0);
 *            with PF_ISLANDS: M floats, all equal (radices (M, m)); with
 *            PF_ISLANDS | PF_ADAPTIVE: m floats, one per island;
 *   scalars  4 doubles: { n, loglik, mu, mu_used }, where mu is the carried
 *            normaliser subtracted from the log-weights at the next step (FP64)
 *            and mu_used its FP32 value the kernels subtract.
 */
pf_status pf_get_state(const pf_handle* h, float* x, float* lV, double* scalars);

/* Ancestor (global particle index, int32) of every particle at the last step;
 * needs PF_RECORD_ANCESTORS.  anc: N int32, host.  Synchronises. */
pf_status pf_get_ancestors(const pf_handle* h, int32_t* anc);

/*
 * The integer prefix sums behind the last step's draws (Algorithm 2; the
 * sampling line of Algorithm 3): prefix[i] = q_0 + ... + q_r for particle i =
 * member r (its digit k) of its group, q_j = floor(e_j 2^B) the quantised
 * weight of member j (B = 24 for groups of at most 256 members, else 32).
 * With the group's total Q and the particle's uniform word(s) r, its ancestor
 * is member #{j : prefix_j <= floor(r Q / 2^W)} (W = 32 or 64), so a checker
 * that is given these integers can redo every draw exactly.  prefix: N
 * uint64, host.  Available with PF_RECORD_DRAWS, and always for global
 * resampling (radices = {N}, N > 1024), whose single group is all N
 * particles.  Synchronises.  Errors: PF_ESTATE when not recorded.
 */
pf_status pf_get_draw_prefix(const pf_handle* h, uint64_t* prefix);

/* Sticky device-side status bits of the handle (0 = none): bit 0 = a
 * non-finite log-weight was seen and treated as weight zero; bit 1 = a group
 * had zero total weight and kept its particles.  Synchronises. */
pf_status pf_get_status(const pf_handle* h, uint32_t* bits);

/*
 * Checkpoint / resume (no counterpart in the paper).  A checkpoint holds the
 * filter's whole device workspace (particles, carried weights, normaliser,
 * FP64 log-likelihood, step counter, pushed observations, output rings) and
 * its host counters, behind a header naming the model, N, radices, seed and
 * options.  The random numbers are counter-based (keyed by seed, step and
 * particle), so a filter resumed from a checkpoint continues bit for bit as
 * the uninterrupted one.
 *   pf_checkpoint_size: bytes a checkpoint of h needs.
 *   pf_save: writes it to buf (host memory, len >= that size); synchronises.
 *   pf_load: restores h from buf; h must have been created with the same
 *            model, N, radices, seed and options (else PF_EINVAL, h unchanged).
 *            Synchronises.
 */
pf_status pf_checkpoint_size(const pf_handle* h, size_t* bytes);
pf_status pf_save(const pf_handle* h, void* buf, size_t len);
pf_status pf_load(pf_handle* h, const void* buf, size_t len);

/* Number of resampling stages executed so far (PF_ADAPTIVE counts only the
 * stages its ESS test let run; otherwise one per stage launched).  Synchronises. */
pf_status pf_stage_count(const pf_handle* h, uint64_t* out);

/*
 * Describe the launch plan as a JSON object (NUL-terminated, truncated to
 * `len` bytes): per digit k its radix, stride, kernel ("group" = the
 * register-resident kernel for power-of-two radices <= 32, "tile" = the
 * general shared-memory tile kernel), lanes per group or tile size, and grid.
 * Host-only; never synchronises.
 */
pf_status pf_describe(const pf_handle* h, char* buf, size_t len);

/* Release the handle and, if the library allocated it, its workspace.
 * Synchronises the stream.  NULL is accepted. */
pf_status pf_destroy(pf_handle* h);

/* Message for the last failed call on `h`, or on the calling thread when
 * h is NULL.  Never NULL; valid until the next call on the same handle/thread. */
const char* pf_last_error(const pf_handle* h);

/*
 * Philox4x32-7 blocks, for checking the device generator against an
 * independent implementation: out[4*j + w] = word w of Philox4x32-7 with
 * key (seed mod 2^32, seed div 2^32) and counter (c0 + j, c1, c2, c3),
 * j = 0..count-1.  out: device pointer to 4*count uint32.  Runs on `stream`
 * (cudaStream_t, may be NULL) and is asynchronous.
 */
pf_status pf_philox_blocks(uint64_t seed, uint32_t c0, uint32_t c1, uint32_t c2, uint32_t c3,
                           int64_t count, uint32_t* out, void* stream);

/*
 * Batches: F independent filters with their own model, N, radices and seed
 * (uneven sizes and state dimensions), advanced together, one time step per
 * kernel launch for the whole batch.  radices is the concatenation of the F
 * radix lists (m[f] entries each).  Every radix must be <= 256, and m[f] == 1
 * needs N[f] <= 1024; otherwise the rules of pf_create apply per filter.
 * Filter f's observation at step n is y[(f*T + n)*dy_max + j] in pf_batch_run,
 * dy_max = the largest dy of the batch; outputs are [F][T] (increments, ESS)
 * and [F][T][d_max] (means), d_max = the largest d.  workspace as in pf_create
 * (NULL: the library allocates).  A filter's results do not depend on the
 * other filters of the batch.  A time step of every filter is a few kernel
 * launches (per class of model kind and d, one for the digits on the
 * register-resident group path and one for the tile path; captured in a CUDA
 * graph per chunk of opts.chunk_len steps); a filter's step is split over
 * max(ceil(N (d + 1) / W), ceil(N / 16384)) thread blocks, at most the fewest
 * tiles of any of its digits, where W = opts.grid if > 0 (particle-dimensions
 * of work per block), else 32768; the blocks of one filter fold their
 * partial sums in a fixed order, so a filter's results depend only on itself, W
 * and opts.tile (particles per tile, 0 = by state dimension).
 */
typedef struct pf_batch pf_batch;
pf_status pf_batch_workspace_size(int32_t F, const pf_model* models, const int64_t* N,
                                  const int32_t* radices, const int32_t* m,
                                  const pf_options* opts, size_t* bytes);
pf_status pf_batch_create(int32_t F, const pf_model* models, const int64_t* N, const int32_t* radices,
                          const int32_t* m, const uint64_t* seeds, const pf_options* opts,
                          void* workspace, size_t workspace_bytes, pf_batch** out);
pf_status pf_batch_run(pf_batch* b, const float* y, int32_t T, double* loglik_incs, float* means,
                       float* ess);
/* Cumulative FP64 log-likelihood of every filter (F doubles, host).  Synchronises. */
pf_status pf_batch_loglik(const pf_batch* b, double* out);
/* State of filter f as pf_get_state (x: N[f]*d floats, lV, scalars {n, loglik, mu, mu_used}). */
pf_status pf_batch_get_state(const pf_batch* b, int32_t f, float* x, float* lV, double* scalars);
pf_status pf_batch_destroy(pf_batch* b);
/* Message for the last failed call on `b` (or on this thread when b is NULL). */
const char* pf_batch_last_error(const pf_batch* b);

/*
 * pf_step_noalloc - one time step on buffers the caller already owns, with no
 * device allocation of any kind.  (The paper has no counterpart: this entry
 * point exists for callers whose device memory is managed by someone else -
 * an engine or framework that owns every allocation, or a real-time loop with
 * a fixed memory budget - and who therefore may not call cudaMalloc, nor keep
 * a pf_create workspace alive.)
 *
 * The step's temporary data (the device state block, per-block partial sums
 * and the per-step outputs) lives in a fixed scratch area compiled into the
 * library: 192 KiB of device memory per GPU that loads the library, held until
 * the process exits.  The step runs at most 2048 thread blocks (the grid is
 * capped there; a larger problem only takes more iterations per block), so N
 * and d stay limited only as for pf_create.
 *
 * Arguments: model, N, radices, m, seed as for pf_create; n = index of this
 * time step (digit n mod m interacts; it keys the random draws); mu = carried
 * normaliser: 0 at n = 0, then out[1] of the previous step.  Device buffers:
 * x (N*d floats, state-major, x[t*N + i]) holds the prediction particles
 * zeta_n and is overwritten with zeta_{n+1}; lV_in (N / a_{(n-1) mod m}
 * floats, all zero at n = 0) the carried log stage weights; lV_out
 * (N / a_{n mod m} floats) receives the new ones.  y_n: dy floats, host.
 * Host outputs: out[3] = { log-likelihood increment, mu for step n + 1, ESS };
 * mean_out (d floats, may be NULL) = the filtering mean; status_out (1 uint32,
 * may be NULL) = this step's status bits as pf_get_status reports them (bit 0:
 * a non-finite log-weight was treated as weight zero; bit 1: a group had zero
 * total weight and kept its particles).  Synchronises `stream`, which must
 * belong to the current device (NULL = the legacy default stream of the
 * current device; another device's stream: PF_EINVAL).
 *
 * The first call on a device resolves the scratch area's device address
 * (cudaGetSymbolAddress) with that device current, so make that first call
 * outside any CUDA stream capture.  Every call on a device shares the one
 * scratch area and the call clears what must start at zero; calls that can
 * overlap on the GPU (different streams, or threads without ordering) race on
 * it and must be serialised by the caller.
 * Errors: PF_EINVAL as pf_create; PF_ECUDA.
 */
pf_status pf_step_noalloc(const pf_model* model, int64_t N, const int32_t* radices, int32_t m,
                          uint64_t seed, uint32_t n, double mu, float* x, const float* lV_in,
                          float* lV_out, const float* y_n, double* out, float* mean_out,
                          uint32_t* status_out, void* stream);

#ifdef __cplusplus
}
#endif
#endif /* BFPF_H */
