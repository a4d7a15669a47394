/*
 * smc.h -- C-ABI of libsmc.so, the GB300 (sm_103a) hot path of one iteration of
 * the SMC sampler with recycling of Varsi, Kekempanos, Thiyagalingam & Maskell,
 * "A Single SMC Sampler on MPI that Outperforms a Single MCMC Sampler"
 * (arXiv:1905.10252).
 *
 * Conventions shared by every entry point
 *  - Pointers named *_dev are DEVICE pointers on the current CUDA device; the
 *    caller allocates and frees them (the library never allocates device
 *    memory).  Host pointers are named *_host.
 *  - Particles are row-major N x D arrays of float (SMC_F32) or double
 *    (SMC_F64); row i is particle x^i (the paper's x_t in R^{N x M}, Sec. 3.1,
 *    with the paper's state dimension M called D here).  Log-weights are
 *    double[N]; the cached log-target log pi(x^i) has the particle dtype.
 *  - Every call only enqueues work on the sampler's stream (or the stream
 *    argument) and returns; results land in device memory.  A call returns
 *    SMC_OK when its launches were accepted.  Errors found on the device
 *    (non-finite weights, an invalid copy-count vector, a bounded wait that
 *    gave up) are recorded in an error word and returned by the next
 *    smc_sync() / smc_ws_status().
 *  - Sizes: 1 <= N < 2^31, 1 <= D <= 32.
 *  - Not thread-safe per handle; distinct handles are independent.
 */
#ifndef SMC_H_
#define SMC_H_

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* A cudaStream_t (identical type); NULL is the legacy default stream. */
typedef struct CUstream_st* smc_stream_t;

typedef enum {
  SMC_OK = 0,
  SMC_EINVAL = 1,      /* bad argument: size, dtype, null pointer, ncopies not summing to N */
  SMC_ENOMEM = 2,      /* workspace too small / admission refused */
  SMC_ECUDA = 3,       /* a CUDA runtime call failed (message in smc_last_error) */
  SMC_ETIMEOUT = 4,    /* a bounded device-side wait gave up */
  SMC_ENONFINITE = 5   /* a log-weight is NaN, or every log-weight is -inf */
} smc_status;

typedef enum { SMC_F32 = 1, SMC_F64 = 2 } smc_dtype;

/* Targets pi(x) of the static SMC sampler (Sec. 3.1.2), normalising
 * constants dropped:
 *  SMC_GAUSS      log pi = -1/2 (x-mu)^T Sigma^-1 (x-mu)
 *  SMC_LOGISTIC   log pi = sum_m [y_m z_m - softplus(z_m)] - |x|^2/(2 prior_var),
 *                 z = X x (Bayesian logistic regression, M data rows)
 *  SMC_STUDENT_T  log pi = -(nu+1)/2 log(1 + (x-mu)^2/nu), D = 1 (Sec. 5.2.3, eq. (14)) */
typedef enum { SMC_GAUSS = 1, SMC_LOGISTIC = 2, SMC_STUDENT_T = 3 } smc_target_kind;

/* When to resample (Sec. 3.1): SMC_RESAMPLE_ESS resamples iff N_eff < N*
 * (smc_config.nstar; N/2 by default), decided exactly on the quantised
 * weights (2 S^2 < N sum W^2 for N/2);
 * SMC_RESAMPLE_ALWAYS is the worst case of Sec. 5.2 (every iteration). */
typedef enum { SMC_RESAMPLE_ESS = 0, SMC_RESAMPLE_ALWAYS = 1, SMC_RESAMPLE_NEVER = 2 } smc_resample_mode;

/* smc_config.flags.  SMC_FLAG_LOGISTIC_CUDA_CORES: an FP32 logistic sampler
 * evaluates its likelihood on the CUDA cores in FP32 (z = X b by FMAs) instead
 * of the default tensor-core contraction (BF16 hi/lo split, FP32 accumulation);
 * FP64 samplers always use the CUDA cores in FP64. */
#define SMC_FLAG_LOGISTIC_CUDA_CORES 1
/* Test hook for the failure path: the tensor-core likelihood never issues its
 * data copies, so every wait on them runs out (after about one second);
 * the kernel then drains, frees its tensor memory and returns, and the next
 * smc_sync reports SMC_ETIMEOUT.  The GPU context stays usable. */
#define SMC_FLAG_TEST_STALL_LIKELIHOOD 2
/* SMC_FLAG_DEFER_REDISTRIBUTE: in smc_step and smc_step_profile, an iteration
 * that resamples does not copy the rows (Algorithm 5) itself; the next
 * iteration's move reads each particle's row from its source (the copy fused
 * into the move kernel, which saves one write and one read of every row), so
 * the rows, log pi and log w in the caller's buffers are the sampler's state
 * only after one of the calls that complete a pending copy: smc_materialize,
 * smc_current, smc_move, smc_reweight, smc_estimate, smc_resample,
 * smc_redistribute, smc_checkpoint_save, smc_checkpoint_load or
 * smc_batch_create.  smc_step, smc_step_profile, smc_sync and smc_read_stats
 * leave it pending (a caller reading x / log w after smc_sync alone sees the
 * rows before the copy and log w before the reset).  The particles, weights, estimates and statistics are bit-identical to those
 * without the flag.  Honoured by FP32 Gaussian samplers with D <= 16 and
 * N > 4096 (whose move kernel forms the eq. (7) sums); ignored otherwise. */
#define SMC_FLAG_DEFER_REDISTRIBUTE 4
/* Test hook for the failure path of the fused small-sampler iterations (see
 * smc_step): their grid barrier waits for one block more than the launch
 * has, so every wait runs out (after about half a second), the kernel
 * returns, and the next smc_sync reports SMC_ETIMEOUT.  The GPU context stays
 * usable. */
#define SMC_FLAG_TEST_STALL_BARRIER 8

typedef struct {
  int64_t n;              /* N particles */
  int32_t d;              /* D state dimension */
  int32_t dtype;          /* smc_dtype of particles and log pi */
  uint64_t seed;          /* Philox4x32-10 key: (seed low 32 bits, seed high 32 bits) */
  int32_t target;         /* smc_target_kind */
  int32_t resample_mode;  /* smc_resample_mode */
  double step;            /* random-walk proposal std eps: x_t = x_{t-1} + eps z (Sec. 5.2.3) */
  double init_scale;      /* q0 = N(0, init_scale^2 I) (Algorithm 2, line 1) */
  /* target parameters, DEVICE pointers, read during smc_init only */
  const double* mu_dev;     /* GAUSS: D; STUDENT_T: 1 */
  const double* sigma_dev;  /* GAUSS: D x D symmetric positive definite, row-major */
  const float* X_dev;       /* LOGISTIC: M x D row-major */
  const float* y_dev;       /* LOGISTIC: M labels in {0, 1} */
  int32_t m;                /* LOGISTIC: M rows */
  int32_t flags;            /* SMC_FLAG_* (0: defaults) */
  double prior_var;         /* LOGISTIC: prior N(0, prior_var I) */
  double nu;                /* STUDENT_T: degrees of freedom */
  int64_t nstar;            /* SMC_RESAMPLE_ESS threshold N* of Algorithm 2: resample iff
                               N_eff < N*, decided exactly as S^2 < N* sum W^2; 0..n, and
                               0 selects the paper's N* = N/2 (2 S^2 < N sum W^2) */
} smc_config;

typedef struct smc_sampler smc_sampler;

/* Per-iteration statistics written by smc_reweight / smc_step (device memory,
 * one record per iteration when a trace buffer is given). */
typedef struct {
  double lse;        /* log sum_i w_t^i (eq. (2) normaliser, log space) */
  double logc;       /* log c_t = LSE_t - LSE_{t-1} (eq. (8)); LSE_{t-1} = 0 after a reset */
  double ess;        /* N_eff = 1 / sum_i (w~_t^i)^2 (eq. (1)), from the quantised weights */
  double max_logw;   /* m = max_i log w_t^i */
  int64_t resampled; /* 1 if N_eff < N* triggered resampling (Algorithm 2, lines 7-9) */
  int64_t t;         /* iteration index */
  int64_t survivors; /* particles with ncopies > 0 when resampled, else 0 */
} smc_iter_stats;

/* Bytes of device workspace a sampler with this configuration needs. */
int smc_workspace_bytes(const smc_config* cfg, size_t* bytes);

/* Algorithm 2, line 1: draws x_0 ~ q0 = N(0, init_scale^2 I) with Philox
 * (seed, t = 0, particle i) and sets w_0 = pi(x_0)/q0(x_0).
 * x_dev/x_alt_dev: two N x D particle buffers (ping-pong: redistribute writes
 * the other one); logpi_dev/logpi_alt_dev: two N buffers of the particle
 * dtype; logw_dev: N doubles; workspace_dev: smc_workspace_bytes() bytes,
 * 256-byte aligned.  All are borrowed until smc_destroy.  On success *out is
 * a new handle.  Errors: SMC_EINVAL (sizes, pointers, alignment, target),
 * SMC_ENOMEM (workspace too small), SMC_ECUDA. */
int smc_init(smc_sampler** out, const smc_config* cfg, void* x_dev, void* x_alt_dev, double* logw_dev,
             void* logpi_dev, void* logpi_alt_dev, void* workspace_dev, size_t workspace_bytes,
             smc_stream_t stream);

/* Algorithm 2, line 4 (proposal): starts iteration t <- t+1 and moves every
 * particle x_t = x_{t-1} + eps z, z ~ N(0, I) from Philox (seed, t, i). */
int smc_move(smc_sampler* h);

/* Eq. (5) with the forward-proposal L-kernel L = q of Sec. 5.2.3 (the L/q
 * factor is exactly 1):  log w_t = log w_{t-1} + log pi(x_t) - log pi(x_{t-1});
 * then eqs. (1), (2), (8): m, LSE_t, N_eff, log c_t and the resampling
 * decision into the device statistics (smc_read_stats). */
int smc_reweight(smc_sampler* h);

/* Eq. (7): f_t = sum_i w~_t^i x_t^i into mean_dev[D] (double) and, if
 * cov_dev is not NULL, the weighted covariance into cov_dev[D*D]. */
int smc_estimate(smc_sampler* h, double* mean_dev, double* cov_dev);

/* Algorithm 4, line 1 (MVR): systematic resampling of the quantised weights
 * W_i = E(log w_i - m) >> (62 - F) into ncopies_dev[N] (int32, sum N, eq. (9)),
 * whatever the decision; did_resample_dev (int32, may be NULL) receives the
 * decision of the last smc_reweight. */
int smc_resample(smc_sampler* h, int32_t* ncopies_dev, int32_t* did_resample_dev);

/* Algorithm 4, lines 2-3 with Algorithm 5 (S-R) as the definition of the
 * result: particle row i and its log pi are written ncopies[i] times, in
 * index order, into the other buffer, which becomes current; every log-weight
 * is reset to -log N.  ncopies_dev must be N non-negative ints summing to N
 * (else SMC_EINVAL at the next smc_sync, and nothing is written). */
int smc_redistribute(smc_sampler* h, const int32_t* ncopies_dev);

/* K iterations of Algorithm 2 (lines 3-10): move, reweight, normalise,
 * estimate, N_eff, and resample + redistribute + reset when N_eff < N*,
 * with no host synchronisation between iterations (the decision stays on the
 * device; the launches of an iteration are replayed from a CUDA graph).  An
 * FP64 sampler with N <= 2048 (Gaussian or Student-t target) runs the K
 * iterations in one cooperative launch instead, with the same per-stage
 * arithmetic (bit-identical results); if its grid cannot be resident it uses
 * the graph. 
 * mean_dev[D] receives f_K, cov_dev[D*D] (may be NULL) the final weighted
 * covariance, trace_dev (may be NULL) K smc_iter_stats records, and
 * fhat_dev[D] (may be NULL) the recycled estimate of eq. (6) over all
 * iterations run so far. */
int smc_step(smc_sampler* h, int32_t k, double* mean_dev, double* cov_dev, smc_iter_stats* trace_dev,
             double* fhat_dev);

/* Tracing: one iteration of smc_step launched directly (not from a graph),
 * with events_host[0] (cudaEvent_t, created by the caller) recorded before it
 * and events_host[j] after stage j: 1 move + reweight, 2 max / mean finalise,
 * 3 quantise reduce, 4 quantise finalise, 5 systematic scan, 6 redistribute,
 * 7 commit.  n_events must be 8, or 0 to record nothing.  The iteration is
 * identical to one iteration of smc_step (mean_dev may be NULL). */
int smc_step_profile(smc_sampler* h, double* mean_dev, void* const* events_host, int32_t n_events);

/* Synchronises the sampler's stream; returns the first error recorded on the
 * device since the last smc_sync (then clears it), or SMC_OK. */
int smc_sync(smc_sampler* h);

/* Copies the last iteration's statistics to the host (synchronising). */
int smc_read_stats(smc_sampler* h, smc_iter_stats* out_host);

/* 0 if x_dev / logpi_dev hold the current particles, 1 if the _alt buffers do
 * (synchronising; completes a deferred redistribution first). */
int smc_current(smc_sampler* h, int32_t* which_host);

/* Completes the redistribution (Algorithm 5 and the log w reset) that a
 * sampler created with SMC_FLAG_DEFER_REDISTRIBUTE left pending, on the
 * sampler's stream; a no-op otherwise.  smc_move, smc_reweight, smc_estimate,
 * smc_resample, smc_redistribute, smc_current, the checkpoint calls and
 * smc_batch_create do it themselves. */
int smc_materialize(smc_sampler* h);

/* Frees the handle (host memory only). */
int smc_destroy(smc_sampler* h);

/* ---------------------------------------------------------------------------
 * Checkpoint / resume.  The state of Algorithm 2 between two iterations is the
 * particles x, their log pi, the log-weights (eq. 5), the iteration index t,
 * LSE_{t-1} and the recycling sums of eq. (6).  Random numbers are
 * counter-based (Philox keyed by seed, t and particle index), so a sampler
 * restored from a checkpoint taken after iteration t continues bit for bit as
 * the original would have.
 *
 * smc_checkpoint_bytes: size of a checkpoint of h (host bytes) in *bytes.
 *   Layout: a 56-byte header (magic "SMCCKPT1", version, D, N, dtype, target,
 *   seed, state-block bytes, row bytes), the device state block, x (N x D, row-major, the sampler's dtype),
 *   log pi (N, the sampler's dtype), log w (N doubles).
 * smc_checkpoint_save: waits for the work queued on the sampler's stream,
 *   then copies the state into host_dst (caller-owned, `bytes` long, any host
 *   memory).  Returns SMC_EINVAL if bytes is too small, the pending device
 *   error (nothing saved) if one is recorded, SMC_ECUDA on a failed copy.
 * smc_checkpoint_load: restores a checkpoint into h, which must have been
 *   created with the same N, D, dtype, target and seed (SMC_EINVAL otherwise,
 *   and h is untouched).  The particles land in x_dev / logpi_dev (buffer 0);
 *   outputs requested from earlier calls are not written.  Synchronous: the
 *   host buffer may be freed when it returns.  The target's parameters are
 *   not part of the checkpoint: h's own are used. */
int smc_checkpoint_bytes(const smc_sampler* h, size_t* bytes);
int smc_checkpoint_save(smc_sampler* h, void* host_dst, size_t bytes);
int smc_checkpoint_load(smc_sampler* h, const void* host_src, size_t bytes);

/* Message of the last error on this handle (or of the last handle-less call
 * when h is NULL); never NULL. */
const char* smc_last_error(const smc_sampler* h);

/* ---------------------------------------------------------------------------
 * Stateless redistribute (the resample + redistribute microbenchmark).
 * Algorithm 5 on raw rows: out row k = in row src(k), src(k) = the i with
 * off_i <= k < off_i + ncopies_i, off = exclusive cumulative sum of ncopies.
 * row_bytes must be a multiple of 4; in/out must not overlap.  ws_dev:
 * smc_redistribute_ws_bytes(n) bytes, 256-byte aligned.  An ncopies vector
 * with a negative entry or a sum other than n writes nothing and records
 * SMC_EINVAL, returned by smc_ws_status. */
int smc_redistribute_ws_bytes(int64_t n, size_t* bytes);
int smc_redistribute_raw(int64_t n, int32_t row_bytes, const int32_t* ncopies_dev, const void* in_dev,
                         void* out_dev, void* ws_dev, smc_stream_t stream);
/* The same call with caller events (cudaEvent_t, n_events = 3, or 0 for
 * none) recorded on stream before it, after the exclusive scan of ncopies
 * (run starts and tile starts written), and after the row copy: the copy
 * kernel's own time is the interval between events 1 and 2. */
int smc_redistribute_raw_profile(int64_t n, int32_t row_bytes, const int32_t* ncopies_dev, const void* in_dev,
                                 void* out_dev, void* ws_dev, smc_stream_t stream, void* const* events_host,
                                 int32_t n_events);

/* Stateless resampling (Algorithm 4, line 1) of logw_dev[n] with Philox
 * (seed, t): writes ncopies_dev[n] and, when stats_dev is not NULL, one
 * smc_iter_stats record (lse, ess, max_logw, resampled decision under mode).
 * ws_dev: smc_redistribute_ws_bytes(n) bytes. */
int smc_resample_raw(int64_t n, const double* logw_dev, uint64_t seed, uint64_t t, int32_t mode,
                     int32_t* ncopies_dev, smc_iter_stats* stats_dev, void* ws_dev, smc_stream_t stream);

/* Algorithm 8 (S-NS, Sec. 4.2), the local step of the paper's nearly-sort
 * based redistribute (N-R, Algorithm 9), as a comparison for the gather
 * design of smc_redistribute_raw.  Scanning i = 0..n-1, a row whose key
 * ncopies_i is positive goes to the next free slot from the right end of the
 * output, any other row to the next free slot from the left end:
 *   slot(i) = n - 1 - P_i if ncopies_i > 0, else i - P_i,
 *   P_i = #{j < i : ncopies_j > 0};
 * ncopies_out_dev[slot(i)] = ncopies_i and out row slot(i) = in row i, so the
 * output keys are an ascending Nearly-Sorted sequence (Definition 1: every
 * zero before every positive key).  Any int32 keys are accepted (no device
 * error).  ncopies_dev: n int32, 16-byte aligned; in_dev / out_dev: n rows of
 * row_bytes (a multiple of 4; rows aligned to 16, 8 or 4 bytes as row_bytes
 * allows); outputs must not overlap inputs.  ws_dev:
 * smc_nearly_sort_ws_bytes(n) bytes, 256-byte aligned.  Errors: SMC_EINVAL
 * (sizes, null or misaligned pointers), SMC_ECUDA. */
int smc_nearly_sort_ws_bytes(int64_t n, size_t* bytes);
int smc_nearly_sort_raw(int64_t n, int32_t row_bytes, const int32_t* ncopies_dev, const void* in_dev,
                        int32_t* ncopies_out_dev, void* out_dev, void* ws_dev, smc_stream_t stream);

/* Synchronises stream and returns (then clears) the error recorded in a
 * stateless workspace. */
int smc_ws_status(void* ws_dev, smc_stream_t stream);

/* ---------------------------------------------------------------------------
 * Allocation-free stateless redistribute.  The paper has no counterpart: this
 * is a deployment convenience.  It computes exactly what smc_redistribute_raw
 * computes, for callers that cannot allocate device memory when they call --
 * for example a plug-in handed only its input and output buffers, code inside
 * a framework whose memory pool owns every device allocation, or a real-time
 * loop that forbids allocation after start-up.  Its scratch is a fixed device
 * array inside the library (about 4.2 MB on every GPU that loads the library,
 * held until the process exits), so:
 *  - n must be at most SMC_NOALLOC_MAX_N, else SMC_EINVAL and nothing runs;
 *  - all calls on a device share the array: calls whose work overlaps on the
 *    GPU (streams with no ordering between them) race and give undefined
 *    results;
 *  - the first call on each device looks up the array's device address with
 *    that device current; make that first call before any stream capture;
 *  - that address is kept for the life of the process: do not call this
 *    entry point on a device after cudaDeviceReset (or any other reset of its
 *    primary context) in the same process -- the kept address would then
 *    name memory that no longer exists.
 * status_dev (device int32, may be NULL) receives SMC_OK, or SMC_EINVAL when
 * ncopies has a negative entry or does not sum to n (then out_dev is not
 * written).  The call allocates nothing: no cudaMalloc, no cudaFree, no
 * allocating library routine. */
#define SMC_NOALLOC_MAX_N 1048576
int smc_redistribute_raw_noalloc(int64_t n, int32_t row_bytes, const int32_t* ncopies_dev, const void* in_dev,
                                 void* out_dev, int32_t* status_dev, smc_stream_t stream);

/* ---------------------------------------------------------------------------
 * Batches: many independent samplers stepped together, one launch per stage
 * for all of them (Algorithm 2, lines 3-10, for every member at once).  The
 * paper runs one sampler at a time; batching is an addition for workloads of
 * many small samplers, where one sampler per launch leaves the GPU idle
 * between tiny kernels.  Every member's results are bit-identical to those
 * of smc_step on that sampler alone: each member keeps its own blocks, tiles,
 * partial sums and reduction order; only the launch is shared.
 *
 * Members are handles from smc_init with dtype SMC_F32 and target SMC_GAUSS
 * (the FP32 move / reweight kernel), all on the current device, each listed
 * once.  A handle must not be stepped by itself, nor be a member of another
 * batch, while the batch is in use.  smc_batch_create makes the batch's
 * stream wait (on the device, no host wait) for the work already queued on
 * every member's stream; afterwards the batch works on its own stream, and
 * a member's own calls must be ordered after the batch's work (smc_batch_sync,
 * or the member's stream waiting on the batch's stream) to see its results.
 *
 * ws_dev: smc_batch_ws_bytes(...) bytes of device memory, 256-byte aligned,
 * owned by the caller and alive until smc_batch_destroy.  It holds the
 * members' kernel arguments and the block maps of the launches. */
typedef struct smc_batch smc_batch;

int smc_batch_ws_bytes(smc_sampler* const* members, int32_t count, size_t* bytes);
int smc_batch_create(smc_batch** out, smc_sampler* const* members, int32_t count, void* ws_dev,
                     size_t ws_bytes, smc_stream_t stream);

/* k iterations for every member.  mean_dev / trace_dev / fhat_dev are NULL or
 * HOST arrays of count DEVICE pointers (entries may be NULL) with the meaning
 * smc_step gives its arguments of those names, per member.  Iterations are
 * replayed from a CUDA graph of one batched iteration (8 launches). */
int smc_batch_step(smc_batch* b, int32_t k, double* const* mean_dev, smc_iter_stats* const* trace_dev,
                   double* const* fhat_dev);

/* Tracing: one batched iteration launched directly (not from a graph), with
 * the caller's 8 CUDA events (cudaEvent_t, may be NULL when n_events == 0)
 * recorded on the batch's stream around the stages, in the order of
 * smc_step_profile.  Results are identical to one iteration of
 * smc_batch_step with no outputs. */
int smc_batch_step_profile(smc_batch* b, void* const* events_host, int32_t n_events);

/* Launch-shape variants.  None changes any result.  move_variant picks how
 * many blocks share the move / reweight launch (0: 2 per SM, 1: 4, 2: 8,
 * 3: 16, 4: one thread per particle), which fixes the particles each warp
 * handles; copy_variant picks the 16-byte loads each thread keeps in flight
 * in the redistribute copy (0: 4, 1: 8, 2: 16).  Defaults: 2 and 1. */
#define SMC_BATCH_MOVE_VARIANTS 5
#define SMC_BATCH_COPY_VARIANTS 3
int smc_batch_set_variant(smc_batch* b, int32_t move_variant, int32_t copy_variant);

/* Autotuner: times every variant reps times (CUDA events, median) on work
 * that leaves every member's state untouched -- the move on the members'
 * spare buffers, the copy as an in-place identity copy -- then keeps the
 * fastest of each.  Writes {move_variant, copy_variant} to choice_host when
 * not NULL.  Synchronises the batch's stream. */
int smc_batch_tune(smc_batch* b, int32_t reps, int32_t* choice_host);

/* Synchronises the batch's stream; returns (then clears) the first device
 * error recorded by any member, with the member's index in which_host
 * (-1 when none; may be NULL). */
int smc_batch_sync(smc_batch* b, int32_t* which_host);

/* Frees the handle (host memory only); members stay valid. */
int smc_batch_destroy(smc_batch* b);
const char* smc_batch_last_error(const smc_batch* b);

/* ---------------------------------------------------------------------------
 * Standing batches of slots (serving).  The batch above is laid out for one
 * member list; a server whose jobs come and go would rebuild it (block maps,
 * CUDA graph) at every change.  A standing batch is laid out once for `count`
 * slots of fixed capacity: slot s holds one FP32 Gaussian sampler of at most
 * cap_n[s] particles (any D), attached and detached between steps by editing
 * a slot table in device memory, with no rebuild and no host
 * synchronisation.  Each step runs, for every slot, the number of
 * iterations (Algorithm 2, lines 3-10) the caller asks for that slot, all
 * slots in one launch per stage (one CUDA graph replay per iteration);
 * slots with fewer iterations, and empty slots, do nothing in the later
 * launches.  A sampler's results in a slot are bit-identical to those of
 * smc_step on it alone (its own blocks, tiles and reduction order).
 *
 * smc_slots_ws_bytes: device workspace for these capacities (1 <= count <=
 *   512, 1 <= cap_n[s] < 2^31).
 * smc_slots_create: ws_dev 256-byte aligned, owned by the caller, alive until
 *   smc_slots_destroy; stream must not be NULL (the legacy default stream
 *   cannot hold the graph).  Synchronises the stream once (layout upload).
 * smc_slots_attach: puts h (an smc_init handle, SMC_F32, SMC_GAUSS, N <=
 *   cap_n[slot], attached nowhere else) into the empty slot; mean_dev (D
 *   doubles), trace_dev (one smc_iter_stats per iteration run in the slot)
 *   and fhat_dev (D doubles) are device outputs with smc_step's meaning, each
 *   may be NULL.  The slots' stream is ordered after the work already queued
 *   on h's stream (device-side; a pending deferred copy is completed first).
 *   h must not be stepped by itself while attached.
 * smc_slots_detach: empties the slot; h's stream is ordered after the slots'
 *   work queued so far, so h's own calls may follow at once.
 * smc_slots_step: iters_host[count] (host array) gives each slot's
 *   iterations for this call (0 for idle and empty slots; a positive count
 *   for an empty slot is SMC_EINVAL); the call enqueues max(iters) batched
 *   iterations on the slots' stream and returns.
 * smc_slots_sync: synchronises the stream; returns (then clears) the first
 *   device error of an attached sampler, its slot in which_host (-1 when
 *   none; may be NULL).
 * Errors: SMC_EINVAL (arguments, as above), SMC_ENOMEM (workspace too
 * small), SMC_ECUDA; messages from smc_slots_last_error (NULL: the last
 * handle-less call). */
typedef struct smc_slots smc_slots;

int smc_slots_ws_bytes(const int64_t* cap_n, int32_t count, size_t* bytes);
int smc_slots_create(smc_slots** out, const int64_t* cap_n, int32_t count, void* ws_dev, size_t ws_bytes,
                     smc_stream_t stream);
int smc_slots_attach(smc_slots* b, int32_t slot, smc_sampler* h, double* mean_dev, smc_iter_stats* trace_dev,
                     double* fhat_dev);
int smc_slots_detach(smc_slots* b, int32_t slot);
int smc_slots_step(smc_slots* b, const int32_t* iters_host);
int smc_slots_sync(smc_slots* b, int32_t* which_host);
int smc_slots_destroy(smc_slots* b);
const char* smc_slots_last_error(const smc_slots* b);

#ifdef __cplusplus
}
#endif

#endif /* SMC_H_ */
