// smc_kernels.h -- host-visible launch interface between the C-ABI layer
// (smc_api.cu) and the kernel translation units of libsmc.so.
#pragma once

#include <cstddef>
#include <cstdint>
#include <cuda_runtime.h>

#include "../../include/smc.h"

namespace smc {

struct DevState;
constexpr int kTgtMaxD = 32;

// Device copy of the target: Gaussian mean, Cholesky factor L (FP64 path),
// its inverse P and FP32 copies (FP32 path), Student-t nu.
struct alignas(256) TargetDev {
  int32_t kind;
  int32_t d;
  double nu;
  double mu[kTgtMaxD];
  float muf[kTgtMaxD];
  double L[kTgtMaxD * kTgtMaxD];
  double P[kTgtMaxD * kTgtMaxD];
  float Pf[kTgtMaxD * kTgtMaxD];
  // Bayesian logistic regression: log pi(b) = sum_m [y_m z_m - log(1 + e^z_m)]
  // - |b|^2 / (2 prior_var), z = X b.  The data live in the sampler's workspace.
  const float* X;         // M x D row-major (FP32 copy of the caller's data)
  const float* y;         // M labels
  const uint16_t* ximg;   // BF16 hi / lo images of X for the tensor-core likelihood
  double v[kTgtMaxD];     // X^T y in FP64
  double xsum[kTgtMaxD];  // column sums of X in FP64
  double prior_var;
  int32_t m;
  int32_t m_pad;          // M rounded up to the likelihood's data tile
};

// Tensor-core logistic likelihood: data tile (rows of X per MMA) and the bytes
// of one tile's BF16 hi + lo images (K = 32 columns, zero padded).
constexpr int kLgRows = 256;
constexpr int kLgK = 32;
constexpr size_t kLgTileBytes = size_t(kLgRows) * kLgK * 2 * 2;

enum { OP_INIT = 0, OP_MOVE = 1, OP_REWEIGHT = 2, OP_MOVE_REWEIGHT = 3, OP_MOVE_REWEIGHT_EST = 4,
       OP_MOVE_REWEIGHT_GATHER = 5 };  // (5: OP_MOVE_REWEIGHT_EST that also gathers a pending resampling's rows)

// FP32 Gaussian target passed by value as a kernel parameter (constant bank):
// the lower triangle of L^-1 packed row by row (row r holds r + 1 entries at
// r (r + 1) / 2) and mu.
// The FP32 Gaussian target of the move / reweight kernels: mu and the
// inverse Cholesky factor P = L^-1 with rows 2p and 2p + 1 interleaved,
// P2[p][c] = {P[2p][c], P[2p+1][c]} (zero above the diagonal), so that one
// packed two-lane FMA advances both rows.
struct GaussParamsF32 {
  float mu[kTgtMaxD];
  float2 P2[kTgtMaxD / 2 * kTgtMaxD];
};

// Lanes that share one particle in the move / reweight kernels: one in every
// path (the FP32 path holds up to 32 coordinates in one lane's registers).
inline int lanes_per_particle(int, int) { return 1; }

// ParticleArgs.flags
enum {
  PA_INIT_SKIP_LOGPI = 1,  // init writes log pi = 0 (a later likelihood pass adds it)
  PA_STALL_COPIES = 2,     // test hook: the tensor-core likelihood issues no data copies
};

struct ParticleArgs {
  int64_t n;
  int32_t d;
  int32_t dtype;
  int32_t kind;
  int32_t flags;
  uint64_t seed;
  double step;
  double init_scale;
  void* x[2];
  void* logpi[2];
  double* logw;
  double* part;   // per-block maximum records (2 doubles each)
  double* epart;  // eq. (7) records {M_r, sum e x} per 256-particle tile (1 + d doubles each)
  const TargetDev* tg;
  DevState* st;
  // a pending resampling's run starts and copy-tile sources (gathering move);
  // rs_alt: the second run-start array (NULL when the sampler has one)
  int32_t* rs;
  int32_t* rs_alt;
  const int32_t* tile_src;
};

struct QuantArgs {
  int64_t n;
  int64_t nstar;       // resampling threshold N* (0: N/2)
  const double* logw;
  uint64_t seed;
  int32_t mode;        // smc_resample_mode
  int32_t force;       // scan even if the decision is "no resample"
  uint64_t* qpart;     // per-block {sumW, sw2 lo, sw2 hi, sumE lo, sumE hi}
  uint64_t* cbase;     // exclusive prefix of the block sums of W
  int32_t* runstart;   // runstart[off_i] = i for every survivor (when write_rs)
  int32_t* runstart_alt;  // second run-start array (NULL: one array); st->rs_w picks
  int32_t write_rs;
  int32_t pad;
  uint64_t* wbuf;      // W_i written by the reduce pass, read by the scan (N words)
  int32_t* ncopies;    // optional output
  int32_t* tile_src;   // source row of the first output row of each redistribute tile
  int32_t nblocks;     // quantise blocks
  int32_t ntiles;      // redistribute tiles
  DevState* st;
  smc_iter_stats* stats_out;  // optional single record (stateless path)
  // eq. (7) in the reduce pass: sum_i E_i x_i over the current rows, when x[0]
  const void* x[2];
  int32_t d;
  int32_t dtype;
  void* xpart;         // nblocks x d partial sums, in the particle dtype
  // est_src = 1: the reduce pass forms the eq. (7) partials from the move
  // kernel's tile records (epart) instead of reading x
  const double* epart;
  int32_t est_src;
  int32_t pad2;
};

// Sequential Nearly Sort (Algorithm 8) as a stable partition (k_nearly_sort.cu).
constexpr int kNsTile = 4096;  // keys per block
struct NearlySortArgs {
  int64_t n;
  int32_t row_bytes;   // multiple of 4
  int32_t ntiles;      // ceil(n / kNsTile)
  const int32_t* ncopies;  // 16-byte aligned
  int32_t* ncopies_out;
  const void* in;
  void* out;
  int32_t* tile_count;  // ntiles
  int32_t* tile_base;   // ntiles, exclusive prefix of tile_count
};

struct RedistArgs {
  int64_t n;
  int32_t row_bytes;
  int32_t lp_bytes;      // 0: no log pi payload
  int32_t* runstart;     // consumed and reset to -1 by the tile that reads it
  int32_t* runstart_alt; // second run-start array (NULL: one array); st->rs_w picks
  const int32_t* tile_src;
  int32_t ntiles;
  int32_t force;         // copy even if the decision is "no resample"
  const void* x_in[2];   // indexed by the current buffer (stateful) or [0]
  void* x_out[2];
  const void* lp_in[2];
  void* lp_out[2];
  double* logw;          // reset to reset_logw (may be NULL)
  double reset_logw;
  DevState* st;
  int32_t stateful;      // 1: choose buffers by st->cur, honour st->flag / st->err
  int32_t use_pending;   // stateful: copy iff st->pending (a deferred resampling), not st->flag
  // stamped calls (see NcScanArgs::stamps): per tile, nonzero when the tile
  // has run starts (its runstart slice is then fully written; otherwise the
  // slice is not read and means -1 throughout); NULL: read every slice
  const int32_t* stamps;
};

struct NcScanArgs {
  int64_t n;
  const int32_t* ncopies;
  uint64_t* part;       // per-block sums
  uint64_t* cbase;      // exclusive block prefixes
  int32_t* runstart;    // must hold -1 everywhere on entry, unless clear_rs
  int32_t* runstart_alt;  // second run-start array (NULL: one array); st->rs_w picks
  int32_t* tile_src;
  int32_t nblocks;
  int32_t ntiles;
  DevState* st;
  int32_t clear_rs;     // the reduce pass sets runstart[0, n) to -1 first (runstart_alt NULL)
  int32_t pad;
  // stamped calls (the stateless entry points; zeroed by the caller before
  // each call): per copy tile, set when a run start lands in it -- runstart
  // then need not be clean on entry (k_nc_scan writes every slice the copy
  // reads); NULL: runstart must hold -1 everywhere on entry
  int32_t* stamps;
};

size_t devstate_bytes();

// Message returned by smc_last_error(NULL) (smc_api.cu).
void set_global_error(const char* msg);

// threads: block size, a multiple of 32 up to kPThreads (small samplers use
// small blocks so that their particles spread over more SMs)
cudaError_t launch_particles(int op, const ParticleArgs& a, int grid, int threads, cudaStream_t s,
                             const GaussParamsF32* gp = nullptr);
cudaError_t launch_target_setup(TargetDev* tg, int kind, double nu, const double* mu, const double* sigma, int d,
                                DevState* st, cudaStream_t s);
// Copies the logistic data into the workspace (Xw: M x D, yw: M), builds the
// BF16 images (ximg: m_pad / kLgRows tiles) and v = X^T y, and points tg at them.
cudaError_t launch_logistic_setup(TargetDev* tg, const float* X, const float* y, int m, int d, double prior_var,
                                  float* Xw, float* yw, uint16_t* ximg, cudaStream_t s);
cudaError_t launch_max_finalize(const double* part, int nb, DevState* st, cudaStream_t s);
// eq. (7) covariance: grid blocks write covpart[grid][D(D+1)/2], then a fixed-order sum
cudaError_t launch_cov(const ParticleArgs& a, double* cov, double* covpart, int grid, cudaStream_t s);
cudaError_t launch_begin(DevState* st, cudaStream_t s);
cudaError_t launch_commit(DevState* st, int d, int force_flip, int recycle, cudaStream_t s, int defer = 0);
// Ends a pending (deferred) redistribution after its copy: the copied rows'
// buffer becomes current.
cudaError_t launch_settle(DevState* st, cudaStream_t s);
cudaError_t launch_copy_mean(const DevState* st, double* out, int d, cudaStream_t s);
cudaError_t launch_step_setup(DevState* st, smc_iter_stats* trace, double* mean_out, double* fhat_out,
                              double* cov_out, cudaStream_t s);

// Logistic likelihood on the tensor cores, fused with the reweight of eq. (5)
// (k_logistic_tc.cu): log pi of the current particles, log w += new - old,
// one max record per CTA in a.part (grid = logistic_tc_grid(n, SMs)).
int logistic_tc_grid(int64_t n, int sms);
cudaError_t launch_logistic_tc(const ParticleArgs& a, int grid, cudaStream_t s);

// batched launches (one per stage for many samplers; int4 map = {sampler, block, blocks, 0}).
// left (standing batches of slots, k_slots): per-member count of iterations
// still to run in this call; members at 0 do nothing, and the commit
// decrements it.  NULL for plain batches (every member runs).
cudaError_t launch_move_reweight_batch(const ParticleArgs* pa, const GaussParamsF32* gps, const int4* map, int nblocks,
                                       cudaStream_t s, const int32_t* left = nullptr);
cudaError_t launch_max_finalize_batch(const ParticleArgs* pa, const int* nb, int count, cudaStream_t s,
                                      const int32_t* left = nullptr);
cudaError_t launch_begin_batch(const ParticleArgs* pa, int count, cudaStream_t s, const int32_t* left = nullptr);
cudaError_t launch_commit_batch(const ParticleArgs* pa, int count, cudaStream_t s, int32_t* left = nullptr);
cudaError_t launch_quant_reduce_batch(const QuantArgs* qa, const int4* map, int nblocks, cudaStream_t s,
                                      const int32_t* left = nullptr);
cudaError_t launch_quant_finalize_batch(const QuantArgs* qa, int count, cudaStream_t s, const int32_t* left = nullptr);
cudaError_t launch_quant_scan_batch(const QuantArgs* qa, const int4* map, int nblocks, cudaStream_t s,
                                    const int32_t* left = nullptr);
cudaError_t launch_redistribute_batch(const RedistArgs* ra, const int4* map, int nblocks, int copy_variant,
                                      cudaStream_t s, const int32_t* left = nullptr);  // copy_variant: 4, 8, 16 loads in flight per thread
cudaError_t launch_identity_runs_batch(const RedistArgs* ra, const int4* map, int nblocks, cudaStream_t s);
cudaError_t launch_step_setup_batch(const ParticleArgs* pa, void* const* outs, int count, cudaStream_t s);
cudaError_t launch_take_errors_batch(const ParticleArgs* pa, int32_t* errs, int count, cudaStream_t s);

// k_resample.cu
cudaError_t upload_expfx_table();  // once per device, outside stream capture
cudaError_t launch_max_logw(const double* logw, int64_t n, double* part, int nb, DevState* st, cudaStream_t s);
cudaError_t launch_quant_reduce(const QuantArgs& a, cudaStream_t s);
cudaError_t launch_quant_finalize(const QuantArgs& a, int set_lse_prev, cudaStream_t s);
cudaError_t launch_quant_scan(const QuantArgs& a, cudaStream_t s);
cudaError_t launch_nc_reduce(const NcScanArgs& a, cudaStream_t s);
cudaError_t launch_nc_finalize(const NcScanArgs& a, cudaStream_t s);
cudaError_t launch_nc_scan(const NcScanArgs& a, cudaStream_t s);
cudaError_t launch_redistribute(const RedistArgs& a, cudaStream_t s);
// one-block samplers: quantise reduce + finalise + scan (N <= 4096), and
// redistribute + commit (N <= 2048), each as one launch
cudaError_t launch_quant_small(const QuantArgs& a, cudaStream_t s);
cudaError_t launch_redistribute_commit(const RedistArgs& a, int d, int force_flip, int recycle, cudaStream_t s);

// k iterations of an FP64 sampler of one quantise block and one copy tile
// (N <= 2048) in one cooperative launch of move_blocks blocks (see
// k_iterate_small).  bar: the grid barrier's zeroed 64-bit count.  stop_last: the
// last iteration ends after its scan (its copy and commit follow as separate
// launches, after the covariance).
struct SmallIterArgs {
  ParticleArgs a;
  QuantArgs q;
  RedistArgs r;
  unsigned long long* bar;
  int32_t k;
  int32_t move_threads;  // threads per block that own particles (the separate move launch's block size)
  int32_t d;
  int32_t stop_last;
  int32_t stall;  // test hook (SMC_FLAG_TEST_STALL_BARRIER): the barrier waits for one block more than the grid
  int32_t pad;
};
bool small_iter_fits(int64_t n, int dtype);
cudaError_t launch_iterate_small(const SmallIterArgs& s, int move_blocks, cudaStream_t st);
int nearly_sort_tiles(int64_t n);
cudaError_t launch_nearly_sort(const NearlySortArgs& a, cudaStream_t s);
cudaError_t launch_state_init(DevState* st, int64_t n, int64_t t, int F, cudaStream_t s);

}  // namespace smc
