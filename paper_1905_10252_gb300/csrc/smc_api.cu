// smc_api.cu -- the C-ABI of libsmc.so (declared in include/smc.h): argument
// checking, the workspace layout, the order of kernel launches for each step
// of the sampler, CUDA-graph replay of whole iterations, and error reporting.
// The library allocates no device memory: every buffer is the caller's.
#include <algorithm>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <new>
#include <string>

#include "smc_host.h"
#include "smc_trace.h"

using namespace smc;

namespace {

thread_local std::string g_err = "ok";

constexpr size_t kAlign = 256;
constexpr int kMaxPartBlocks = 4096;  // particle-kernel grid cap (partials buffer)

size_t align_up(size_t v) { return (v + kAlign - 1) / kAlign * kAlign; }

int64_t div_up(int64_t a, int64_t b) { return (a + b - 1) / b; }

int quant_shift(int64_t n) {
  int c = 0;
  while ((int64_t(1) << c) < n) ++c;
  const int F = 63 - c;
  return F > 62 ? 62 : F;
}

// two_rs: a second run-start array (SMC_FLAG_DEFER_REDISTRIBUTE samplers)
Layout layout_for(int64_t n, int d, int m = 0, bool two_rs = false) {
  Layout L{};
  L.qblocks = int(div_up(n, kQTile));
  L.ntiles = int(div_up(n, kRTile));
  size_t p = 0;
  L.st = p;
  p = align_up(p + sizeof(DevState));
  L.tg = p;
  p = align_up(p + sizeof(TargetDev));
  L.part = p;
  const size_t part_blocks = size_t(std::max(kMaxPartBlocks, L.qblocks));
  p = align_up(p + part_blocks * 2 * sizeof(double));
  // eq. (7) records of the move kernel, one per 256-particle tile: {M_r, sum e x}
  L.epart = p;
  p = align_up(p + size_t(div_up(n, kEstTile)) * (1 + size_t(d < 1 ? 1 : d)) * sizeof(double));
  L.qpart = p;
  p = align_up(p + size_t(L.qblocks) * 5 * sizeof(uint64_t));
  L.cbase = p;
  p = align_up(p + size_t(L.qblocks) * sizeof(uint64_t));
  L.xpart = p;
  p = align_up(p + size_t(L.qblocks) * size_t(d < 1 ? 1 : d) * sizeof(double));
  L.rs = p;
  p = align_up(p + size_t(n) * sizeof(int32_t));
  L.rs_alt = 0;
  if (two_rs) {
    L.rs_alt = p;
    p = align_up(p + size_t(n) * sizeof(int32_t));
  }
  L.wbuf = p;
  p = align_up(p + size_t(n) * sizeof(uint64_t));
  L.tile_src = p;
  p = align_up(p + size_t(L.ntiles + 1) * sizeof(int32_t));
  // the grid barrier of the fused small-sampler iterations (a 64-bit count)
  L.gbar = p;
  p = align_up(p + sizeof(unsigned long long));
  // logistic data: X, y and the BF16 tile images
  const size_t m_pad = size_t(m + kLgRows - 1) / kLgRows * kLgRows;
  L.lg_x = p;
  p = align_up(p + size_t(m) * size_t(d) * sizeof(float));
  L.lg_y = p;
  p = align_up(p + size_t(m) * sizeof(float));
  L.lg_img = p;
  p = align_up(p + m_pad / kLgRows * kLgTileBytes);
  // per-block covariance partials
  L.cov_blocks = int(std::min<int64_t>(kCovMaxBlocks, div_up(n, 128)));
  L.covpart = p;
  p = align_up(p + size_t(L.cov_blocks) * size_t(d * (d + 1) / 2) * sizeof(double));
  L.total = p;
  return L;
}

int logistic_rows(const smc_config* c) { return c->target == SMC_LOGISTIC ? c->m : 0; }

bool wants_two_rs(const smc_config* c) { return (c->flags & SMC_FLAG_DEFER_REDISTRIBUTE) != 0; }

bool aligned(const void* p, size_t a) { return (reinterpret_cast<uintptr_t>(p) % a) == 0; }

}  // namespace

void smc::set_global_error(const char* msg) { g_err = msg; }

int smc::sm_count() {
  static int cached[64] = {0};
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return 132;
  if (dev >= 0 && dev < 64 && cached[dev]) return cached[dev];
  int v = 0;
  if (cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || v <= 0) v = 132;
  if (dev >= 0 && dev < 64) cached[dev] = v;
  return v;
}


namespace {

int fail(smc_sampler* h, int code, const std::string& msg) {
  if (h)
    h->err = msg;
  else
    g_err = msg;
  return code;
}

int cuda_fail(smc_sampler* h, cudaError_t e, const char* where) {
  return fail(h, SMC_ECUDA, std::string(where) + ": " + cudaGetErrorString(e));
}

#define SMC_TRY(h, expr)                                  \
  do {                                                    \
    cudaError_t _e = (expr);                              \
    if (_e != cudaSuccess) return cuda_fail((h), _e, #expr); \
  } while (0)

// (fetch_gp must have run: an FP32 Gaussian sampler launched without its
// factor would take the generic kernel)
const GaussParamsF32* gauss_params(const smc_sampler* h) { return h->gp_ready ? &h->gp : nullptr; }

}  // namespace

namespace smc {

ParticleArgs particle_args(const smc_sampler* h) {
  ParticleArgs a{};
  a.n = h->n;
  a.d = h->d;
  a.dtype = h->dtype;
  a.kind = h->cfg.target;
  a.seed = h->cfg.seed;
  a.step = h->cfg.step;
  a.init_scale = h->cfg.init_scale;
  a.x[0] = h->x[0];
  a.x[1] = h->x[1];
  a.logpi[0] = h->lp[0];
  a.logpi[1] = h->lp[1];
  a.logw = h->logw;
  a.part = h->part;
  a.epart = reinterpret_cast<double*>(h->ws + h->L.epart);
  a.tg = h->tg;
  a.st = h->st;
  a.rs = h->rs;
  a.rs_alt = h->rs_alt;
  a.tile_src = h->tile_src;
  if (h->cfg.flags & SMC_FLAG_TEST_STALL_LIKELIHOOD) a.flags |= PA_STALL_COPIES;
  return a;
}

QuantArgs quant_args(const smc_sampler* h, int force, int32_t* ncopies) {
  QuantArgs q{};
  q.n = h->n;
  q.nstar = h->cfg.nstar;
  q.logw = h->logw;
  q.seed = h->cfg.seed;
  q.mode = h->cfg.resample_mode;
  q.force = force;
  q.qpart = h->qpart;
  q.cbase = h->cbase;
  q.runstart = h->rs;
  q.runstart_alt = h->rs_alt;
  q.write_rs = force ? 0 : 1;  // the fused step feeds redistribute; smc_resample does not
  q.wbuf = h->wbuf;
  q.ncopies = ncopies;
  q.x[0] = h->x[0];
  q.x[1] = h->x[1];
  q.d = h->d;
  q.dtype = h->dtype;
  q.xpart = h->xpart;
  q.tile_src = h->tile_src;
  q.epart = reinterpret_cast<const double*>(h->ws + h->L.epart);
  q.est_src = 0;
  q.nblocks = h->L.qblocks;
  q.ntiles = h->L.ntiles;
  q.st = h->st;
  q.stats_out = nullptr;
  return q;
}

// A deferred resampling's rows copied (Algorithm 5, the log w reset) and
// their buffer made current; both kernels do nothing unless one is pending.
cudaError_t materialize(smc_sampler* h) {
  if (!h->defer) return cudaSuccess;
  RedistArgs r = redist_args(h, 0);
  r.use_pending = 1;
  cudaError_t e = launch_redistribute(r, h->stream);
  if (e == cudaSuccess) e = launch_settle(h->st, h->stream);
  return e;
}

// The FP32 factor of an FP32 Gaussian sampler as host-side kernel
// parameters (mu and the interleaved row pairs of L^-1), copied from the
// device the first time a direct launch needs it: synchronises h's stream
// that once.  Never called during stream capture.
cudaError_t fetch_gp(smc_sampler* h) {
  if (!h->have_gp || h->gp_ready) return cudaSuccess;
  static thread_local float Pf[kTgtMaxD * kTgtMaxD], muf[kTgtMaxD];
  cudaError_t e = cudaMemcpyAsync(Pf, h->tg->Pf, sizeof Pf, cudaMemcpyDeviceToHost, h->stream);
  if (e == cudaSuccess) e = cudaMemcpyAsync(muf, h->tg->muf, sizeof muf, cudaMemcpyDeviceToHost, h->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
  if (e != cudaSuccess) return e;
  for (int c = 0; c < kTgtMaxD; ++c) h->gp.mu[c] = muf[c];
  for (int p = 0; p < kTgtMaxD / 2; ++p)
    for (int c = 0; c < kTgtMaxD; ++c)
      h->gp.P2[p * kTgtMaxD + c] = make_float2(c <= 2 * p ? Pf[2 * p * kTgtMaxD + c] : 0.0f,
                                               c <= 2 * p + 1 ? Pf[(2 * p + 1) * kTgtMaxD + c] : 0.0f);
  h->gp_ready = true;
  return cudaSuccess;
}

RedistArgs redist_args(const smc_sampler* h, int force) {
  RedistArgs r{};
  r.n = h->n;
  r.row_bytes = int32_t(h->esize * h->d);
  r.lp_bytes = int32_t(h->esize);
  r.runstart = h->rs;
  r.runstart_alt = h->rs_alt;
  r.tile_src = h->tile_src;
  r.ntiles = h->L.ntiles;
  r.force = force;
  r.x_in[0] = h->x[0];
  r.x_in[1] = h->x[1];
  r.x_out[0] = h->x[1];
  r.x_out[1] = h->x[0];
  r.lp_in[0] = h->lp[0];
  r.lp_in[1] = h->lp[1];
  r.lp_out[0] = h->lp[1];
  r.lp_out[1] = h->lp[0];
  r.logw = h->logw;
  r.reset_logw = 0.0;
  r.st = h->st;
  r.stateful = 1;
  return r;
}

}  // namespace smc

namespace {

// Weighted statistics after a reweight: max, quantised sums with the mean of
// eq. (7), decision.  nb: max records written by the reweighting kernel.
cudaError_t launch_stats(smc_sampler* h, int set_lse_prev, int nb) {
  cudaError_t e = launch_max_finalize(h->part, nb, h->st, h->stream);
  if (e != cudaSuccess) return e;
  const QuantArgs q = quant_args(h, 0, nullptr);
  e = launch_quant_reduce(q, h->stream);
  if (e != cudaSuccess) return e;
  return launch_quant_finalize(q, set_lse_prev, h->stream);
}

// FP32 Gaussian samplers with D <= 16: the fused move/reweight kernel also
// forms the eq. (7) sums of its blocks (the particles are in its registers),
// so the quantise pass does not read them again.  (For D > 16 the kernel has
// no registers to spare.)
bool est_in_move(const smc_sampler* h) { return h->have_gp && !h->lg_tc && h->d <= 16; }

// Move and reweight of one iteration (Algorithm 2, line 4; eq. (5)); returns
// the number of max records written.
cudaError_t launch_move_reweight(smc_sampler* h, const ParticleArgs& a, int* nb) {
  if (h->lg_tc) {
    cudaError_t e = launch_particles(OP_MOVE, a, h->grid_p, h->threads_p, h->stream);
    if (e == cudaSuccess) e = launch_logistic_tc(a, h->grid_lg, h->stream);
    *nb = h->grid_lg;
    return e;
  }
  *nb = h->grid_p;
  const int op = h->defer ? OP_MOVE_REWEIGHT_GATHER : (est_in_move(h) ? OP_MOVE_REWEIGHT_EST : OP_MOVE_REWEIGHT);
  return launch_particles(op, a, h->grid_p, h->threads_p, h->stream, gauss_params(h));
}

// One iteration of Algorithm 2 (lines 3-10), all on h->stream.
cudaError_t launch_iteration(smc_sampler* h, bool with_cov) {
  const ParticleArgs a = particle_args(h);
  int nb = 0;
  cudaError_t e = launch_begin(h->st, h->stream);
  if (e == cudaSuccess) e = launch_move_reweight(h, a, &nb);
  if (e == cudaSuccess) e = launch_max_finalize(h->part, nb, h->st, h->stream);
  QuantArgs q = quant_args(h, 0, nullptr);
  q.est_src = est_in_move(h) ? 1 : 0;
  // (a sampler of one quantise block / one copy tile: the same bodies fused
  // into fewer launches; the covariance reads nothing the scan writes)
  const bool one_q = h->L.qblocks == 1, one_r = h->L.ntiles == 1;
  if (one_q) {
    if (e == cudaSuccess) e = launch_quant_small(q, h->stream);
  } else {
    if (e == cudaSuccess) e = launch_quant_reduce(q, h->stream);
    if (e == cudaSuccess) e = launch_quant_finalize(q, 0, h->stream);
  }
  if (e == cudaSuccess && with_cov)
    e = launch_cov(a, nullptr, reinterpret_cast<double*>(h->ws + h->L.covpart), h->L.cov_blocks, h->stream);
  if (!one_q && e == cudaSuccess) e = launch_quant_scan(q, h->stream);
  if (h->defer) {  // the next move gathers the rows (smc_materialize, if none follows)
    if (e == cudaSuccess) e = launch_commit(h->st, h->d, 0, 1, h->stream, 1);
  } else if (one_r) {
    if (e == cudaSuccess) e = launch_redistribute_commit(redist_args(h, 0), h->d, 0, 1, h->stream);
  } else {
    if (e == cudaSuccess) e = launch_redistribute(redist_args(h, 0), h->stream);
    if (e == cudaSuccess) e = launch_commit(h->st, h->d, 0, 1, h->stream);
  }
  return e;
}

// k iterations of a small FP64 sampler in one cooperative launch: the bodies
// of launch_iteration's kernels in its order (bit-identical results); with
// the covariance, the last iteration's copy and commit follow the covariance
// as separate launches, as in launch_iteration.  Returns
// cudaErrorCooperativeLaunchTooLarge (nothing launched but the barrier reset)
// when the grid cannot be resident.
cudaError_t launch_small_iterations(smc_sampler* h, int32_t k, bool with_cov) {
  SmallIterArgs s{};
  s.a = particle_args(h);
  s.q = quant_args(h, 0, nullptr);
  s.r = redist_args(h, 0);
  s.bar = reinterpret_cast<unsigned long long*>(h->ws + h->L.gbar);
  s.k = k;
  s.move_threads = h->threads_p;
  s.d = h->d;
  s.stop_last = with_cov ? 1 : 0;
  s.stall = (h->cfg.flags & SMC_FLAG_TEST_STALL_BARRIER) ? 1 : 0;
  cudaError_t e = cudaMemsetAsync(s.bar, 0, sizeof(unsigned long long), h->stream);
  if (e == cudaSuccess) e = launch_iterate_small(s, h->grid_p, h->stream);
  if (e == cudaSuccess && with_cov)
    e = launch_cov(s.a, nullptr, reinterpret_cast<double*>(h->ws + h->L.covpart), h->L.cov_blocks, h->stream);
  if (e == cudaSuccess && with_cov) e = launch_redistribute_commit(redist_args(h, 0), h->d, 0, 1, h->stream);
  return e;
}

cudaError_t build_graph(smc_sampler* h, bool with_cov, cudaGraphExec_t* out) {
  cudaGraph_t g = nullptr;
  cudaError_t e = cudaStreamBeginCapture(h->stream, cudaStreamCaptureModeThreadLocal);
  if (e != cudaSuccess) return e;
  cudaError_t le = launch_iteration(h, with_cov);
  e = cudaStreamEndCapture(h->stream, &g);
  if (le != cudaSuccess) {
    if (g) cudaGraphDestroy(g);
    return le;
  }
  if (e != cudaSuccess) return e;
  e = cudaGraphInstantiate(out, g, 0);
  cudaGraphDestroy(g);
  return e;
}

int check_config(const smc_config* c) {
  if (!c) return fail(nullptr, SMC_EINVAL, "null config");
  if (c->n < 1 || c->n > 2147483647LL) return fail(nullptr, SMC_EINVAL, "n must be in [1, 2^31)");
  if (c->d < 1 || c->d > kMaxD) return fail(nullptr, SMC_EINVAL, "d must be in [1, 32]");
  if (c->dtype != SMC_F32 && c->dtype != SMC_F64) return fail(nullptr, SMC_EINVAL, "dtype must be SMC_F32 or SMC_F64");
  if (c->target != SMC_GAUSS && c->target != SMC_STUDENT_T && c->target != SMC_LOGISTIC)
    return fail(nullptr, SMC_EINVAL, "unknown target kind");
  if (c->target == SMC_LOGISTIC && (!c->X_dev || !c->y_dev || c->m < 1 || !(c->prior_var > 0.0)))
    return fail(nullptr, SMC_EINVAL, "logistic target needs X_dev, y_dev, m >= 1 and prior_var > 0");
  if (c->target == SMC_STUDENT_T && (c->d != 1 || !(c->nu > 0.0)))
    return fail(nullptr, SMC_EINVAL, "Student-t target needs d == 1 and nu > 0");
  if (c->target == SMC_GAUSS && (!c->mu_dev || !c->sigma_dev))
    return fail(nullptr, SMC_EINVAL, "Gaussian target needs mu_dev and sigma_dev");
  if (c->target == SMC_STUDENT_T && !c->mu_dev) return fail(nullptr, SMC_EINVAL, "Student-t target needs mu_dev");
  if (c->resample_mode < 0 || c->resample_mode > 2) return fail(nullptr, SMC_EINVAL, "bad resample_mode");
  if (c->nstar < 0 || c->nstar > c->n) return fail(nullptr, SMC_EINVAL, "nstar must be in [0, n]");
  if (!(c->step >= 0.0) || !(c->init_scale > 0.0)) return fail(nullptr, SMC_EINVAL, "bad step / init_scale");
  return SMC_OK;
}

}  // namespace

extern "C" {

int smc_workspace_bytes(const smc_config* cfg, size_t* bytes) {
  int rc = check_config(cfg);
  if (rc) return rc;
  if (!bytes) return fail(nullptr, SMC_EINVAL, "null bytes");
  *bytes = layout_for(cfg->n, cfg->d, logistic_rows(cfg), wants_two_rs(cfg)).total;
  return SMC_OK;
}

int smc_init(smc_sampler** out, const smc_config* cfg, void* x_dev, void* x_alt_dev, double* logw_dev,
             void* logpi_dev, void* logpi_alt_dev, void* workspace_dev, size_t workspace_bytes,
             smc_stream_t stream) {
  SMC_RANGE("smc_init");
  if (!out) return fail(nullptr, SMC_EINVAL, "null out");
  *out = nullptr;
  int rc = check_config(cfg);
  if (rc) return rc;
  if (!x_dev || !x_alt_dev || !logw_dev || !logpi_dev || !logpi_alt_dev || !workspace_dev)
    return fail(nullptr, SMC_EINVAL, "null buffer");
  if (!aligned(workspace_dev, kAlign)) return fail(nullptr, SMC_EINVAL, "workspace must be 256-byte aligned");
  const size_t es = cfg->dtype == SMC_F64 ? 8 : 4;
  if (!aligned(x_dev, 16) || !aligned(x_alt_dev, 16) || !aligned(logw_dev, 8) || !aligned(logpi_dev, es) ||
      !aligned(logpi_alt_dev, es))
    return fail(nullptr, SMC_EINVAL, "particle buffers must be 16-byte aligned");
  const Layout L = layout_for(cfg->n, cfg->d, logistic_rows(cfg), wants_two_rs(cfg));
  if (workspace_bytes < L.total) return fail(nullptr, SMC_ENOMEM, "workspace too small");
  cudaError_t e = upload_expfx_table();
  if (e != cudaSuccess) return cuda_fail(nullptr, e, "upload_expfx_table");

  smc_sampler* h = new (std::nothrow) smc_sampler();
  if (!h) return fail(nullptr, SMC_ENOMEM, "host allocation failed");
  h->cfg = *cfg;
  h->n = cfg->n;
  h->d = cfg->d;
  h->dtype = cfg->dtype;
  h->esize = es;
  h->x[0] = x_dev;
  h->x[1] = x_alt_dev;
  h->lp[0] = logpi_dev;
  h->lp[1] = logpi_alt_dev;
  h->logw = logw_dev;
  h->ws = static_cast<char*>(workspace_dev);
  h->L = L;
  h->stream = reinterpret_cast<cudaStream_t>(stream);
  h->st = reinterpret_cast<DevState*>(h->ws + L.st);
  h->tg = reinterpret_cast<TargetDev*>(h->ws + L.tg);
  h->part = reinterpret_cast<double*>(h->ws + L.part);
  h->qpart = reinterpret_cast<uint64_t*>(h->ws + L.qpart);
  h->cbase = reinterpret_cast<uint64_t*>(h->ws + L.cbase);
  h->xpart = h->ws + L.xpart;
  h->rs = reinterpret_cast<int32_t*>(h->ws + L.rs);
  h->rs_alt = L.rs_alt ? reinterpret_cast<int32_t*>(h->ws + L.rs_alt) : nullptr;
  h->wbuf = reinterpret_cast<uint64_t*>(h->ws + L.wbuf);
  h->tile_src = reinterpret_cast<int32_t*>(h->ws + L.tile_src);
  // particle kernels: 256-thread blocks, at most 8 per SM (grid-stride);
  // samplers of fewer than 256 particles per SM use one-warp blocks so that
  // their work (FP64 in particular) spreads over the SMs
  {
    const int64_t units = h->n * lanes_per_particle(h->dtype, h->d);
    const int64_t sms = sm_count();
    h->threads_p = units < int64_t(kPThreads) * sms ? 32 : kPThreads;
    h->grid_p = int(std::min<int64_t>(div_up(units, h->threads_p), sms * 8));
    if (h->grid_p > kMaxPartBlocks) h->grid_p = kMaxPartBlocks;
  }
  h->lg_tc = cfg->target == SMC_LOGISTIC && cfg->dtype == SMC_F32 && !(cfg->flags & SMC_FLAG_LOGISTIC_CUDA_CORES);
  h->grid_lg = logistic_tc_grid(h->n, sm_count());
  h->g_iter[0] = h->g_iter[1] = nullptr;
  h->have_gp = false;
  h->gp_ready = false;
  h->err = "ok";

  // Algorithm 2, line 1, then the statistics of w_0 (LSE_0 becomes LSE_{t-1})
  e = cudaMemsetAsync(h->tg, 0, sizeof(TargetDev), h->stream);
  if (e == cudaSuccess) e = cudaMemsetAsync(h->rs, 0xFF, size_t(h->n) * sizeof(int32_t), h->stream);
  if (e == cudaSuccess && h->rs_alt)
    e = cudaMemsetAsync(h->rs_alt, 0xFF, size_t(h->n) * sizeof(int32_t), h->stream);
  if (e == cudaSuccess) e = launch_state_init(h->st, h->n, 0, quant_shift(h->n), h->stream);
  if (e == cudaSuccess) {
    if (cfg->target == SMC_LOGISTIC)
      e = launch_logistic_setup(h->tg, cfg->X_dev, cfg->y_dev, cfg->m, h->d, cfg->prior_var,
                                reinterpret_cast<float*>(h->ws + L.lg_x), reinterpret_cast<float*>(h->ws + L.lg_y),
                                reinterpret_cast<uint16_t*>(h->ws + L.lg_img), h->stream);
    else
      e = launch_target_setup(h->tg, cfg->target, cfg->nu, cfg->mu_dev, cfg->sigma_dev, h->d, h->st, h->stream);
  }
  // with the tensor-core likelihood, init leaves log pi(x_0) = 0 and the
  // likelihood pass adds it (log w_0 = log pi - log q0 either way), so every
  // later difference of eq. (5) compares values of one method
  ParticleArgs ia = particle_args(h);
  if (h->lg_tc) ia.flags |= PA_INIT_SKIP_LOGPI;
  if (e == cudaSuccess) e = launch_particles(OP_INIT, ia, h->grid_p, h->threads_p, h->stream);
  if (e == cudaSuccess && h->lg_tc) e = launch_logistic_tc(particle_args(h), h->grid_lg, h->stream);
  if (e == cudaSuccess) e = launch_stats(h, 1, h->lg_tc ? h->grid_lg : h->grid_p);
  // FP32 Gaussian samplers: the FP32 factor the set-up kernel wrote becomes
  // a kernel parameter of the move / reweight kernel; it is fetched by the
  // first direct launch that needs it (fetch_gp), so smc_init returns
  // without waiting for its own work
  h->have_gp = cfg->target == SMC_GAUSS && h->dtype == SMC_F32;
  h->gp_ready = false;
  // deferred redistribution: the gathering move is the records kernel's, and
  // the quantise and copy passes span several blocks
  h->defer = (cfg->flags & SMC_FLAG_DEFER_REDISTRIBUTE) && est_in_move(h) && h->L.qblocks > 1 && h->L.ntiles > 1;
  // small FP64 samplers (generic move kernel, one quantise block, one copy
  // tile): smc_step fuses their iterations into one cooperative launch
  h->small_iter = small_iter_fits(h->n, h->dtype) && cfg->target != SMC_LOGISTIC && !h->defer &&
                  h->L.qblocks == 1 && h->L.ntiles == 1;
  if (e != cudaSuccess) {
    int r = cuda_fail(nullptr, e, "smc_init launch");
    delete h;
    return r;
  }
  *out = h;
  return SMC_OK;
}

int smc_move(smc_sampler* h) {
  SMC_RANGE("smc_move");
  if (!h) return fail(nullptr, SMC_EINVAL, "null handle");
  SMC_TRY(h, fetch_gp(h));
  SMC_TRY(h, materialize(h));
  SMC_TRY(h, launch_begin(h->st, h->stream));
  SMC_TRY(h, launch_particles(OP_MOVE, particle_args(h), h->grid_p, h->threads_p, h->stream, gauss_params(h)));
  return SMC_OK;
}

int smc_reweight(smc_sampler* h) {
  SMC_RANGE("smc_reweight");
  if (!h) return fail(nullptr, SMC_EINVAL, "null handle");
  SMC_TRY(h, fetch_gp(h));
  SMC_TRY(h, materialize(h));
  if (h->lg_tc) {
    SMC_TRY(h, launch_logistic_tc(particle_args(h), h->grid_lg, h->stream));
    SMC_TRY(h, launch_stats(h, 0, h->grid_lg));
  } else {
    SMC_TRY(h, launch_particles(OP_REWEIGHT, particle_args(h), h->grid_p, h->threads_p, h->stream, gauss_params(h)));
    SMC_TRY(h, launch_stats(h, 0, h->grid_p));
  }
  return SMC_OK;
}

int smc_estimate(smc_sampler* h, double* mean_dev, double* cov_dev) {
  SMC_RANGE("smc_estimate");
  if (!h) return fail(nullptr, SMC_EINVAL, "null handle");
  SMC_TRY(h, materialize(h));
  if (mean_dev) SMC_TRY(h, launch_copy_mean(h->st, mean_dev, h->d, h->stream));
  if (cov_dev)
    SMC_TRY(h, launch_cov(particle_args(h), cov_dev, reinterpret_cast<double*>(h->ws + h->L.covpart),
                          h->L.cov_blocks, h->stream));
  return SMC_OK;
}

int smc_resample(smc_sampler* h, int32_t* ncopies_dev, int32_t* did_resample_dev) {
  SMC_RANGE("smc_resample");
  if (!h) return fail(nullptr, SMC_EINVAL, "null handle");
  SMC_TRY(h, materialize(h));
  if (ncopies_dev) SMC_TRY(h, launch_quant_scan(quant_args(h, 1, ncopies_dev), h->stream));
  if (did_resample_dev)
    SMC_TRY(h, cudaMemcpyAsync(did_resample_dev, &h->st->flag, sizeof(int32_t), cudaMemcpyDeviceToDevice,
                               h->stream));
  return SMC_OK;
}

int smc_redistribute(smc_sampler* h, const int32_t* ncopies_dev) {
  SMC_RANGE("smc_redistribute");
  if (!h) return fail(nullptr, SMC_EINVAL, "null handle");
  if (!ncopies_dev) return fail(h, SMC_EINVAL, "null ncopies");
  SMC_TRY(h, materialize(h));
  NcScanArgs s{};
  s.n = h->n;
  s.ncopies = ncopies_dev;
  s.part = h->qpart;
  s.cbase = h->cbase;
  s.runstart = h->rs;
  s.runstart_alt = h->rs_alt;
  s.tile_src = h->tile_src;
  s.nblocks = h->L.qblocks;
  s.ntiles = h->L.ntiles;
  s.st = h->st;
  SMC_TRY(h, launch_nc_reduce(s, h->stream));
  SMC_TRY(h, launch_nc_finalize(s, h->stream));
  SMC_TRY(h, launch_nc_scan(s, h->stream));
  SMC_TRY(h, launch_redistribute(redist_args(h, 1), h->stream));
  SMC_TRY(h, launch_commit(h->st, h->d, 1, 0, h->stream));
  return SMC_OK;
}

int smc_step(smc_sampler* h, int32_t k, double* mean_dev, double* cov_dev, smc_iter_stats* trace_dev,
             double* fhat_dev) {
  SMC_RANGE("smc_step");
  if (!h) return fail(nullptr, SMC_EINVAL, "null handle");
  if (k < 0) return fail(h, SMC_EINVAL, "k must be >= 0");
  if (k == 0) return SMC_OK;
  SMC_TRY(h, fetch_gp(h));  // (before any stream capture)
  SMC_TRY(h, launch_step_setup(h->st, trace_dev, mean_dev, fhat_dev, cov_dev, h->stream));
  if (h->small_iter) {
    const cudaError_t e = launch_small_iterations(h, k, cov_dev != nullptr);
    if (e != cudaErrorCooperativeLaunchTooLarge) {
      SMC_TRY(h, e);
      return SMC_OK;
    }
    (void)cudaGetLastError();  // the grid cannot be resident here: separate launches below
  }
  const bool use_graph = h->stream != nullptr;
  for (int32_t it = 0; it < k; ++it) {
    const bool with_cov = cov_dev && it == k - 1;
    if (use_graph) {
      cudaGraphExec_t& g = h->g_iter[with_cov ? 1 : 0];
      if (!g) SMC_TRY(h, build_graph(h, with_cov, &g));
      SMC_TRY(h, cudaGraphLaunch(g, h->stream));
    } else {
      SMC_TRY(h, launch_iteration(h, with_cov));
    }
  }
  return SMC_OK;
}

int smc_step_profile(smc_sampler* h, double* mean_dev, void* const* events_host, int32_t n_events) {
  SMC_RANGE("smc_step_profile");
  if (!h) return fail(nullptr, SMC_EINVAL, "null handle");
  if (n_events != 0 && n_events != 8) return fail(h, SMC_EINVAL, "n_events must be 0 or 8");
  if (n_events && !events_host) return fail(h, SMC_EINVAL, "null events");
  cudaStream_t s = h->stream;
  auto rec = [&](int j) -> cudaError_t {
    return n_events ? cudaEventRecord(static_cast<cudaEvent_t>(events_host[j]), s) : cudaSuccess;
  };
  SMC_TRY(h, fetch_gp(h));
  SMC_TRY(h, launch_step_setup(h->st, nullptr, mean_dev, nullptr, nullptr, s));
  const ParticleArgs a = particle_args(h);
  QuantArgs q = quant_args(h, 0, nullptr);
  q.est_src = est_in_move(h) ? 1 : 0;
  int nb = 0;
  SMC_TRY(h, rec(0));
  {
    SMC_RANGE("move+reweight");
    SMC_TRY(h, launch_begin(h->st, s));
    SMC_TRY(h, launch_move_reweight(h, a, &nb));
  }
  SMC_TRY(h, rec(1));
  {
    SMC_RANGE("max finalise");
    SMC_TRY(h, launch_max_finalize(h->part, nb, h->st, s));
  }
  SMC_TRY(h, rec(2));
  {
    SMC_RANGE("quantise reduce");
    SMC_TRY(h, launch_quant_reduce(q, s));
  }
  SMC_TRY(h, rec(3));
  {
    SMC_RANGE("quantise finalise");
    SMC_TRY(h, launch_quant_finalize(q, 0, s));
  }
  SMC_TRY(h, rec(4));
  {
    SMC_RANGE("systematic scan");
    SMC_TRY(h, launch_quant_scan(q, s));
  }
  SMC_TRY(h, rec(5));
  if (!h->defer) {  // (deferred: the next iteration's move gathers the rows)
    SMC_RANGE("redistribute");
    SMC_TRY(h, launch_redistribute(redist_args(h, 0), s));
  }
  SMC_TRY(h, rec(6));
  {
    SMC_RANGE("commit");
    SMC_TRY(h, launch_commit(h->st, h->d, 0, 1, s, h->defer ? 1 : 0));
  }
  SMC_TRY(h, rec(7));
  return SMC_OK;
}

int smc_sync(smc_sampler* h) {
  SMC_RANGE("smc_sync");
  if (!h) return fail(nullptr, SMC_EINVAL, "null handle");
  SMC_TRY(h, cudaStreamSynchronize(h->stream));
  int32_t err = 0;
  SMC_TRY(h, cudaMemcpy(&err, &h->st->err, sizeof err, cudaMemcpyDeviceToHost));
  if (err) {
    SMC_TRY(h, cudaMemset(&h->st->err, 0, sizeof err));
    static const char* names[] = {"ok", "invalid argument on the device", "out of memory", "cuda",
                                  "a bounded device wait timed out", "non-finite log-weights"};
    return fail(h, err, err >= 0 && err <= 5 ? names[err] : "device error");
  }
  return SMC_OK;
}

int smc_read_stats(smc_sampler* h, smc_iter_stats* out_host) {
  if (!h || !out_host) return fail(h, SMC_EINVAL, "null argument");
  SMC_TRY(h, cudaStreamSynchronize(h->stream));
  SMC_TRY(h, cudaMemcpy(out_host, &h->st->last, sizeof(smc_iter_stats), cudaMemcpyDeviceToHost));
  return SMC_OK;
}

int smc_current(smc_sampler* h, int32_t* which_host) {
  if (!h || !which_host) return fail(h, SMC_EINVAL, "null argument");
  SMC_TRY(h, materialize(h));
  SMC_TRY(h, cudaStreamSynchronize(h->stream));
  SMC_TRY(h, cudaMemcpy(which_host, &h->st->cur, sizeof(int32_t), cudaMemcpyDeviceToHost));
  return SMC_OK;
}

int smc_materialize(smc_sampler* h) {
  SMC_RANGE("smc_materialize");
  if (!h) return fail(nullptr, SMC_EINVAL, "null handle");
  SMC_TRY(h, materialize(h));
  return SMC_OK;
}

int smc_destroy(smc_sampler* h) {
  if (!h) return SMC_OK;
  for (auto& g : h->g_iter)
    if (g) cudaGraphExecDestroy(g);
  delete h;
  return SMC_OK;
}

const char* smc_last_error(const smc_sampler* h) { return h ? h->err.c_str() : g_err.c_str(); }

// ------------------------------------------------------------------ stateless
namespace {
struct RawLayout {
  size_t st, part, qpart, cbase, rs, wbuf, tile_src, stamps, total;
  int qblocks, ntiles;
};
RawLayout raw_layout(int64_t n) {
  RawLayout L{};
  L.qblocks = int(div_up(n, kQTile));
  L.ntiles = int(div_up(n, kRTile));
  size_t p = 0;
  L.st = p;
  p = align_up(p + sizeof(DevState));
  L.part = p;
  p = align_up(p + size_t(L.qblocks) * 2 * sizeof(double));
  L.qpart = p;
  p = align_up(p + size_t(L.qblocks) * 5 * sizeof(uint64_t));
  L.cbase = p;
  p = align_up(p + size_t(L.qblocks) * sizeof(uint64_t));
  L.rs = p;
  p = align_up(p + size_t(n) * sizeof(int32_t));
  L.wbuf = p;
  p = align_up(p + size_t(n) * sizeof(uint64_t));
  L.tile_src = p;
  p = align_up(p + size_t(L.ntiles + 1) * sizeof(int32_t));
  // per copy tile: run starts were written there (zeroed by each
  // redistribute call)
  L.stamps = p;
  p = align_up(p + size_t(L.ntiles) * sizeof(int32_t));
  L.total = p;
  return L;
}
}  // namespace

int smc_redistribute_ws_bytes(int64_t n, size_t* bytes) {
  if (n < 1 || n > 2147483647LL || !bytes) return fail(nullptr, SMC_EINVAL, "n must be in [1, 2^31)");
  *bytes = raw_layout(n).total;
  return SMC_OK;
}

namespace {

// Algorithm 5 on raw rows; with n_events = 3, caller events are recorded
// before the call, after the ncopies scan, and after the copy.
int redistribute_raw_impl(int64_t n, int32_t row_bytes, const int32_t* ncopies_dev, const void* in_dev,
                          void* out_dev, void* ws_dev, smc_stream_t stream, void* const* events_host,
                          int32_t n_events) {
  if (n < 1 || n > 2147483647LL) return fail(nullptr, SMC_EINVAL, "n must be in [1, 2^31)");
  if (row_bytes < 4 || row_bytes % 4) return fail(nullptr, SMC_EINVAL, "row_bytes must be a positive multiple of 4");
  if (!ncopies_dev || !in_dev || !out_dev || !ws_dev) return fail(nullptr, SMC_EINVAL, "null pointer");
  if (!aligned(ws_dev, kAlign)) return fail(nullptr, SMC_EINVAL, "workspace must be 256-byte aligned");
  if (n_events != 0 && (n_events != 3 || !events_host)) return fail(nullptr, SMC_EINVAL, "n_events must be 0 or 3");
  const size_t va = row_bytes % 16 == 0 ? 16 : (row_bytes % 8 == 0 ? 8 : 4);
  if (!aligned(in_dev, va) || !aligned(out_dev, va)) return fail(nullptr, SMC_EINVAL, "rows misaligned");
  const RawLayout L = raw_layout(n);
  char* ws = static_cast<char*>(ws_dev);
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  auto rec = [&](int j) -> cudaError_t {
    return n_events ? cudaEventRecord(static_cast<cudaEvent_t>(events_host[j]), s) : cudaSuccess;
  };
  DevState* st = reinterpret_cast<DevState*>(ws + L.st);
  NcScanArgs a{};
  a.n = n;
  a.ncopies = ncopies_dev;
  a.part = reinterpret_cast<uint64_t*>(ws + L.qpart);
  a.cbase = reinterpret_cast<uint64_t*>(ws + L.cbase);
  a.runstart = reinterpret_cast<int32_t*>(ws + L.rs);
  a.tile_src = reinterpret_cast<int32_t*>(ws + L.tile_src);
  a.nblocks = L.qblocks;
  a.ntiles = L.ntiles;
  a.st = st;
  // stamped: the run-start array is not cleared; the copy reads the slices
  // of the stamped tiles only, which the scan writes whole
  a.stamps = reinterpret_cast<int32_t*>(ws + L.stamps);
  RedistArgs r{};
  r.n = n;
  r.row_bytes = row_bytes;
  r.lp_bytes = 0;
  r.runstart = a.runstart;
  r.tile_src = a.tile_src;
  r.ntiles = L.ntiles;
  r.force = 1;
  r.x_in[0] = r.x_in[1] = in_dev;
  r.x_out[0] = r.x_out[1] = out_dev;
  r.logw = nullptr;
  r.st = st;
  r.stateful = 0;
  r.stamps = a.stamps;
  cudaError_t e = rec(0);
  if (e == cudaSuccess) e = cudaMemsetAsync(&st->err, 0, sizeof(int32_t), s);
  if (e == cudaSuccess) e = cudaMemsetAsync(a.stamps, 0, size_t(L.ntiles) * sizeof(int32_t), s);
  if (e == cudaSuccess) e = launch_nc_reduce(a, s);
  if (e == cudaSuccess) e = launch_nc_finalize(a, s);
  if (e == cudaSuccess) e = launch_nc_scan(a, s);
  if (e == cudaSuccess) e = rec(1);
  if (e == cudaSuccess) e = launch_redistribute(r, s);
  if (e == cudaSuccess) e = rec(2);
  if (e != cudaSuccess) return cuda_fail(nullptr, e, "smc_redistribute_raw");
  return SMC_OK;
}

}  // namespace

int smc_redistribute_raw(int64_t n, int32_t row_bytes, const int32_t* ncopies_dev, const void* in_dev,
                         void* out_dev, void* ws_dev, smc_stream_t stream) {
  SMC_RANGE("smc_redistribute_raw");
  return redistribute_raw_impl(n, row_bytes, ncopies_dev, in_dev, out_dev, ws_dev, stream, nullptr, 0);
}

int smc_redistribute_raw_profile(int64_t n, int32_t row_bytes, const int32_t* ncopies_dev, const void* in_dev,
                                 void* out_dev, void* ws_dev, smc_stream_t stream, void* const* events_host,
                                 int32_t n_events) {
  SMC_RANGE("smc_redistribute_raw_profile");
  return redistribute_raw_impl(n, row_bytes, ncopies_dev, in_dev, out_dev, ws_dev, stream, events_host, n_events);
}

int smc_resample_raw(int64_t n, const double* logw_dev, uint64_t seed, uint64_t t, int32_t mode,
                     int32_t* ncopies_dev, smc_iter_stats* stats_dev, void* ws_dev, smc_stream_t stream) {
  SMC_RANGE("smc_resample_raw");
  if (n < 1 || n > 2147483647LL) return fail(nullptr, SMC_EINVAL, "n must be in [1, 2^31)");
  if (!logw_dev || !ncopies_dev || !ws_dev) return fail(nullptr, SMC_EINVAL, "null pointer");
  if (mode < 0 || mode > 2) return fail(nullptr, SMC_EINVAL, "bad mode");
  if (!aligned(ws_dev, kAlign)) return fail(nullptr, SMC_EINVAL, "workspace must be 256-byte aligned");
  cudaError_t e = upload_expfx_table();
  if (e != cudaSuccess) return cuda_fail(nullptr, e, "upload_expfx_table");
  const RawLayout L = raw_layout(n);
  char* ws = static_cast<char*>(ws_dev);
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  DevState* st = reinterpret_cast<DevState*>(ws + L.st);
  double* part = reinterpret_cast<double*>(ws + L.part);
  QuantArgs q{};
  q.n = n;
  q.logw = logw_dev;
  q.seed = seed;
  q.mode = mode;
  q.force = 1;
  q.qpart = reinterpret_cast<uint64_t*>(ws + L.qpart);
  q.cbase = reinterpret_cast<uint64_t*>(ws + L.cbase);
  q.runstart = reinterpret_cast<int32_t*>(ws + L.rs);
  q.write_rs = 0;
  q.wbuf = reinterpret_cast<uint64_t*>(ws + L.wbuf);
  q.ncopies = ncopies_dev;
  q.tile_src = reinterpret_cast<int32_t*>(ws + L.tile_src);
  q.nblocks = L.qblocks;
  q.ntiles = L.ntiles;
  q.st = st;
  q.stats_out = stats_dev;
  e = launch_state_init(st, n, int64_t(t), quant_shift(n), s);
  if (e == cudaSuccess) e = launch_max_logw(logw_dev, n, part, L.qblocks, st, s);
  if (e == cudaSuccess) e = launch_max_finalize(part, L.qblocks, st, s);
  if (e == cudaSuccess) e = launch_quant_reduce(q, s);
  if (e == cudaSuccess) e = launch_quant_finalize(q, 0, s);
  if (e == cudaSuccess) e = launch_quant_scan(q, s);
  if (e != cudaSuccess) return cuda_fail(nullptr, e, "smc_resample_raw");
  return SMC_OK;
}

int smc_nearly_sort_ws_bytes(int64_t n, size_t* bytes) {
  if (n < 1 || n > 2147483647LL || !bytes) return fail(nullptr, SMC_EINVAL, "n must be in [1, 2^31)");
  *bytes = 2 * align_up(size_t(nearly_sort_tiles(n)) * sizeof(int32_t));
  return SMC_OK;
}

int smc_nearly_sort_raw(int64_t n, int32_t row_bytes, const int32_t* ncopies_dev, const void* in_dev,
                        int32_t* ncopies_out_dev, void* out_dev, void* ws_dev, smc_stream_t stream) {
  SMC_RANGE("smc_nearly_sort_raw");
  if (n < 1 || n > 2147483647LL) return fail(nullptr, SMC_EINVAL, "n must be in [1, 2^31)");
  if (row_bytes < 4 || row_bytes % 4) return fail(nullptr, SMC_EINVAL, "row_bytes must be a positive multiple of 4");
  if (!ncopies_dev || !in_dev || !ncopies_out_dev || !out_dev || !ws_dev) return fail(nullptr, SMC_EINVAL, "null pointer");
  if (!aligned(ws_dev, kAlign)) return fail(nullptr, SMC_EINVAL, "workspace must be 256-byte aligned");
  if (!aligned(ncopies_dev, 16)) return fail(nullptr, SMC_EINVAL, "ncopies must be 16-byte aligned");
  const size_t va = row_bytes % 16 == 0 ? 16 : (row_bytes % 8 == 0 ? 8 : 4);
  if (!aligned(in_dev, va) || !aligned(out_dev, va)) return fail(nullptr, SMC_EINVAL, "rows misaligned");
  NearlySortArgs a{};
  a.n = n;
  a.row_bytes = row_bytes;
  a.ntiles = nearly_sort_tiles(n);
  a.ncopies = ncopies_dev;
  a.ncopies_out = ncopies_out_dev;
  a.in = in_dev;
  a.out = out_dev;
  a.tile_count = static_cast<int32_t*>(ws_dev);
  a.tile_base = reinterpret_cast<int32_t*>(static_cast<char*>(ws_dev) + align_up(size_t(a.ntiles) * sizeof(int32_t)));
  cudaError_t e = launch_nearly_sort(a, reinterpret_cast<cudaStream_t>(stream));
  if (e != cudaSuccess) return cuda_fail(nullptr, e, "smc_nearly_sort_raw");
  return SMC_OK;
}

int smc_ws_status(void* ws_dev, smc_stream_t stream) {
  if (!ws_dev) return fail(nullptr, SMC_EINVAL, "null workspace");
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  cudaError_t e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return cuda_fail(nullptr, e, "smc_ws_status");
  DevState* st = reinterpret_cast<DevState*>(ws_dev);
  int32_t err = 0;
  e = cudaMemcpy(&err, &st->err, sizeof err, cudaMemcpyDeviceToHost);
  if (e != cudaSuccess) return cuda_fail(nullptr, e, "smc_ws_status");
  if (err) {
    cudaMemset(&st->err, 0, sizeof err);
    return fail(nullptr, err, "device-side error in stateless call");
  }
  return SMC_OK;
}

}  // extern "C"
