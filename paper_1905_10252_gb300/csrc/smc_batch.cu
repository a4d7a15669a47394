// smc_batch.cu -- the batch part of the C-ABI (include/smc.h): many samplers
// stepped with one launch per stage.  Each launch walks a block map whose
// entry b names (member, block of that member, blocks of that member); every
// member keeps the blocks, tiles and reduction order it has when stepped
// alone, so its results are bit-identical to smc_step.  The map order, the
// move launch's block budget and the copy's loads in flight are launch
// shapes only; the autotuner picks them by timing work that leaves every
// member's state untouched.
#include <algorithm>
#include <cmath>
#include <new>
#include <string>
#include <vector>

#include "smc_host.h"
#include "smc_trace.h"

using namespace smc;

namespace {

constexpr size_t kAl = 256;
constexpr int kMoveBudget[SMC_BATCH_MOVE_VARIANTS] = {2, 4, 8, 16, 0};  // blocks per SM; 0: one per particle
constexpr int kMaxMoveBlocks = 4096;  // per member: the size of its partials buffer
constexpr int kDefaultMove = 2, kDefaultCopy = 1;

size_t up(size_t v) { return (v + kAl - 1) / kAl * kAl; }
int64_t div_up(int64_t a, int64_t b) { return (a + b - 1) / b; }

thread_local std::string g_batch_err = "ok";

// Host-side block maps of a member list (independent of device addresses).
struct Plan {
  int count = 0;
  std::vector<int4> qmap;                               // quantise / scan blocks
  std::vector<int4> rmap;                               // copy tiles
  std::vector<int4> mmap[SMC_BATCH_MOVE_VARIANTS];      // move / reweight blocks
  std::vector<int32_t> nb[SMC_BATCH_MOVE_VARIANTS];     // move blocks per member
};

int move_blocks_full(const smc_sampler* h) {
  const int64_t b = div_up(h->n * lanes_per_particle(h->dtype, h->d), kPThreads);
  return int(std::min<int64_t>(b, kMaxMoveBlocks));
}

Plan make_plan(smc_sampler* const* m, int count, int sms) {
  Plan p;
  p.count = count;
  // members with the most work first, so the last blocks of a launch are short
  std::vector<int> order(count);
  std::vector<double> w(count);
  double wsum = 0.0;
  for (int s = 0; s < count; ++s) {
    order[s] = s;
    w[s] = double(m[s]->n) * double(m[s]->d + 8);  // ~ bytes and flops of the move per member
    wsum += w[s];
  }
  std::stable_sort(order.begin(), order.end(), [&](int a, int b) { return w[a] > w[b]; });
  for (int s : order) {
    const int nq = int(div_up(m[s]->n, kQTile));
    for (int j = 0; j < nq; ++j) p.qmap.push_back(make_int4(s, j, nq, 0));
    const int nr = int(div_up(m[s]->n, kRTile));
    for (int j = 0; j < nr; ++j) p.rmap.push_back(make_int4(s, j, nr, 0));
  }
  for (int v = 0; v < SMC_BATCH_MOVE_VARIANTS; ++v) {
    p.nb[v].assign(count, 1);
    const double total = double(kMoveBudget[v]) * sms;
    for (int s = 0; s < count; ++s) {
      const int full = move_blocks_full(m[s]);
      int b = full;
      if (kMoveBudget[v] > 0) b = int(std::llround(total * w[s] / wsum));
      p.nb[v][s] = std::max(1, std::min(b, full));
    }
    for (int s : order)
      for (int j = 0; j < p.nb[v][s]; ++j) p.mmap[v].push_back(make_int4(s, j, p.nb[v][s], 0));
  }
  return p;
}

// Byte offsets in the batch workspace.
struct BatchLayout {
  size_t pa, pa_dry, qa, ra, ra_dry, gp, outs, errs, nb, qmap, rmap, mmap[SMC_BATCH_MOVE_VARIANTS], dry_st, total;
};

BatchLayout batch_layout(const Plan& p) {
  BatchLayout L{};
  const size_t c = size_t(p.count);
  size_t o = 0;
  auto take = [&](size_t bytes) {
    const size_t at = o;
    o = up(o + bytes);
    return at;
  };
  L.pa = take(c * sizeof(ParticleArgs));
  L.pa_dry = take(c * sizeof(ParticleArgs));
  L.qa = take(c * sizeof(QuantArgs));
  L.ra = take(c * sizeof(RedistArgs));
  L.ra_dry = take(c * sizeof(RedistArgs));
  L.gp = take(c * sizeof(GaussParamsF32));
  L.outs = take(3 * c * sizeof(void*));
  L.errs = take(c * sizeof(int32_t));
  L.nb = take(SMC_BATCH_MOVE_VARIANTS * c * sizeof(int32_t));
  L.qmap = take(p.qmap.size() * sizeof(int4));
  L.rmap = take(p.rmap.size() * sizeof(int4));
  for (int v = 0; v < SMC_BATCH_MOVE_VARIANTS; ++v) L.mmap[v] = take(p.mmap[v].size() * sizeof(int4));
  L.dry_st = take(devstate_bytes());
  L.total = o;
  return L;
}

int check_members(smc_sampler* const* m, int32_t count) {
  if (!m || count < 1) {
    g_batch_err = "members must be a non-empty array";
    return SMC_EINVAL;
  }
  for (int s = 0; s < count; ++s) {
    if (!m[s]) {
      g_batch_err = "null member " + std::to_string(s);
      return SMC_EINVAL;
    }
    if (m[s]->dtype != SMC_F32 || m[s]->cfg.target != SMC_GAUSS || !m[s]->have_gp) {
      g_batch_err = "member " + std::to_string(s) + " is not an FP32 Gaussian sampler";
      return SMC_EINVAL;
    }
    for (int r = 0; r < s; ++r)
      if (m[r] == m[s]) {
        g_batch_err = "member " + std::to_string(s) + " is listed twice";
        return SMC_EINVAL;
      }
  }
  return SMC_OK;
}

}  // namespace

struct smc_batch {
  std::vector<smc_sampler*> m;
  int count;
  Plan plan;
  BatchLayout L;
  char* ws;
  cudaStream_t stream;
  int move_v, copy_v;
  cudaGraphExec_t graph;
  int graph_move_v, graph_copy_v;
  std::vector<void*> outs_host;
  std::vector<int32_t> errs_host;
  std::string err;

  template <typename T>
  T* at(size_t off) const {
    return reinterpret_cast<T*>(ws + off);
  }
};

namespace {

int bfail(smc_batch* b, int code, const std::string& msg) {
  if (b)
    b->err = msg;
  else
    g_batch_err = msg;
  return code;
}

#define BATCH_TRY(b, expr)                                                              \
  do {                                                                                  \
    cudaError_t _e = (expr);                                                            \
    if (_e != cudaSuccess) return bfail((b), SMC_ECUDA, std::string(#expr) + ": " + cudaGetErrorString(_e)); \
  } while (0)

// One iteration of Algorithm 2 (lines 3-10) for every member: 8 launches.
cudaError_t launch_batch_iteration(const smc_batch* b) {
  const int c = b->count, mv = b->move_v;
  cudaStream_t s = b->stream;
  const ParticleArgs* pa = b->at<ParticleArgs>(b->L.pa);
  const QuantArgs* qa = b->at<QuantArgs>(b->L.qa);
  const int4* qmap = b->at<int4>(b->L.qmap);
  const int nq = int(b->plan.qmap.size());
  cudaError_t e = launch_begin_batch(pa, c, s);
  if (e == cudaSuccess)
    e = launch_move_reweight_batch(pa, b->at<GaussParamsF32>(b->L.gp), b->at<int4>(b->L.mmap[mv]),
                                   int(b->plan.mmap[mv].size()), s);
  if (e == cudaSuccess) e = launch_max_finalize_batch(pa, b->at<int32_t>(b->L.nb) + size_t(mv) * c, c, s);
  if (e == cudaSuccess) e = launch_quant_reduce_batch(qa, qmap, nq, s);
  if (e == cudaSuccess) e = launch_quant_finalize_batch(qa, c, s);
  if (e == cudaSuccess) e = launch_quant_scan_batch(qa, qmap, nq, s);
  if (e == cudaSuccess)
    e = launch_redistribute_batch(b->at<RedistArgs>(b->L.ra), b->at<int4>(b->L.rmap), int(b->plan.rmap.size()),
                                  b->copy_v, s);
  if (e == cudaSuccess) e = launch_commit_batch(pa, c, s);
  return e;
}

cudaError_t build_batch_graph(smc_batch* b) {
  if (b->graph) {
    cudaGraphExecDestroy(b->graph);
    b->graph = nullptr;
  }
  cudaGraph_t g = nullptr;
  cudaError_t e = cudaStreamBeginCapture(b->stream, cudaStreamCaptureModeThreadLocal);
  if (e != cudaSuccess) return e;
  const cudaError_t le = launch_batch_iteration(b);
  e = cudaStreamEndCapture(b->stream, &g);
  if (le != cudaSuccess) {
    if (g) cudaGraphDestroy(g);
    return le;
  }
  if (e != cudaSuccess) return e;
  e = cudaGraphInstantiate(&b->graph, g, 0);
  cudaGraphDestroy(g);
  if (e == cudaSuccess) {
    b->graph_move_v = b->move_v;
    b->graph_copy_v = b->copy_v;
  }
  return e;
}

float median(std::vector<float> v) {
  std::sort(v.begin(), v.end());
  return v.empty() ? 0.0f : v[v.size() / 2];
}

}  // namespace

extern "C" {

int smc_batch_ws_bytes(smc_sampler* const* members, int32_t count, size_t* bytes) {
  const int rc = check_members(members, count);
  if (rc) return rc;
  if (!bytes) return bfail(nullptr, SMC_EINVAL, "null bytes");
  *bytes = batch_layout(make_plan(members, count, sm_count())).total;
  return SMC_OK;
}

int smc_batch_create(smc_batch** out, smc_sampler* const* members, int32_t count, void* ws_dev, size_t ws_bytes,
                     smc_stream_t stream) {
  SMC_RANGE("smc_batch_create");
  if (!out) return bfail(nullptr, SMC_EINVAL, "null out");
  *out = nullptr;
  const int rc = check_members(members, count);
  if (rc) return rc;
  if (!ws_dev || (reinterpret_cast<uintptr_t>(ws_dev) % kAl))
    return bfail(nullptr, SMC_EINVAL, "workspace must be non-null and 256-byte aligned");
  Plan plan = make_plan(members, count, sm_count());
  const BatchLayout L = batch_layout(plan);
  if (ws_bytes < L.total) return bfail(nullptr, SMC_ENOMEM, "workspace too small");
  // the batch's stream waits for the members' queued work (device-side
  // ordering: one event, recorded on each member stream in turn), after any
  // redistribution a member left pending is completed on its stream
  {
    cudaEvent_t ev = nullptr;
    cudaError_t e = cudaSuccess;
    for (int s = 0; s < count && e == cudaSuccess; ++s) e = fetch_gp(members[s]);
    for (int s = 0; s < count && e == cudaSuccess; ++s) e = materialize(members[s]);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&ev, cudaEventDisableTiming);
    const cudaStream_t bs = reinterpret_cast<cudaStream_t>(stream);
    for (int s = 0; s < count && e == cudaSuccess; ++s) {
      if (members[s]->stream == bs) continue;
      e = cudaEventRecord(ev, members[s]->stream);
      if (e == cudaSuccess) e = cudaStreamWaitEvent(bs, ev, 0);
    }
    if (ev) {
      const cudaError_t e2 = cudaEventDestroy(ev);
      if (e == cudaSuccess) e = e2;
    }
    if (e != cudaSuccess) return bfail(nullptr, SMC_ECUDA, std::string("member stream order: ") + cudaGetErrorString(e));
  }
  smc_batch* b = new (std::nothrow) smc_batch();
  if (!b) return bfail(nullptr, SMC_ENOMEM, "host allocation failed");
  b->m.assign(members, members + count);
  b->count = count;
  b->plan = std::move(plan);
  b->L = L;
  b->ws = static_cast<char*>(ws_dev);
  b->stream = reinterpret_cast<cudaStream_t>(stream);
  b->move_v = kDefaultMove;
  b->copy_v = kDefaultCopy;
  b->graph = nullptr;
  b->graph_move_v = b->graph_copy_v = -1;
  b->outs_host.assign(3 * size_t(count), nullptr);
  b->errs_host.assign(count, 0);
  b->err = "ok";

  std::vector<ParticleArgs> pa(count);
  std::vector<QuantArgs> qa(count);
  std::vector<RedistArgs> ra(count), rdry(count);
  std::vector<GaussParamsF32> gp(count);
  DevState* dry_st = b->at<DevState>(L.dry_st);
  for (int s = 0; s < count; ++s) {
    const smc_sampler* h = members[s];
    pa[s] = particle_args(h);
    qa[s] = quant_args(h, 0, nullptr);
    qa[s].est_src = h->d <= 16 ? 1 : 0;  // the batched move kernel writes the eq. (7) tile records
    ra[s] = redist_args(h, 0);
    gp[s] = h->gp;
    // the copy autotuner's input: an in-place identity copy of buffer 0
    // (every row rewritten with its own bytes), no payload, no log w reset
    RedistArgs r = ra[s];
    r.stateful = 0;
    r.force = 1;
    r.x_in[0] = r.x_in[1] = h->x[0];
    r.x_out[0] = r.x_out[1] = h->x[0];
    r.lp_bytes = 0;
    r.logw = nullptr;
    r.st = dry_st;
    rdry[s] = r;
  }
  std::vector<int32_t> nb(size_t(SMC_BATCH_MOVE_VARIANTS) * count);
  for (int v = 0; v < SMC_BATCH_MOVE_VARIANTS; ++v)
    std::copy(b->plan.nb[v].begin(), b->plan.nb[v].end(), nb.begin() + size_t(v) * count);
  // pageable sources: each copy is staged before cudaMemcpyAsync returns
  cudaStream_t st = b->stream;
  cudaError_t e = cudaMemcpyAsync(b->ws + L.pa, pa.data(), count * sizeof(ParticleArgs), cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess) e = cudaMemcpyAsync(b->ws + L.qa, qa.data(), count * sizeof(QuantArgs), cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess) e = cudaMemcpyAsync(b->ws + L.ra, ra.data(), count * sizeof(RedistArgs), cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(b->ws + L.ra_dry, rdry.data(), count * sizeof(RedistArgs), cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(b->ws + L.gp, gp.data(), count * sizeof(GaussParamsF32), cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess) e = cudaMemcpyAsync(b->ws + L.nb, nb.data(), nb.size() * sizeof(int32_t), cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(b->ws + L.qmap, b->plan.qmap.data(), b->plan.qmap.size() * sizeof(int4), cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(b->ws + L.rmap, b->plan.rmap.data(), b->plan.rmap.size() * sizeof(int4), cudaMemcpyHostToDevice, st);
  for (int v = 0; v < SMC_BATCH_MOVE_VARIANTS && e == cudaSuccess; ++v)
    e = cudaMemcpyAsync(b->ws + L.mmap[v], b->plan.mmap[v].data(), b->plan.mmap[v].size() * sizeof(int4),
                        cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess) e = cudaMemsetAsync(dry_st, 0, devstate_bytes(), st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) {
    delete b;
    return bfail(nullptr, SMC_ECUDA, std::string("smc_batch_create: ") + cudaGetErrorString(e));
  }
  *out = b;
  return SMC_OK;
}

int smc_batch_step(smc_batch* b, int32_t k, double* const* mean_dev, smc_iter_stats* const* trace_dev,
                   double* const* fhat_dev) {
  SMC_RANGE("smc_batch_step");
  if (!b) return bfail(nullptr, SMC_EINVAL, "null handle");
  if (k < 0) return bfail(b, SMC_EINVAL, "k must be >= 0");
  if (k == 0) return SMC_OK;
  const int c = b->count;
  for (int s = 0; s < c; ++s) {
    b->outs_host[s] = trace_dev ? static_cast<void*>(trace_dev[s]) : nullptr;
    b->outs_host[c + s] = mean_dev ? static_cast<void*>(mean_dev[s]) : nullptr;
    b->outs_host[2 * c + s] = fhat_dev ? static_cast<void*>(fhat_dev[s]) : nullptr;
  }
  BATCH_TRY(b, cudaMemcpyAsync(b->ws + b->L.outs, b->outs_host.data(), 3 * size_t(c) * sizeof(void*),
                               cudaMemcpyHostToDevice, b->stream));
  BATCH_TRY(b, launch_step_setup_batch(b->at<ParticleArgs>(b->L.pa), b->at<void*>(b->L.outs), c, b->stream));
  const bool use_graph = b->stream != nullptr;
  for (int32_t it = 0; it < k; ++it) {
    if (use_graph) {
      if (!b->graph || b->graph_move_v != b->move_v || b->graph_copy_v != b->copy_v)
        BATCH_TRY(b, build_batch_graph(b));
      BATCH_TRY(b, cudaGraphLaunch(b->graph, b->stream));
    } else {
      BATCH_TRY(b, launch_batch_iteration(b));
    }
  }
  return SMC_OK;
}

int smc_batch_step_profile(smc_batch* b, void* const* events_host, int32_t n_events) {
  SMC_RANGE("smc_batch_step_profile");
  if (!b) return bfail(nullptr, SMC_EINVAL, "null handle");
  if (n_events != 0 && n_events != 8) return bfail(b, SMC_EINVAL, "n_events must be 0 or 8");
  if (n_events && !events_host) return bfail(b, SMC_EINVAL, "null events");
  const int c = b->count, mv = b->move_v;
  cudaStream_t s = b->stream;
  auto rec = [&](int j) -> cudaError_t {
    return n_events ? cudaEventRecord(static_cast<cudaEvent_t>(events_host[j]), s) : cudaSuccess;
  };
  std::fill(b->outs_host.begin(), b->outs_host.end(), nullptr);
  const ParticleArgs* pa = b->at<ParticleArgs>(b->L.pa);
  const QuantArgs* qa = b->at<QuantArgs>(b->L.qa);
  const int4* qmap = b->at<int4>(b->L.qmap);
  const int nq = int(b->plan.qmap.size());
  BATCH_TRY(b, cudaMemcpyAsync(b->ws + b->L.outs, b->outs_host.data(), 3 * size_t(c) * sizeof(void*),
                               cudaMemcpyHostToDevice, s));
  BATCH_TRY(b, launch_step_setup_batch(pa, b->at<void*>(b->L.outs), c, s));
  BATCH_TRY(b, rec(0));
  BATCH_TRY(b, launch_begin_batch(pa, c, s));
  BATCH_TRY(b, launch_move_reweight_batch(pa, b->at<GaussParamsF32>(b->L.gp), b->at<int4>(b->L.mmap[mv]),
                                          int(b->plan.mmap[mv].size()), s));
  BATCH_TRY(b, rec(1));
  BATCH_TRY(b, launch_max_finalize_batch(pa, b->at<int32_t>(b->L.nb) + size_t(mv) * c, c, s));
  BATCH_TRY(b, rec(2));
  BATCH_TRY(b, launch_quant_reduce_batch(qa, qmap, nq, s));
  BATCH_TRY(b, rec(3));
  BATCH_TRY(b, launch_quant_finalize_batch(qa, c, s));
  BATCH_TRY(b, rec(4));
  BATCH_TRY(b, launch_quant_scan_batch(qa, qmap, nq, s));
  BATCH_TRY(b, rec(5));
  BATCH_TRY(b, launch_redistribute_batch(b->at<RedistArgs>(b->L.ra), b->at<int4>(b->L.rmap),
                                         int(b->plan.rmap.size()), b->copy_v, s));
  BATCH_TRY(b, rec(6));
  BATCH_TRY(b, launch_commit_batch(pa, c, s));
  BATCH_TRY(b, rec(7));
  return SMC_OK;
}

int smc_batch_set_variant(smc_batch* b, int32_t move_variant, int32_t copy_variant) {
  if (!b) return bfail(nullptr, SMC_EINVAL, "null handle");
  if (move_variant < 0 || move_variant >= SMC_BATCH_MOVE_VARIANTS || copy_variant < 0 ||
      copy_variant >= SMC_BATCH_COPY_VARIANTS)
    return bfail(b, SMC_EINVAL, "variant out of range");
  b->move_v = move_variant;
  b->copy_v = copy_variant;
  return SMC_OK;
}

int smc_batch_tune(smc_batch* b, int32_t reps, int32_t* choice_host) {
  SMC_RANGE("smc_batch_tune");
  if (!b) return bfail(nullptr, SMC_EINVAL, "null handle");
  if (reps < 1) return bfail(b, SMC_EINVAL, "reps must be >= 1");
  const int c = b->count;
  cudaStream_t s = b->stream;
  // The move is timed on each member's spare buffers: the particle buffer and
  // log pi buffer that the current iteration does not hold, and the W buffer
  // of the quantise pass (rewritten before every use) in place of log w.  A
  // zeroed state block supplies t = 0 and buffer 0.
  BATCH_TRY(b, cudaStreamSynchronize(s));
  std::vector<ParticleArgs> dry(c);
  for (int q = 0; q < c; ++q) {
    const smc_sampler* h = b->m[q];
    int32_t cur = 0;
    BATCH_TRY(b, cudaMemcpy(&cur, &h->st->cur, sizeof cur, cudaMemcpyDeviceToHost));
    ParticleArgs a = particle_args(h);
    a.x[0] = a.x[1] = h->x[cur ? 0 : 1];
    a.logpi[0] = a.logpi[1] = h->lp[cur ? 0 : 1];
    a.logw = reinterpret_cast<double*>(h->wbuf);
    a.st = b->at<DevState>(b->L.dry_st);
    dry[q] = a;
  }
  BATCH_TRY(b, cudaMemcpyAsync(b->ws + b->L.pa_dry, dry.data(), c * sizeof(ParticleArgs), cudaMemcpyHostToDevice, s));
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  BATCH_TRY(b, cudaEventCreate(&e0));
  cudaError_t e = cudaEventCreate(&e1);
  auto cleanup = [&]() {
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
  };
  float best_move = 0.0f, best_copy = 0.0f;
  int pick_move = b->move_v, pick_copy = b->copy_v;
  const ParticleArgs* pdry = b->at<ParticleArgs>(b->L.pa_dry);
  const GaussParamsF32* gp = b->at<GaussParamsF32>(b->L.gp);
  for (int v = 0; v < SMC_BATCH_MOVE_VARIANTS && e == cudaSuccess; ++v) {
    std::vector<float> t;
    for (int r = 0; r <= reps && e == cudaSuccess; ++r) {  // r == 0 warms up
      e = cudaEventRecord(e0, s);
      if (e == cudaSuccess)
        e = launch_move_reweight_batch(pdry, gp, b->at<int4>(b->L.mmap[v]), int(b->plan.mmap[v].size()), s);
      if (e == cudaSuccess) e = cudaEventRecord(e1, s);
      if (e == cudaSuccess) e = cudaEventSynchronize(e1);
      float ms = 0.0f;
      if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
      if (r > 0) t.push_back(ms);
    }
    const float md = median(t);
    if (e == cudaSuccess && (v == 0 || md < best_move)) {
      best_move = md;
      pick_move = v;
    }
  }
  // the move's garbage inputs may have flagged the zeroed state; the copy
  // needs it clear
  if (e == cudaSuccess) e = cudaMemsetAsync(b->at<DevState>(b->L.dry_st), 0, devstate_bytes(), s);
  const RedistArgs* rdry = b->at<RedistArgs>(b->L.ra_dry);
  const int4* rmap = b->at<int4>(b->L.rmap);
  const int nr = int(b->plan.rmap.size());
  for (int v = 0; v < SMC_BATCH_COPY_VARIANTS && e == cudaSuccess; ++v) {
    std::vector<float> t;
    for (int r = 0; r <= reps && e == cudaSuccess; ++r) {
      e = launch_identity_runs_batch(rdry, rmap, nr, s);
      if (e == cudaSuccess) e = cudaEventRecord(e0, s);
      if (e == cudaSuccess) e = launch_redistribute_batch(rdry, rmap, nr, v, s);
      if (e == cudaSuccess) e = cudaEventRecord(e1, s);
      if (e == cudaSuccess) e = cudaEventSynchronize(e1);
      float ms = 0.0f;
      if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
      if (r > 0) t.push_back(ms);
    }
    const float md = median(t);
    if (e == cudaSuccess && (v == 0 || md < best_copy)) {
      best_copy = md;
      pick_copy = v;
    }
  }
  cleanup();
  if (e != cudaSuccess) return bfail(b, SMC_ECUDA, std::string("smc_batch_tune: ") + cudaGetErrorString(e));
  b->move_v = pick_move;
  b->copy_v = pick_copy;
  if (choice_host) {
    choice_host[0] = pick_move;
    choice_host[1] = pick_copy;
  }
  return SMC_OK;
}

int smc_batch_sync(smc_batch* b, int32_t* which_host) {
  SMC_RANGE("smc_batch_sync");
  if (!b) return bfail(nullptr, SMC_EINVAL, "null handle");
  if (which_host) *which_host = -1;
  const int c = b->count;
  BATCH_TRY(b, launch_take_errors_batch(b->at<ParticleArgs>(b->L.pa), b->at<int32_t>(b->L.errs), c, b->stream));
  BATCH_TRY(b, cudaMemcpyAsync(b->errs_host.data(), b->ws + b->L.errs, c * sizeof(int32_t), cudaMemcpyDeviceToHost,
                               b->stream));
  BATCH_TRY(b, cudaStreamSynchronize(b->stream));
  for (int s = 0; s < c; ++s) {
    const int32_t code = b->errs_host[s];
    if (code) {
      if (which_host) *which_host = s;
      static const char* names[] = {"ok", "invalid argument on the device", "out of memory", "cuda",
                                    "a bounded device wait timed out", "non-finite log-weights"};
      return bfail(b, code,
                   std::string("member ") + std::to_string(s) + ": " + (code >= 0 && code <= 5 ? names[code] : "device error"));
    }
  }
  return SMC_OK;
}

int smc_batch_destroy(smc_batch* b) {
  if (!b) return SMC_OK;
  if (b->graph) cudaGraphExecDestroy(b->graph);
  delete b;
  return SMC_OK;
}

const char* smc_batch_last_error(const smc_batch* b) { return b ? b->err.c_str() : g_batch_err.c_str(); }

}  // extern "C"
