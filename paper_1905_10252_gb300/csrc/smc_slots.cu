// smc_slots.cu -- a standing batch of slots (C-ABI, include/smc.h): the batch
// of smc_batch.cu with a fixed launch layout, for serving.
//
// Each slot has a capacity (the most particles a sampler in it may have).
// The block maps of every stage are sized once, at creation, from the
// capacities -- a slot's quantise, scan and copy blocks cover its capacity,
// its move blocks are a share of a fixed budget -- and one batched iteration
// is captured in a CUDA graph then.  While membership is unchanged the maps
// and the graph are reused as they are; after an attach or detach the next
// step writes compact maps of the attached slots' own blocks (from pinned
// staging, double buffered) and sets the grid sizes of the graph's four
// map-driven kernel nodes to match (no re-instantiation).  Samplers are attached to and detached
// from slots afterwards by editing the slot table in device memory (their
// kernel arguments, an attached flag, their outputs); a step sets, per slot,
// how many iterations to run, and replays the graph.  Every kernel reads a
// slot's count first: a slot with none left (or empty) does nothing, and
// blocks past a member's own block count exit, so a member runs exactly the
// blocks, tiles and reduction order it has alone and its results are
// bit-identical to smc_step.  No host synchronisation: table edits are
// kernel launches that carry their values as parameters, ordered on the
// slots' stream.
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
constexpr int kSlotMax = 512;          // slots per standing batch (the per-step counts travel as one parameter block)
constexpr int kSlotMoveBudget = 8;     // move blocks per SM shared by the slots, in proportion to capacity
constexpr int kSlotMaxMoveBlocks = 4096;
constexpr int kSlotCopyVariant = 1;    // 8 loads in flight per thread in the copy

size_t up(size_t v) { return (v + kAl - 1) / kAl * kAl; }
int64_t div_up(int64_t a, int64_t b) { return (a + b - 1) / b; }

thread_local std::string g_slots_err = "ok";

struct SlotsPlan {
  std::vector<int4> qmap, rmap, mmap;
  std::vector<int32_t> nb;  // move blocks (max records) per slot
};

SlotsPlan make_slots_plan(const int64_t* cap, int count, int sms) {
  SlotsPlan p;
  std::vector<int> order(count);
  double csum = 0.0;
  for (int s = 0; s < count; ++s) {
    order[s] = s;
    csum += double(cap[s]);
  }
  // largest slots first, so that the last blocks of a launch are short
  std::stable_sort(order.begin(), order.end(), [&](int a, int b) { return cap[a] > cap[b]; });
  p.nb.assign(count, 1);
  const double budget = double(kSlotMoveBudget) * sms;
  for (int s = 0; s < count; ++s) {
    const int full = int(std::min<int64_t>(div_up(cap[s], kPThreads), kSlotMaxMoveBlocks));
    const int b = int(std::llround(budget * double(cap[s]) / csum));
    p.nb[s] = std::max(1, std::min(b, full));
  }
  for (int s : order) {
    const int nq = int(div_up(cap[s], kQTile)), nr = int(div_up(cap[s], kRTile));
    for (int j = 0; j < nq; ++j) p.qmap.push_back(make_int4(s, j, nq, 0));
    for (int j = 0; j < nr; ++j) p.rmap.push_back(make_int4(s, j, nr, 0));
    for (int j = 0; j < p.nb[s]; ++j) p.mmap.push_back(make_int4(s, j, p.nb[s], 0));
  }
  return p;
}

struct SlotsLayout {
  size_t pa, qa, ra, gp, nb, left, attached, errs, qmap, rmap, mmap, total;
};

SlotsLayout slots_layout(const SlotsPlan& p, int count) {
  SlotsLayout L{};
  const size_t c = size_t(count);
  size_t o = 0;
  auto take = [&](size_t bytes) {
    const size_t at = o;
    o = up(o + bytes);
    return at;
  };
  L.pa = take(c * sizeof(ParticleArgs));
  L.qa = take(c * sizeof(QuantArgs));
  L.ra = take(c * sizeof(RedistArgs));
  L.gp = take(c * sizeof(GaussParamsF32));
  L.nb = take(c * sizeof(int32_t));
  L.left = take(c * sizeof(int32_t));
  L.attached = take(c * sizeof(int32_t));
  L.errs = take(c * sizeof(int32_t));
  L.qmap = take(p.qmap.size() * sizeof(int4));
  L.rmap = take(p.rmap.size() * sizeof(int4));
  L.mmap = take(p.mmap.size() * sizeof(int4));
  L.total = o;
  return L;
}

int check_caps(const int64_t* cap, int32_t count) {
  if (!cap || count < 1 || count > kSlotMax) {
    g_slots_err = "count must be in [1, 512] and cap_n non-null";
    return SMC_EINVAL;
  }
  for (int s = 0; s < count; ++s)
    if (cap[s] < 1 || cap[s] > 2147483647LL) {
      g_slots_err = "slot " + std::to_string(s) + ": capacity must be in [1, 2^31)";
      return SMC_EINVAL;
    }
  return SMC_OK;
}

// ---------------------------------------------------------------- slot-table kernels
// The kernel arguments of one slot's sampler, passed by value.
struct SlotEntry {
  ParticleArgs pa;
  QuantArgs qa;
  RedistArgs ra;
};

// Installs a sampler: its arguments, and its FP32 factor built from the
// device copy of its target (mu and the row pairs of L^-1 interleaved as the
// move kernel reads them: the same floats smc_step passes as parameters).
__global__ void k_slots_install(ParticleArgs* pa, QuantArgs* qa, RedistArgs* ra, GaussParamsF32* gp,
                                int32_t* attached, int32_t* left, int slot, const SlotEntry e,
                                const TargetDev* __restrict__ tg) {
  GaussParamsF32* g = gp + slot;
  for (int q = threadIdx.x; q < kTgtMaxD / 2 * kTgtMaxD; q += blockDim.x) {
    const int p = q / kTgtMaxD, c = q % kTgtMaxD;
    g->P2[q] = make_float2(c <= 2 * p ? tg->Pf[2 * p * kTgtMaxD + c] : 0.0f,
                           c <= 2 * p + 1 ? tg->Pf[(2 * p + 1) * kTgtMaxD + c] : 0.0f);
  }
  for (int c = threadIdx.x; c < kTgtMaxD; c += blockDim.x) g->mu[c] = tg->muf[c];
  if (threadIdx.x != 0) return;
  pa[slot] = e.pa;
  qa[slot] = e.qa;
  ra[slot] = e.ra;
  left[slot] = 0;
  attached[slot] = 1;
}

__global__ void k_slots_clear(int32_t* attached, int32_t* left, int slot) {
  if (threadIdx.x != 0) return;
  attached[slot] = 0;
  left[slot] = 0;
}

struct SlotCounts {
  int32_t v[kSlotMax];
};

__global__ void k_slots_set_left(int32_t* left, int count, const SlotCounts c) {
  for (int s = threadIdx.x; s < count; s += blockDim.x) left[s] = c.v[s];
}

__global__ void k_slots_take_errors(const ParticleArgs* __restrict__ pa, const int32_t* __restrict__ attached,
                                    int32_t* errs, int count) {
  const int s = blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= count) return;
  if (!attached[s]) {
    errs[s] = 0;
    return;
  }
  errs[s] = pa[s].st->err;
  pa[s].st->err = 0;
}

}  // namespace

struct smc_slots {
  int count;
  std::vector<int64_t> cap;
  std::vector<smc_sampler*> m;  // attached sampler per slot, NULL when empty
  SlotsPlan plan;
  SlotsLayout L;
  char* ws;
  cudaStream_t stream;
  cudaGraph_t tmpl;             // the captured iteration (kept: its nodes are updated)
  cudaGraphExec_t graph;
  cudaGraphNode_t map_node[4];  // move, quantise reduce, scan, copy: kernels launched over a map
  cudaEvent_t ev;
  // compact maps: pinned staging (two buffers of qmap | rmap | mmap, each at
  // its full size) and the event after each buffer's last upload
  int4* stage[2];
  cudaEvent_t stage_ev[2];
  int stage_next;
  bool dirty;                   // membership changed since the maps were written
  std::vector<int32_t> errs_host;
  std::string err;

  template <typename T>
  T* at(size_t off) const {
    return reinterpret_cast<T*>(ws + off);
  }
};

namespace {

int sfail(smc_slots* b, int code, const std::string& msg) {
  if (b)
    b->err = msg;
  else
    g_slots_err = msg;
  return code;
}

#define SLOTS_TRY(b, expr)                                                                \
  do {                                                                                    \
    cudaError_t _e = (expr);                                                              \
    if (_e != cudaSuccess) return sfail((b), SMC_ECUDA, std::string(#expr) + ": " + cudaGetErrorString(_e)); \
  } while (0)

// One iteration of Algorithm 2 (lines 3-10) for every slot with iterations
// left: the 8 launches of a batched iteration, each gated on the counts.
cudaError_t launch_slots_iteration(const smc_slots* b) {
  const int c = b->count;
  cudaStream_t s = b->stream;
  const ParticleArgs* pa = b->at<ParticleArgs>(b->L.pa);
  const QuantArgs* qa = b->at<QuantArgs>(b->L.qa);
  int32_t* left = b->at<int32_t>(b->L.left);
  const int4* qmap = b->at<int4>(b->L.qmap);
  const int nq = int(b->plan.qmap.size());
  cudaError_t e = launch_begin_batch(pa, c, s, left);
  if (e == cudaSuccess)
    e = launch_move_reweight_batch(pa, b->at<GaussParamsF32>(b->L.gp), b->at<int4>(b->L.mmap),
                                   int(b->plan.mmap.size()), s, left);
  if (e == cudaSuccess) e = launch_max_finalize_batch(pa, b->at<int32_t>(b->L.nb), c, s, left);
  if (e == cudaSuccess) e = launch_quant_reduce_batch(qa, qmap, nq, s, left);
  if (e == cudaSuccess) e = launch_quant_finalize_batch(qa, c, s, left);
  if (e == cudaSuccess) e = launch_quant_scan_batch(qa, qmap, nq, s, left);
  if (e == cudaSuccess)
    e = launch_redistribute_batch(b->at<RedistArgs>(b->L.ra), b->at<int4>(b->L.rmap), int(b->plan.rmap.size()),
                                  kSlotCopyVariant, s, left);
  if (e == cudaSuccess) e = launch_commit_batch(pa, c, s, left);
  return e;
}

cudaError_t build_slots_graph(smc_slots* b) {
  cudaGraph_t g = nullptr;
  cudaError_t e = cudaStreamBeginCapture(b->stream, cudaStreamCaptureModeThreadLocal);
  if (e != cudaSuccess) return e;
  const cudaError_t le = launch_slots_iteration(b);
  e = cudaStreamEndCapture(b->stream, &g);
  if (le != cudaSuccess) {
    if (g) cudaGraphDestroy(g);
    return le;
  }
  if (e != cudaSuccess) return e;
  // the captured launches form one chain in launch order: begin, move, max,
  // quantise reduce, quantise finalise, scan, copy, commit
  cudaGraphNode_t chain[8];
  size_t nroot = 1;
  e = cudaGraphGetRootNodes(g, chain, &nroot);
  for (int k = 1; e == cudaSuccess && k < 8; ++k) {
    size_t nd = 1;
    e = cudaGraphNodeGetDependentNodes(chain[k - 1], &chain[k], nullptr, &nd);
    if (e == cudaSuccess && nd != 1) e = cudaErrorInvalidValue;
  }
  if (e == cudaSuccess && nroot != 1) e = cudaErrorInvalidValue;
  if (e == cudaSuccess) {
    b->map_node[0] = chain[1];
    b->map_node[1] = chain[3];
    b->map_node[2] = chain[5];
    b->map_node[3] = chain[6];
    e = cudaGraphInstantiate(&b->graph, g, 0);
  }
  if (e != cudaSuccess) {
    cudaGraphDestroy(g);
    return e;
  }
  b->tmpl = g;
  return cudaSuccess;
}

// Compact maps of the attached slots (their own quantise / copy blocks and
// the slot's move blocks), uploaded on the slots' stream, and the grid sizes
// of the map-driven kernel nodes set to the new entry counts.
cudaError_t write_compact_maps(smc_slots* b) {
  const size_t fq = b->plan.qmap.size(), fr = b->plan.rmap.size(), fm = b->plan.mmap.size();
  const int sb = b->stage_next;
  b->stage_next ^= 1;
  cudaError_t e = cudaEventSynchronize(b->stage_ev[sb]);  // (that buffer's previous upload is done)
  if (e != cudaSuccess) return e;
  int4* q = b->stage[sb];
  int4* r = q + fq;
  int4* m = r + fr;
  size_t nq = 0, nr = 0, nm = 0;
  // the creation order (largest capacity first), attached slots only
  std::vector<int> order(b->count);
  for (int s = 0; s < b->count; ++s) order[s] = s;
  std::stable_sort(order.begin(), order.end(), [&](int x, int y) { return b->cap[x] > b->cap[y]; });
  for (int s : order) {
    const smc_sampler* h = b->m[s];
    if (!h) continue;
    const int hq = h->L.qblocks, hr = h->L.ntiles, hm = b->plan.nb[s];
    for (int j = 0; j < hq; ++j) q[nq++] = make_int4(s, j, hq, 0);
    for (int j = 0; j < hr; ++j) r[nr++] = make_int4(s, j, hr, 0);
    for (int j = 0; j < hm; ++j) m[nm++] = make_int4(s, j, hm, 0);
  }
  if (nq == 0) {  // (no slot attached: the maps are not launched)
    b->dirty = false;
    return cudaSuccess;
  }
  e = cudaMemcpyAsync(b->ws + b->L.qmap, q, nq * sizeof(int4), cudaMemcpyHostToDevice, b->stream);
  if (e == cudaSuccess) e = cudaMemcpyAsync(b->ws + b->L.rmap, r, nr * sizeof(int4), cudaMemcpyHostToDevice, b->stream);
  if (e == cudaSuccess) e = cudaMemcpyAsync(b->ws + b->L.mmap, m, nm * sizeof(int4), cudaMemcpyHostToDevice, b->stream);
  if (e == cudaSuccess) e = cudaEventRecord(b->stage_ev[sb], b->stream);
  const size_t counts[4] = {nm, nq, nq, nr};
  for (int k = 0; k < 4 && e == cudaSuccess; ++k) {
    cudaKernelNodeParams kp{};
    e = cudaGraphKernelNodeGetParams(b->map_node[k], &kp);
    if (e != cudaSuccess) break;
    kp.gridDim = dim3(unsigned(counts[k]), 1, 1);
    e = cudaGraphExecKernelNodeSetParams(b->graph, b->map_node[k], &kp);
  }
  if (e == cudaSuccess) b->dirty = false;
  return e;
}

}  // namespace

extern "C" {

int smc_slots_ws_bytes(const int64_t* cap_n, int32_t count, size_t* bytes) {
  const int rc = check_caps(cap_n, count);
  if (rc) return rc;
  if (!bytes) return sfail(nullptr, SMC_EINVAL, "null bytes");
  *bytes = slots_layout(make_slots_plan(cap_n, count, sm_count()), count).total;
  return SMC_OK;
}

int smc_slots_create(smc_slots** out, const int64_t* cap_n, int32_t count, void* ws_dev, size_t ws_bytes,
                     smc_stream_t stream) {
  SMC_RANGE("smc_slots_create");
  if (!out) return sfail(nullptr, SMC_EINVAL, "null out");
  *out = nullptr;
  const int rc = check_caps(cap_n, count);
  if (rc) return rc;
  if (!stream) return sfail(nullptr, SMC_EINVAL, "a standing batch needs a non-default stream (its iteration is a CUDA graph)");
  if (!ws_dev || (reinterpret_cast<uintptr_t>(ws_dev) % kAl))
    return sfail(nullptr, SMC_EINVAL, "workspace must be non-null and 256-byte aligned");
  SlotsPlan plan = make_slots_plan(cap_n, count, sm_count());
  const SlotsLayout L = slots_layout(plan, count);
  if (ws_bytes < L.total) return sfail(nullptr, SMC_ENOMEM, "workspace too small");
  smc_slots* b = new (std::nothrow) smc_slots();
  if (!b) return sfail(nullptr, SMC_ENOMEM, "host allocation failed");
  b->count = count;
  b->cap.assign(cap_n, cap_n + count);
  b->m.assign(count, nullptr);
  b->plan = std::move(plan);
  b->L = L;
  b->ws = static_cast<char*>(ws_dev);
  b->stream = reinterpret_cast<cudaStream_t>(stream);
  b->tmpl = nullptr;
  b->graph = nullptr;
  b->ev = nullptr;
  b->stage[0] = b->stage[1] = nullptr;
  b->stage_ev[0] = b->stage_ev[1] = nullptr;
  b->stage_next = 0;
  b->dirty = true;
  b->errs_host.assign(count, 0);
  b->err = "ok";
  cudaStream_t st = b->stream;
  cudaError_t e = cudaMemsetAsync(b->ws, 0, L.total, st);  // every slot empty, no counts
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(b->ws + L.nb, b->plan.nb.data(), count * sizeof(int32_t), cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(b->ws + L.qmap, b->plan.qmap.data(), b->plan.qmap.size() * sizeof(int4),
                        cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(b->ws + L.rmap, b->plan.rmap.data(), b->plan.rmap.size() * sizeof(int4),
                        cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(b->ws + L.mmap, b->plan.mmap.data(), b->plan.mmap.size() * sizeof(int4),
                        cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);  // (the host vectors are pageable)
  if (e == cudaSuccess) e = cudaEventCreateWithFlags(&b->ev, cudaEventDisableTiming);
  const size_t maps = b->plan.qmap.size() + b->plan.rmap.size() + b->plan.mmap.size();
  for (int k = 0; k < 2 && e == cudaSuccess; ++k) {
    e = cudaHostAlloc(reinterpret_cast<void**>(&b->stage[k]), maps * sizeof(int4), cudaHostAllocDefault);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&b->stage_ev[k], cudaEventDisableTiming);
  }
  if (e == cudaSuccess) e = build_slots_graph(b);
  if (e != cudaSuccess) {
    if (b->graph) cudaGraphExecDestroy(b->graph);
    if (b->tmpl) cudaGraphDestroy(b->tmpl);
    if (b->ev) cudaEventDestroy(b->ev);
    for (int k = 0; k < 2; ++k) {
      if (b->stage[k]) cudaFreeHost(b->stage[k]);
      if (b->stage_ev[k]) cudaEventDestroy(b->stage_ev[k]);
    }
    delete b;
    return sfail(nullptr, SMC_ECUDA, std::string("smc_slots_create: ") + cudaGetErrorString(e));
  }
  *out = b;
  return SMC_OK;
}

int smc_slots_attach(smc_slots* b, int32_t slot, smc_sampler* h, double* mean_dev, smc_iter_stats* trace_dev,
                     double* fhat_dev) {
  SMC_RANGE("smc_slots_attach");
  if (!b) return sfail(nullptr, SMC_EINVAL, "null handle");
  if (slot < 0 || slot >= b->count) return sfail(b, SMC_EINVAL, "slot out of range");
  if (!h) return sfail(b, SMC_EINVAL, "null sampler");
  if (b->m[slot]) return sfail(b, SMC_EINVAL, "slot " + std::to_string(slot) + " is not empty");
  if (h->dtype != SMC_F32 || h->cfg.target != SMC_GAUSS || !h->have_gp)
    return sfail(b, SMC_EINVAL, "only FP32 Gaussian samplers can be attached");
  if (h->n > b->cap[slot]) return sfail(b, SMC_EINVAL, "sampler larger than the slot's capacity");
  for (int s = 0; s < b->count; ++s)
    if (b->m[s] == h) return sfail(b, SMC_EINVAL, "sampler already attached to slot " + std::to_string(s));
  SlotEntry en{};
  en.pa = particle_args(h);
  en.qa = quant_args(h, 0, nullptr);
  en.qa.est_src = h->d <= 16 ? 1 : 0;  // the batched move kernel writes the eq. (7) tile records
  en.ra = redist_args(h, 0);
  // the slots' stream after the sampler's queued work (a pending
  // redistribution first completed on the sampler's stream)
  SLOTS_TRY(b, materialize(h));
  SLOTS_TRY(b, cudaEventRecord(b->ev, h->stream));
  SLOTS_TRY(b, cudaStreamWaitEvent(b->stream, b->ev, 0));
  k_slots_install<<<1, 256, 0, b->stream>>>(b->at<ParticleArgs>(b->L.pa), b->at<QuantArgs>(b->L.qa),
                                            b->at<RedistArgs>(b->L.ra), b->at<GaussParamsF32>(b->L.gp),
                                            b->at<int32_t>(b->L.attached), b->at<int32_t>(b->L.left), slot, en,
                                            h->tg);
  SLOTS_TRY(b, cudaGetLastError());
  SLOTS_TRY(b, launch_step_setup(h->st, trace_dev, mean_dev, fhat_dev, nullptr, b->stream));
  b->m[slot] = h;
  b->dirty = true;
  return SMC_OK;
}

int smc_slots_detach(smc_slots* b, int32_t slot) {
  SMC_RANGE("smc_slots_detach");
  if (!b) return sfail(nullptr, SMC_EINVAL, "null handle");
  if (slot < 0 || slot >= b->count) return sfail(b, SMC_EINVAL, "slot out of range");
  smc_sampler* h = b->m[slot];
  if (!h) return sfail(b, SMC_EINVAL, "slot " + std::to_string(slot) + " is empty");
  k_slots_clear<<<1, 32, 0, b->stream>>>(b->at<int32_t>(b->L.attached), b->at<int32_t>(b->L.left), slot);
  SLOTS_TRY(b, cudaGetLastError());
  // the sampler's own later calls come after the slots' work on it
  SLOTS_TRY(b, cudaEventRecord(b->ev, b->stream));
  SLOTS_TRY(b, cudaStreamWaitEvent(h->stream, b->ev, 0));
  b->m[slot] = nullptr;
  b->dirty = true;
  return SMC_OK;
}

int smc_slots_step(smc_slots* b, const int32_t* iters_host) {
  SMC_RANGE("smc_slots_step");
  if (!b) return sfail(nullptr, SMC_EINVAL, "null handle");
  if (!iters_host) return sfail(b, SMC_EINVAL, "null iteration counts");
  SlotCounts c{};
  int k = 0;
  for (int s = 0; s < b->count; ++s) {
    const int32_t v = iters_host[s];
    if (v < 0) return sfail(b, SMC_EINVAL, "negative iteration count for slot " + std::to_string(s));
    if (v > 0 && !b->m[s]) return sfail(b, SMC_EINVAL, "iterations requested for empty slot " + std::to_string(s));
    c.v[s] = v;
    k = std::max(k, int(v));
  }
  if (k == 0) return SMC_OK;
  if (b->dirty) SLOTS_TRY(b, write_compact_maps(b));
  k_slots_set_left<<<1, 256, 0, b->stream>>>(b->at<int32_t>(b->L.left), b->count, c);
  SLOTS_TRY(b, cudaGetLastError());
  for (int it = 0; it < k; ++it) SLOTS_TRY(b, cudaGraphLaunch(b->graph, b->stream));
  return SMC_OK;
}

int smc_slots_sync(smc_slots* b, int32_t* which_host) {
  SMC_RANGE("smc_slots_sync");
  if (!b) return sfail(nullptr, SMC_EINVAL, "null handle");
  if (which_host) *which_host = -1;
  const int c = b->count;
  k_slots_take_errors<<<(c + 127) / 128, 128, 0, b->stream>>>(b->at<ParticleArgs>(b->L.pa),
                                                             b->at<int32_t>(b->L.attached),
                                                             b->at<int32_t>(b->L.errs), c);
  SLOTS_TRY(b, cudaGetLastError());
  SLOTS_TRY(b, cudaMemcpyAsync(b->errs_host.data(), b->ws + b->L.errs, c * sizeof(int32_t), cudaMemcpyDeviceToHost,
                               b->stream));
  SLOTS_TRY(b, cudaStreamSynchronize(b->stream));
  for (int s = 0; s < c; ++s) {
    const int32_t code = b->errs_host[s];
    if (code) {
      if (which_host) *which_host = s;
      return sfail(b, code, "slot " + std::to_string(s) + ": device error " + std::to_string(code));
    }
  }
  return SMC_OK;
}

int smc_slots_destroy(smc_slots* b) {
  if (!b) return SMC_OK;
  cudaStreamSynchronize(b->stream);  // (the pinned staging may still feed an upload)
  if (b->graph) cudaGraphExecDestroy(b->graph);
  if (b->tmpl) cudaGraphDestroy(b->tmpl);
  if (b->ev) cudaEventDestroy(b->ev);
  for (int k = 0; k < 2; ++k) {
    if (b->stage[k]) cudaFreeHost(b->stage[k]);
    if (b->stage_ev[k]) cudaEventDestroy(b->stage_ev[k]);
  }
  delete b;
  return SMC_OK;
}

const char* smc_slots_last_error(const smc_slots* b) { return b ? b->err.c_str() : g_slots_err.c_str(); }

}  // extern "C"
