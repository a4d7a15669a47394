// smc_checkpoint.cu -- checkpoint / resume of a sampler (C-ABI in
// include/smc.h).  The state of Algorithm 2 between iterations is the
// particles, their log-weights and log-targets, and the device state block
// (iteration index t, LSE_{t-1}, the recycling sums of eq. (6), the last
// statistics).  Random numbers are counter-based (Philox keyed by seed,
// iteration and particle), so a sampler restored from a checkpoint taken at
// iteration t continues exactly as the original would have: same bits.
//
// Host buffer layout: CkptHeader | DevState | x (N x D) | log pi (N) | log w (N).
#include <cstring>
#include <string>

#include "smc_host.h"
#include "smc_trace.h"

using namespace smc;

namespace {

struct CkptHeader {
  char magic[8];
  uint32_t version;
  int32_t d;
  int64_t n;
  int32_t dtype;
  int32_t target;
  uint64_t seed;
  uint64_t state_bytes;
  uint64_t row_bytes;
};

static_assert(sizeof(CkptHeader) == 56, "checkpoint header layout");

constexpr char kMagic[8] = {'S', 'M', 'C', 'C', 'K', 'P', 'T', '1'};

size_t ckpt_bytes(const smc_sampler* h) {
  return sizeof(CkptHeader) + sizeof(DevState) + size_t(h->n) * (h->esize * h->d + h->esize + sizeof(double));
}

int ck_fail(smc_sampler* h, int code, const char* msg) {
  if (h) h->err = msg;
  return code;
}

}  // namespace

extern "C" {

int smc_checkpoint_bytes(const smc_sampler* h, size_t* bytes) {
  if (!h || !bytes) return SMC_EINVAL;
  *bytes = ckpt_bytes(h);
  return SMC_OK;
}

int smc_checkpoint_save(smc_sampler* h, void* host_dst, size_t bytes) {
  SMC_RANGE("smc_checkpoint_save");
  if (!h || !host_dst) return ck_fail(h, SMC_EINVAL, "null argument");
  if (bytes < ckpt_bytes(h)) return ck_fail(h, SMC_EINVAL, "checkpoint buffer too small");
  char* p = static_cast<char*>(host_dst);
  CkptHeader hd{};
  std::memcpy(hd.magic, kMagic, sizeof kMagic);
  hd.version = 1;
  hd.d = h->d;
  hd.n = h->n;
  hd.dtype = h->dtype;
  hd.target = h->cfg.target;
  hd.seed = h->cfg.seed;
  hd.state_bytes = sizeof(DevState);
  hd.row_bytes = h->esize * h->d;
  std::memcpy(p, &hd, sizeof hd);
  p += sizeof hd;
  // the state block first (it says which buffer holds the particles); all
  // copies are ordered after the work already queued on the sampler's stream
  DevState* st = reinterpret_cast<DevState*>(p);
  cudaError_t e = materialize(h);  // (a deferred redistribution completed first)
  if (e == cudaSuccess) e = cudaMemcpyAsync(st, h->st, sizeof(DevState), cudaMemcpyDeviceToHost, h->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
  if (e != cudaSuccess) return ck_fail(h, SMC_ECUDA, cudaGetErrorString(e));
  if (st->err != SMC_OK) return ck_fail(h, st->err, "the sampler holds an unreported error: nothing saved");
  p += sizeof(DevState);
  const int cur = st->cur;
  const size_t xb = size_t(h->n) * h->esize * h->d, lb = size_t(h->n) * h->esize;
  e = cudaMemcpyAsync(p, h->x[cur], xb, cudaMemcpyDeviceToHost, h->stream);
  if (e == cudaSuccess) e = cudaMemcpyAsync(p + xb, h->lp[cur], lb, cudaMemcpyDeviceToHost, h->stream);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(p + xb + lb, h->logw, size_t(h->n) * sizeof(double), cudaMemcpyDeviceToHost, h->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
  if (e != cudaSuccess) return ck_fail(h, SMC_ECUDA, cudaGetErrorString(e));
  return SMC_OK;
}

int smc_checkpoint_load(smc_sampler* h, const void* host_src, size_t bytes) {
  SMC_RANGE("smc_checkpoint_load");
  if (!h || !host_src) return ck_fail(h, SMC_EINVAL, "null argument");
  if (bytes < ckpt_bytes(h)) return ck_fail(h, SMC_EINVAL, "checkpoint buffer too small for this sampler");
  const char* p = static_cast<const char*>(host_src);
  CkptHeader hd;
  std::memcpy(&hd, p, sizeof hd);
  if (std::memcmp(hd.magic, kMagic, sizeof kMagic) != 0 || hd.version != 1)
    return ck_fail(h, SMC_EINVAL, "not a checkpoint of this format");
  if (hd.n != h->n || hd.d != h->d || hd.dtype != h->dtype || hd.target != h->cfg.target ||
      hd.seed != h->cfg.seed || hd.state_bytes != sizeof(DevState) || hd.row_bytes != h->esize * h->d)
    return ck_fail(h, SMC_EINVAL, "checkpoint taken from a sampler of another configuration");
  p += sizeof hd;
  // the state block as saved, the particles in buffer 0, no pending outputs
  DevState st;
  std::memcpy(&st, p, sizeof st);
  p += sizeof st;
  st.cur = 0;
  st.err = 0;
  st.pending = 0;
  // the run-start arrays of this sampler are reset below (both clean, the
  // first in use), whatever the saving sampler's were
  st.rs_dirty = 0;
  st.rs_w = 0;
  st.trace = nullptr;
  st.mean_out = nullptr;
  st.fhat_out = nullptr;
  st.cov_out = nullptr;
  const size_t xb = size_t(h->n) * h->esize * h->d, lb = size_t(h->n) * h->esize;
  // stream-ordered copies, complete before the call returns (the host buffer
  // may be released afterwards)
  // (a redistribution this sampler left pending is completed first, which
  // also clears its run starts)
  cudaError_t e = materialize(h);
  if (e == cudaSuccess) e = cudaMemsetAsync(h->rs, 0xFF, size_t(h->n) * sizeof(int32_t), h->stream);
  if (e == cudaSuccess && h->rs_alt)
    e = cudaMemsetAsync(h->rs_alt, 0xFF, size_t(h->n) * sizeof(int32_t), h->stream);
  if (e == cudaSuccess) e = cudaMemcpyAsync(h->st, &st, sizeof st, cudaMemcpyHostToDevice, h->stream);
  if (e == cudaSuccess) e = cudaMemcpyAsync(h->x[0], p, xb, cudaMemcpyHostToDevice, h->stream);
  if (e == cudaSuccess) e = cudaMemcpyAsync(h->lp[0], p + xb, lb, cudaMemcpyHostToDevice, h->stream);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(h->logw, p + xb + lb, size_t(h->n) * sizeof(double), cudaMemcpyHostToDevice, h->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
  if (e != cudaSuccess) return ck_fail(h, SMC_ECUDA, cudaGetErrorString(e));
  return SMC_OK;
}

}  // extern "C"
