// smc_noalloc.cu -- a stateless redistribute that needs no workspace from the
// caller.
//
// smc_redistribute_raw wants a device workspace (the exclusive offsets of the
// copy counts, the block sums and the first source row of every output tile).
// Some callers cannot provide one: a plug-in that is handed only its input and
// output buffers, code running inside a framework whose memory pool owns every
// device allocation, or a real-time loop that forbids allocation once it has
// started.  For them this file keeps that scratch in a file-scope device array
// of fixed size, so the entry point below performs no allocation of any kind.
//
// Limits and sharing rules:
//  * n <= SMC_NOALLOC_MAX_N (2^20 rows); larger n is rejected with SMC_EINVAL.
//  * The array (about 4.2 MB) exists once per GPU that loads the library and
//    stays resident until the process exits.
//  * Every call on a device uses the same array and leaves its contents behind;
//    the only word that has to start at zero (the error word) is cleared by
//    each call.  Calls whose work overlaps on the GPU (different streams, no
//    ordering between them) race on the array and give undefined results.
//  * The first call on each device looks up the array's device address
//    (cudaGetSymbolAddress) with that device current; make that first call
//    before any stream capture.
//  * That address is kept for the rest of the process.  A device reset
//    (cudaDeviceReset, or any other reset of the primary context) frees the
//    array's old storage, so this entry point must not be used on a device
//    after such a reset.
#include <mutex>
#include <string>

#include "smc_internal.cuh"
#include "smc_kernels.h"

namespace {

constexpr size_t kAl = 256;
constexpr size_t up(size_t v) { return (v + kAl - 1) / kAl * kAl; }
constexpr int64_t kMaxN = SMC_NOALLOC_MAX_N;
constexpr int64_t kBlocks = (kMaxN + smc::kQTile - 1) / smc::kQTile;
constexpr int64_t kTiles = (kMaxN + smc::kRTile - 1) / smc::kRTile;
// fixed layout, sized for kMaxN: state | block sums | block prefixes | run starts | tile starts
constexpr size_t kAtState = 0;
constexpr size_t kAtPart = up(sizeof(smc::DevState));
constexpr size_t kAtBase = kAtPart + up(size_t(kBlocks) * 8);
constexpr size_t kAtRun = kAtBase + up(size_t(kBlocks) * 8);
constexpr size_t kAtTile = kAtRun + up(size_t(kMaxN) * 4);
constexpr size_t kBytes = kAtTile + up(size_t(kTiles + 1) * 4);

}  // namespace

// The scratch.  In host code this name is only a host-side stand-in; kernels
// must be given the device address obtained below.
static __device__ __align__(256) unsigned char g_redistribute_scratch[kBytes];

namespace {

// Device address of the scratch on the current device, looked up once per
// device with that device current.
cudaError_t scratch_address(char** out) {
  static std::mutex mu;
  static char* addr[128] = {nullptr};
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= 128) return cudaErrorInvalidDevice;
  std::lock_guard<std::mutex> lock(mu);
  if (!addr[dev]) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_redistribute_scratch);
    if (e != cudaSuccess) return e;
    addr[dev] = static_cast<char*>(p);
  }
  *out = addr[dev];
  return cudaSuccess;
}

int noalloc_fail(int code, const std::string& msg) {
  smc::set_global_error(msg.c_str());  // reported by smc_last_error(NULL)
  return code;
}

}  // namespace

extern "C" int smc_redistribute_raw_noalloc(int64_t n, int32_t row_bytes, const int32_t* ncopies_dev,
                                            const void* in_dev, void* out_dev, int32_t* status_dev,
                                            smc_stream_t stream) {
  using namespace smc;
  if (n < 1) return noalloc_fail(SMC_EINVAL, "n must be >= 1");
  if (n > kMaxN)
    return noalloc_fail(SMC_EINVAL, "n exceeds SMC_NOALLOC_MAX_N (1048576) for the allocation-free redistribute; "
                                    "use smc_redistribute_raw with a caller-provided workspace");
  if (row_bytes < 4 || row_bytes % 4) return noalloc_fail(SMC_EINVAL, "row_bytes must be a positive multiple of 4");
  if (!ncopies_dev || !in_dev || !out_dev) return noalloc_fail(SMC_EINVAL, "null pointer");
  const uintptr_t va = row_bytes % 16 == 0 ? 16 : (row_bytes % 8 == 0 ? 8 : 4);
  if ((reinterpret_cast<uintptr_t>(in_dev) % va) || (reinterpret_cast<uintptr_t>(out_dev) % va))
    return noalloc_fail(SMC_EINVAL, "rows misaligned");
  char* ws = nullptr;
  cudaError_t e = scratch_address(&ws);
  if (e != cudaSuccess) return noalloc_fail(SMC_ECUDA, std::string("cudaGetSymbolAddress: ") + cudaGetErrorString(e));
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  DevState* st = reinterpret_cast<DevState*>(ws + kAtState);
  NcScanArgs a{};
  a.n = n;
  a.ncopies = ncopies_dev;
  a.part = reinterpret_cast<uint64_t*>(ws + kAtPart);
  a.cbase = reinterpret_cast<uint64_t*>(ws + kAtBase);
  a.runstart = reinterpret_cast<int32_t*>(ws + kAtRun);
  a.tile_src = reinterpret_cast<int32_t*>(ws + kAtTile);
  a.clear_rs = 1;  // (the reduce pass resets the run starts: no separate pass)
  a.nblocks = int32_t((n + kQTile - 1) / kQTile);
  a.ntiles = int32_t((n + kRTile - 1) / kRTile);
  a.st = st;
  RedistArgs r{};
  r.n = n;
  r.row_bytes = row_bytes;
  r.lp_bytes = 0;
  r.runstart = a.runstart;
  r.tile_src = a.tile_src;
  r.ntiles = a.ntiles;
  r.force = 1;
  r.x_in[0] = r.x_in[1] = in_dev;
  r.x_out[0] = r.x_out[1] = out_dev;
  r.logw = nullptr;
  r.st = st;
  r.stateful = 0;
  e = cudaMemsetAsync(&st->err, 0, sizeof(int32_t), s);
  if (e == cudaSuccess) e = launch_nc_reduce(a, s);
  if (e == cudaSuccess) e = launch_nc_finalize(a, s);
  if (e == cudaSuccess) e = launch_nc_scan(a, s);
  if (e == cudaSuccess) e = launch_redistribute(r, s);
  if (e == cudaSuccess && status_dev)
    e = cudaMemcpyAsync(status_dev, &st->err, sizeof(int32_t), cudaMemcpyDeviceToDevice, s);
  if (e != cudaSuccess) return noalloc_fail(SMC_ECUDA, std::string("launch: ") + cudaGetErrorString(e));
  return SMC_OK;
}
