// k_nearly_sort.cu -- Sequential Nearly Sort (Algorithm 8, Sec. 4.2) as a
// data-parallel stable partition, the local step of the paper's N-R
// redistribute (Algorithm 9), kept as a comparison for the gather design.
//
// Algorithm 8 walks the keys once with two cursors: a positive key (and its
// row) goes to the next free slot from the right end, any other key to the
// next free slot from the left end.  With P_i = #{j < i : ncopies_j > 0} the
// slot of element i is therefore
//     N - 1 - P_i  if ncopies_i > 0,      i - P_i  otherwise,
// which every element computes independently once P_i is known: a
// reduce-then-scan over tiles of 4096 keys (count, scan of the tile counts,
// scatter), no waits between blocks.  The scatter pass copies the rows
// warp-cooperatively: consecutive lanes move consecutive 16/8/4-byte words of
// consecutive source rows, whose destinations are runs of consecutive slots
// (ascending for the left part, descending for the right part).
#include "smc_internal.cuh"
#include "smc_kernels.h"

namespace smc {

namespace {

constexpr int kNsThreads = 256;
constexpr int kNsPerThread = kNsTile / kNsThreads;  // 16 consecutive keys per thread
static_assert(kNsPerThread == 16, "four int4 loads per thread");

// Loads the thread's 16 keys (guarded at the ragged end); returns the number
// of positive ones.
__device__ __forceinline__ int load_keys(const int32_t* __restrict__ nc, int64_t n, int64_t first, int k[16]) {
  int cnt = 0;
  if (first + 16 <= n) {
    const int4* p = reinterpret_cast<const int4*>(nc + first);
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const int4 v = __ldg(p + q);
      k[4 * q] = v.x;
      k[4 * q + 1] = v.y;
      k[4 * q + 2] = v.z;
      k[4 * q + 3] = v.w;
    }
  } else {
#pragma unroll
    for (int j = 0; j < 16; ++j) k[j] = first + j < n ? nc[first + j] : 0;
  }
#pragma unroll
  for (int j = 0; j < 16; ++j) cnt += (first + j < n && k[j] > 0) ? 1 : 0;
  return cnt;
}

__global__ void __launch_bounds__(kNsThreads) k_ns_count(NearlySortArgs a) {
  __shared__ int s_w[kNsThreads / 32];
  const int64_t first = int64_t(blockIdx.x) * kNsTile + int64_t(threadIdx.x) * kNsPerThread;
  int k[16];
  int c = load_keys(a.ncopies, a.n, first, k);
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) c += __shfl_xor_sync(0xffffffffu, c, o);
  if ((threadIdx.x & 31) == 0) s_w[threadIdx.x >> 5] = c;
  __syncthreads();
  if (threadIdx.x == 0) {
    int t = 0;
    for (int w = 0; w < kNsThreads / 32; ++w) t += s_w[w];
    a.tile_count[blockIdx.x] = t;
  }
}

// Exclusive scan of the tile counts by one block: thread t sums a contiguous
// chunk of tiles, the chunk sums are scanned, the chunk is rewritten as
// prefixes.
__global__ void __launch_bounds__(1024) k_ns_scan(NearlySortArgs a) {
  __shared__ uint64_t scratch[33];
  const int per = (a.ntiles + blockDim.x - 1) / blockDim.x;
  const int lo = min(a.ntiles, int(threadIdx.x) * per), hi = min(a.ntiles, lo + per);
  uint64_t s = 0;
  for (int j = lo; j < hi; ++j) s += uint64_t(a.tile_count[j]);
  uint64_t total;
  uint64_t run = block_excl_scan_u64(s, scratch, &total);
  for (int j = lo; j < hi; ++j) {
    const int c = a.tile_count[j];
    a.tile_base[j] = int32_t(run);
    run += uint64_t(c);
  }
}

template <typename VT>
__global__ void __launch_bounds__(kNsThreads) k_ns_scatter(NearlySortArgs a) {
  __shared__ uint64_t scratch[33];
  __shared__ int32_t s_dst[kNsTile];
  const int64_t tile0 = int64_t(blockIdx.x) * kNsTile;
  const int64_t first = tile0 + int64_t(threadIdx.x) * kNsPerThread;
  int k[16];
  const int c = load_keys(a.ncopies, a.n, first, k);
  uint64_t tot;
  const int64_t before = int64_t(a.tile_base[blockIdx.x]) + int64_t(block_excl_scan_u64(uint64_t(c), scratch, &tot));
  // slots of the thread's keys; the keys themselves travel with them
  int64_t p = before;
#pragma unroll
  for (int j = 0; j < 16; ++j) {
    const int64_t i = first + j;
    if (i < a.n) {
      const bool right = k[j] > 0;
      const int64_t dst = right ? a.n - 1 - p : i - p;
      p += right ? 1 : 0;
      s_dst[threadIdx.x * kNsPerThread + j] = int32_t(dst);
      a.ncopies_out[dst] = k[j];
    }
  }
  __syncthreads();
  // rows: warp w moves source rows [w * 512, (w + 1) * 512) of the tile
  const int rows_tile = int(a.n - tile0 < kNsTile ? a.n - tile0 : int64_t(kNsTile));
  constexpr int kRowsPerWarp = kNsTile / (kNsThreads / 32);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int r0 = warp * kRowsPerWarp;
  const int rows_w = max(0, min(kRowsPerWarp, rows_tile - r0));
  const int vpr = a.row_bytes / int(sizeof(VT));
  const int units = rows_w * vpr;
  const VT* __restrict__ in = static_cast<const VT*>(a.in);
  VT* __restrict__ out = static_cast<VT*>(a.out);
  constexpr int kU = 4;  // words in flight per lane
  for (int u0 = 0; u0 < units; u0 += 32 * kU) {
    VT v[kU];
    int64_t d[kU];
#pragma unroll
    for (int q = 0; q < kU; ++q) {
      const int u = u0 + q * 32 + lane;
      d[q] = -1;
      if (u < units) {
        const int r = u / vpr, w = u - r * vpr;
        const int lr = r0 + r;
        v[q] = in[size_t(tile0 + lr) * size_t(vpr) + size_t(w)];
        d[q] = int64_t(s_dst[lr]) * vpr + w;
      }
    }
#pragma unroll
    for (int q = 0; q < kU; ++q)
      if (d[q] >= 0) out[d[q]] = v[q];
  }
}

}  // namespace

int nearly_sort_tiles(int64_t n) { return int((n + kNsTile - 1) / kNsTile); }

cudaError_t launch_nearly_sort(const NearlySortArgs& a, cudaStream_t s) {
  k_ns_count<<<a.ntiles, kNsThreads, 0, s>>>(a);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  k_ns_scan<<<1, 1024, 0, s>>>(a);
  e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  if (a.row_bytes % 16 == 0)
    k_ns_scatter<uint4><<<a.ntiles, kNsThreads, 0, s>>>(a);
  else if (a.row_bytes % 8 == 0)
    k_ns_scatter<uint2><<<a.ntiles, kNsThreads, 0, s>>>(a);
  else
    k_ns_scatter<uint32_t><<<a.ntiles, kNsThreads, 0, s>>>(a);
  return cudaGetLastError();
}

}  // namespace smc
