// k_resample.cu -- resampling and redistribute on sm_103a.
//
//  * Quantisation of the weights to 64-bit fixed point, W_i = E(log w_i - m)
//    >> (62 - F), with exact 128-bit sums S, sum W^2, sum E (reduce pass; the
//    partial sums of eq. (7) from the rows, or from the move kernel's tile
//    records), the N_eff decision S^2 < N* sum W^2 (eq. (1) against the
//    threshold N* of Algorithm 2; 2 S^2 < N sum W^2 for N* = N/2), LSE_t and
//    log c_t (eqs. (2), (8)) in a single-block finaliser.
//  * Systematic resampling (MVR, Algorithm 4 line 1) on the integer CDF:
//    off_i = floor((N C_{i-1} + U)/S) is the exclusive cumulative sum of
//    ncopies and ncopies_i = off_{i+1} - off_i (eq. (9) holds by telescoping);
//    a block-local scan of W plus the block prefix gives C_i.
//  * Redistribute (Algorithm 5 as the definition of the output): output-tile
//    parallel gather.  The scan pass writes runstart[off_i] = i for every
//    survivor (a run of ncopies_i output rows starts at off_i) and the source
//    row of each tile's first output row; a tile of 2048 output rows loads its
//    slice of runstart (resetting it to -1 for the next iteration), a block
//    max-scan turns it into src(k), and the rows are copied with 16-byte
//    vector loads/stores.  Every tile does the same bounded work whatever the
//    weights.  Replaces the paper's MPI nearly-sort and rotational shifts
//    (Sec. 4) with O(1) passes over the data.
#include <cmath>

#include "particle_bodies.cuh"
#include "smc_internal.cuh"
#include "smc_kernels.h"

namespace smc {

// Tables of the fixed-point exponential: [0, 64) ~2^63 2^(-j/64),
// [64, 128) ~2^63 2^(-j/4096).
__constant__ uint64_t c_T[128];

// floor(sqrt(n)) for n < 2^126 by Newton's iteration from above.
static uint64_t isqrt_newton(u128 n) {
  if (n == 0) return 0;
  u128 x = u128(1) << 64;  // >= sqrt(n) for n < 2^128
  while (true) {
    const u128 y = (x + n / x) >> 1;
    if (y >= x) break;
    x = y;
  }
  return uint64_t(x);
}

// c_0 = 2^62, c_b = isqrt(c_{b-1} 2^63) ~= 2^63 2^(-2^-b) for b = 1..12;
// T1[j] (T[j]) is the product of c_1..c_6 over the set bits of j (c_1 for the
// top bit), T2[j] (T[64 + j]) the same with c_7..c_12; every product is
// floored to 2^63 fixed point.
static void build_table(uint64_t T[128]) {
  uint64_t c[13];
  c[0] = 1ull << 62;
  for (int b = 1; b <= 12; ++b) c[b] = isqrt_newton(u128(c[b - 1]) << 63);
  for (int half = 0; half < 2; ++half) {
    for (int j = 0; j < 64; ++j) {
      uint64_t acc = 1ull << 63;
      for (int b = 1; b <= 6; ++b)
        if (j & (1 << (6 - b))) acc = uint64_t((u128(acc) * c[6 * half + b]) >> 63);
      T[64 * half + j] = acc;
    }
  }
}

cudaError_t upload_expfx_table() {
  static bool done[64] = {false};
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev >= 0 && dev < 64 && done[dev]) return cudaSuccess;
  uint64_t T[128];
  build_table(T);
  e = cudaMemcpyToSymbol(c_T, T, sizeof T);
  if (e == cudaSuccess && dev >= 0 && dev < 64) done[dev] = true;
  return e;
}

__device__ __forceinline__ void load_table(uint64_t* T) {
  if (threadIdx.x < 128) T[threadIdx.x] = c_T[threadIdx.x];
  __syncthreads();
}


// ---------------------------------------------------------------- state init
// reset value of Algorithm 4 line 3, -log N, from the exact log so that both
// implementations agree bit for bit
__global__ void k_state_init(DevState* st, int64_t n, int64_t t, int F) {
  if (threadIdx.x != 0) return;
  const double reset_logw = -det_log(double(n));
  st->t = t;
  st->cur = 0;
  st->flag = 0;
  st->err = 0;
  st->F = F;
  st->L = 1;
  st->m = 0.0;
  st->lse = 0.0;
  st->lse_prev = 0.0;
  st->logc = 0.0;
  st->ess = 0.0;
  st->reset_logw = reset_logw;
  st->S = st->U = 0;
  st->sw2_lo = st->sw2_hi = st->se_lo = st->se_hi = 0;
  st->recip = 0;
  st->rc_max = -INFINITY;
  st->rc_den = 0.0;
  for (int c = 0; c < kMaxD; ++c) st->rc_num[c] = st->mean[c] = 0.0;
  st->est_s = 0.0;
  st->trace = nullptr;
  st->trace_t0 = 0;
  st->mean_out = st->fhat_out = st->cov_out = nullptr;
  st->want_cov = 0;
  st->w_uniform = 0;
  st->est_ready = 0;
  st->pending = 0;
  st->rs_dirty = 0;
  st->rs_w = 0;
}

// ---------------------------------------------------------------- max of log w (stateless path)
// part[b] = {max, number of finite entries}; NaN is an error.
__global__ void __launch_bounds__(kQThreads) k_max_logw(const double* __restrict__ logw, int64_t n,
                                                       double* __restrict__ part, DevState* st) {
  __shared__ double shm[kQThreads / 32], shc[kQThreads / 32];
  double m = -INFINITY, cnt = 0.0;
  bool nan = false;
  const int64_t base = int64_t(blockIdx.x) * kQTile;
#pragma unroll 4
  for (int k = 0; k < kQItems; ++k) {
    const int64_t i = base + k * kQThreads + threadIdx.x;
    if (i < n) {
      const double v = logw[i];
      nan |= isnan(v);
      if (v > -INFINITY) cnt += 1.0;
      m = fmax(m, v);
    }
  }
  if (nan) record_error(st, SMC_ENONFINITE);
  m = warp_max(m);
  cnt = warp_sum(cnt);
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  if (lane == 0) {
    shm[wid] = m;
    shc[wid] = cnt;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    double mm = -INFINITY, cc = 0.0;
    for (int w = 0; w < kQThreads / 32; ++w) {
      mm = fmax(mm, shm[w]);
      cc += shc[w];
    }
    part[2 * blockIdx.x] = mm;
    part[2 * blockIdx.x + 1] = cc;
  }
}

// ---------------------------------------------------------------- quantise: reduce
// Per block of 4096 weights: the exact sums S = sum W, sum W^2, sum E, and
// (EST) the partial sums sum_i E_i x_i of the estimate of eq. (7), whose
// normalised weights are E_i / sum E (the fixed-point exp of log w_i - m).
__device__ __forceinline__ float u64_to_float_trunc(uint64_t v) {
  if (v == 0) return 0.0f;
  const int e = 63 - __clzll((long long)v);
  const uint32_t mant = e >= 23 ? uint32_t(v >> (e - 23)) : uint32_t(v << (23 - e));
  return __uint_as_float((uint32_t(e + 127) << 23) | (mant & 0x7FFFFFu));
}
__device__ __forceinline__ void weight_of(uint64_t E, float* w) { *w = u64_to_float_trunc(E); }
__device__ __forceinline__ void weight_of(uint64_t E, double* w) { *w = __ull2double_rn(E); }

// Loads of rows the kernel only reads (read-only path), or, in a kernel whose
// other blocks wrote them before a grid barrier, at the coherent level (L2).
template <bool COH, typename V>
__device__ __forceinline__ V ld_rows(const V* p) {
  if constexpr (COH)
    return __ldcg(p);
  else
    return __ldg(p);
}

template <bool COH, typename V>
__device__ __forceinline__ V ld_plain(const V* p) {
  if constexpr (COH)
    return __ldcg(p);
  else
    return *p;
}

// Shared memory of one quantise-reduce block (declared by the calling kernel).
struct QuantReduceSmem {
  uint64_t T[128];
  uint64_t sh[kQThreads / 32][5];
  double shx[kQThreads / 32][32];
};

template <typename ST, int DMAX, bool EST, bool COH = false>
__device__ __forceinline__ void quant_reduce_body(const QuantArgs& a, const int blk, QuantReduceSmem& sm) {
  uint64_t* const T = sm.T;
  uint64_t (*const sh)[5] = sm.sh;
  double (*const shx)[32] = sm.shx;
  load_table(T);
  const DevState* st = a.st;
  uint64_t sw = 0;
  u128 sw2 = 0, se = 0;
  ST acc[DMAX];
#pragma unroll
  for (int c = 0; c < DMAX; ++c) acc[c] = ST(0);
  const int d = a.d;
  // eq. (7) from the move kernel's tile records when it wrote them this
  // iteration, else from the rows
  const bool use_rec = EST && a.est_src && st->est_ready;
  if (!st->err) {
    const double m = st->m;
    const int sh_w = 62 - st->F;
    const int64_t base = int64_t(blk) * kQTile;
    const ST* __restrict__ x = static_cast<const ST*>(st->cur ? a.x[1] : a.x[0]);
    bool done = false;
    if constexpr (sizeof(ST) == 4) {  // (records exist for FP32 samplers only)
      if (use_rec) {
        // only log w is read: every load of the thread first (more bytes in
        // flight), then the arithmetic
        double lv[kQItems];
#pragma unroll
        for (int k = 0; k < kQItems; ++k) {
          const int64_t i = base + k * kQThreads + threadIdx.x;
          lv[k] = i < a.n ? a.logw[i] : 0.0;
        }
#pragma unroll
        for (int k = 0; k < kQItems; ++k) {
          const int64_t i = base + k * kQThreads + threadIdx.x;
          if (i < a.n) {
            const uint64_t E = expfx_a(__dsub_rn(m, lv[k]), T);
            const uint64_t W = E >> sh_w;
            a.wbuf[i] = W;
            sw += W;
            sw2 += u128(W) * W;
            se += E;
          }
        }
        done = true;
      }
    }
    if constexpr (COH && EST && DMAX <= 8) {
      // (the fused small-sampler iteration, rows written by other blocks of
      // the same launch: coherent loads, latency-bound) each group of four
      // items' log w and rows loaded first, then the arithmetic in the
      // same order as below
      if (!done && !use_rec) {
        for (int k0 = 0; k0 < kQItems; k0 += 4) {
          double lv[4];
          ST xr[4][DMAX];
#pragma unroll
          for (int u = 0; u < 4; ++u) {
            const int64_t i = base + (k0 + u) * kQThreads + threadIdx.x;
            lv[u] = i < a.n ? __ldcg(a.logw + i) : 0.0;
#pragma unroll
            for (int c = 0; c < DMAX; ++c) xr[u][c] = (i < a.n && c < d) ? __ldcg(x + i * d + c) : ST(0);
          }
#pragma unroll
          for (int u = 0; u < 4; ++u) {
            const int64_t i = base + (k0 + u) * kQThreads + threadIdx.x;
            if (i < a.n) {
              const uint64_t E = expfx_a(__dsub_rn(m, lv[u]), T);
              const uint64_t W = E >> sh_w;
              a.wbuf[i] = W;
              sw += W;
              sw2 += u128(W) * W;
              se += E;
              ST w;
              weight_of(E, &w);
#pragma unroll
              for (int c = 0; c < DMAX; ++c)
                if (c < d) acc[c] = fma(w, xr[u][c], acc[c]);
            }
          }
        }
        done = true;
      }
    }
    if (!done)
#pragma unroll 4
    for (int k = 0; k < kQItems; ++k) {
      const int64_t i = base + k * kQThreads + threadIdx.x;
      if (i < a.n) {
        const uint64_t E = expfx_a(__dsub_rn(m, ld_plain<COH>(a.logw + i)), T);
        const uint64_t W = E >> sh_w;
        a.wbuf[i] = W;
        sw += W;
        sw2 += u128(W) * W;
        se += E;
        if (EST && !use_rec) {
          ST w;
          weight_of(E, &w);
          const ST* row = x + i * d;
          if (d == DMAX && (DMAX * sizeof(ST)) % 16 == 0) {
#pragma unroll
            for (int v = 0; v < int(DMAX * sizeof(ST) / 16); ++v) {
              const float4 f = ld_rows<COH>(reinterpret_cast<const float4*>(row) + v);
              const ST* fv = reinterpret_cast<const ST*>(&f);
#pragma unroll
              for (int u = 0; u < int(16 / sizeof(ST)); ++u) {
                const int c = v * int(16 / sizeof(ST)) + u;
                acc[c] = fma(w, fv[u], acc[c]);
              }
            }
          } else {
#pragma unroll
            for (int c = 0; c < DMAX; ++c)
              if (c < d) acc[c] = fma(w, ld_plain<COH>(row + c), acc[c]);
          }
        }
      }
    }
  }
  sw = warp_sum(sw);
  sw2 = warp_sum_u128(sw2);
  se = warp_sum_u128(se);
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  if (lane == 0) {
    sh[wid][0] = sw;
    sh[wid][1] = uint64_t(sw2);
    sh[wid][2] = uint64_t(sw2 >> 64);
    sh[wid][3] = uint64_t(se);
    sh[wid][4] = uint64_t(se >> 64);
  }
  if (EST && !use_rec) {
    // warp sums in the state precision (the FP64 pipe is scarce), then FP64
#pragma unroll
    for (int c = 0; c < DMAX; ++c) {
      if (c < d) {
        const ST v = warp_sum(acc[c]);
        if (lane == 0) shx[wid][c] = double(v);
      }
    }
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    uint64_t tw = 0;
    u128 t2 = 0, te = 0;
    for (int w = 0; w < kQThreads / 32; ++w) {
      tw += sh[w][0];
      t2 += (u128(sh[w][2]) << 64) | sh[w][1];
      te += (u128(sh[w][4]) << 64) | sh[w][3];
    }
    uint64_t* q = a.qpart + 5 * int64_t(blk);
    q[0] = tw;
    q[1] = uint64_t(t2);
    q[2] = uint64_t(t2 >> 64);
    q[3] = uint64_t(te);
    q[4] = uint64_t(te >> 64);
  }
  if (EST && !use_rec && threadIdx.x < d) {
    double v = 0.0;
    for (int w = 0; w < kQThreads / 32; ++w) v += shx[w][threadIdx.x];
    static_cast<ST*>(a.xpart)[int64_t(blk) * d + threadIdx.x] = ST(v);
  }
  if (use_rec && wid == 0) {
    // eq. (7) partials of this block from the move kernel's tile records
    // {M_r, sum e^{log w - M_r} x}: scaled to the units of E_i (2^62 e^{log w - m})
    // and added over the block's tiles by a fixed shuffle tree
    constexpr int kTiles = kQTile / kEstTile;
    static_assert(kTiles <= 32, "one lane per tile record");
    const int64_t ntile = (a.n + kEstTile - 1) / kEstTile;
    const int64_t jt = int64_t(blk) * kTiles + lane;
    const bool have = lane < kTiles && jt < ntile && !st->err;
    const double* rec = a.epart + jt * (1 + d);
    const double Mr = have ? rec[0] : -INFINITY;
    const float f = Mr == -INFINITY ? 0.0f : __expf(float(Mr - st->m)) * 0x1p62f;
    for (int c = 0; c < d; ++c) {
      const ST v = warp_sum(ST(have ? f * float(rec[1 + c]) : 0.0f));
      if (lane == 0) static_cast<ST*>(a.xpart)[int64_t(blk) * d + c] = v;
    }
  }
}

template <typename ST, int DMAX, bool EST>
__global__ void __launch_bounds__(kQThreads) k_quant_reduce(QuantArgs a) {
  __shared__ QuantReduceSmem sm;
  quant_reduce_body<ST, DMAX, EST>(a, blockIdx.x, sm);
}

__device__ __forceinline__ double u128_to_double(u128 v) {
  return double(uint64_t(v >> 64)) * 0x1p64 + double(uint64_t(v));
}

// ---------------------------------------------------------------- quantise: finalise
// Single block: totals, exclusive prefix of the block sums (the CDF base of
// each scan block), decision, systematic offset U, division constants, LSE,
// N_eff, log c_t, and the statistics record.
__device__ __forceinline__ void quant_finalize_body(const QuantArgs& a, const int set_lse_prev) {
  __shared__ uint64_t scratch[33];
  __shared__ uint64_t shw[32], sh2l[32], sh2h[32], shel[32], sheh[32];
  DevState* st = a.st;
  const int nb = a.nblocks;
  uint64_t tw = 0;
  u128 t2 = 0, te = 0;
#pragma unroll 4
  for (int b = threadIdx.x; b < nb; b += blockDim.x) {
    const uint64_t* q = a.qpart + 5 * int64_t(b);
    tw += q[0];
    t2 += (u128(q[2]) << 64) | q[1];
    te += (u128(q[4]) << 64) | q[3];
  }
  tw = warp_sum(tw);
  t2 = warp_sum_u128(t2);
  te = warp_sum_u128(te);
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
  if (lane == 0) {
    shw[wid] = tw;
    sh2l[wid] = uint64_t(t2);
    sh2h[wid] = uint64_t(t2 >> 64);
    shel[wid] = uint64_t(te);
    sheh[wid] = uint64_t(te >> 64);
  }
  // exclusive scan of the block sums of W: contiguous chunk per thread
  const int chunk = (nb + blockDim.x - 1) / blockDim.x;
  const int b0 = threadIdx.x * chunk, b1 = min(nb, b0 + chunk);
  uint64_t local = 0;
#pragma unroll 4
  for (int b = b0; b < b1; ++b) local += a.qpart[5 * int64_t(b)];
  uint64_t total;
  uint64_t pre = block_excl_scan_u64(local, scratch, &total);  // contains __syncthreads
  for (int b = b0; b < b1; ++b) {
    a.cbase[b] = pre;
    pre += a.qpart[5 * int64_t(b)];
  }
  // eq. (7): f_t = sum_i E_i x_i / sum_i E_i from the per-block partial sums
  __shared__ double sxsum[kMaxD];
  const bool est = a.x[0] != nullptr && a.d > 0;
  if (est) {
    // logical thread j (of kFinThreads, whatever the block size) sums column
    // j % d over rows j / d, j / d + stride / d, ... in a fixed order
    // (deterministic, and the same in one-sampler and batched launches), in
    // the particle precision (the FP64 pipe is scarce); the per-thread
    // partials are then added in order per column
    const int stride = (kFinThreads / a.d) * a.d;
    const int64_t total_words = int64_t(nb) * a.d;
    __shared__ double tpart[kFinThreads];
    for (int lt = threadIdx.x; lt < kFinThreads; lt += blockDim.x) {
      double part = 0.0;
      if (lt < stride) {
        if (a.dtype == SMC_F64) {
          const double* xp = static_cast<const double*>(a.xpart);
          for (int64_t j = lt; j < total_words; j += stride) part += xp[j];
        } else {
          const float* xp = static_cast<const float*>(a.xpart);
          float v[8] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
          int64_t j = lt;
          const int64_t s1 = int64_t(stride), s8 = 8 * s1;
          // four rounds' loads in flight at once, then their additions in
          // round order (the same sums as one round at a time)
          for (; j + 3 * s8 + 7 * s1 < total_words; j += 4 * s8) {
            float tv[32];
#pragma unroll
            for (int r = 0; r < 32; ++r) tv[r] = xp[j + r * s1];
#pragma unroll
            for (int q = 0; q < 4; ++q)
#pragma unroll
              for (int u = 0; u < 8; ++u) v[u] += tv[8 * q + u];
          }
          for (; j + 7 * s1 < total_words; j += s8) {
#pragma unroll
            for (int u = 0; u < 8; ++u) v[u] += xp[j + u * s1];
          }
          for (; j < total_words; j += stride) v[0] += xp[j];
          part = double(((v[0] + v[1]) + (v[2] + v[3])) + ((v[4] + v[5]) + (v[6] + v[7])));
        }
      }
      tpart[lt] = part;
    }
    __syncthreads();
    // column c's stride / d partials (tpart[c + d j]) summed by warps
    // c, c + nw, ...: lane l adds j = l, l + 32, ... in order, then a fixed
    // shuffle tree -- deterministic, and a short FP64 dependency chain
    {
      const int per_col = stride / a.d;
      const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nwarps = blockDim.x >> 5;
      for (int c = wid; c < a.d; c += nwarps) {
        double t = 0.0;
        for (int j = lane; j < per_col; j += 32) t += tpart[c + a.d * j];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
        if (lane == 0) sxsum[c] = t;
      }
    }
    __syncthreads();
  }
  // eq. (7): the weighted mean, one column per thread
  {
    u128 se_all = 0;
    for (int w = 0; w < nw; ++w) se_all += (u128(sheh[w]) << 64) | shel[w];
    const double se_all_d = u128_to_double(se_all);
    if (est && !st->err && se_all_d > 0.0 && int(threadIdx.x) < a.d) {
      double* const mean_out = st->mean_out;  // (loaded before the store below)
      const double mc = sxsum[threadIdx.x] / se_all_d;
      st->mean[threadIdx.x] = mc;
      if (mean_out) mean_out[threadIdx.x] = mc;
    }
  }
  // the totals, then three independent chains on three lanes of warp 0 (the
  // same operations as one thread would do: the 128-bit division for the
  // copy counts, the logarithm of LSE, the division of N_eff), each a long
  // latency chain on this GPU
  if (threadIdx.x >= 32) return;
  // the state the record needs, loaded before the first store (one round
  // trip, overlapping the chains below; nothing else writes these fields
  // while this block finalises)
  const int err0 = st->err;
  const int64_t t_now = st->t, trace_t0 = st->trace_t0;
  const double m = st->m, lse_prev = st->lse_prev;
  smc_iter_stats* const trace = st->trace;
  uint64_t S = 0;
  u128 sw2 = 0, se = 0;
  for (int w = 0; w < nw; ++w) {
    S += shw[w];
    sw2 += (u128(sh2h[w]) << 64) | sh2l[w];
    se += (u128(sheh[w]) << 64) | shel[w];
  }
  const uint64_t n = uint64_t(a.n);
  const int lane0 = threadIdx.x;
  uint64_t R = 0;
  double lse = 0.0, se_d = 0.0, ess = 0.0;
  if (lane0 == 0) {
    // S >= 2^F = 2^(63 - ceil(log2 N)), so floor(N 2^64 / S) <= 2^(2 ceil(log2 N) + 1) fits 64 bits
    R = S ? uint64_t((u128(n) << 64) / S) : 0;
  } else if (lane0 == 1) {
    se_d = u128_to_double(se);
    lse = m + log(se_d * 0x1p-62);
  } else if (lane0 == 2) {
    const double Sd = double(S);
    ess = (S && sw2) ? Sd * Sd / u128_to_double(sw2) : 0.0;
  }
  lse = __shfl_sync(0xffffffffu, lse, 1);
  se_d = __shfl_sync(0xffffffffu, se_d, 1);
  ess = __shfl_sync(0xffffffffu, ess, 2);
  if (lane0 != 0) return;
  int flag = 0;
  if (!err0 && S > 0) {
    if (a.mode == SMC_RESAMPLE_ALWAYS)
      flag = 1;
    else if (a.mode == SMC_RESAMPLE_NEVER)
      flag = 0;
    else if (a.nstar > 0)  // N_eff < N*  <=>  S^2 < N* sum W^2 (Algorithm 2, line 7)
      flag = u128(S) * S < u128(uint64_t(a.nstar)) * sw2;
    else  // N* = N/2
      flag = (u128(S) * S * 2) < u128(n) * sw2;
  }
  const P4 r = stream_block(a.seed, uint64_t(t_now), kPurposeResample, 0xFFFFFFFFull, 0);
  const uint64_t r64 = (uint64_t(r.v[0]) << 32) | r.v[1];
  const uint64_t U = S ? __umul64hi(r64, S) : 0;
  const int L = S ? 64 - __clzll((long long)S) : 1;
  st->est_s = se_d * 0x1p-62;
  st->S = S;
  st->U = U;
  st->L = L;
  st->recip = R;
  st->sw2_lo = uint64_t(sw2);
  st->sw2_hi = uint64_t(sw2 >> 64);
  st->se_lo = uint64_t(se);
  st->se_hi = uint64_t(se >> 64);
  st->flag = flag;
  st->lse = lse;
  st->ess = ess;
  const double logc = lse - lse_prev;
  st->logc = logc;
  if (set_lse_prev) st->lse_prev = lse;
  smc_iter_stats rec;
  rec.lse = lse;
  rec.logc = logc;
  rec.ess = ess;
  rec.max_logw = m;
  rec.resampled = flag;
  rec.t = t_now;
  rec.survivors = 0;
  st->survivors = 0;
  st->last = rec;
  if (trace) {
    const int64_t idx = t_now - trace_t0 - 1;
    if (idx >= 0) trace[idx] = rec;
  }
  if (a.stats_out) *a.stats_out = rec;
}

__global__ void __launch_bounds__(kFinThreads) k_quant_finalize(QuantArgs a, int set_lse_prev) {
  quant_finalize_body(a, set_lse_prev);
}

// ---------------------------------------------------------------- copy-tile sources
// Every redistribute tile whose first output row k lies in a survivor's run
// [lo, hi) gets src = that survivor.  A thread writes the tile starts of its
// own short runs; a run spanning more than kBigRun tile starts (a heavily
// copied particle: in the one-hot case one run covers all N rows) is queued
// and written by the whole block after a barrier.  Every thread of the block
// must call tile_starts_flush.
constexpr int kBigRun = 4;
constexpr int kBigRuns = 64;
struct BigRuns {
  int count;
  int32_t src[kBigRuns];
  int64_t first[kBigRuns];  // first tile index
  int64_t tiles[kBigRuns];  // tile starts in the run
};

__device__ __forceinline__ void tile_starts_of_run(int32_t* __restrict__ tile_src, uint64_t lo, uint64_t hi,
                                                   uint64_t n, int32_t i, BigRuns& big) {
  const uint64_t kb0 = ((lo + kRTile - 1) / kRTile) * kRTile;
  const uint64_t end = hi < n ? hi : n;
  if (kb0 >= end) return;
  const uint64_t tiles = (end - kb0 + kRTile - 1) / kRTile;
  if (tiles > uint64_t(kBigRun)) {
    const int slot = atomicAdd(&big.count, 1);
    if (slot < kBigRuns) {
      big.src[slot] = i;
      big.first[slot] = int64_t(kb0 / kRTile);
      big.tiles[slot] = int64_t(tiles);
      return;
    }
  }
  for (uint64_t kb = kb0; kb < end; kb += kRTile) tile_src[kb / kRTile] = i;  // (short run, or the queue is full)
}

__device__ __forceinline__ void tile_starts_flush(int32_t* __restrict__ tile_src, BigRuns& big) {
  __syncthreads();
  const int nb = min(big.count, kBigRuns);
  for (int r = 0; r < nb; ++r)
    for (int64_t t = threadIdx.x; t < big.tiles[r]; t += blockDim.x) tile_src[big.first[r] + t] = big.src[r];
}

// ---------------------------------------------------------------- quantise: scan + ncopies
// Shared memory of the scan: the block's W staged for a blocked layout (then
// its copy counts), the block scan's scratch and the long-run queue.
struct ScanSmem {
  union {
    uint64_t w[kQThreads * 17];
    uint32_t o[kQThreads * 17];
  } buf;
  uint64_t scratch[33];
  BigRuns big;
};

// ITEMS consecutive items per thread (a block covers kQThreads ITEMS items):
// kQItems for the quantise blocks of kQTile; fewer for a sampler whose N fits
// one block of kQThreads ITEMS items (shorter per-thread chains, the same
// exact integers).
template <int ITEMS = kQItems>
__device__ __forceinline__ void quant_scan_body(const QuantArgs& a, const int blk, ScanSmem& sm) {
  static_assert(ITEMS >= 1 && ITEMS <= kQItems, "items per thread");
  const DevState* st = a.st;
  if (st->err || !(a.force || st->flag)) return;
  auto& buf = sm.buf;
  uint64_t* const scratch = sm.scratch;
  BigRuns& big = sm.big;
  if (threadIdx.x == 0) big.count = 0;
  const int64_t n = a.n;
  const int64_t base = int64_t(blk) * kQTile;
  // the quantised weights of the reduce pass, staged for a blocked layout
#pragma unroll 4
  for (int k = 0; k < ITEMS; ++k) {
    const int idx = k * kQThreads + threadIdx.x;
    const int64_t i = base + idx;
    buf.w[(idx / ITEMS) * (ITEMS + 1) + idx % ITEMS] = i < n ? a.wbuf[i] : 0ull;
  }
  __syncthreads();
  const uint64_t S = st->S, U = st->U;
  uint64_t W[ITEMS];
  uint64_t tsum = 0;
#pragma unroll
  for (int q = 0; q < ITEMS; ++q) {
    W[q] = buf.w[threadIdx.x * (ITEMS + 1) + q];
    tsum += W[q];
  }
  uint64_t btot;
  uint64_t C = a.cbase[blk] + block_excl_scan_u64(tsum, scratch, &btot);
  uint32_t ncv[ITEMS];
  unsigned nsurv = 0;
  // off_i = floor((N C_{i-1} + U) / S) for every item independently (no
  // serial dependency between items): the estimate mulhi(C, floor(N 2^64/S))
  // is at most 2 below floor(N C / S), and floor((N C + U)/S) is at most 1
  // above that; exact 128-bit comparisons fix the result.
  const uint64_t Rn = st->recip;  // floor(N 2^64 / S)
  // the run-start array, chosen once (its choice does not change during the
  // pass; read per store, it was a load after every store)
  int32_t* const rsa = rs_now(a.runstart, a.runstart_alt, st);
  auto quot = [&](uint64_t c) -> uint64_t {
    const u128 X = u128(n) * c + U;
    uint64_t qq = __umul64hi(c, Rn);
    u128 nxt = u128(qq + 1) * S;
#pragma unroll
    for (int it = 0; it < 3; ++it)
      if (nxt <= X) {
        ++qq;
        nxt += S;
      }
    return qq;
  };
  if (!a.ncopies) {
    // no copy counts to return (the sampler's own resampling): the items
    // one after another, each offset computed as it is needed -- the same
    // integers as below, from a short loop instead of ITEMS + 1 unrolled
    // quotients (which overflowed the instruction cache)
    const int64_t i0 = base + int64_t(threadIdx.x) * ITEMS;
    uint64_t cp = C, op = quot(C);
#pragma unroll 4
    for (int q = 0; q < ITEMS; ++q) {
      const uint64_t cn = cp + buf.w[threadIdx.x * (ITEMS + 1) + q];
      const uint64_t on = quot(cn);
      const int64_t i = i0 + q;
      if (on > op && i < n) {
        ++nsurv;
        if (a.write_rs) rsa[op] = int32_t(i);
        tile_starts_of_run(a.tile_src, op, on, uint64_t(n), int32_t(i), big);
      }
      cp = cn;
      op = on;
    }
    tile_starts_flush(a.tile_src, big);
    unsigned v = nsurv;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    if ((threadIdx.x & 31) == 0 && v) atomicAdd(&const_cast<DevState*>(st)->survivors, (unsigned long long)v);
    return;
  }
  uint64_t Cx[ITEMS + 1];
  Cx[0] = C;
#pragma unroll
  for (int q = 0; q < ITEMS; ++q) Cx[q + 1] = Cx[q] + W[q];
  uint64_t offs[ITEMS + 1];
#pragma unroll
  for (int q = 0; q <= ITEMS; ++q) offs[q] = quot(Cx[q]);
  const int64_t i0 = base + int64_t(threadIdx.x) * ITEMS;
#pragma unroll
  for (int q = 0; q < ITEMS; ++q) {
    const uint64_t lo = offs[q], hi = offs[q + 1];
    ncv[q] = uint32_t(hi - lo);
    const int64_t i = i0 + q;
    if (hi > lo && i < n) {
      ++nsurv;
      if (a.write_rs) rsa[lo] = int32_t(i);
      // every redistribute tile whose first output row lies in [lo, hi)
      tile_starts_of_run(a.tile_src, lo, hi, uint64_t(n), int32_t(i), big);
    }
  }
  tile_starts_flush(a.tile_src, big);
  {
    unsigned v = nsurv;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    if ((threadIdx.x & 31) == 0 && v) atomicAdd(&const_cast<DevState*>(st)->survivors, (unsigned long long)v);
  }
  __syncthreads();  // buf.w no longer read
  if (a.ncopies) {
#pragma unroll
    for (int q = 0; q < ITEMS; ++q) buf.o[threadIdx.x * (ITEMS + 1) + q] = ncv[q];
    __syncthreads();
#pragma unroll 4
    for (int k = 0; k < ITEMS; ++k) {
      const int idx = k * kQThreads + threadIdx.x;
      const int64_t i = base + idx;
      if (i < n) a.ncopies[i] = int32_t(buf.o[(idx / ITEMS) * (ITEMS + 1) + idx % ITEMS]);
    }
  }
}

__global__ void __launch_bounds__(kQThreads, 4) k_quant_scan(QuantArgs a) {
  __shared__ ScanSmem sm;
  quant_scan_body(a, blockIdx.x, sm);
}

// ---------------------------------------------------------------- standalone ncopies scan
// Thread t of a block owns the 16 consecutive entries [base + 16 t, +16) of
// the caller's ncopies, read with 16-byte loads when the vector is 16-byte
// aligned and the group is complete (scalar loads otherwise).
__device__ __forceinline__ void load_counts(const int32_t* __restrict__ nc, int64_t n, int64_t first, int32_t c[16]) {
  const bool vec = ((reinterpret_cast<uintptr_t>(nc) & 15) == 0) && first + 16 <= n;
  if (vec) {
    const int4* p = reinterpret_cast<const int4*>(nc + first);
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const int4 v = __ldg(p + q);
      c[4 * q] = v.x;
      c[4 * q + 1] = v.y;
      c[4 * q + 2] = v.z;
      c[4 * q + 3] = v.w;
    }
  } else {
#pragma unroll
    for (int q = 0; q < 16; ++q) c[q] = first + q < n ? nc[first + q] : 0;
  }
}

// Exclusive prefix of the block sums (cbase) and the check sum == n.
__device__ __forceinline__ void nc_finalize_body(const NcScanArgs& a) {
  __shared__ uint64_t scratch[33];
  const int nb = a.nblocks;
  const int chunk = (nb + blockDim.x - 1) / blockDim.x;
  const int b0 = threadIdx.x * chunk, b1 = min(nb, b0 + chunk);
  uint64_t local = 0;
  for (int b = b0; b < b1; ++b) local += a.part[b];
  uint64_t total;
  uint64_t pre = block_excl_scan_u64(local, scratch, &total);
  for (int b = b0; b < b1; ++b) {
    a.cbase[b] = pre;
    pre += a.part[b];
  }
  if (threadIdx.x == 0 && total != uint64_t(a.n)) record_error(a.st, SMC_EINVAL);
}

__global__ void __launch_bounds__(kQThreads) k_nc_reduce(NcScanArgs a) {
  __shared__ uint64_t sh[kQThreads / 32];
  __shared__ int bad;
  if (threadIdx.x == 0) bad = 0;
  __syncthreads();
  const int64_t first = int64_t(blockIdx.x) * kQTile + int64_t(threadIdx.x) * kQItems;
  int32_t c[kQItems];
  load_counts(a.ncopies, a.n, first, c);
  if (a.clear_rs) {
    // the run-start array starts at -1 for the scan: this block's slice
    // [4096 b, 4096 b + 4096) of it, with 16-byte stores (the array is
    // 256-byte aligned) and single stores for a partial last vector
    int4* rs4 = reinterpret_cast<int4*>(a.runstart);
    const int64_t v0 = int64_t(blockIdx.x) * (kQTile / 4);
#pragma unroll
    for (int u = 0; u < kQTile / 4 / kQThreads; ++u) {
      const int64_t v = v0 + u * kQThreads + threadIdx.x;
      if (4 * v + 3 < a.n)
        rs4[v] = make_int4(-1, -1, -1, -1);
      else
        for (int64_t k = 4 * v; k < a.n; ++k) a.runstart[k] = -1;
    }
  }
  uint64_t s = 0;
  bool neg = false;
#pragma unroll
  for (int q = 0; q < kQItems; ++q) {
    neg |= c[q] < 0;
    s += uint64_t(uint32_t(max(c[q], 0)));
  }
  if (neg) bad = 1;
  s = warp_sum(s);
  if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x == 0) {
    uint64_t t = 0;
    for (int w = 0; w < kQThreads / 32; ++w) t += sh[w];
    a.part[blockIdx.x] = t;
    if (bad) record_error(a.st, SMC_EINVAL);
  }
}

__global__ void __launch_bounds__(kFinThreads) k_nc_finalize(NcScanArgs a) { nc_finalize_body(a); }

// Run starts of the block's items.  The block's outputs form the window
// [cbase, cbase + total); the windows of the blocks are disjoint and tile
// [0, n).  A window that fits shared memory is assembled there (-1, then the
// run starts) and written out with coalesced stores.  A larger one, when the
// run-start array holds -1 everywhere on entry (a sampler's, kept clean by
// the copy that consumes it), gets its run starts stored one by one.
// Stamped calls (a.stamps set; the stateless entry points, whose array is
// not cleared): every copy tile that receives a run start is stamped, and
// the copy reads the run starts of stamped tiles only, so a larger window
// sets -1 over all of itself when it has at most kFillAll rows, else over
// its part of its two edge copy tiles and of every copy tile where it puts a
// run start (over all of itself if those overflow a queue), before its run
// starts -- every slice the copy reads is then written in this call.
constexpr int kNcWin = 8192;
constexpr int kFillTiles = 128;
constexpr uint64_t kFillAll = 1u << 17;

__global__ void __launch_bounds__(kQThreads) k_nc_scan(NcScanArgs a) {
  if (a.st->err) return;
  __shared__ int32_t win[kNcWin];
  __shared__ uint64_t scratch[33];
  __shared__ BigRuns big;
  __shared__ int s_nfill;
  __shared__ int64_t s_fill[kFillTiles];
  __shared__ int s_has[kNcWin / kRTile + 2];  // staged window: its tiles that receive a run start
  if (threadIdx.x == 0) {
    big.count = 0;
    s_nfill = 0;
  }
  if (threadIdx.x < kNcWin / kRTile + 2) s_has[threadIdx.x] = 0;
  const int64_t n = a.n;
  const uint64_t un = uint64_t(n);
  const int64_t base = int64_t(blockIdx.x) * kQTile;
  const int64_t i0 = base + int64_t(threadIdx.x) * kQItems;
  int32_t c[kQItems];
  load_counts(a.ncopies, n, i0, c);
  uint64_t tsum = 0;
#pragma unroll
  for (int q = 0; q < kQItems; ++q) tsum += uint32_t(c[q]);
  uint64_t btot;
  const uint64_t w0 = a.cbase[blockIdx.x];
  const uint64_t excl = block_excl_scan_u64(tsum, scratch, &btot);  // (block barriers inside)
  const uint64_t wend = min(w0 + btot, un);
  const bool staged = btot <= uint64_t(kNcWin);
  const bool stamped = a.stamps != nullptr;
  const bool fill_all = stamped && !staged && btot <= kFillAll;
  int32_t* __restrict__ rsa = rs_now(a.runstart, a.runstart_alt, a.st);
  if (staged) {
    for (int k = threadIdx.x; k < int(btot); k += blockDim.x) win[k] = -1;
  } else if (stamped && !fill_all && threadIdx.x == 0 && w0 < wend) {
    s_fill[0] = int64_t(w0 / kRTile);  // the edge tiles, shared with the neighbouring windows
    s_fill[1] = int64_t((wend - 1) / kRTile);
    s_nfill = 2;
  }
  __syncthreads();
  uint64_t o = w0 + excl;
  if (stamped && !staged) {
    if (!fill_all) {
      int64_t last = -1;
#pragma unroll
      for (int q = 0; q < kQItems; ++q) {
        if (c[q] > 0 && i0 + q < n && o < un && int64_t(o / kRTile) != last) {
          last = int64_t(o / kRTile);
          const int slot = atomicAdd(&s_nfill, 1);
          if (slot < kFillTiles) s_fill[slot] = last;
        }
        o += uint32_t(c[q]);
      }
      __syncthreads();
    }
    if (fill_all || s_nfill > kFillTiles) {
      for (uint64_t k = w0 + threadIdx.x; k < wend; k += blockDim.x) rsa[k] = -1;
    } else {
      for (int f = 0; f < s_nfill; ++f) {
        const uint64_t t0 = max(w0, uint64_t(s_fill[f]) * kRTile);
        const uint64_t t1 = min(wend, uint64_t(s_fill[f]) * kRTile + kRTile);
        for (uint64_t k = t0 + threadIdx.x; k < t1; k += blockDim.x) rsa[k] = -1;
      }
    }
    __syncthreads();  // every -1 before any run start
    o = w0 + excl;
  }
  const uint64_t tfirst = w0 / kRTile;
  int64_t stamped_tile = -1;  // (a thread's items are consecutive: one stamp per tile it reaches)
#pragma unroll
  for (int q = 0; q < kQItems; ++q) {
    const int64_t i = i0 + q;
    if (c[q] > 0 && i < n && o < un) {
      if (staged) {
        win[o - w0] = int32_t(i);
        if (stamped) s_has[o / kRTile - tfirst] = 1;
      } else {
        rsa[o] = int32_t(i);
        if (stamped && int64_t(o / kRTile) != stamped_tile) {
          stamped_tile = int64_t(o / kRTile);
          a.stamps[stamped_tile] = 1;
        }
      }
      tile_starts_of_run(a.tile_src, o, o + uint32_t(c[q]), un, int32_t(i), big);
    }
    o += uint32_t(c[q]);
  }
  tile_starts_flush(a.tile_src, big);  // (block barrier inside)
  if (staged) {
    int32_t* __restrict__ rs = rsa + w0;
    for (int k = threadIdx.x; w0 + uint64_t(k) < wend; k += blockDim.x) rs[k] = win[k];
    if (stamped && threadIdx.x < kNcWin / kRTile + 2 && s_has[threadIdx.x]) a.stamps[tfirst + threadIdx.x] = 1;
  }
}

// ---------------------------------------------------------------- redistribute
// Shared memory of one redistribute block, declared by the calling kernel so
// that kernels dispatching to several row sizes hold one copy.
struct RedistSmem {
  int32_t mark[kRTile];
  int32_t wsc[kRThreads / 32];
};

template <typename V, int CPR, int KU = 8, bool COH = false>
__device__ __forceinline__ void redistribute_body(const RedistArgs& a, const int blk, RedistSmem& sm) {
  int cur = 0;
  if (a.stateful) {
    if (a.use_pending ? !a.st->pending : !(a.force || a.st->flag)) return;
    cur = a.st->cur;
  }
  // after an error nothing is copied, but the runstart slice is still reset
  const bool failed = a.st->err != 0;
  int32_t* const mark = sm.mark;
  int32_t* const wsc = sm.wsc;
  const int64_t n = a.n;
  const int64_t k0 = int64_t(blk) * kRTile;
  const int len = int(n - k0 < kRTile ? n - k0 : int64_t(kRTile));
  // this tile's slice of runstart (survivor runs starting here), reset to -1
  // for the next resampling
  int32_t* __restrict__ rs = rs_now(a.runstart, a.runstart_alt, a.st) + k0;
  // (a stamped stateless call: an unstamped tile has no run starts, and its
  // slice is neither read nor reset)
  const bool read = !a.stamps || a.stamps[blk];
  {
    constexpr int kItems = kRTile / kRThreads;
    int32_t v[kItems];
#pragma unroll
    for (int u = 0; u < kItems; ++u) {
      const int k = threadIdx.x + u * kRThreads;
      v[u] = (read && k < len) ? rs[k] : -1;
    }
#pragma unroll
    for (int u = 0; u < kItems; ++u) {
      const int k = threadIdx.x + u * kRThreads;
      // reset only the entries that were set (rewriting the whole slice was
      // measured slower); stamped calls need no reset
      if (!a.stamps && k < len && v[u] >= 0) rs[k] = -1;
      mark[k] = v[u] < int32_t(n) ? v[u] : int32_t(n - 1);
    }
  }
  __syncthreads();
  if (failed) return;
  // the run covering the first output row may have started in an earlier tile
  if (threadIdx.x == 0) {
    const int32_t first = min(max(a.tile_src[blk], 0), int32_t(n - 1));
    mark[0] = max(mark[0], first);
  }
  __syncthreads();
  // inclusive max-scan of mark[0, kRTile): 16 consecutive entries per thread
  {
    constexpr int kItems = kRTile / kRThreads;
    const int b = threadIdx.x * kItems;
    int run = -1;
#pragma unroll
    for (int q = 0; q < kItems; ++q) run = max(run, mark[b + q]);
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    int incl = warp_incl_max_i32(run);
    if (lane == 31) wsc[wid] = incl;
    __syncthreads();
    int carry = -1;
    for (int w = 0; w < wid; ++w) carry = max(carry, wsc[w]);
    int excl = __shfl_up_sync(0xffffffffu, incl, 1);
    if (lane == 0) excl = -1;
    run = max(carry, excl);
#pragma unroll
    for (int q = 0; q < kItems; ++q) {
      run = max(run, mark[b + q]);
      mark[b + q] = run;
    }
  }
  __syncthreads();
  // copy rows: element e of the tile is chunk (e % cpr) of row (e / cpr)
  const int cpr = CPR > 0 ? CPR : a.row_bytes / int(sizeof(V));
  const V* __restrict__ in = static_cast<const V*>(cur ? a.x_in[1] : a.x_in[0]);
  V* __restrict__ out = static_cast<V*>(cur ? a.x_out[1] : a.x_out[0]) + k0 * cpr;
  const int total = len * cpr;
  constexpr int kU = KU;  // loads in flight per thread
  for (int e0 = threadIdx.x; e0 < total; e0 += kRThreads * kU) {
    V v[kU];
#pragma unroll
    for (int u = 0; u < kU; ++u) {
      const int e = e0 + u * kRThreads;
      if (e < total) {
        const int k = e / cpr, c = e - k * cpr;
        v[u] = ld_rows<COH>(in + int64_t(mark[k]) * cpr + c);
      }
    }
#pragma unroll
    for (int u = 0; u < kU; ++u) {
      const int e = e0 + u * kRThreads;
      if (e < total) out[e] = v[u];
    }
  }
  if (a.lp_bytes == 4) {
    const uint32_t* __restrict__ li = static_cast<const uint32_t*>(cur ? a.lp_in[1] : a.lp_in[0]);
    uint32_t* __restrict__ lo = static_cast<uint32_t*>(cur ? a.lp_out[1] : a.lp_out[0]) + k0;
    for (int k = threadIdx.x; k < len; k += kRThreads) lo[k] = ld_plain<COH>(li + mark[k]);
  } else if (a.lp_bytes == 8) {
    const uint64_t* __restrict__ li = static_cast<const uint64_t*>(cur ? a.lp_in[1] : a.lp_in[0]);
    uint64_t* __restrict__ lo = static_cast<uint64_t*>(cur ? a.lp_out[1] : a.lp_out[0]) + k0;
    for (int k = threadIdx.x; k < len; k += kRThreads) lo[k] = ld_plain<COH>(li + mark[k]);
  }
  if (a.logw) {
    const double reset = a.stateful ? a.st->reset_logw : a.reset_logw;
    double* __restrict__ lw = a.logw + k0;
    for (int k = threadIdx.x; k < len; k += kRThreads) lw[k] = reset;
  }
}

template <typename V, int CPR>
__global__ void __launch_bounds__(kRThreads) k_redistribute(RedistArgs a) {
  __shared__ RedistSmem sm;
  redistribute_body<V, CPR>(a, blockIdx.x, sm);
}

// ---------------------------------------------------------------- one-block samplers
// A sampler whose N fits one quantise block (N <= 4096) runs the reduce,
// finalise and scan passes as one kernel of one block, with the same bodies in
// the same order (the results are those of the three launches); one whose N
// fits one copy tile (N <= 2048) runs redistribute and commit as one kernel.
// For such samplers the launches, not the work, set the iteration's time.
template <typename ST, int DMAX, bool EST>
__global__ void __launch_bounds__(kQThreads) k_quant_small(QuantArgs a) {
  __shared__ QuantReduceSmem sm;
  quant_reduce_body<ST, DMAX, EST>(a, 0, sm);
  __syncthreads();  // the block's sums, W and estimate partials are written
  quant_finalize_body(a, 0);
  __syncthreads();  // S, U, the decision and the block base are written
  __shared__ ScanSmem ssm;
  quant_scan_body(a, 0, ssm);
}

template <typename V, int CPR>
__global__ void __launch_bounds__(kRThreads) k_redistribute_commit(RedistArgs a, int d, int force_flip, int recycle) {
  __shared__ RedistSmem sm;
  redistribute_body<V, CPR>(a, 0, sm);
  __syncthreads();
  if (threadIdx.x < 32) commit_warp(a.st, d, force_flip, recycle);
}

// ---------------------------------------------------------------- fused small-sampler iterations
// FP64 samplers of one quantise block and one copy tile (N <= 2048): k
// iterations of Algorithm 2 in one cooperative launch.  Every block runs its
// share of the move + reweight with the particle-to-thread map of the
// separate move launch (move_threads per block own particles); then block 0
// alone runs, in the order of the separate launches, t += 1, the maximum, the
// quantise reduce / finalise / scan, the copy and the commit -- the bodies of
// k_max_finalize, k_quant_small and k_redistribute_commit -- so the results
// are bit for bit those of the separate launches.  At this size an iteration
// is a chain of dependent FP64 operations (tens to thousands of cycles each
// on this GPU) and kernel boundaries; two grid barriers per iteration replace
// the five boundaries.
//
// The grid barrier (every block is resident: cooperative launch): one 64-bit
// count of arrivals, zeroed before the launch; a block's b-th barrier of the
// launch (b = 1, 2, ...) completes when the count reaches b (grid + extra).
// A block adds its arrival (release) and polls the count (acquire) -- for at
// most half a second of the global timer (and at most 2^24 polls), after
// which it records SMC_ETIMEOUT and the kernel returns.  extra: arrivals
// expected beyond the grid (0; 1 only in the stall test, where every wait
// runs out).
constexpr unsigned long long kBarrierNs = 500000000ull;
constexpr long long kBarrierPolls = 1ll << 24;

__device__ __forceinline__ unsigned long long ld_acquire_u64(const unsigned long long* p) {
  unsigned long long v;
  asm volatile("ld.acquire.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
  return v;
}

__device__ __forceinline__ void red_release_add_u64(unsigned long long* p, unsigned long long v) {
  asm volatile("red.release.gpu.global.add.u64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}

__device__ __forceinline__ unsigned long long global_ns() {
  unsigned long long v;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(v));
  return v;
}

__device__ __forceinline__ bool grid_barrier(unsigned long long* bar, unsigned long long& nbar, DevState* st,
                                             unsigned extra) {
  __shared__ int s_ok;
  ++nbar;
  __syncthreads();
  if (threadIdx.x == 0) {
    const unsigned long long target = nbar * (gridDim.x + extra);
    red_release_add_u64(bar, 1ull);
    int ok = 1;
    const unsigned long long t0 = global_ns();
    for (long long polls = 0; ld_acquire_u64(bar) < target; ++polls) {
      if (polls > kBarrierPolls || global_ns() - t0 > kBarrierNs) {
        record_error(st, SMC_ETIMEOUT);
        ok = 0;
        break;
      }
      __nanosleep(64);
    }
    __threadfence();
    s_ok = ok;
  }
  __syncthreads();
  return s_ok != 0;
}

// The stages' shared memory overlaps (each phase writes what it reads before
// reading it, and phases are separated by block barriers).
union SmallIterSmem {
  TargetSmem<double> ts;
  QuantReduceSmem q;
  ScanSmem sc;
  RedistSmem r;
};

template <int DMAX, typename V>
__global__ void __launch_bounds__(kQThreads) k_iterate_small(SmallIterArgs s) {
  __shared__ SmallIterSmem sm;
  TargetSmem<double>& ts = sm.ts;
  QuantReduceSmem& qsm = sm.q;
  RedistSmem& rsm = sm.r;
  DevState* st = s.a.st;
  unsigned long long* const bar = s.bar;
  unsigned long long nbar = 0;
  const unsigned extra = s.stall ? 1u : 0u;
  for (int it = 0; it < s.k; ++it) {
    move_reweight_generic_body<double, DMAX, true, true>(s.a, ts, blockIdx.x, gridDim.x, s.move_threads, 1);
    if (!grid_barrier(bar, nbar, st, extra)) return;
    if (blockIdx.x == 0) {
      if (threadIdx.x == 0) st->t += 1;
      __syncthreads();
      max_finalize_body(s.a.part, gridDim.x, st);
      __syncthreads();
      quant_reduce_body<double, DMAX, true, true>(s.q, 0, qsm);
      __syncthreads();
      quant_finalize_body(s.q, 0);
      __syncthreads();
      if (s.a.n <= kQThreads * 4)
        quant_scan_body<4>(s.q, 0, sm.sc);
      else
        quant_scan_body<8>(s.q, 0, sm.sc);
      if (!(s.stop_last && it + 1 == s.k)) {
        __syncthreads();
        redistribute_body<V, 0, 8, true>(s.r, 0, rsm);
        __syncthreads();
        if (threadIdx.x < 32) commit_warp(st, s.d, 0, 1);
      }
    }
    if (it + 1 < s.k && !grid_barrier(bar, nbar, st, extra)) return;
  }
}

bool small_iter_fits(int64_t n, int dtype) { return dtype == SMC_F64 && n <= kRTile && n <= kQTile; }

template <int DMAX>
static cudaError_t iterate_small_d(const SmallIterArgs& s, int blocks, cudaStream_t st) {
  SmallIterArgs a = s;
  void* args[] = {&a};
  const void* fn = (s.r.row_bytes % 16 == 0) ? reinterpret_cast<const void*>(&k_iterate_small<DMAX, uint4>)
                                             : reinterpret_cast<const void*>(&k_iterate_small<DMAX, uint2>);
  return cudaLaunchCooperativeKernel(fn, dim3(blocks), dim3(kQThreads), args, 0, st);
}

cudaError_t launch_iterate_small(const SmallIterArgs& s, int move_blocks, cudaStream_t st) {
  if (!small_iter_fits(s.a.n, s.a.dtype) || s.k < 1 || move_blocks < 1 || s.move_threads < 1 ||
      s.move_threads > kQThreads || s.d < 1 || s.d > kMaxD || s.r.row_bytes % 8 != 0)
    return cudaErrorInvalidValue;
  if (s.d <= 4) return iterate_small_d<4>(s, move_blocks, st);
  if (s.d <= 8) return iterate_small_d<8>(s, move_blocks, st);
  if (s.d <= 16) return iterate_small_d<16>(s, move_blocks, st);
  return iterate_small_d<32>(s, move_blocks, st);
}

// ---------------------------------------------------------------- batched launches
// One launch per stage for many samplers: block b of the launch runs block
// map[b].y of sampler map[b].x with that sampler's own arguments, so every
// sampler's blocks, reductions and results are those of its own launch.
__device__ __forceinline__ int dclass(int d) { return d <= 4 ? 0 : (d <= 8 ? 1 : (d <= 16 ? 2 : 3)); }

// left (standing batches of slots; NULL otherwise): see k_move_reweight_batch.
// A slot's map covers its capacity; blocks past the member's own count exit.
__global__ void __launch_bounds__(kQThreads) k_quant_reduce_batch(const QuantArgs* __restrict__ qa,
                                                                 const int4* __restrict__ map,
                                                                 const int32_t* __restrict__ left) {
  __shared__ QuantReduceSmem sm;
  const int4 m = map[blockIdx.x];
  if (left && left[m.x] <= 0) return;
  const QuantArgs a = qa[m.x];
  if (m.y >= a.nblocks) return;
  switch (dclass(a.d)) {
    case 0: quant_reduce_body<float, 4, true>(a, m.y, sm); break;
    case 1: quant_reduce_body<float, 8, true>(a, m.y, sm); break;
    case 2: quant_reduce_body<float, 16, true>(a, m.y, sm); break;
    default: quant_reduce_body<float, 32, true>(a, m.y, sm); break;
  }
}

__global__ void __launch_bounds__(kFinBatchThreads) k_quant_finalize_batch(const QuantArgs* __restrict__ qa,
                                                                     const int32_t* __restrict__ left) {
  if (left && left[blockIdx.x] <= 0) return;
  const QuantArgs a = qa[blockIdx.x];
  quant_finalize_body(a, 0);
}

__global__ void __launch_bounds__(kQThreads, 4) k_quant_scan_batch(const QuantArgs* __restrict__ qa,
                                                               const int4* __restrict__ map,
                                                               const int32_t* __restrict__ left) {
  const int4 m = map[blockIdx.x];
  if (left && left[m.x] <= 0) return;
  const QuantArgs a = qa[m.x];
  if (m.y >= a.nblocks) return;
  __shared__ ScanSmem sm;
  quant_scan_body(a, m.y, sm);
}

template <int KU>
__global__ void __launch_bounds__(kRThreads) k_redistribute_batch(const RedistArgs* __restrict__ ra,
                                                                 const int4* __restrict__ map,
                                                                 const int32_t* __restrict__ left) {
  __shared__ RedistSmem sm;
  const int4 m = map[blockIdx.x];
  if (left && left[m.x] <= 0) return;
  const RedistArgs a = ra[m.x];
  if (m.y >= a.ntiles) return;
  switch (a.row_bytes) {
    case 8: redistribute_body<uint2, 1, KU>(a, m.y, sm); break;
    case 16: redistribute_body<uint4, 1, KU>(a, m.y, sm); break;
    case 32: redistribute_body<uint4, 2, KU>(a, m.y, sm); break;
    case 64: redistribute_body<uint4, 4, KU>(a, m.y, sm); break;
    case 128: redistribute_body<uint4, 8, KU>(a, m.y, sm); break;
    default:
      if (a.row_bytes % 16 == 0)
        redistribute_body<uint4, 0, KU>(a, m.y, sm);
      else if (a.row_bytes % 8 == 0)
        redistribute_body<uint2, 0, KU>(a, m.y, sm);
      else
        redistribute_body<uint32_t, 0, KU>(a, m.y, sm);
      break;
  }
}

// Timing input for the copy stage: every tile's run starts set to the
// identity (each row its own single copy), which the copy consumes and resets
// to -1 as usual.
__global__ void __launch_bounds__(kRThreads) k_identity_runs_batch(const RedistArgs* __restrict__ ra,
                                                                  const int4* __restrict__ map) {
  const int4 m = map[blockIdx.x];
  const RedistArgs a = ra[m.x];
  const int64_t k0 = int64_t(m.y) * kRTile;
  const int len = int(a.n - k0 < kRTile ? a.n - k0 : int64_t(kRTile));
  int32_t* __restrict__ rs = rs_now(a.runstart, a.runstart_alt, a.st);
  for (int k = threadIdx.x; k < len; k += kRThreads) rs[k0 + k] = int32_t(k0 + k);
  if (threadIdx.x == 0) const_cast<int32_t*>(a.tile_src)[m.y] = int32_t(k0);
}

cudaError_t launch_quant_reduce_batch(const QuantArgs* qa, const int4* map, int nblocks, cudaStream_t s,
                                      const int32_t* left) {
  k_quant_reduce_batch<<<nblocks, kQThreads, 0, s>>>(qa, map, left);
  return cudaGetLastError();
}
cudaError_t launch_quant_finalize_batch(const QuantArgs* qa, int count, cudaStream_t s, const int32_t* left) {
  k_quant_finalize_batch<<<count, kFinBatchThreads, 0, s>>>(qa, left);
  return cudaGetLastError();
}
cudaError_t launch_quant_scan_batch(const QuantArgs* qa, const int4* map, int nblocks, cudaStream_t s,
                                    const int32_t* left) {
  k_quant_scan_batch<<<nblocks, kQThreads, 0, s>>>(qa, map, left);
  return cudaGetLastError();
}
cudaError_t launch_redistribute_batch(const RedistArgs* ra, const int4* map, int nblocks, int copy_variant,
                                      cudaStream_t s, const int32_t* left) {
  switch (copy_variant) {
    case 0: k_redistribute_batch<4><<<nblocks, kRThreads, 0, s>>>(ra, map, left); break;
    case 1: k_redistribute_batch<8><<<nblocks, kRThreads, 0, s>>>(ra, map, left); break;
    case 2: k_redistribute_batch<16><<<nblocks, kRThreads, 0, s>>>(ra, map, left); break;
    default: return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}
cudaError_t launch_identity_runs_batch(const RedistArgs* ra, const int4* map, int nblocks, cudaStream_t s) {
  k_identity_runs_batch<<<nblocks, kRThreads, 0, s>>>(ra, map);
  return cudaGetLastError();
}

// ---------------------------------------------------------------- launchers
static int qblocks(int64_t n) { return int((n + kQTile - 1) / kQTile); }

cudaError_t launch_state_init(DevState* st, int64_t n, int64_t t, int F, cudaStream_t s) {
  k_state_init<<<1, 32, 0, s>>>(st, n, t, F);
  return cudaGetLastError();
}

cudaError_t launch_max_logw(const double* logw, int64_t n, double* part, int nb, DevState* st, cudaStream_t s) {
  k_max_logw<<<nb, kQThreads, 0, s>>>(logw, n, part, st);
  return cudaGetLastError();
}

template <typename ST>
static cudaError_t quant_reduce_t(const QuantArgs& a, cudaStream_t s) {
  const int g = qblocks(a.n);
  if (!a.x[0] || a.d < 1)
    k_quant_reduce<ST, 1, false><<<g, kQThreads, 0, s>>>(a);
  else if (a.d <= 4)
    k_quant_reduce<ST, 4, true><<<g, kQThreads, 0, s>>>(a);
  else if (a.d <= 8)
    k_quant_reduce<ST, 8, true><<<g, kQThreads, 0, s>>>(a);
  else if (a.d <= 16)
    k_quant_reduce<ST, 16, true><<<g, kQThreads, 0, s>>>(a);
  else
    k_quant_reduce<ST, 32, true><<<g, kQThreads, 0, s>>>(a);
  return cudaGetLastError();
}

cudaError_t launch_quant_reduce(const QuantArgs& a, cudaStream_t s) {
  return a.dtype == SMC_F64 ? quant_reduce_t<double>(a, s) : quant_reduce_t<float>(a, s);
}

cudaError_t launch_quant_finalize(const QuantArgs& a, int set_lse_prev, cudaStream_t s) {
  k_quant_finalize<<<1, kFinThreads, 0, s>>>(a, set_lse_prev);
  return cudaGetLastError();
}

cudaError_t launch_quant_scan(const QuantArgs& a, cudaStream_t s) {
  k_quant_scan<<<qblocks(a.n), kQThreads, 0, s>>>(a);
  return cudaGetLastError();
}

cudaError_t launch_nc_reduce(const NcScanArgs& a, cudaStream_t s) {
  k_nc_reduce<<<qblocks(a.n), kQThreads, 0, s>>>(a);
  return cudaGetLastError();
}

cudaError_t launch_nc_finalize(const NcScanArgs& a, cudaStream_t s) {
  k_nc_finalize<<<1, kFinThreads, 0, s>>>(a);
  return cudaGetLastError();
}

cudaError_t launch_nc_scan(const NcScanArgs& a, cudaStream_t s) {
  k_nc_scan<<<qblocks(a.n), kQThreads, 0, s>>>(a);
  return cudaGetLastError();
}

cudaError_t launch_redistribute(const RedistArgs& a, cudaStream_t s) {
  const int grid = int((a.n + kRTile - 1) / kRTile);
  const int rb = a.row_bytes;
  if (rb % 16 == 0) {
    switch (rb / 16) {
      case 1: k_redistribute<uint4, 1><<<grid, kRThreads, 0, s>>>(a); break;
      case 2: k_redistribute<uint4, 2><<<grid, kRThreads, 0, s>>>(a); break;
      case 4: k_redistribute<uint4, 4><<<grid, kRThreads, 0, s>>>(a); break;
      case 8: k_redistribute<uint4, 8><<<grid, kRThreads, 0, s>>>(a); break;
      default: k_redistribute<uint4, 0><<<grid, kRThreads, 0, s>>>(a); break;
    }
  } else if (rb % 8 == 0) {
    if (rb == 8)
      k_redistribute<uint2, 1><<<grid, kRThreads, 0, s>>>(a);
    else
      k_redistribute<uint2, 0><<<grid, kRThreads, 0, s>>>(a);
  } else {
    if (rb == 4)
      k_redistribute<uint32_t, 1><<<grid, kRThreads, 0, s>>>(a);
    else
      k_redistribute<uint32_t, 0><<<grid, kRThreads, 0, s>>>(a);
  }
  return cudaGetLastError();
}

template <typename ST>
static cudaError_t quant_small_t(const QuantArgs& a, cudaStream_t s) {
  if (!a.x[0] || a.d < 1)
    k_quant_small<ST, 1, false><<<1, kQThreads, 0, s>>>(a);
  else if (a.d <= 4)
    k_quant_small<ST, 4, true><<<1, kQThreads, 0, s>>>(a);
  else if (a.d <= 8)
    k_quant_small<ST, 8, true><<<1, kQThreads, 0, s>>>(a);
  else if (a.d <= 16)
    k_quant_small<ST, 16, true><<<1, kQThreads, 0, s>>>(a);
  else
    k_quant_small<ST, 32, true><<<1, kQThreads, 0, s>>>(a);
  return cudaGetLastError();
}

cudaError_t launch_quant_small(const QuantArgs& a, cudaStream_t s) {
  if (qblocks(a.n) != 1) return cudaErrorInvalidValue;
  return a.dtype == SMC_F64 ? quant_small_t<double>(a, s) : quant_small_t<float>(a, s);
}

cudaError_t launch_redistribute_commit(const RedistArgs& a, int d, int force_flip, int recycle, cudaStream_t s) {
  if (a.n > kRTile) return cudaErrorInvalidValue;
  const int rb = a.row_bytes;
  if (rb % 16 == 0) {
    switch (rb / 16) {
      case 1: k_redistribute_commit<uint4, 1><<<1, kRThreads, 0, s>>>(a, d, force_flip, recycle); break;
      case 2: k_redistribute_commit<uint4, 2><<<1, kRThreads, 0, s>>>(a, d, force_flip, recycle); break;
      case 4: k_redistribute_commit<uint4, 4><<<1, kRThreads, 0, s>>>(a, d, force_flip, recycle); break;
      default: k_redistribute_commit<uint4, 0><<<1, kRThreads, 0, s>>>(a, d, force_flip, recycle); break;
    }
  } else if (rb % 8 == 0) {
    k_redistribute_commit<uint2, 0><<<1, kRThreads, 0, s>>>(a, d, force_flip, recycle);
  } else {
    k_redistribute_commit<uint32_t, 0><<<1, kRThreads, 0, s>>>(a, d, force_flip, recycle);
  }
  return cudaGetLastError();
}

size_t devstate_bytes() { return sizeof(DevState); }

}  // namespace smc
