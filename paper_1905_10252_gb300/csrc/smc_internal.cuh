// smc_internal.cuh -- device-side building blocks of libsmc.so (sm_103a).
//
// Shared by the kernel translation units of the library only.  Contents:
//  * DevState: the sampler's device-resident control block (iteration t,
//    current ping-pong buffer, resampling decision, error word, statistics).
//  * Philox4x32-10 (Salmon et al., SC'11) for counter-based normals keyed by
//    (seed, iteration, particle).
//  * IEEE-exact log and sincos(2 pi a) for the FP64 Box-Muller transform: only
//    correctly rounded basic operations, each written with an explicit
//    rounding intrinsic so nvcc cannot contract or reorder them.
//  * The integer fixed-point exponential that quantises the weights before
//    systematic resampling, and the 128-bit helpers around it.
//  * Warp / block reductions and scans.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

#include "../../include/smc.h"

namespace smc {

typedef unsigned __int128 u128;

// ---------------------------------------------------------------- constants
constexpr int kMaxD = 32;
constexpr int kQTile = 4096;          // elements per block of the quantise / scan passes
constexpr int kQThreads = 256;        // 16 consecutive elements per thread
constexpr int kQItems = kQTile / kQThreads;
constexpr int kRTile = 2048;          // output rows per block of the redistribute copy
constexpr int kRThreads = 256;
constexpr int kPThreads = 256;        // particle kernels (init / move / reweight)
constexpr int kFinThreads = 1024;     // single-block finalisers
constexpr int kEstTile = 256;         // particles per eq. (7) record of the move kernel (one warp tile)
static_assert(kQTile % kEstTile == 0, "a quantise block covers whole estimate tiles");
constexpr int kFinBatchThreads = 256; // one finaliser block per sampler of a batch

// Random-stream purposes (third Philox counter word = purpose << 32 | block).
constexpr uint32_t kPurposeInit = 1;
constexpr uint32_t kPurposeMove = 2;
constexpr uint32_t kPurposeResample = 3;

// ---------------------------------------------------------------- device state
struct alignas(256) DevState {
  int64_t t;            // iteration index (0 after smc_init)
  int32_t cur;          // 0: x/logpi hold the particles, 1: the _alt buffers
  int32_t flag;         // resampling decision of iteration t
  int32_t err;          // first smc_status recorded on the device, 0 if none
  int32_t F;            // fixed-point scale of the weights
  int32_t L;            // bit length of S (ncopies division)
  int32_t w_uniform;    // 1: every log w equals reset_logw (the last iteration resampled)
  // deferred redistribution (samplers created with SMC_FLAG_DEFER_REDISTRIBUTE):
  // pending = 1: iteration t resampled but its rows still sit in buffer cur, to
  // be gathered through the run starts rs / tile_src by the next move (or by
  // smc_materialize); log w is then reset_logw for every particle whatever
  // the array holds.
  // Such samplers keep two run-start arrays.  rs_w names the one the next
  // scan writes and the next copy reads; it holds -1 everywhere between
  // resamplings.  A gathering move reads rs_w's array without resetting it
  // (other warps of the same launch still search it), so the array it
  // consumed is left dirty: the move resets the OTHER array when rs_dirty
  // says that one is dirty, and the max pass that follows makes the other
  // array current (rs_w ^= 1) and marks the consumed one dirty.  A copy
  // kernel resets the entries it consumed, so rs_w's array stays clean.
  int32_t pending;
  int32_t rs_dirty;
  int32_t rs_w;
  int32_t rs_pad;
  double m;             // max_i log w
  double lse;           // LSE_t
  double lse_prev;      // LSE_{t-1} (0 after a reset)
  double logc;          // log c_t
  double ess;           // N_eff
  double reset_logw;    // -log N
  uint64_t S, U;        // sum W, systematic offset
  uint64_t sw2_lo, sw2_hi, se_lo, se_hi;
  uint64_t recip;       // floor(N 2^64 / S) (ncopies quotients)
  // recycling (eq. (6)): running log-max of log c_t and the scaled sums
  double rc_max;
  double rc_den;
  double rc_num[kMaxD];
  double mean[kMaxD];   // f_t of the current iteration
  double est_s;         // sum_i exp(log w_i - m) behind mean (estimate kernel)
  // output pointers of the running smc_step (set before a graph replay)
  smc_iter_stats* trace;
  int64_t trace_t0;
  double* mean_out;
  double* fhat_out;
  double* cov_out;
  int32_t want_cov;
  int32_t est_ready;    // 1: this iteration's move kernel wrote the eq. (7) tile records
  unsigned long long survivors;  // particles with ncopies > 0 in the current resampling
  smc_iter_stats last;  // statistics of the last finalised iteration
};

// The run-start array in use: rs1 (the second array of a sampler that has
// one) when st->rs_w says so, else rs0.
__device__ __forceinline__ int32_t* rs_now(int32_t* rs0, int32_t* rs1, const DevState* st) {
  return (rs1 && st->rs_w) ? rs1 : rs0;
}

__device__ __forceinline__ void record_error(DevState* st, int code) {
  atomicCAS(&st->err, 0, code);
}

// ---------------------------------------------------------------- Philox4x32-10
struct P4 {
  uint32_t v[4];
};

__device__ __forceinline__ P4 philox(uint32_t c0, uint32_t c1, uint32_t c2, uint32_t c3, uint32_t k0,
                                     uint32_t k1) {
  const uint32_t M0 = 0xD2511F53u, M1 = 0xCD9E8D57u;
  const uint32_t W0 = 0x9E3779B9u, W1 = 0xBB67AE85u;
#pragma unroll
  for (int r = 0; r < 10; ++r) {
    const uint32_t lo0 = M0 * c0, hi0 = __umulhi(M0, c0);
    const uint32_t lo1 = M1 * c2, hi1 = __umulhi(M1, c2);
    const uint32_t n0 = hi1 ^ c1 ^ k0, n2 = hi0 ^ c3 ^ k1;
    c0 = n0;
    c1 = lo1;
    c2 = n2;
    c3 = lo0;
    k0 += W0;
    k1 += W1;
  }
  P4 o;
  o.v[0] = c0;
  o.v[1] = c1;
  o.v[2] = c2;
  o.v[3] = c3;
  return o;
}

// Block b of the stream of particle i at iteration t: counter
// (i, t, purpose << 24 | b, 0), key (seed low, seed high); 32-bit word w of the
// stream is output w % 4 of block w / 4.
__device__ __forceinline__ P4 stream_block(uint64_t seed, uint64_t t, uint32_t purpose, uint64_t i,
                                           uint32_t b) {
  return philox(uint32_t(i), uint32_t(t), (purpose << 24) | b, 0u, uint32_t(seed), uint32_t(seed >> 32));
}

// ---------------------------------------------------------------- exact FP64 helpers
// ln 2 split so that e * kLn2Hi is exact for |e| < 2^11.
__device__ __forceinline__ double ln2_hi() { return __longlong_as_double(0x3FE62E42FEE00000ll); }
__device__ __forceinline__ double ln2_lo() { return __longlong_as_double(0x3DEA39EF35793C76ll); }

// log(u), u finite, normal, > 0: u = 2^e m, m in [sqrt(1/2), sqrt(2)),
// log m = 2 atanh(s), s = (m-1)/(m+1), series to s^22.
__device__ __forceinline__ double det_log(double u) {
  const long long b = __double_as_longlong(u);
  int e = int((b >> 52) & 0x7ff) - 1023;
  double m = __longlong_as_double((b & 0x000FFFFFFFFFFFFFll) | 0x3FF0000000000000ll);
  if (m > __longlong_as_double(0x3FF6A09E667F3BCDll)) {
    m = __dmul_rn(m, 0.5);
    e += 1;
  }
  const double s = __ddiv_rn(__dsub_rn(m, 1.0), __dadd_rn(m, 1.0));
  const double s2 = __dmul_rn(s, s);
  double p = 1.0 / 23.0;
  p = __fma_rn(p, s2, 1.0 / 21.0);
  p = __fma_rn(p, s2, 1.0 / 19.0);
  p = __fma_rn(p, s2, 1.0 / 17.0);
  p = __fma_rn(p, s2, 1.0 / 15.0);
  p = __fma_rn(p, s2, 1.0 / 13.0);
  p = __fma_rn(p, s2, 1.0 / 11.0);
  p = __fma_rn(p, s2, 1.0 / 9.0);
  p = __fma_rn(p, s2, 1.0 / 7.0);
  p = __fma_rn(p, s2, 1.0 / 5.0);
  p = __fma_rn(p, s2, 1.0 / 3.0);
  p = __fma_rn(p, s2, 1.0);
  const double logm = __dmul_rn(__dmul_rn(2.0, s), p);
  const double de = double(e);
  return __fma_rn(de, ln2_hi(), __fma_rn(de, ln2_lo(), logm));
}

// sin and cos of 2 pi v 2^-53 (0 <= v < 2^53): exact quarter-turn reduction on
// the integer, Taylor series to degree 17 / 18 on [-pi/4, pi/4].
__device__ __forceinline__ void det_sincos2pi(uint64_t v, double* s_out, double* c_out) {
  const uint64_t q = (v + (1ull << 50)) >> 51;
  const long long vr = (long long)v - (long long)(q << 51);
  const double x = __dmul_rn(double(vr), 0x1p-53);
  const double t = __dmul_rn(x, __longlong_as_double(0x401921FB54442D18ll));  // 2 pi
  const double t2 = __dmul_rn(t, t);
  double ps = -1.0 / 121645100408832000.0;
  ps = __fma_rn(ps, t2, 1.0 / 355687428096000.0);
  ps = __fma_rn(ps, t2, -1.0 / 1307674368000.0);
  ps = __fma_rn(ps, t2, 1.0 / 6227020800.0);
  ps = __fma_rn(ps, t2, -1.0 / 39916800.0);
  ps = __fma_rn(ps, t2, 1.0 / 362880.0);
  ps = __fma_rn(ps, t2, -1.0 / 5040.0);
  ps = __fma_rn(ps, t2, 1.0 / 120.0);
  ps = __fma_rn(ps, t2, -1.0 / 6.0);
  ps = __fma_rn(ps, t2, 1.0);
  const double sn = __dmul_rn(t, ps);
  double pc = 1.0 / 6402373705728000.0;
  pc = __fma_rn(pc, t2, -1.0 / 20922789888000.0);
  pc = __fma_rn(pc, t2, 1.0 / 87178291200.0);
  pc = __fma_rn(pc, t2, -1.0 / 479001600.0);
  pc = __fma_rn(pc, t2, 1.0 / 3628800.0);
  pc = __fma_rn(pc, t2, -1.0 / 40320.0);
  pc = __fma_rn(pc, t2, 1.0 / 720.0);
  pc = __fma_rn(pc, t2, -1.0 / 24.0);
  pc = __fma_rn(pc, t2, 1.0 / 2.0);
  const double cs = __fma_rn(-pc, t2, 1.0);
  switch (q & 3) {
    case 0: *s_out = sn; *c_out = cs; break;
    case 1: *s_out = cs; *c_out = -sn; break;
    case 2: *s_out = -sn; *c_out = -cs; break;
    default: *s_out = -cs; *c_out = sn; break;
  }
}

// D standard normals (FP64 path): pair p uses block p, whose four 32-bit words
// make the 64-bit words (w0 w1) and (w2 w3); their top 53 bits are a and b;
// u1 = 1 - a, r = sqrt(-2 log u1), (z0, z1) = r (cos, sin)(2 pi b).
template <int DMAX>
__device__ __forceinline__ void normals_f64(uint64_t seed, uint64_t t, uint32_t purpose, uint64_t i, int d,
                                            double (&z)[DMAX]) {
#pragma unroll
  for (int p = 0; 2 * p < DMAX; ++p) {
    if (2 * p < d) {
      const P4 w = stream_block(seed, t, purpose, i, uint32_t(p));
      const uint64_t va = ((uint64_t(w.v[0]) << 32) | w.v[1]) >> 11;
      const uint64_t vb = ((uint64_t(w.v[2]) << 32) | w.v[3]) >> 11;
      const double u1 = __dmul_rn(double((1ull << 53) - va), 0x1p-53);
      const double r = __dsqrt_rn(__dmul_rn(-2.0, det_log(u1)));
      double sn, cs;
      det_sincos2pi(vb, &sn, &cs);
      z[2 * p] = __dmul_rn(r, cs);
      if (2 * p + 1 < DMAX) z[2 * p + 1] = __dmul_rn(r, sn);
    }
  }
}

// D standard normals (FP32 path): pair p uses 32-bit words 2p, 2p+1 (block
// p / 2), the top 24 bits of each giving the uniforms a, b.
template <int DMAX>
__device__ __forceinline__ void normals_f32(uint64_t seed, uint64_t t, uint32_t purpose, uint64_t i, int d,
                                            float (&z)[DMAX]) {
#pragma unroll
  for (int blk = 0; blk < (DMAX + 3) / 4; ++blk) {
    if (4 * blk < d) {
      const P4 w = stream_block(seed, t, purpose, i, uint32_t(blk));
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        const int p = 2 * blk + h;
        if (2 * p < d && 2 * p < DMAX) {
          const uint32_t h0 = w.v[2 * h], h1 = w.v[2 * h + 1];
          const float u1 = float((1u << 24) - (h0 >> 8)) * 0x1p-24f;
          const float b2 = float(h1 >> 8) * 0x1p-23f;  // 2b, exact
          const float r = sqrtf(-2.0f * logf(u1));
          float sn, cs;
          sincospif(b2, &sn, &cs);
          z[2 * p] = r * cs;
          if (2 * p + 1 < DMAX) z[2 * p + 1] = r * sn;
        }
      }
    }
  }
}

// ---------------------------------------------------------------- fixed-point exp
// E(y) ~= 2^62 exp(y) for y <= 0, an integer in [0, 2^62]:
//   a = -y; A = floor(a 2^57) from the bits of a; Z = A round(log2(e) 2^62)
//   (z = a log2 e = Z 2^-119); k = integer part, f = 64 fraction bits;
//   2^-f = T1[top 6 bits] T2[next 6 bits] exp(-g ln 2) for the low 52 bits g;
//   exp(-h) = C0 - h(C1 - h(C2 - h(C3 - h C4))) in 2^63 fixed point with
//   C_k = floor(2^63 / k!);  E = ((T1 T2 >> 63) P 2^-64) >> k.
// T (128 entries: T1 ~= 2^63 2^(-j/64), T2 ~= 2^63 2^(-j/4096)) is built on
// the host from integer square roots and lives in shared memory while a
// kernel uses it.
// Takes a = m - log w >= 0 (one IEEE subtraction, equal to -(log w - m)); the
// range test is done on the bits (a >= 44, +inf and NaN give 0) so that the
// only FP64 operation per weight is the caller's subtraction.
__device__ __forceinline__ uint64_t expfx_a(double a, const uint64_t* __restrict__ T) {
  const uint64_t bits = (uint64_t)__double_as_longlong(a);
  if (bits >= 0x4046000000000000ull) return 0;  // 44.0 and above (a is never negative)
  const int e = int((bits >> 52) & 0x7ff);
  uint64_t A = 0;
  if (e != 0) {
    const uint64_t mant = (bits & 0x000FFFFFFFFFFFFFull) | (1ull << 52);
    const int sh = e - 1018;
    A = sh >= 0 ? (mant << sh) : (sh > -64 ? (mant >> (-sh)) : 0);
  }
  const uint64_t L2E = 0x5C551D94AE0BF85Eull;  // round(log2(e) 2^62)
  const uint64_t LN2 = 0xB17217F7D1CF79ACull;  // round(ln(2) 2^64)
  const uint64_t zlo = A * L2E, zhi = __umul64hi(A, L2E);
  const unsigned k = unsigned(zhi >> 55);
  const uint64_t f = (zhi << 9) | (zlo >> 55);
  const unsigned j1 = unsigned(f >> 58);
  const unsigned j2 = unsigned((f >> 52) & 63);
  const uint64_t g = f & ((1ull << 52) - 1);
  const uint64_t H = __umul64hi(g << 12, LN2);
  constexpr uint64_t ONE = 1ull << 63;
  uint64_t P = ONE / 24;
  P = ONE / 6 - (__umul64hi(H, P) >> 12);
  P = ONE / 2 - (__umul64hi(H, P) >> 12);
  P = ONE - (__umul64hi(H, P) >> 12);
  P = ONE - (__umul64hi(H, P) >> 12);
  const uint64_t t1 = T[j1], t2 = T[64 + j2];
  const uint64_t Tm = (__umul64hi(t1, t2) << 1) | ((t1 * t2) >> 63);
  return __umul64hi(Tm, P) >> k;
}

__device__ __forceinline__ uint64_t expfx(double y, const uint64_t* __restrict__ T) {
  return expfx_a(-y, T);
}

// ---------------------------------------------------------------- reductions
template <typename T>
__device__ __forceinline__ T warp_sum(T v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

__device__ __forceinline__ double warp_max(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
  return v;
}

__device__ __forceinline__ u128 shfl_xor_u128(u128 v, int o) {
  const uint64_t lo = __shfl_xor_sync(0xffffffffu, uint64_t(v), o);
  const uint64_t hi = __shfl_xor_sync(0xffffffffu, uint64_t(v >> 64), o);
  return (u128(hi) << 64) | lo;
}

__device__ __forceinline__ u128 warp_sum_u128(u128 v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += shfl_xor_u128(v, o);
  return v;
}

// Inclusive warp scan (Hillis-Steele) of 64-bit values.
__device__ __forceinline__ uint64_t warp_incl_scan_u64(uint64_t v) {
  const int lane = threadIdx.x & 31;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const uint64_t n = __shfl_up_sync(0xffffffffu, v, o);
    if (lane >= o) v += n;
  }
  return v;
}

__device__ __forceinline__ int warp_incl_max_i32(int v) {
  const int lane = threadIdx.x & 31;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const int n = __shfl_up_sync(0xffffffffu, v, o);
    if (lane >= o) v = max(v, n);
  }
  return v;
}

// Exclusive block scan of one 64-bit value per thread; returns the exclusive
// prefix and writes the block total.  scratch: blockDim/32 + 1 words.
__device__ __forceinline__ uint64_t block_excl_scan_u64(uint64_t v, uint64_t* scratch, uint64_t* total) {
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
  const uint64_t incl = warp_incl_scan_u64(v);
  if (lane == 31) scratch[wid] = incl;
  __syncthreads();
  if (wid == 0) {
    uint64_t s = lane < nw ? scratch[lane] : 0;
    const uint64_t si = warp_incl_scan_u64(s);
    if (lane < nw) scratch[lane] = si - s;
    if (lane == nw - 1) scratch[32] = si;
  }
  __syncthreads();
  const uint64_t r = scratch[wid] + incl - v;
  *total = scratch[32];
  __syncthreads();
  return r;
}

// ---------------------------------------------------------------- running maximum of log w
// Doubles compared as integers (order-preserving map of the bit pattern): the
// FP64 pipe of GB300 runs at a small fraction of its integer rate.
__device__ __forceinline__ long long ordered_key(double v) {
  const long long b = __double_as_longlong(v);
  return b >= 0 ? b : (b ^ 0x7FFFFFFFFFFFFFFFll);
}
__device__ __forceinline__ double from_ordered_key(long long k) {
  return __longlong_as_double(k >= 0 ? k : (k ^ 0x7FFFFFFFFFFFFFFFll));
}

struct MaxTracker {
  long long best;
  bool nan;
  __device__ __forceinline__ void init() {
    best = ordered_key(-INFINITY);
    nan = false;
  }
  __device__ __forceinline__ void add(double v) {
    const long long b = __double_as_longlong(v);
    if ((b & 0x7FF0000000000000ll) == 0x7FF0000000000000ll && (b & 0x000FFFFFFFFFFFFFll)) {
      nan = true;
      return;
    }
    const long long k = b >= 0 ? b : (b ^ 0x7FFFFFFFFFFFFFFFll);
    best = k > best ? k : best;
  }
};

__device__ __forceinline__ long long warp_max_ll(long long v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    const long long w = __shfl_xor_sync(0xffffffffu, v, o);
    v = w > v ? w : v;
  }
  return v;
}


// ---------------------------------------------------------------- end of an iteration
// Ends iteration t, executed by one full warp: swap buffers if resampled (or
// if forced by an explicit redistribute), LSE_t becomes the next LSE_{t-1}
// (0 after a reset), and the recycling sums of eq. (6) take f_t with weight
// c_t -- one column per lane, each with explicitly rounded FP64 operations
// (the same bits whichever kernel runs it).
// defer: a resampled iteration leaves its rows in place and marks them
// pending instead of swapping (the next move gathers them).
// Every field the commit reads is loaded before its first store (one round
// trip to memory instead of a chain of them; the values are those the
// original order reads, as no field is read after the commit writes it).
__device__ __forceinline__ void commit_warp(DevState* st, int d, int force_flip, int recycle, int defer = 0) {
  const int lane = threadIdx.x & 31;
  const int err = st->err, flag = st->flag, cur = st->cur;
  const double lc = st->logc, rmax = st->rc_max, rden = st->rc_den, lse = st->lse;
  double* const fh = st->fhat_out;
  smc_iter_stats* const trace = st->trace;
  const int64_t t = st->t, t0 = st->trace_t0;
  const unsigned long long surv = st->survivors;
  constexpr int kLanesD = kMaxD / 32;  // columns per lane
  double rnum[kLanesD], mc[kLanesD];
#pragma unroll
  for (int j = 0; j < kLanesD; ++j) {
    const int c = lane + 32 * j;
    rnum[j] = c < d ? st->rc_num[c] : 0.0;
    mc[j] = c < d ? st->mean[c] : 0.0;
  }
  const bool pend = defer && flag && !err;
  const bool flip = force_flip || (flag && !err && !defer);
  double M = 0.0, den = 0.0;
  if (recycle && !err) {
    M = fmax(rmax, lc);
    const double sc = (rmax == -INFINITY) ? 0.0 : exp(__dsub_rn(rmax, M));
    const double e = exp(__dsub_rn(lc, M));
    den = __fma_rn(rden, sc, e);
#pragma unroll
    for (int j = 0; j < kLanesD; ++j) {
      const int c = lane + 32 * j;
      if (c < d) {
        const double num = __fma_rn(rnum[j], sc, __dmul_rn(e, mc[j]));
        st->rc_num[c] = num;
        if (fh) fh[c] = __ddiv_rn(num, den);
      }
    }
  }
  __syncwarp();  // every lane has read the state before lane 0 writes it
  if (lane != 0) return;
  if (recycle && !err) {
    st->rc_den = den;
    st->rc_max = M;
  }
  if (flag && !err) {
    st->last.survivors = (int64_t)surv;
    if (trace) {
      const int64_t idx = t - t0 - 1;
      if (idx >= 0) trace[idx].survivors = (int64_t)surv;
    }
  }
  if (flip) st->cur = cur ^ 1;
  st->pending = pend ? 1 : 0;
  st->lse_prev = (flip || pend) ? 0.0 : lse;
  // a resampled iteration leaves every log w at reset_logw
  st->w_uniform = ((flip || pend) && !err) ? 1 : 0;
}

}  // namespace smc
