// k_particles.cu -- element-wise stages of one SMC iteration on sm_103a:
//   * target set-up (Cholesky of Sigma, its inverse, FP32 copies),
//   * initialisation (Algorithm 2, line 1),
//   * random-walk move and importance reweighting (Algorithm 2, line 4; eq. (5)),
//     fused in one pass over the particle rows,
//   * the per-block maxima of log w (integer-ordered compares, no FP64 pipe),
//     combined by a single-block finaliser,
//   * the sums of eq. (7) for FP32 Gaussian samplers whose iteration starts
//     from equal weights, one record per 256-particle warp tile (otherwise
//     the quantisation pass forms them from the fixed-point weights),
//   * the weighted covariance (diagnostic),
//   * the iteration bookkeeping kernels (begin / commit, eq. (6) recycling).
//
// One thread owns one particle row at a time (grid-stride over N; the FP32
// Gaussian kernel strides over warp tiles of 256 consecutive rows); rows are
// read and written with the widest aligned vector the row allows.  The FP64
// path uses explicitly rounded operations only, in the same order as the
// paper's definitions, so its results are reproducible bit for bit.
#include <cfloat>
#include <cmath>

#include "particle_bodies.cuh"
#include "smc_internal.cuh"
#include "smc_kernels.h"

namespace smc {

// ---------------------------------------------------------------- target set-up
// One thread: Cholesky-Banachiewicz of Sigma (row by row, fma accumulation),
// then P = L^-1 by forward substitution on the identity, and FP32 copies.
__global__ void k_target_setup(TargetDev* tg, int kind, double nu, const double* __restrict__ mu,
                               const double* __restrict__ sigma, int d, DevState* st) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  tg->kind = kind;
  tg->d = d;
  tg->nu = nu;
  for (int c = 0; c < d; ++c) {
    tg->mu[c] = mu[c];
    tg->muf[c] = float(mu[c]);
  }
  if (tg->kind == SMC_STUDENT_T) return;
  double* L = tg->L;
  for (int i = 0; i < d * kMaxD; ++i) L[i] = 0.0;
  for (int i = 0; i < d; ++i) {
    for (int j = 0; j <= i; ++j) {
      double s = 0.0;
      for (int k = 0; k < j; ++k) s = __fma_rn(L[i * kMaxD + k], L[j * kMaxD + k], s);
      if (i == j) {
        const double dd = __dsub_rn(sigma[i * d + i], s);
        if (!(dd > 0.0)) {
          record_error(st, SMC_EINVAL);
          return;
        }
        L[i * kMaxD + i] = __dsqrt_rn(dd);
      } else {
        L[i * kMaxD + j] = __ddiv_rn(__dsub_rn(sigma[i * d + j], s), L[j * kMaxD + j]);
      }
    }
  }
  // P = L^-1 (lower triangular), column by column
  for (int c = 0; c < d; ++c) {
    for (int r = 0; r < d; ++r) {
      double acc = (r == c) ? 1.0 : 0.0;
      for (int k = c; k < r; ++k) acc -= L[r * kMaxD + k] * tg->P[k * kMaxD + c];
      tg->P[r * kMaxD + c] = (r < c) ? 0.0 : acc / L[r * kMaxD + r];
    }
  }
  for (int i = 0; i < kMaxD * kMaxD; ++i) tg->Pf[i] = float(tg->P[i]);
}

// Logistic data: FP32 copies, BF16 hi / lo images of X log2(e) (the tensor-core
// likelihood works in base 2) and v = X^T y.  Image of
// data tile j (rows 256 j ..): kLgTileBytes bytes, hi then lo, each 256 rows x
// 32 columns of BF16 in the tensor cores' K-major core-matrix order: element
// (r, k) at byte (r / 8) * 512 + (k / 8) * 128 + (r % 8) * 16 + (k % 8) * 2.
// Rows >= M and columns >= D are zero.  lo = bf16(x' - float(hi)), x' = x log2 e.
// BF16 = the top 16 bits of an FP32, rounded to nearest even (finite inputs).
__device__ __forceinline__ uint16_t bf16_rn(float f) {
  const uint32_t u = __float_as_uint(f);
  return uint16_t((u + 0x7FFFu + ((u >> 16) & 1u)) >> 16);
}
__device__ __forceinline__ float bf16_to_f32(uint16_t h) { return __uint_as_float(uint32_t(h) << 16); }

__global__ void k_logistic_copy(TargetDev* tg, const float* __restrict__ X, const float* __restrict__ y, int m, int d,
                                double prior_var, float* __restrict__ Xw, float* __restrict__ yw,
                                uint16_t* __restrict__ ximg) {
  const int m_pad = (m + kLgRows - 1) / kLgRows * kLgRows;
  const int64_t total = int64_t(m_pad) * kLgK;
  for (int64_t e = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; e < total; e += int64_t(gridDim.x) * blockDim.x) {
    const int r = int(e / kLgK), k = int(e % kLgK);
    const float xv = (r < m && k < d) ? X[int64_t(r) * d + k] : 0.0f;
    if (r < m && k < d) Xw[int64_t(r) * d + k] = xv;
    const float v = xv * 1.4426950408889634f;  // the images hold X log2(e)
    if (k == 0 && r < m) yw[r] = y[r];
    const uint16_t hi = bf16_rn(v);
    const uint16_t lo = bf16_rn(v - bf16_to_f32(hi));
    const int tile = r / kLgRows, rr = r % kLgRows;
    const size_t off = (size_t(rr / 8) * 512 + size_t(k / 8) * 128 + size_t(rr % 8) * 16 + size_t(k % 8) * 2) / 2;
    uint16_t* img = ximg + size_t(tile) * (kLgTileBytes / 2);
    img[off] = hi;
    img[off + kLgTileBytes / 4] = lo;
  }
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    tg->kind = SMC_LOGISTIC;
    tg->d = d;
    tg->X = Xw;
    tg->y = yw;
    tg->ximg = ximg;
    tg->prior_var = prior_var;
    tg->m = m;
    tg->m_pad = m_pad;
  }
}

// v_c = sum_m y_m X_mc and the column sums of X, in FP64, row order (one
// thread per column).
__global__ void k_logistic_v(TargetDev* tg, const float* __restrict__ X, const float* __restrict__ y, int m, int d) {
  const int c = threadIdx.x;
  if (c >= kTgtMaxD) return;
  double acc = 0.0, sum = 0.0;
  if (c < d)
    for (int r = 0; r < m; ++r) {
      const double xv = double(X[int64_t(r) * d + c]);
      acc = fma(double(y[r]), xv, acc);
      sum += xv;
    }
  tg->v[c] = acc;
  tg->xsum[c] = sum;
}

// ---------------------------------------------------------------- init
// x0 = s z (z from the INIT stream at t = 0), log w0 = log pi(x0) - log q0(x0),
// log q0(x) = (-1/2 |x|^2) / s^2.
template <typename T, int DMAX>
__global__ void __launch_bounds__(kPThreads) k_init(ParticleArgs a) {
  __shared__ TargetSmem<T> ts;
  load_target<T>(a.tg, a.d, ts);
  MaxTracker mt;
  mt.init();
  T* __restrict__ x = static_cast<T*>(a.x[0]);
  T* __restrict__ lp = static_cast<T*>(a.logpi[0]);
  const T nu = T(a.tg->nu);
  for (int64_t i = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; i < a.n; i += int64_t(gridDim.x) * blockDim.x) {
    T xr[DMAX];
    double lw;
    if constexpr (sizeof(T) == 8) {
      double z[DMAX];
      normals_f64<DMAX>(a.seed, 0, kPurposeInit, uint64_t(i), a.d, z);
      double q = 0.0;
#pragma unroll
      for (int c = 0; c < DMAX; ++c) {
        xr[c] = c < a.d ? __dmul_rn(a.init_scale, z[c]) : 0.0;
        if (c < a.d) q = __fma_rn(xr[c], xr[c], q);
      }
      const double lpi = (a.flags & PA_INIT_SKIP_LOGPI) ? 0.0 : eval_logpi<T, DMAX>(xr, a.d, a.kind, ts, nu, a.tg);
      const double lq0 = __ddiv_rn(__dmul_rn(-0.5, q), __dmul_rn(a.init_scale, a.init_scale));
      lw = __dsub_rn(lpi, lq0);
      lp[i] = lpi;
    } else {
      float z[DMAX];
      normals_f32<DMAX>(a.seed, 0, kPurposeInit, uint64_t(i), a.d, z);
      const float s = float(a.init_scale);
      float q = 0.0f;
#pragma unroll
      for (int c = 0; c < DMAX; ++c) {
        xr[c] = c < a.d ? s * z[c] : 0.0f;
        if (c < a.d) q = fmaf(xr[c], xr[c], q);
      }
      const float lpi = (a.flags & PA_INIT_SKIP_LOGPI) ? 0.0f : eval_logpi<T, DMAX>(xr, a.d, a.kind, ts, nu, a.tg);
      const float lq0 = (-0.5f * q) / (s * s);
      lw = double(lpi) - double(lq0);
      lp[i] = lpi;
    }
    store_row<T, DMAX>(x + i * a.d, a.d, xr);
    a.logw[i] = lw;
    mt.add(lw);
  }
  block_write_max(mt, a.part + 2 * blockIdx.x, a.st);
}

// ---------------------------------------------------------------- move + reweight
// The generic kernel (one thread per particle; FP64 samplers and non-Gaussian
// FP32 targets): move_reweight_generic_body over the whole launch.
template <typename T, int DMAX, bool MOVE, bool REWEIGHT>
__global__ void __launch_bounds__(kPThreads) k_move_reweight(ParticleArgs a) {
  __shared__ TargetSmem<T> ts;
  move_reweight_generic_body<T, DMAX, MOVE, REWEIGHT>(a, ts, blockIdx.x, gridDim.x, blockDim.x, 0);
}

// ---------------------------------------------------------------- move + reweight, FP32 fast path
// The FP32 path gives each lane one particle of up to DPL coordinates (DPL/4
// Philox blocks: four 32-bit words, two Box-Muller pairs per block).
// Box-Muller uses the multi-function unit: (eps r)^2 = -2 eps^2 ln(1-a) from
// log2 (ln y = ln 2 log2 y), or from its series when a < 1/16 (where the
// approximate log2's absolute error would dominate), and __sincosf on
// 2 pi (b - 1/2) in [-pi, pi).  The step eps is folded into the constants, so
// a pair costs one multiply for each of a, the radius and the angle, and the
// move itself is two FMAs; the moved coordinates differ from the exactly
// rounded x + eps z by a few 1e-6 at most, and since the random-walk proposal
// stays symmetric the weights of eq. (5) are unaffected.
// Up to 16 coordinates, the next particle's row, log pi and log w are loaded
// while the current one is computed.
struct BmStep {
  float s4, s3, s2, s1, s0;  // eps^2 (2/5, 1/2, 2/3, 1, 2): -2 eps^2 ln(1-a) / a as a series in a
  float slog;                // -2 eps^2 ln 2
};
__device__ __forceinline__ BmStep bm_step(float eps) {
  const float e2 = eps * eps;
  return BmStep{0.4f * e2, 0.5f * e2, (2.0f / 3.0f) * e2, e2, 2.0f * e2, -1.38629436111989061883f * e2};
}
// x0 += eps z0, x1 += eps z1 for the normal pair (z0, z1) of the words h0, h1.
__device__ __forceinline__ void bm_pair_step(uint32_t h0, uint32_t h1, const BmStep& k, float& x0, float& x1) {
  const float a = float(h0 >> 8) * 0x1p-24f;  // u1 = 1 - a
  // -ln(1 - a) = a (1 + a/2 + a^2/3 + a^3/4 + a^4/5 + ...): for a < 1/16 the
  // truncation error is below 1.7e-7 relative (about 1.4 FP32 ulp)
  float p = fmaf(a, k.s4, k.s3);
  p = fmaf(a, p, k.s2);
  p = fmaf(a, p, k.s1);
  p = fmaf(a, p, k.s0);
  const float r2s = a * p;  // (eps r)^2, a < 1/16
  const float r2l = __log2f(1.0f - a) * k.slog;
  const float r2 = a < 0.0625f ? r2s : r2l;
  const float r = r2 > 0.0f ? r2 * rsqrtf(r2) : 0.0f;  // eps r
  const float th = float(int(h1 >> 8) - (1 << 23)) * (0x1p-24f * 6.28318530717958647692f);
  float sn, cs;
  __sincosf(th, &sn, &cs);  // (sin, cos)(2 pi b - pi) = -(sin, cos)(2 pi b)
  x0 = fmaf(-r, cs, x0);
  x1 = fmaf(-r, sn, x1);
}

template <int DPL>
__device__ __forceinline__ void load_seg(const float* __restrict__ row, bool vec, int nvalid, float (&xr)[DPL]) {
  if (vec) {
#pragma unroll
    for (int v = 0; v < DPL / 4; ++v) {
      const float4 f = reinterpret_cast<const float4*>(row)[v];
      xr[4 * v] = f.x;
      xr[4 * v + 1] = f.y;
      xr[4 * v + 2] = f.z;
      xr[4 * v + 3] = f.w;
    }
  } else {
#pragma unroll
    for (int c = 0; c < DPL; ++c) xr[c] = c < nvalid ? row[c] : 0.0f;
  }
}

// Where the FP32 factor comes from: the kernel parameters (one sampler per
// launch; the FMAs read the constant bank) or shared memory (batched
// launches).  row(r, dv) = sum_{c <= r} P[r][c] dv[c], accumulated with one
// FMA per term in the order c = 0, 1, ..., r in both cases, so both give the
// same bits.
// Packed two-lane FP32 arithmetic (sm_100 family): each lane of fma.rn.f32x2
// is an IEEE fused multiply-add rounded to nearest, bit for bit the fmaf of
// that lane, so pairing changes no result, only the instruction count.
__device__ __forceinline__ uint64_t pack2(float a, float b) {
  uint64_t r;
  asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(a), "f"(b));
  return r;
}
__device__ __forceinline__ float2 unpack2(uint64_t v) {
  float a, b;
  asm("mov.b64 {%0, %1}, %2;" : "=f"(a), "=f"(b) : "l"(v));
  return make_float2(a, b);
}
__device__ __forceinline__ uint64_t ffma2(uint64_t a, uint64_t b, uint64_t c) {
  uint64_t d;
  asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(d) : "l"(a), "l"(b), "l"(c));
  return d;
}

struct FactorParam {
  const GaussParamsF32& g;
  __device__ __forceinline__ float mu(int c) const { return g.mu[c]; }
  // rows r and r + 1 (r even) at once, from the interleaved copy: the same
  // FMAs in the same order per row (row r's extra term at c = r + 1 has a
  // zero coefficient and adds +0)
  template <int DMAX>
  __device__ __forceinline__ float2 row2(int r, const uint64_t (&dd)[DMAX]) const {
    uint64_t acc = 0;
#pragma unroll
    for (int c = 0; c < DMAX; ++c)
      if (c <= r + 1) acc = ffma2(*reinterpret_cast<const uint64_t*>(&g.P2[(r / 2) * kTgtMaxD + c]), dd[c], acc);
    return unpack2(acc);
  }
};


// Shared-memory layout of the factor for batched launches: the interleaved
// row pairs of GaussParamsF32::P2, pair p (rows 2p, 2p + 1) holding columns
// 0 .. 2p + 1 from float2 offset p (p + 1), read with 16-byte loads.
constexpr int kPairedFactor = (kTgtMaxD / 2) * (kTgtMaxD / 2 + 1);  // float2 entries

struct FactorSmem {
  static constexpr bool kPaired = true;
  const float4* p;  // the pairs, two columns per 16-byte load
  const float* m;
  __device__ __forceinline__ float mu(int c) const { return m[c]; }
  template <int DMAX>
  __device__ __forceinline__ float2 row2(int r, const uint64_t (&dd)[DMAX]) const {
    const int pr = r / 2;
    const float4* rp = p + pr * (pr + 1) / 2;
    uint64_t acc = 0;
#pragma unroll
    for (int j = 0; j < DMAX / 2; ++j) {
      if (j <= pr) {
        const float4 v = rp[j];
        acc = ffma2(pack2(v.x, v.y), dd[2 * j], acc);
        acc = ffma2(pack2(v.z, v.w), dd[2 * j + 1], acc);
      }
    }
    return unpack2(acc);
  }
};

// Stages the row pairs of rows < d into the layout of FactorSmem.
__device__ __forceinline__ void stage_pairs(const float2* __restrict__ P2, const float* __restrict__ mu, int d,
                                            float2* pr, float* m) {
  const int np = (d + 1) / 2;
  for (int q = threadIdx.x; q < np; q += blockDim.x)
    for (int c = 0; c <= 2 * q + 1; ++c) pr[q * (q + 1) + c] = P2[q * kTgtMaxD + c];
  for (int c = threadIdx.x; c < kTgtMaxD; c += blockDim.x) m[c] = mu[c];
}

// eq. (7) record of one warp tile (kEstTile consecutive particles) whose
// starting log weights all equal R: rec = {M, sum_i e^{dlt_i - Mf} x_i} with
// M = R + Mf, dlt_i the particle's log pi difference and Mf the largest of
// the lanes' references em (every dlt_i < Mf + 16).  Each lane's sums are
// rescaled from its em to Mf and added over the warp by a transposing halving
// tree (a fixed order: the record does not depend on the launch shape).
template <int DMAX>
__device__ __forceinline__ void warp_write_est(float em, double R, float (&v)[DMAX], int d,
                                               double* __restrict__ rec) {
  const int lane = threadIdx.x & 31;
  float Mf = em;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) Mf = fmaxf(Mf, __shfl_xor_sync(0xffffffffu, Mf, o));
  const float sc = (em == -INFINITY) ? 0.0f : __expf(em - Mf);
#pragma unroll
  for (int c = 0; c < DMAX; ++c) v[c] *= sc;
  // halving: at the step with offset o, a lane keeps the upper half of its
  // columns if (lane & o), the lower half otherwise, and adds its partner's
  // copy of the kept half
  int col = 0;
#pragma unroll
  for (int h = DMAX / 2, o = 16; h >= 1; h >>= 1, o >>= 1) {
    const bool up = lane & o;
#pragma unroll
    for (int k = 0; k < h; ++k) {
      const float send = up ? v[k] : v[k + h];
      const float keep = up ? v[k + h] : v[k];
      v[k] = keep + __shfl_xor_sync(0xffffffffu, send, o);
    }
    col += up ? h : 0;
  }
  // DMAX halvings used offsets 16 .. 32 / DMAX; the lanes that still share
  // a column add up with the remaining offsets
#pragma unroll
  for (int o = 16 / DMAX; o >= 1; o >>= 1) v[0] += __shfl_xor_sync(0xffffffffu, v[0], o);
  if ((lane & (32 / DMAX - 1)) == 0 && col < d) rec[1 + col] = double(v[0]);
  // the record's reference log w, formed as the reweight forms every log w
  if (lane == 0) rec[0] = Mf == -INFINITY ? -INFINITY : R + double(Mf);
}

// Algorithm 5 as a gather, for the 256 particles of move tile jt: row k of
// the resampled set is row src(k) = the last run start at or before k
// (rs[off_i] = i for every survivor i, -1 elsewhere).  tile_src holds src at
// the first row of each 2048-row copy tile; run starts between that row and
// the move tile's first row are found by a backward search 32 rows at a time
// (in all but heavily duplicated regions the 32 rows just before hold one).
//
// The tile's run starts are staged into shared memory one tile ahead of use
// with asynchronous copies (cp.async), so that resolving a tile's sources
// does not wait on memory:
//   stage[0, 256)   rs[k0 .. k0 + 256)    (entries at or beyond n: masked)
//   stage[256, 288) rs[k0 - 32 .. k0)     (the first step of the backward search)
//   stage[288]      tile_src[k0 / 2048]
// tile_sources_issue starts the copies; tile_sources_finish waits for them
// and writes the tile's 256 sources to out[] (clamped into [0, n), as the copy
// kernel clamps them).  Every lane of the warp takes part in both.
constexpr int kStage = kEstTile + 32 + 4;

__device__ __forceinline__ void cp_async16(int32_t* smem, const int32_t* gmem, int src_bytes) {
  const unsigned sa = static_cast<unsigned>(__cvta_generic_to_shared(smem));
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;" ::"r"(sa), "l"(gmem), "r"(src_bytes) : "memory");
}
__device__ __forceinline__ void cp_async4(int32_t* smem, const int32_t* gmem) {
  const unsigned sa = static_cast<unsigned>(__cvta_generic_to_shared(smem));
  asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"(sa), "l"(gmem) : "memory");
}

__device__ __forceinline__ void tile_sources_issue(const int32_t* __restrict__ rs,
                                                   const int32_t* __restrict__ tile_src, int64_t n, int64_t jt,
                                                   int32_t* __restrict__ stage) {
  const int lane = threadIdx.x & 31;
  const int64_t k0 = jt * kEstTile;
  const int64_t t0 = (k0 / kRTile) * kRTile;
  // lane l: entries [8l, 8l + 8) as two 16-byte pieces.  rs is 256-byte
  // aligned and padded to a multiple of 256 bytes, so a piece that starts
  // below n stays inside the array; pieces at or beyond n copy nothing
  // (zero-filled, masked when the sources are resolved).
#pragma unroll
  for (int h = 0; h < 2; ++h) {
    const int64_t k = k0 + 8 * lane + 4 * h;
    const bool in = k < n;
    cp_async16(stage + 8 * lane + 4 * h, rs + (in ? k : 0), in ? 16 : 0);
  }
  if (k0 > t0) cp_async4(stage + kEstTile + lane, rs + (k0 - 32 + lane));
  if (lane == 0) cp_async4(stage + kEstTile + 32, tile_src + k0 / kRTile);
  asm volatile("cp.async.commit_group;" ::: "memory");
}

__device__ __forceinline__ void tile_sources_finish(const int32_t* __restrict__ rs, int64_t n, int64_t jt,
                                                    const int32_t* __restrict__ stage, int32_t* __restrict__ out) {
  asm volatile("cp.async.wait_all;" ::: "memory");
  __syncwarp();  // every lane's copies have landed
  const int lane = threadIdx.x & 31;
  const int64_t k0 = jt * kEstTile;
  const int64_t t0 = (k0 / kRTile) * kRTile;
  int carry = stage[kEstTile + 32];
  if (k0 > t0) {
    int m = stage[kEstTile + lane];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) m = max(m, __shfl_xor_sync(0xffffffffu, m, o));
    if (m >= 0) {
      carry = max(carry, m);
    } else {
      // a long run of copies: continue the search from global memory
      for (int64_t q = k0 - 64; q >= t0; q -= 32) {
        int mm = rs[q + lane];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) mm = max(mm, __shfl_xor_sync(0xffffffffu, mm, o));
        if (mm >= 0) {
          carry = max(carry, mm);
          break;
        }
      }
    }
  }
  const int last = int(n - 1);
#pragma unroll
  for (int r = 0; r < kEstTile / 32; ++r) {
    const int64_t k = k0 + r * 32 + lane;
    const int v = k < n ? stage[r * 32 + lane] : -1;
    const int sk = min(max(max(warp_incl_max_i32(v), carry), 0), last);
    out[r * 32 + lane] = sk;
    carry = __shfl_sync(0xffffffffu, sk, 31);
  }
  __syncwarp();  // out[] written, stage[] read: the next issue may overwrite it
}

// FULL: the sampler's D equals DPL, so every coordinate loop, row test and
// store width is known at compile time (the same arithmetic in the same
// order as the general kernel: the results are bit for bit the same).
template <int DPL, bool MOVE, bool REWEIGHT, typename FS, bool EST = false, bool GATHER = false, bool FULL = false>
__device__ __forceinline__ void move_reweight_body(const ParticleArgs& a, const FS gp, const int blk, const int nblk) {
  constexpr int DMAX = DPL;
  static_assert(!EST || DPL <= 16, "eq. (7) records: D <= 16");
  static_assert(!GATHER || EST, "the gathering move is the records kernel's");
  // the next particle's data is loaded during the current one's arithmetic
  // when the registers allow it (up to 16 coordinates per lane)
  constexpr bool PF = DPL <= 16;
  MaxTracker mt;
  mt.init();
  // EST: eq. (7) sums of the lane's particles in the current warp tile.  They
  // are formed only when every starting log w is the same value R (the last
  // iteration resampled): then log w_i - log w_j = (lpi_i - lpc_i) - (lpi_j -
  // lpc_j) up to one FP64 rounding, so the weights need only the FP32 log pi
  // differences dlt.  The lane's sums are relative to a reference em, raised
  // (and the sums rescaled) only when a dlt exceeds it by more than 16, so
  // every term stays below e^16 and the rescale is rare.  Otherwise (weights
  // not uniform) the quantise pass reads the rows.
  const bool est_on = EST && a.st->w_uniform;
  const double R = a.st->reset_logw;
  float em = -INFINITY;
  // (est_on: the maximum of log w from the FP32 differences, see below)
  int dkey = __float_as_int(-INFINITY) ^ 0x7FFFFFFF;
  bool dnan = false;
  float eacc[EST ? DMAX : 1];
#pragma unroll
  for (int c = 0; c < (EST ? DMAX : 1); ++c) eacc[c] = 0.0f;
  const int cur = a.st->cur;
  const uint64_t t = uint64_t(a.st->t);
  float* __restrict__ x = static_cast<float*>(cur ? a.x[1] : a.x[0]);
  float* __restrict__ lp = static_cast<float*>(cur ? a.logpi[1] : a.logpi[0]);
  double* __restrict__ logw = a.logw;
  // GATHER with a pending resampling (Algorithm 5 fused into this move):
  // particle k starts from row src(k) of buffer cur with log w = reset_logw,
  // and is written to row k of the other buffer.  Otherwise in place.
  const bool gat = GATHER && a.st->pending;
  float* xd = gat ? static_cast<float*>(cur ? a.x[0] : a.x[1]) : x;
  float* lpd = gat ? static_cast<float*>(cur ? a.logpi[0] : a.logpi[1]) : lp;
  __shared__ int32_t s_src[GATHER ? kPThreads / 32 : 1][GATHER ? kEstTile : 1];
  __shared__ __align__(16) int32_t s_stage[GATHER ? kPThreads / 32 : 1][GATHER ? kStage : 4];
  int32_t* const wsrc = s_src[GATHER ? (threadIdx.x >> 5) : 0];
  int32_t* const wstage = s_stage[GATHER ? (threadIdx.x >> 5) : 0];
  // the run starts this move reads, and the other array (reset to -1 here
  // when a previous gather left it dirty; see DevState)
  const int32_t* rs_rd = nullptr;
  int32_t* rs_clr = nullptr;
  if constexpr (GATHER) {
    if (gat) {
      rs_rd = rs_now(a.rs, a.rs_alt, a.st);
      if (a.rs_alt && a.st->rs_dirty) rs_clr = a.st->rs_w ? a.rs : a.rs_alt;
    }
  }
  const int d = FULL ? DPL : a.d;
  constexpr int q = 0, c0 = 0;  // one lane per particle: it owns coordinates [0, d)
  const int nvalid = d;
  const bool vec = ((d & 3) == 0) && (nvalid >= DPL);
  const BmStep bs = bm_step(float(a.step));
  // Warp tiles of kEstTile consecutive particles (kEstChunks chunks of 32,
  // lane l takes particle 32 r + l of chunk r), tile j to warp j mod W.  The
  // loop bound is warp-uniform; lanes past the end are predicated.
  constexpr int kChunks = kEstTile / 32;
  const int64_t gw = (int64_t(blk) * blockDim.x + threadIdx.x) >> 5;
  const int64_t W = int64_t(nblk) * (blockDim.x >> 5);
  const int64_t ntile = (a.n + kEstTile - 1) / kEstTile;
  const int grp = threadIdx.x & 31;
  int64_t j = gw;
  int r = 0;
  // prologue: the first particle's data
  float xo[DPL];
  double lwc = 0.0;
  float lpc = 0.0f;
  {
    const int64_t i = j * kEstTile + grp;
    int64_t si = i;
    if constexpr (GATHER) {
      if (gat && j < ntile) {
        tile_sources_issue(rs_rd, a.tile_src, a.n, j, wstage);
        tile_sources_finish(rs_rd, a.n, j, wstage, wsrc);
        si = wsrc[grp];
        // the warp's next tile, staged while this one is processed
        if (j + W < ntile) tile_sources_issue(rs_rd, a.tile_src, a.n, j + W, wstage);
      }
    }
    if (j < ntile && i < a.n && nvalid > 0) load_seg<DPL>(x + si * d + c0, vec, nvalid, xo);
    else
#pragma unroll
      for (int c = 0; c < DPL; ++c) xo[c] = 0.0f;
    if (REWEIGHT && j < ntile && i < a.n && q == 0) {
      lwc = gat ? R : logw[i];
      lpc = lp[si];
    }
  }
  bool first = true;
  while (j < ntile) {
    const int64_t i = j * kEstTile + r * 32 + grp;
    const bool valid = i < a.n;
    if (!PF && !first) {  // (the prologue loaded the first)
      if (valid && nvalid > 0) load_seg<DPL>(x + i * d + c0, vec, nvalid, xo);
      if (REWEIGHT && valid && q == 0) {
        lwc = logw[i];
        lpc = lp[i];
      }
    }
    first = false;
    // the next particle: next chunk of this tile, or the first of the next
    const int rn = r + 1 == kChunks ? 0 : r + 1;
    const int64_t jn = r + 1 == kChunks ? j + W : j;
    const int64_t inx = jn * kEstTile + rn * 32 + grp;
    const bool vn = jn < ntile && inx < a.n;
    constexpr int kPF = PF ? DPL : 1;
    float xn[kPF];
    double lwn = 0.0;
    float lpn = 0.0f;
    if constexpr (PF) {
      int64_t sn = inx;
      if constexpr (GATHER) {
        if (gat && jn < ntile) {
          // the current tile's sources are no longer needed once its last
          // chunk is loaded: the next tile's (staged since this tile began)
          // replace them, and the tile after that is staged
          if (rn == 0) {
            tile_sources_finish(rs_rd, a.n, jn, wstage, wsrc);
            if (jn + W < ntile) tile_sources_issue(rs_rd, a.tile_src, a.n, jn + W, wstage);
          }
          sn = wsrc[rn * 32 + grp];
        }
      }
      if (vn && nvalid > 0) load_seg<kPF>(x + sn * d + c0, vec, nvalid, xn);
      else
#pragma unroll
        for (int c = 0; c < kPF; ++c) xn[c] = 0.0f;
      if (REWEIGHT && vn && q == 0) {
        lwn = gat ? R : logw[inx];
        lpn = lp[sn];
      }
    }
    if (MOVE && valid && nvalid > 0) {
      // all of the lane's Philox blocks first: independent 10-round chains
      // that the scheduler interleaves
      P4 w[DPL / 4];
#pragma unroll
      for (int b4 = 0; b4 < DPL / 4; ++b4)
        if (DPL != 8 || 4 * b4 < nvalid)  // wider classes: unconditional (interleaves better)
          w[b4] = stream_block(a.seed, t, kPurposeMove, uint64_t(i), uint32_t(c0 / 4 + b4));
#pragma unroll
      for (int b4 = 0; b4 < DPL / 4; ++b4) {
        if (4 * b4 < nvalid) {
#pragma unroll
          for (int h = 0; h < 2; ++h) {
            if (DPL == 8 && 4 * b4 + 2 * h >= nvalid) continue;  // this pair's normals are not used
            bm_pair_step(w[b4].v[2 * h], w[b4].v[2 * h + 1], bs, xo[4 * b4 + 2 * h], xo[4 * b4 + 2 * h + 1]);
          }
        }
      }
      float* row = xd + i * d + c0;
      if (vec) {
#pragma unroll
        for (int v = 0; v < DPL / 4; ++v)
          reinterpret_cast<float4*>(row)[v] = make_float4(xo[4 * v], xo[4 * v + 1], xo[4 * v + 2], xo[4 * v + 3]);
      } else {
#pragma unroll
        for (int c = 0; c < DPL; ++c)
          if (c < nvalid) row[c] = xo[c];
      }
    }
    if (REWEIGHT && valid) {
      // y = L^-1 (x - mu) row by row
      float dv[DMAX];
#pragma unroll
      for (int c = 0; c < DMAX; ++c) dv[c] = xo[c] - gp.mu(c);
      // rows 2p and 2p + 1 advance together in packed two-lane FMAs, each
      // row's terms in column order (as a scalar loop would add them)
      float qs = 0.0f;
      uint64_t dd[DMAX];
#pragma unroll
      for (int c = 0; c < DMAX; ++c) dd[c] = pack2(dv[c], dv[c]);
#pragma unroll
      for (int rr = 0; rr < DMAX; rr += 2) {
        if (rr < d) {
          const float2 acc = gp.row2(rr, dd);
          qs = fmaf(acc.x, acc.x, qs);
          if (rr + 1 < d) qs = fmaf(acc.y, acc.y, qs);
        }
      }
      // eq. (5): the log-target difference in FP32 (exact when the two
      // values are within a factor of two), one FP64 addition
      const float lpi = -0.5f * qs;
      const float dlt = lpi - lpc;
      const double lw = lwc + double(dlt);
      lpd[i] = lpi;
      logw[i] = lw;
      if constexpr (GATHER) {
        if (rs_clr) rs_clr[i] = -1;
      }
      if (EST && est_on) {
        // every log w started at R: max lw = R + double(max dlt) (R + double(x)
        // does not decrease with x), so the maximum is tracked on the FP32
        // differences with integer-ordered keys -- the same value
        const int b = __float_as_int(dlt);
        if (dlt != dlt)
          dnan = true;
        else
          dkey = max(dkey, b >= 0 ? b : (b ^ 0x7FFFFFFF));
      } else {
        mt.add(lw);
      }
      if constexpr (EST) {
        if (est_on) {
          float dl = dlt - em;
          if (dl > 16.0f) {  // the lane's reference exceeded by e^16 (always for its first particle)
            const float sc = __expf(-dl);
#pragma unroll
            for (int c = 0; c < DMAX; ++c) eacc[c] *= sc;
            em = dlt;
            dl = 0.0f;
          }
          const float e = dl == dl ? __expf(dl) : 0.0f;  // NaN only with a NaN log pi (reported)
#pragma unroll
          for (int c = 0; c < DMAX; ++c)
            if (c < d) eacc[c] = fmaf(e, xo[c], eacc[c]);
        }
      }
    }
    if constexpr (EST) {
      if (est_on && r + 1 == kChunks) {  // the tile is complete: its record, then fresh sums
        warp_write_est<DMAX>(em, R, eacc, d, a.epart + j * (1 + d));
        em = -INFINITY;
#pragma unroll
        for (int c = 0; c < DMAX; ++c) eacc[c] = 0.0f;
      }
    }
    if constexpr (PF) {
#pragma unroll
      for (int c = 0; c < kPF; ++c) xo[c] = xn[c];
      lwc = lwn;
      lpc = lpn;
    }
    r = rn;
    j = jn;
  }
  if (REWEIGHT) {
    if (EST && est_on) {
      const int b = dkey >= 0 ? dkey : (dkey ^ 0x7FFFFFFF);
      mt.add(R + double(__int_as_float(b)));
      mt.nan = mt.nan || dnan;
    }
    block_write_max(mt, a.part + 2 * blk, a.st);
  }
}

// One sampler per launch: the factor's entries are kernel parameters, read by
// the FMAs straight from the constant bank.
template <int DPL, bool MOVE, bool REWEIGHT, bool EST = false, bool GATHER = false, bool FULL = false>
__global__ void __launch_bounds__(kPThreads, 2) k_move_reweight_lanes(ParticleArgs a, const GaussParamsF32 gp) {
  move_reweight_body<DPL, MOVE, REWEIGHT, FactorParam, EST, GATHER, FULL>(a, FactorParam{gp}, blockIdx.x, gridDim.x);
}

// Batched: block b runs block map[b].y of map[b].z of sampler map[b].x; the
// sampler's factor is staged in shared memory (padded rows, 16-byte loads).
// left (standing batches of slots; NULL otherwise): a member whose count is
// not positive does nothing in this iteration, and its arguments are not
// read (an empty slot's are not valid).
__global__ void __launch_bounds__(kPThreads, 2) k_move_reweight_batch(const ParticleArgs* __restrict__ pa,
                                                                     const GaussParamsF32* __restrict__ gps,
                                                                     const int4* __restrict__ map,
                                                                     const int32_t* __restrict__ left) {
  const int4 m = map[blockIdx.x];
  if (left && left[m.x] <= 0) return;
  const ParticleArgs a = pa[m.x];
  __shared__ float4 sfac[kPairedFactor / 2];
  __shared__ float smu[kTgtMaxD];
  stage_pairs(gps[m.x].P2, gps[m.x].mu, a.d, reinterpret_cast<float2*>(sfac), smu);
  __syncthreads();
  const FactorSmem fs{sfac, smu};
  // (no D-exact instances here: with them this kernel needs more registers
  // than it has and spills, and ran slower)
  if (a.d <= 8)
    move_reweight_body<8, true, true, FactorSmem, true>(a, fs, m.y, m.z);
  else if (a.d <= 16)
    move_reweight_body<16, true, true, FactorSmem, true>(a, fs, m.y, m.z);
  else  // (D > 16: no register room for the estimate; the quantise pass forms it)
    move_reweight_body<32, true, true, FactorSmem, false>(a, fs, m.y, m.z);
}

// ---------------------------------------------------------------- finalise the maximum
// (max_finalize_body: particle_bodies.cuh)
__global__ void __launch_bounds__(kFinThreads) k_max_finalize(const double* __restrict__ part, int nb,
                                                             DevState* st) {
  max_finalize_body(part, nb, st);
}

// Batched: block s finalises sampler s over its nb[s] move blocks.
__global__ void __launch_bounds__(kFinBatchThreads) k_max_finalize_batch(const ParticleArgs* __restrict__ pa,
                                                                   const int* __restrict__ nb,
                                                                   const int32_t* __restrict__ left) {
  if (left && left[blockIdx.x] <= 0) return;
  const ParticleArgs a = pa[blockIdx.x];
  max_finalize_body(a.part, nb[blockIdx.x], a.st);
}

// ---------------------------------------------------------------- covariance
// cov_ab = sum_i w~_i (x_ia - mean_a)(x_ib - mean_b), w~_i = e^{log w_i - m} / s.
// A block stages 128 rows at a time; each thread owns up to three (a <= b)
// pairs and writes its block's sums to covpart[block][pair]; k_cov_finalize
// adds the blocks in index order (no atomics: the result does not depend on
// the order in which blocks run).
__device__ __forceinline__ void cov_pair(int p, int d, int& pa, int& pb) {
  int r = 0;
  while (p >= d - r) {
    p -= d - r;
    ++r;
  }
  pa = r;
  pb = r + p;
}

template <typename T>
__global__ void __launch_bounds__(kPThreads) k_cov(ParticleArgs a, double* cov, double* __restrict__ covpart) {
  constexpr int kChunk = 128;
  if (!cov) cov = a.st->cov_out;
  if (!cov || a.st->err) return;
  __shared__ T rows[kChunk][kMaxD + 1];
  __shared__ double wts[kChunk];
  const int cur = a.st->cur;
  const T* __restrict__ x = static_cast<const T*>(cur ? a.x[1] : a.x[0]);
  const double m = a.st->m, s = a.st->est_s;
  const int d = a.d;
  const int npairs = d * (d + 1) / 2;
  double acc[3] = {0.0, 0.0, 0.0};
  int pa[3], pb[3];
  for (int k = 0; k < 3; ++k) {
    const int p = threadIdx.x + k * blockDim.x;
    pa[k] = pb[k] = -1;
    if (p < npairs) cov_pair(p, d, pa[k], pb[k]);
  }
  for (int64_t base = int64_t(blockIdx.x) * kChunk; base < a.n; base += int64_t(gridDim.x) * kChunk) {
    if (threadIdx.x < kChunk) {
      const int64_t i = base + threadIdx.x;
      if (i < a.n) {
        for (int c = 0; c < d; ++c) rows[threadIdx.x][c] = T(double(x[i * d + c]) - a.st->mean[c]);
        const double lw = a.logw[i];
        wts[threadIdx.x] = (lw == -INFINITY) ? 0.0 : exp(lw - m) / s;
      } else {
        wts[threadIdx.x] = 0.0;
        for (int c = 0; c < d; ++c) rows[threadIdx.x][c] = T(0);
      }
    }
    __syncthreads();
    for (int k = 0; k < 3; ++k) {
      if (pa[k] < 0) continue;
      double v = 0.0;
      for (int r = 0; r < kChunk; ++r) v += wts[r] * double(rows[r][pa[k]]) * double(rows[r][pb[k]]);
      acc[k] += v;
    }
    __syncthreads();
  }
  for (int k = 0; k < 3; ++k)
    if (pa[k] >= 0) covpart[size_t(blockIdx.x) * npairs + threadIdx.x + k * blockDim.x] = acc[k];
}

// Sums the per-block covariance partials in block order; fills both triangles.
__global__ void k_cov_finalize(const DevState* st, double* cov, const double* __restrict__ covpart, int nblocks,
                               int d) {
  if (!cov) cov = st->cov_out;
  if (!cov || st->err) return;
  const int npairs = d * (d + 1) / 2;
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= npairs) return;
  double v = 0.0;
  for (int b = 0; b < nblocks; ++b) v += covpart[size_t(b) * npairs + p];
  int pa, pb;
  cov_pair(p, d, pa, pb);
  cov[pa * d + pb] = v;
  cov[pb * d + pa] = v;
}

// ---------------------------------------------------------------- bookkeeping
__global__ void k_begin(DevState* st) {
  if (threadIdx.x == 0) st->t += 1;
}

__global__ void k_commit(DevState* st, int d, int force_flip, int recycle, int defer) {
  if (threadIdx.x < 32) commit_warp(st, d, force_flip, recycle, defer);
}

__global__ void k_settle(DevState* st) {
  if (threadIdx.x == 0 && st->pending) {
    if (!st->err) st->cur ^= 1;
    st->pending = 0;
  }
}

// Batched bookkeeping: thread s handles sampler s.
__global__ void k_begin_batch(const ParticleArgs* __restrict__ pa, int count, const int32_t* __restrict__ left) {
  const int s = blockIdx.x * blockDim.x + threadIdx.x;
  if (s < count && (!left || left[s] > 0)) pa[s].st->t += 1;
}

// Batched: one warp (block) per sampler.
// (left: the member's count of iterations still to run is decremented here,
// after every other kernel of the iteration has read it)
__global__ void k_commit_batch(const ParticleArgs* __restrict__ pa, int count, int32_t* __restrict__ left) {
  const int s = blockIdx.x;
  if (s >= count || (left && left[s] <= 0)) return;
  commit_warp(pa[s].st, pa[s].d, 0, 1);
  if (left && threadIdx.x == 0) left[s] -= 1;
}

// Points every sampler's step outputs; outs holds three arrays of count
// pointers: traces, means, recycled estimates (NULL entries allowed).
__global__ void k_step_setup_batch(const ParticleArgs* __restrict__ pa, void* const* __restrict__ outs, int count) {
  const int s = blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= count) return;
  DevState* st = pa[s].st;
  st->trace = static_cast<smc_iter_stats*>(outs[s]);
  st->trace_t0 = st->t;
  st->mean_out = static_cast<double*>(outs[count + s]);
  st->fhat_out = static_cast<double*>(outs[2 * count + s]);
  st->cov_out = nullptr;
}

// Gathers and clears every sampler's device error word.
__global__ void k_take_errors_batch(const ParticleArgs* __restrict__ pa, int32_t* errs, int count) {
  const int s = blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= count) return;
  errs[s] = pa[s].st->err;
  pa[s].st->err = 0;
}

// Copies f_t out (piecewise API).
__global__ void k_copy_mean(const DevState* st, double* out, int d) {
  if (threadIdx.x < d) out[threadIdx.x] = st->mean[threadIdx.x];
}

// Points the running smc_step's outputs (read by graph-replayed kernels).
__global__ void k_step_setup(DevState* st, smc_iter_stats* trace, double* mean_out, double* fhat_out,
                             double* cov_out) {
  if (threadIdx.x != 0) return;
  st->trace = trace;
  st->trace_t0 = st->t;
  st->mean_out = mean_out;
  st->fhat_out = fhat_out;
  st->cov_out = cov_out;
}

// ---------------------------------------------------------------- launchers
template <typename T, int DMAX>
static cudaError_t launch_particles_t(int op, const ParticleArgs& a, int grid, int threads, cudaStream_t s) {
  switch (op) {
    case OP_INIT: k_init<T, DMAX><<<grid, threads, 0, s>>>(a); break;
    case OP_MOVE: k_move_reweight<T, DMAX, true, false><<<grid, threads, 0, s>>>(a); break;
    case OP_REWEIGHT: k_move_reweight<T, DMAX, false, true><<<grid, threads, 0, s>>>(a); break;
    case OP_MOVE_REWEIGHT: k_move_reweight<T, DMAX, true, true><<<grid, threads, 0, s>>>(a); break;
    default: return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

template <typename T>
static cudaError_t launch_particles_d(int op, const ParticleArgs& a, int grid, int threads, cudaStream_t s) {
  if (a.d <= 1) return launch_particles_t<T, 1>(op, a, grid, threads, s);
  if (a.d <= 2) return launch_particles_t<T, 2>(op, a, grid, threads, s);
  if (a.d <= 4) return launch_particles_t<T, 4>(op, a, grid, threads, s);
  if (a.d <= 8) return launch_particles_t<T, 8>(op, a, grid, threads, s);
  if (a.d <= 16) return launch_particles_t<T, 16>(op, a, grid, threads, s);
  return launch_particles_t<T, 32>(op, a, grid, threads, s);
}

// The iteration's kernels (move + reweight, with the eq. (7) records, with the
// gather) have a FULL instance for D equal to the width class.
template <int DPL>
static cudaError_t launch_lanes(int op, const ParticleArgs& a, int grid, int threads, cudaStream_t s,
                                const GaussParamsF32& gp) {
  const bool full = a.d == DPL;
  switch (op) {
    case OP_MOVE: k_move_reweight_lanes<DPL, true, false><<<grid, threads, 0, s>>>(a, gp); break;
    case OP_REWEIGHT: k_move_reweight_lanes<DPL, false, true><<<grid, threads, 0, s>>>(a, gp); break;
    case OP_MOVE_REWEIGHT:
      if (full)
        k_move_reweight_lanes<DPL, true, true, false, false, true><<<grid, threads, 0, s>>>(a, gp);
      else
        k_move_reweight_lanes<DPL, true, true><<<grid, threads, 0, s>>>(a, gp);
      break;
    case OP_MOVE_REWEIGHT_EST:  // D <= 16 only (register room)
      if constexpr (DPL <= 16) {
        if (full)
          k_move_reweight_lanes<DPL, true, true, true, false, true><<<grid, threads, 0, s>>>(a, gp);
        else
          k_move_reweight_lanes<DPL, true, true, true><<<grid, threads, 0, s>>>(a, gp);
        break;
      } else {
        return cudaErrorInvalidValue;
      }
    case OP_MOVE_REWEIGHT_GATHER:  // (the same, and gathers a pending resampling's rows)
      if constexpr (DPL <= 16) {
        if (full)
          k_move_reweight_lanes<DPL, true, true, true, true, true><<<grid, threads, 0, s>>>(a, gp);
        else
          k_move_reweight_lanes<DPL, true, true, true, true><<<grid, threads, 0, s>>>(a, gp);
        break;
      } else {
        return cudaErrorInvalidValue;
      }
    default: return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

cudaError_t launch_particles(int op, const ParticleArgs& a, int grid, int threads, cudaStream_t s,
                             const GaussParamsF32* gp) {
  if (threads < 32 || threads > kPThreads || threads % 32) return cudaErrorInvalidValue;
  if (a.dtype == SMC_F32 && op != OP_INIT && a.kind == SMC_GAUSS && gp) {
    if (a.d <= 8) return launch_lanes<8>(op, a, grid, threads, s, *gp);
    if (a.d <= 16) return launch_lanes<16>(op, a, grid, threads, s, *gp);
    return launch_lanes<32>(op, a, grid, threads, s, *gp);
  }
  return a.dtype == SMC_F64 ? launch_particles_d<double>(op, a, grid, threads, s)
                            : launch_particles_d<float>(op, a, grid, threads, s);
}

cudaError_t launch_target_setup(TargetDev* tg, int kind, double nu, const double* mu, const double* sigma, int d,
                                DevState* st, cudaStream_t s) {
  k_target_setup<<<1, 32, 0, s>>>(tg, kind, nu, mu, sigma, d, st);
  return cudaGetLastError();
}

cudaError_t launch_logistic_setup(TargetDev* tg, const float* X, const float* y, int m, int d, double prior_var,
                                  float* Xw, float* yw, uint16_t* ximg, cudaStream_t s) {
  k_logistic_copy<<<256, 256, 0, s>>>(tg, X, y, m, d, prior_var, Xw, yw, ximg);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  k_logistic_v<<<1, 32, 0, s>>>(tg, X, y, m, d);
  return cudaGetLastError();
}

cudaError_t launch_max_finalize(const double* part, int nb, DevState* st, cudaStream_t s) {
  k_max_finalize<<<1, kFinThreads, 0, s>>>(part, nb, st);
  return cudaGetLastError();
}

cudaError_t launch_cov(const ParticleArgs& a, double* cov, double* covpart, int grid, cudaStream_t s) {
  if (a.dtype == SMC_F64)
    k_cov<double><<<grid, kPThreads, 0, s>>>(a, cov, covpart);
  else
    k_cov<float><<<grid, kPThreads, 0, s>>>(a, cov, covpart);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  const int npairs = a.d * (a.d + 1) / 2;
  k_cov_finalize<<<(npairs + 127) / 128, 128, 0, s>>>(a.st, cov, covpart, grid, a.d);
  return cudaGetLastError();
}

cudaError_t launch_move_reweight_batch(const ParticleArgs* pa, const GaussParamsF32* gps, const int4* map, int nblocks,
                                       cudaStream_t s, const int32_t* left) {
  k_move_reweight_batch<<<nblocks, kPThreads, 0, s>>>(pa, gps, map, left);
  return cudaGetLastError();
}
cudaError_t launch_max_finalize_batch(const ParticleArgs* pa, const int* nb, int count, cudaStream_t s,
                                      const int32_t* left) {
  k_max_finalize_batch<<<count, kFinBatchThreads, 0, s>>>(pa, nb, left);
  return cudaGetLastError();
}
cudaError_t launch_begin_batch(const ParticleArgs* pa, int count, cudaStream_t s, const int32_t* left) {
  k_begin_batch<<<(count + 127) / 128, 128, 0, s>>>(pa, count, left);
  return cudaGetLastError();
}
cudaError_t launch_step_setup_batch(const ParticleArgs* pa, void* const* outs, int count, cudaStream_t s) {
  k_step_setup_batch<<<(count + 127) / 128, 128, 0, s>>>(pa, outs, count);
  return cudaGetLastError();
}
cudaError_t launch_take_errors_batch(const ParticleArgs* pa, int32_t* errs, int count, cudaStream_t s) {
  k_take_errors_batch<<<(count + 127) / 128, 128, 0, s>>>(pa, errs, count);
  return cudaGetLastError();
}
cudaError_t launch_commit_batch(const ParticleArgs* pa, int count, cudaStream_t s, int32_t* left) {
  k_commit_batch<<<count, 32, 0, s>>>(pa, count, left);
  return cudaGetLastError();
}

cudaError_t launch_begin(DevState* st, cudaStream_t s) {
  k_begin<<<1, 32, 0, s>>>(st);
  return cudaGetLastError();
}

cudaError_t launch_commit(DevState* st, int d, int force_flip, int recycle, cudaStream_t s, int defer) {
  k_commit<<<1, 32, 0, s>>>(st, d, force_flip, recycle, defer);
  return cudaGetLastError();
}

cudaError_t launch_settle(DevState* st, cudaStream_t s) {
  k_settle<<<1, 32, 0, s>>>(st);
  return cudaGetLastError();
}

cudaError_t launch_copy_mean(const DevState* st, double* out, int d, cudaStream_t s) {
  k_copy_mean<<<1, 32, 0, s>>>(st, out, d);
  return cudaGetLastError();
}

cudaError_t launch_step_setup(DevState* st, smc_iter_stats* trace, double* mean_out, double* fhat_out,
                              double* cov_out, cudaStream_t s) {
  k_step_setup<<<1, 32, 0, s>>>(st, trace, mean_out, fhat_out, cov_out);
  return cudaGetLastError();
}

}  // namespace smc
