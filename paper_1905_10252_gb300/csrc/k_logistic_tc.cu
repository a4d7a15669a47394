// k_logistic_tc.cu -- the Bayesian logistic-regression log-likelihood of every
// particle on the 5th-generation tensor cores (sm_103a), fused with the
// importance reweighting of eq. (5):
//
//   log pi(b) = b . v - sum_m softplus(z_m) - |b|^2 / (2 prior_var),
//   z = X b,  v = X^T y  (so sum_m y_m z_m = b . v needs no per-row work).
//
// Contraction.  A CTA owns a tile of 128 particles (MMA M = 128) and streams
// the data matrix through shared memory in tiles of 256 rows (MMA N = 256,
// K = 32 features, zero padded).  FP32 accuracy from BF16 tensor cores by the
// split x = hi + lo (hi = bf16(x), lo = bf16(x - hi)) on both operands:
//   z ~= B_hi X_hi + B_lo X_hi + B_hi X_lo   (FP32 accumulation in TMEM),
// dropping only B_lo X_lo (relative size 2^-16 of the product).
//
// Epilogue (the real cost: one transcendental per matrix element).  The data
// images hold X log2(e), so the accumulator holds z' = z log2 e and, with
// a = |z'|:  softplus(z) = (z + a ln 2) / 2 + ln(1 + 2^-a), so
//   sum_m softplus(z_m) = (b . w + ln 2 sum_m a_m) / 2 + ln 2 sum_m log2(1 + e_m),
// w = column sums of X (FP64, once), e_m = ex2.approx(-a_m) on the
// multi-function unit (three instructions per element: |.| accumulate, ex2,
// product); the log2 is taken once per 16 rows of a running FP32
// product prod(1 + e_m) (each factor in (1, 2], so the product stays below
// 2^16).  Zero padding rows give z = 0 exactly and contribute exactly 1 to the
// log2 sum, removed as (m_pad - m).
//
// Warp roles (20 warps): warp 0 lane 0 issues the bulk copies of the data
// tiles (4-stage ring, mbarrier complete_tx); warp 1 owns the TMEM allocation
// (512 columns: two 128 x 256 FP32 accumulators) and lane 0 issues the MMAs;
// warps 2-3 stage each particle tile's BF16 hi / lo images (double buffered,
// so the next tile is staged while the current one is contracted); warps
// 4-19 run the epilogue, four warps per TMEM lane quarter (64 columns each).
// Every
// mbarrier wait is bounded: on a timeout the CTA records SMC_ETIMEOUT, every
// role drains its remaining loop iterations without waiting (so the named
// barriers still match), waits (bounded) for its own copies in flight, frees
// TMEM and returns.
#include <atomic>

#include "smc_internal.cuh"
#include "smc_kernels.h"

namespace smc {
namespace {

constexpr int kTcPT = 128;                                  // particles per tile
constexpr int kTcStages = 4;                                // data tile ring
constexpr int kTcWarps = 20;
constexpr int kTcThreads = 32 * kTcWarps;
constexpr int kTcStageThreads = 64;                         // warps 2..3
constexpr int kTcEpiWarps = 16;                             // warps 4..19
constexpr int kTcEpiThreads = 32 * kTcEpiWarps;
constexpr int kTcEpiCols = 256 / (kTcEpiWarps / 4);         // accumulator columns per epilogue warp
constexpr uint32_t kTcCols = 512;                           // TMEM columns
constexpr size_t kTcAImg = size_t(kTcPT) * kLgK * 2;        // one BF16 A image (8 KB)
constexpr size_t kTcHalf = kLgTileBytes / 2;                // one BF16 data image (16 KB)
// data ring + two (hi, lo) A image pairs + two partial sums per particle of
// the column groups 1..3 + the ring of per-particle constant terms +
// barriers / TMEM slot / flags / warp maxima (1 KB) + alignment slack
constexpr size_t kTcSmem = kTcStages * kLgTileBytes + 4 * kTcAImg +
                           (2 * (kTcEpiWarps / 4 - 1) + 4) * kTcPT * sizeof(double) + 1024 + 1024;
constexpr long long kWaitCycles = 1ll << 31;                // ~1 s at 2 GHz

__device__ __forceinline__ uint32_t su32(const void* p) { return uint32_t(__cvta_generic_to_shared(p)); }

// tcgen05 shared-memory matrix descriptor: K-major, no swizzle; LBO = byte
// distance between core matrices adjacent in K, SBO = between 8-row groups.
__device__ __forceinline__ uint64_t mat_desc(uint32_t saddr, uint32_t lbo, uint32_t sbo) {
  return uint64_t((saddr >> 4) & 0x3FFF) | (uint64_t((lbo >> 4) & 0x3FFF) << 16) |
         (uint64_t((sbo >> 4) & 0x3FFF) << 32) | (uint64_t(1) << 46);
}

// kind::f16 instruction descriptor: FP32 accumulator, BF16 A and B, both
// K-major, N = 256, M = 128.
constexpr uint32_t kIdesc = (1u << 4) | (1u << 7) | (1u << 10) | ((256u >> 3) << 17) | ((128u >> 4) << 24);

__device__ __forceinline__ void mbar_init(uint64_t* b, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(su32(b)), "r"(count) : "memory");
}
__device__ __forceinline__ bool mbar_try(uint64_t* b, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(ok)
      : "r"(su32(b)), "r"(parity)
      : "memory");
  return ok != 0;
}
// Bounded wait; false after ~1 s (or at once when the CTA is already aborting).
__device__ __forceinline__ bool mbar_wait(uint64_t* b, uint32_t parity, volatile int* abort_flag) {
  if (*abort_flag) return false;
  if (mbar_try(b, parity)) return true;
  const long long t0 = clock64();
  while (!mbar_try(b, parity)) {
    if (*abort_flag) return false;
    if (clock64() - t0 > kWaitCycles) {
      *abort_flag = 1;
      return false;
    }
  }
  return true;
}
__device__ __forceinline__ void mbar_arrive(uint64_t* b) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(su32(b)) : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint64_t* b, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(su32(b)), "r"(bytes) : "memory");
}
__device__ __forceinline__ void bulk_g2s(void* dst, const void* src, uint32_t bytes, uint64_t* bar) {
  asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                   su32(dst)),
               "l"(src), "r"(bytes), "r"(su32(bar))
               : "memory");
}
__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void named_sync(int id, int threads) {
  asm volatile("bar.sync %0, %1;" ::"r"(id), "r"(threads) : "memory");
}
__device__ __forceinline__ void mma_bf16(uint32_t tmem_d, uint64_t da, uint64_t db, uint32_t accumulate) {
  asm volatile(
      "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
      " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(tmem_d),
      "l"(da), "l"(db), "r"(kIdesc), "r"(accumulate)
      : "memory");
}
__device__ __forceinline__ void mma_commit(uint64_t* bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(su32(bar))
               : "memory");
}
__device__ __forceinline__ void tmem_ld32(uint32_t taddr, float (&v)[32]) {
  uint32_t r[32];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
      "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];\n"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
        "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]),
        "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]),
        "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
  for (int j = 0; j < 32; ++j) v[j] = __uint_as_float(r[j]);
}
__device__ __forceinline__ float ex2_approx(float x) {
  float y;
  asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}
__device__ __forceinline__ float lg2_approx(float x) {
  float y;
  asm("lg2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}
__device__ __forceinline__ uint16_t bf16_rn(float f) {
  const uint32_t u = __float_as_uint(f);
  return uint16_t((u + 0x7FFFu + ((u >> 16) & 1u)) >> 16);
}
// byte offset of element (row r, column k) in a K-major core-matrix image
__device__ __forceinline__ uint32_t img_off(int r, int k) {
  return uint32_t((r >> 3) * 512 + (k >> 3) * 128 + (r & 7) * 16 + (k & 7) * 2);
}

__global__ void __launch_bounds__(kTcThreads, 1) k_logistic_tc(ParticleArgs a) {
  extern __shared__ uint8_t smem_raw[];
  uint8_t* sm = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  uint8_t* xs = sm;                                         // kTcStages x (hi | lo) data tiles
  uint8_t* aimg = xs + kTcStages * kLgTileBytes;            // [2] x (hi, lo) particle tile images
  constexpr int kGroups = kTcEpiWarps / 4;                  // column groups per lane quarter
  // [kGroups - 1][128][2]: |z| and log2 sums of the column groups 1..3
  double* s_part = reinterpret_cast<double*>(aimg + 4 * kTcAImg);
  // [4][128]: per particle b.v - b.w / 2 - |b|^2 / (2 prior_var), a ring of
  // 4 particle tiles written by the stager warps
  double* s_pre = s_part + (kGroups - 1) * kTcPT * 2;
  uint64_t* full = reinterpret_cast<uint64_t*>(s_pre + 4 * kTcPT);
  uint64_t* empty = full + kTcStages;
  uint64_t* tfull = empty + kTcStages;
  uint64_t* tempty = tfull + 2;
  uint64_t* afull = tempty + 2;
  uint64_t* aempty = afull + 2;
  uint64_t* prefull = aempty + 2;  // [4]
  uint32_t* tslot = reinterpret_cast<uint32_t*>(prefull + 4);
  volatile int* abort_flag = reinterpret_cast<volatile int*>(tslot + 1);
  long long* wmax = reinterpret_cast<long long*>(tslot + 4);  // [kTcWarps]
  int* wnan = reinterpret_cast<int*>(wmax + kTcWarps);

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const TargetDev* __restrict__ tg = a.tg;
  const int cur = a.st->cur;
  const float* __restrict__ x = static_cast<const float*>(cur ? a.x[1] : a.x[0]);
  float* __restrict__ lp = static_cast<float*>(cur ? a.logpi[1] : a.logpi[0]);
  const int64_t n = a.n;
  const int d = a.d;
  const int nx = tg->m_pad / kLgRows;
  const int64_t npt = (n + kTcPT - 1) / kTcPT;

  if (threadIdx.x == 0) {
    for (int s = 0; s < kTcStages; ++s) {
      mbar_init(&full[s], 1);
      mbar_init(&empty[s], 1);
    }
    for (int b = 0; b < 2; ++b) {
      mbar_init(&tfull[b], 1);
      mbar_init(&tempty[b], kTcEpiWarps);
      mbar_init(&afull[b], kTcStageThreads);
      mbar_init(&aempty[b], 1);
    }
    for (int r = 0; r < 4; ++r) mbar_init(&prefull[r], kTcStageThreads);
    *abort_flag = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 1) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(su32(tslot)),
                 "r"(kTcCols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *tslot;

  MaxTracker mt;
  mt.init();

  if (warp == 0) {
    // ------------------------------------------------------------ producer
    if (lane == 0) {
      uint32_t g = 0;
      const uint8_t* img = reinterpret_cast<const uint8_t*>(tg->ximg);
      for (int64_t pt = blockIdx.x; pt < npt; pt += gridDim.x) {
        for (int j = 0; j < nx; ++j, ++g) {
          if (a.flags & PA_STALL_COPIES) continue;  // test hook: the consumers' waits run out
          const int s = int(g % kTcStages);
          const uint32_t r = g / kTcStages;
          if (!mbar_wait(&empty[s], (r & 1) ^ 1, abort_flag)) continue;
          mbar_expect_tx(&full[s], uint32_t(kLgTileBytes));
          bulk_g2s(xs + size_t(s) * kLgTileBytes, img + size_t(j) * kLgTileBytes, uint32_t(kLgTileBytes), &full[s]);
        }
      }
      // after an abort: let copies still in flight land before the CTA exits
      if (*abort_flag) {
        const uint32_t last = g;
        for (uint32_t k = (last > kTcStages ? last - kTcStages : 0); k < last; ++k) {
          const int s = int(k % kTcStages);
          const long long t0 = clock64();
          while (!mbar_try(&full[s], (k / kTcStages) & 1) && clock64() - t0 < kWaitCycles) {
          }
        }
      }
    }
    __syncwarp();
  } else if (warp == 1) {
    // ------------------------------------------------------------ MMA issuer
    if (lane == 0) {
      uint32_t g = 0, u = 0, v = 0;
      for (int64_t pt = blockIdx.x; pt < npt; pt += gridDim.x, ++v) {
        const int ab = int(v & 1);
        const bool have_a = mbar_wait(&afull[ab], (v >> 1) & 1, abort_flag);
        tc_fence_after();
        const uint32_t ah = su32(aimg + size_t(2 * ab) * kTcAImg), al = ah + uint32_t(kTcAImg);
        for (int j = 0; j < nx; ++j, ++g, ++u) {
          const int s = int(g % kTcStages);
          const int b = int(u & 1);
          if (!have_a) continue;
          if (!mbar_wait(&full[s], (g / kTcStages) & 1, abort_flag)) continue;
          if (!mbar_wait(&tempty[b], ((u >> 1) & 1) ^ 1, abort_flag)) continue;
          tc_fence_after();
          const uint32_t dcol = tmem + uint32_t(b) * 256;
          const uint32_t xh = su32(xs + size_t(s) * kLgTileBytes), xl = xh + uint32_t(kTcHalf);
          uint32_t acc = 0;
#pragma unroll
          for (int kk = 0; kk < 2; ++kk) {
            mma_bf16(dcol, mat_desc(ah + kk * 256, 128, 512), mat_desc(xh + kk * 256, 128, 512), acc);
            acc = 1;
            mma_bf16(dcol, mat_desc(al + kk * 256, 128, 512), mat_desc(xh + kk * 256, 128, 512), 1);
            mma_bf16(dcol, mat_desc(ah + kk * 256, 128, 512), mat_desc(xl + kk * 256, 128, 512), 1);
          }
          mma_commit(&empty[s]);
          mma_commit(&tfull[b]);
        }
        // the A images of this tile are free once its MMAs have completed
        if (have_a) mma_commit(&aempty[ab]);
      }
    }
    __syncwarp();
  } else if (warp < 4) {
    // ------------------------------------------------------------ A image stager
    const int t = threadIdx.x - 64;
    uint32_t v = 0;
    for (int64_t pt = blockIdx.x; pt < npt; pt += gridDim.x, ++v) {
      const int ab = int(v & 1);
      const bool free_buf = __all_sync(0xffffffffu, mbar_wait(&aempty[ab], ((v >> 1) & 1) ^ 1, abort_flag));
      if (free_buf) {
        uint8_t* ahi = aimg + size_t(2 * ab) * kTcAImg;
        uint8_t* alo = ahi + kTcAImg;
        // every load of the thread is issued before the conversions, so the
        // tile's memory latency is paid about once (with few data tiles per
        // particle tile -- small M -- this staging sets the kernel's pace)
        if ((d & 3) == 0) {
          // 16-byte loads: thread t takes the groups e = t + 64 u of four
          // consecutive features (r = e / 8, k = 4 (e % 8)); a row of d
          // features is d / 4 such groups, the rest of the 32 are zero
          constexpr int kG = kTcPT * kLgK / 4 / kTcStageThreads;  // 16
          float4 vals[kG];
#pragma unroll
          for (int u = 0; u < kG; ++u) {
            const int e = t + kTcStageThreads * u;
            const int r = e >> 3, k = (e & 7) << 2;
            const int64_t i = pt * kTcPT + r;
            vals[u] = (i < n && k < d) ? *reinterpret_cast<const float4*>(x + i * d + k)
                                       : make_float4(0.0f, 0.0f, 0.0f, 0.0f);
          }
#pragma unroll
          for (int u = 0; u < kG; ++u) {
            const int e = t + kTcStageThreads * u;
            const int r = e >> 3, k = (e & 7) << 2;
            const float f[4] = {vals[u].x, vals[u].y, vals[u].z, vals[u].w};
            uint16_t hi[4], lo[4];
#pragma unroll
            for (int c = 0; c < 4; ++c) {
              hi[c] = bf16_rn(f[c]);
              lo[c] = bf16_rn(f[c] - __uint_as_float(uint32_t(hi[c]) << 16));
            }
            // features k .. k + 3 are adjacent in the core-matrix image
            *reinterpret_cast<uint2*>(ahi + img_off(r, k)) =
                make_uint2(uint32_t(hi[0]) | (uint32_t(hi[1]) << 16), uint32_t(hi[2]) | (uint32_t(hi[3]) << 16));
            *reinterpret_cast<uint2*>(alo + img_off(r, k)) =
                make_uint2(uint32_t(lo[0]) | (uint32_t(lo[1]) << 16), uint32_t(lo[2]) | (uint32_t(lo[3]) << 16));
          }
        } else {
          constexpr int kB = 8;  // loads in flight per thread
          for (int e0 = t; e0 < kTcPT * kLgK; e0 += kTcStageThreads * kB) {
            float vals[kB];
#pragma unroll
            for (int u = 0; u < kB; ++u) {
              const int e = e0 + kTcStageThreads * u;
              const int r = e / kLgK, k = e % kLgK;
              const int64_t i = pt * kTcPT + r;
              vals[u] = (i < n && k < d) ? x[i * d + k] : 0.0f;
            }
#pragma unroll
            for (int u = 0; u < kB; ++u) {
              const int e = e0 + kTcStageThreads * u;
              const int r = e / kLgK, k = e % kLgK;
              const uint16_t hi = bf16_rn(vals[u]);
              const uint16_t lo = bf16_rn(vals[u] - __uint_as_float(uint32_t(hi) << 16));
              *reinterpret_cast<uint16_t*>(ahi + img_off(r, k)) = hi;
              *reinterpret_cast<uint16_t*>(alo + img_off(r, k)) = lo;
            }
          }
        }
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
      }
      mbar_arrive(&afull[ab]);
      // the FP64 part of log pi for each particle (two per thread), kept off
      // the epilogue warps: b.v - (b.w) / 2 - |b|^2 / (2 prior_var).  Slot
      // v % 4 is free: writing tile v requires the MMAs of tile v - 2 to have
      // completed, hence the epilogue to have finished tile v - 4.
      if (!*abort_flag) {
        double* pre = s_pre + size_t(v & 3) * kTcPT;
        for (int r = t; r < kTcPT; r += kTcStageThreads) {
          const int64_t i = pt * kTcPT + r;
          double bv = 0.0, bw = 0.0, b2 = 0.0;
          if (i < n)
            for (int c = 0; c < d; ++c) {
              const double bc = double(x[i * d + c]);
              bv = fma(bc, tg->v[c], bv);
              bw = fma(bc, tg->xsum[c], bw);
              b2 = fma(bc, bc, b2);
            }
          pre[r] = bv - 0.5 * bw - b2 / (2.0 * tg->prior_var);
        }
      }
      mbar_arrive(&prefull[v & 3]);
    }
  } else {
    // ------------------------------------------------------------ epilogue
    const int q = warp & 3, h = (warp - 4) >> 2;
    const int row = 32 * q + lane;
    uint32_t u = 0, v = 0;
    const double log2_pad = double(tg->m_pad - tg->m);
    for (int64_t pt = blockIdx.x; pt < npt; pt += gridDim.x, ++v) {
      const int64_t i = pt * kTcPT + row;
      double acc_abs = 0.0, acc_lg = 0.0;
      float fabs4 = 0.0f, flg4 = 0.0f;  // FP32 sums over up to 8 data tiles
      for (int j = 0; j < nx; ++j, ++u) {
        const int b = int(u & 1);
        // warp-uniform outcome: tcgen05.ld below is a warp-collective
        const bool ready = __all_sync(0xffffffffu, mbar_wait(&tfull[b], (u >> 1) & 1, abort_flag));
        if (ready) {
          tc_fence_after();
#pragma unroll 1
          for (int c = 0; c < kTcEpiCols / 32; ++c) {
            float z[32];
            tmem_ld32(tmem + (uint32_t(32 * q) << 16) + uint32_t(b * 256 + h * kTcEpiCols + c * 32), z);
#pragma unroll
            for (int g16 = 0; g16 < 2; ++g16) {
              float prod = 1.0f;
#pragma unroll
              for (int e = 0; e < 16; ++e) {
                const float az = fabsf(z[16 * g16 + e]);  // |z| log2 e (the images are scaled)
                fabs4 += az;
                prod = fmaf(prod, ex2_approx(-az), prod);
              }
              flg4 += lg2_approx(prod);
            }
          }
        }
        tc_fence_before();
        __syncwarp();
        if (lane == 0) mbar_arrive(&tempty[b]);
        if ((j & 7) == 7 || j == nx - 1) {
          acc_abs += double(fabs4);
          acc_lg += double(flg4);
          fabs4 = flg4 = 0.0f;
        }
      }
      if (h > 0) {
        double* sp = s_part + ((h - 1) * kTcPT + row) * 2;
        sp[0] = acc_abs;
        sp[1] = acc_lg;
      }
      named_sync(2, kTcEpiThreads);
      if (h == 0) {
        // the constant term of this tile (written by the stager warps)
        const bool have_pre = __all_sync(0xffffffffu, mbar_wait(&prefull[v & 3], (v >> 2) & 1, abort_flag));
        if (i < n && have_pre && !*abort_flag) {
          double sum_abs = acc_abs, sum_lg = acc_lg - log2_pad;
#pragma unroll
          for (int g2 = 0; g2 < kGroups - 1; ++g2) {
            const double* sp = s_part + (g2 * kTcPT + row) * 2;
            sum_abs += sp[0];
            sum_lg += sp[1];
          }
          const double ln2 = 0.6931471805599453;
          const float lpn = float(s_pre[(v & 3) * kTcPT + row] - 0.5 * ln2 * sum_abs - ln2 * sum_lg);
          // eq. (5): the log-target difference in FP32 (exact when the two
          // values are within a factor of two), one FP64 addition
          const double lw = a.logw[i] + double(lpn - lp[i]);
          lp[i] = lpn;
          a.logw[i] = lw;
          mt.add(lw);
        }
      }
      named_sync(2, kTcEpiThreads);  // partial sums read before the next tile writes them
    }
  }

  // ------------------------------------------------------------ block maximum, teardown
  __syncwarp();
  {
    const long long wm = warp_max_ll(mt.best);
    const int wn = __any_sync(0xffffffffu, mt.nan);
    if (lane == 0) {
      wmax[warp] = wm;
      wnan[warp] = wn;
    }
  }
  tc_fence_before();
  __syncthreads();
  if (threadIdx.x == 0) {
    long long v = wmax[0];
    int nan = wnan[0];
    for (int w = 1; w < kTcWarps; ++w) {
      v = wmax[w] > v ? wmax[w] : v;
      nan |= wnan[w];
    }
    a.part[2 * blockIdx.x] = from_ordered_key(v);
    a.part[2 * blockIdx.x + 1] = 1.0;
    if (nan) record_error(a.st, SMC_ENONFINITE);
    if (*abort_flag) record_error(a.st, SMC_ETIMEOUT);
  }
  if (warp == 1) {
    tc_fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(kTcCols) : "memory");
  }
}

}  // namespace

int logistic_tc_grid(int64_t n, int sms) {
  const int64_t npt = (n + kTcPT - 1) / kTcPT;
  return int(npt < sms ? npt : sms);
}

cudaError_t launch_logistic_tc(const ParticleArgs& a, int grid, cudaStream_t s) {
  // the dynamic shared-memory limit is a per-device attribute of the kernel
  static std::atomic<bool> configured[64];
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= 64) return cudaErrorInvalidDevice;
  if (!configured[dev].load()) {
    e = cudaFuncSetAttribute(k_logistic_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, int(kTcSmem));
    if (e != cudaSuccess) return e;
    configured[dev].store(true);
  }
  k_logistic_tc<<<grid, kTcThreads, kTcSmem, s>>>(a);
  return cudaGetLastError();
}

}  // namespace smc
