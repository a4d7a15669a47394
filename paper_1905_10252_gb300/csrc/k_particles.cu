// k_particles.cu -- element-wise stages of one SMC iteration on sm_103a:
//   * target set-up (Cholesky of Sigma, its inverse, FP32 copies),
//   * initialisation (Algorithm 2, line 1),
//   * random-walk move and importance reweighting (Algorithm 2, line 4; eq. (5)),
//     fused in one pass over the particle rows,
//   * the per-block partials of max log w and of the weighted mean (eq. (7)),
//     combined by a single-block finaliser,
//   * the weighted covariance (diagnostic),
//   * the iteration bookkeeping kernels (begin / commit, eq. (6) recycling).
//
// One thread owns one particle row at a time (grid-stride over N); rows are
// read and written with the widest aligned vector the row allows.  The FP64
// path uses explicitly rounded operations only, in the same order as the
// paper's definitions, so its results are reproducible bit for bit.
#include <cfloat>
#include <cmath>

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

// ---------------------------------------------------------------- log targets
// Gaussian, FP64: forward substitution z = L^-1 (x - mu), log pi = -1/2 |z|^2.
template <int DMAX>
__device__ __forceinline__ double logpi_gauss(const double (&x)[DMAX], int d, const double* __restrict__ L,
                                              const double* __restrict__ mu) {
  double z[DMAX];
  double q = 0.0;
#pragma unroll
  for (int r = 0; r < DMAX; ++r) {
    if (r < d) {
      double acc = __dsub_rn(x[r], mu[r]);
#pragma unroll
      for (int c = 0; c < r; ++c) acc = __fma_rn(-L[r * kMaxD + c], z[c], acc);
      z[r] = __ddiv_rn(acc, L[r * kMaxD + r]);
      q = __fma_rn(z[r], z[r], q);
    }
  }
  return __dmul_rn(-0.5, q);
}

// Gaussian, FP32: y = P (x - mu) with the precomputed inverse factor.
template <int DMAX>
__device__ __forceinline__ float logpi_gauss(const float (&x)[DMAX], int d, const float* __restrict__ P,
                                             const float* __restrict__ mu) {
  float dv[DMAX];
#pragma unroll
  for (int c = 0; c < DMAX; ++c) dv[c] = c < d ? x[c] - mu[c] : 0.0f;
  float q = 0.0f;
#pragma unroll
  for (int r = 0; r < DMAX; ++r) {
    if (r < d) {
      float acc = 0.0f;
#pragma unroll
      for (int c = 0; c <= r; ++c) acc = fmaf(P[r * kMaxD + c], dv[c], acc);
      q = fmaf(acc, acc, q);
    }
  }
  return -0.5f * q;
}

// Student-t, D = 1 (eq. (14) up to its constant).
__device__ __forceinline__ double logpi_student(double x, double mu, double nu) {
  const double dd = x - mu;
  return -0.5 * (nu + 1.0) * log1p(dd * dd / nu);
}
__device__ __forceinline__ float logpi_student(float x, float mu, float nu) {
  const float dd = x - mu;
  return -0.5f * (nu + 1.0f) * log1pf(dd * dd / nu);
}

// ---------------------------------------------------------------- row I/O
template <typename T, int DMAX>
__device__ __forceinline__ void load_row(const T* __restrict__ p, int d, T (&x)[DMAX]) {
  if (d == DMAX && (DMAX * sizeof(T)) % 16 == 0) {
    const float4* q = reinterpret_cast<const float4*>(p);
#pragma unroll
    for (int v = 0; v < int(DMAX * sizeof(T) / 16); ++v) {
      const float4 f = q[v];
      reinterpret_cast<float4*>(x)[v] = f;
    }
  } else {
#pragma unroll
    for (int c = 0; c < DMAX; ++c) x[c] = c < d ? p[c] : T(0);
  }
}

template <typename T, int DMAX>
__device__ __forceinline__ void store_row(T* __restrict__ p, int d, const T (&x)[DMAX]) {
  if (d == DMAX && (DMAX * sizeof(T)) % 16 == 0) {
    float4* q = reinterpret_cast<float4*>(p);
#pragma unroll
    for (int v = 0; v < int(DMAX * sizeof(T) / 16); ++v) q[v] = reinterpret_cast<const float4*>(x)[v];
  } else {
#pragma unroll
    for (int c = 0; c < DMAX; ++c)
      if (c < d) p[c] = x[c];
  }
}

// ---------------------------------------------------------------- online weighted sums
// Per-thread running (max m, sum e, sum e x) with e = exp(log w - m); the
// accumulators are rescaled when a larger log-weight arrives.
template <typename A, int DMAX>
struct Online {
  double m;
  A s;
  A sx[DMAX];
  bool nan;
  __device__ __forceinline__ void init() {
    m = -INFINITY;
    s = A(0);
#pragma unroll
    for (int c = 0; c < DMAX; ++c) sx[c] = A(0);
    nan = false;
  }
  template <typename T>
  __device__ __forceinline__ void add(double lw, const T (&x)[DMAX]) {
    if (isnan(lw)) {
      nan = true;
      return;
    }
    if (lw == -INFINITY) return;
    if (lw > m) {
      const A sc = (m == -INFINITY) ? A(0) : A(exp_a(A(m - lw)));
      s = s * sc + A(1);
#pragma unroll
      for (int c = 0; c < DMAX; ++c) sx[c] = sx[c] * sc + A(x[c]);
      m = lw;
    } else {
      const A e = exp_a(A(lw - m));
      s += e;
#pragma unroll
      for (int c = 0; c < DMAX; ++c) sx[c] += e * A(x[c]);
    }
  }
  __device__ __forceinline__ static float exp_a(float v) { return __expf(v); }
  __device__ __forceinline__ static double exp_a(double v) { return exp(v); }
};

// Block-combine the online partials and write one record per block:
// part[b * (2 + d) + {0: m, 1: s, 2..: s x}].
template <typename A, int DMAX>
__device__ __forceinline__ void block_write_partial(Online<A, DMAX>& on, int d, double* __restrict__ part,
                                                    DevState* st) {
  __shared__ double sh[kPThreads / 32][DMAX + 2];
  __shared__ double shm[kPThreads / 32];
  __shared__ double mb;
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
  if (on.nan) record_error(st, SMC_ENONFINITE);
  double wm = warp_max(on.m);
  if (lane == 0) shm[wid] = wm;
  __syncthreads();
  if (threadIdx.x == 0) {
    double v = -INFINITY;
    for (int w = 0; w < nw; ++w) v = fmax(v, shm[w]);
    mb = v;
  }
  __syncthreads();
  const double scale = (on.m == -INFINITY) ? 0.0 : exp(on.m - mb);
  double v = double(on.s) * scale;
  v = warp_sum(v);
  if (lane == 0) sh[wid][0] = v;
#pragma unroll
  for (int c = 0; c < DMAX; ++c) {
    if (c < d) {
      double u = warp_sum(double(on.sx[c]) * scale);
      if (lane == 0) sh[wid][1 + c] = u;
    }
  }
  __syncthreads();
  if (threadIdx.x < d + 1) {
    double acc = 0.0;
    for (int w = 0; w < nw; ++w) acc += sh[w][threadIdx.x];
    part[blockIdx.x * (2 + d) + 1 + threadIdx.x] = acc;
  }
  if (threadIdx.x == 0) part[blockIdx.x * (2 + d)] = mb;
}

template <typename T>
struct TargetSmem {
  T mu[kMaxD];
  T F[kMaxD * kMaxD];  // L (FP64 path) or P (FP32 path)
};

template <typename T>
__device__ __forceinline__ void load_target(const TargetDev* __restrict__ tg, int d, TargetSmem<T>& s);
template <>
__device__ __forceinline__ void load_target<double>(const TargetDev* __restrict__ tg, int d,
                                                    TargetSmem<double>& s) {
  for (int i = threadIdx.x; i < kMaxD * kMaxD; i += blockDim.x) s.F[i] = tg->L[i];
  for (int i = threadIdx.x; i < kMaxD; i += blockDim.x) s.mu[i] = tg->mu[i];
  __syncthreads();
}
template <>
__device__ __forceinline__ void load_target<float>(const TargetDev* __restrict__ tg, int d, TargetSmem<float>& s) {
  for (int i = threadIdx.x; i < kMaxD * kMaxD; i += blockDim.x) s.F[i] = tg->Pf[i];
  for (int i = threadIdx.x; i < kMaxD; i += blockDim.x) s.mu[i] = tg->muf[i];
  __syncthreads();
}

template <typename T, int DMAX>
__device__ __forceinline__ T eval_logpi(const T (&x)[DMAX], int d, int kind, const TargetSmem<T>& ts, T nu) {
  if (kind == SMC_STUDENT_T) return logpi_student(x[0], ts.mu[0], nu);
  return logpi_gauss<DMAX>(x, d, ts.F, ts.mu);
}

// ---------------------------------------------------------------- init
// x0 = s z (z from the INIT stream at t = 0), log w0 = log pi(x0) - log q0(x0),
// log q0(x) = (-1/2 |x|^2) / s^2.
template <typename T, int DMAX>
__global__ void __launch_bounds__(kPThreads) k_init(ParticleArgs a) {
  __shared__ TargetSmem<T> ts;
  load_target<T>(a.tg, a.d, ts);
  using A = T;
  Online<A, DMAX> on;
  on.init();
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
      const double lpi = eval_logpi<T, DMAX>(xr, a.d, a.kind, ts, nu);
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
      const float lpi = eval_logpi<T, DMAX>(xr, a.d, a.kind, ts, nu);
      const float lq0 = (-0.5f * q) / (s * s);
      lw = double(lpi) - double(lq0);
      lp[i] = lpi;
    }
    store_row<T, DMAX>(x + i * a.d, a.d, xr);
    a.logw[i] = lw;
    on.add(lw, xr);
  }
  block_write_partial<A, DMAX>(on, a.d, a.part, a.st);
}

// ---------------------------------------------------------------- move + reweight
// MOVE:     x_t = x_{t-1} + eps z, z from the MOVE stream at iteration t.
// REWEIGHT: log w_t = log w_{t-1} + (log pi(x_t) - log pi(x_{t-1})); the
//           forward-kernel L/q factor of eq. (5) is exactly one.
// Works in place on the current buffers.
template <typename T, int DMAX, bool MOVE, bool REWEIGHT>
__global__ void __launch_bounds__(kPThreads) k_move_reweight(ParticleArgs a) {
  __shared__ TargetSmem<T> ts;
  if (REWEIGHT) load_target<T>(a.tg, a.d, ts);
  using A = T;
  Online<A, DMAX> on;
  on.init();
  const int cur = a.st->cur;
  const uint64_t t = uint64_t(a.st->t);
  T* __restrict__ x = static_cast<T*>(cur ? a.x[1] : a.x[0]);
  T* __restrict__ lp = static_cast<T*>(cur ? a.logpi[1] : a.logpi[0]);
  const T nu = T(a.tg->nu);
  for (int64_t i = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; i < a.n; i += int64_t(gridDim.x) * blockDim.x) {
    T xr[DMAX];
    load_row<T, DMAX>(x + i * a.d, a.d, xr);
    if (MOVE) {
      if constexpr (sizeof(T) == 8) {
        double z[DMAX];
        normals_f64<DMAX>(a.seed, t, kPurposeMove, uint64_t(i), a.d, z);
#pragma unroll
        for (int c = 0; c < DMAX; ++c)
          if (c < a.d) xr[c] = __fma_rn(a.step, z[c], xr[c]);
      } else {
        float z[DMAX];
        normals_f32<DMAX>(a.seed, t, kPurposeMove, uint64_t(i), a.d, z);
        const float eps = float(a.step);
#pragma unroll
        for (int c = 0; c < DMAX; ++c)
          if (c < a.d) xr[c] = fmaf(eps, z[c], xr[c]);
      }
      store_row<T, DMAX>(x + i * a.d, a.d, xr);
    }
    if (REWEIGHT) {
      const T lpi = eval_logpi<T, DMAX>(xr, a.d, a.kind, ts, nu);
      const T lpp = lp[i];
      double lw;
      if constexpr (sizeof(T) == 8)
        lw = __dadd_rn(a.logw[i], __dsub_rn(lpi, lpp));
      else
        lw = a.logw[i] + (double(lpi) - double(lpp));
      lp[i] = lpi;
      a.logw[i] = lw;
      on.add(lw, xr);
    }
  }
  if (REWEIGHT) block_write_partial<A, DMAX>(on, a.d, a.part, a.st);
}

// ---------------------------------------------------------------- finalise max + mean
// Single block: m = max_b m_b, s = sum_b s_b e^{m_b - m}, mean = sum_b sx_b e^{m_b-m} / s.
__global__ void __launch_bounds__(kFinThreads) k_est_finalize(const double* __restrict__ part, int nb, int d,
                                                             DevState* st, int write_mean_out) {
  __shared__ double shm[32];
  __shared__ double sh[32][kMaxD + 1];
  __shared__ double mall;
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
  const int stride = 2 + d;
  double m = -INFINITY;
  for (int b = threadIdx.x; b < nb; b += blockDim.x) m = fmax(m, part[b * stride]);
  m = warp_max(m);
  if (lane == 0) shm[wid] = m;
  __syncthreads();
  if (threadIdx.x == 0) {
    double v = -INFINITY;
    for (int w = 0; w < nw; ++w) v = fmax(v, shm[w]);
    mall = v;
  }
  __syncthreads();
  const double M = mall;
  double acc[kMaxD + 1];
#pragma unroll
  for (int c = 0; c <= kMaxD; ++c) acc[c] = 0.0;
  for (int b = threadIdx.x; b < nb; b += blockDim.x) {
    const double mb = part[b * stride];
    const double sc = (mb == -INFINITY) ? 0.0 : exp(mb - M);
#pragma unroll
    for (int c = 0; c <= kMaxD; ++c)
      if (c <= d) acc[c] += part[b * stride + 1 + c] * sc;
  }
#pragma unroll
  for (int c = 0; c <= kMaxD; ++c) {
    if (c <= d) {
      const double v = warp_sum(acc[c]);
      if (lane == 0) sh[wid][c] = v;
    }
  }
  __syncthreads();
  if (threadIdx.x <= d) {
    double v = 0.0;
    for (int w = 0; w < nw; ++w) v += sh[w][threadIdx.x];
    sh[0][threadIdx.x] = v;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    const double s = sh[0][0];
    st->m = M;
    st->est_s = s;
    if (!(M > -INFINITY && M < INFINITY) || !(s > 0.0 && s < INFINITY)) record_error(st, SMC_ENONFINITE);
  }
  if (threadIdx.x < d) {
    const double mean = sh[0][1 + threadIdx.x] / sh[0][0];
    st->mean[threadIdx.x] = mean;
    if (write_mean_out && st->mean_out) st->mean_out[threadIdx.x] = mean;
  }
}

// ---------------------------------------------------------------- covariance
// cov_ab = sum_i w~_i (x_ia - mean_a)(x_ib - mean_b), w~_i = e^{log w_i - m} / s;
// a block stages 256 rows, each thread owns (a, b) pairs; atomics into cov.
template <typename T>
__global__ void __launch_bounds__(kPThreads) k_cov(ParticleArgs a, double* cov) {
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
    int p = threadIdx.x + k * blockDim.x;
    pa[k] = pb[k] = -1;
    if (p < npairs) {
      int r = 0;
      while (p >= d - r) {
        p -= d - r;
        ++r;
      }
      pa[k] = r;
      pb[k] = r + p;
    }
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
  for (int k = 0; k < 3; ++k) {
    if (pa[k] < 0) continue;
    atomicAdd(&cov[pa[k] * d + pb[k]], acc[k]);
    if (pa[k] != pb[k]) atomicAdd(&cov[pb[k] * d + pa[k]], acc[k]);
  }
}

// ---------------------------------------------------------------- bookkeeping
__global__ void k_begin(DevState* st) {
  if (threadIdx.x == 0) st->t += 1;
}

// Ends iteration t: swap buffers if resampled (or if forced by an explicit
// redistribute), LSE_{t} becomes the next LSE_{t-1} (0 after a reset), and
// the recycling sums of eq. (6) take f_t with weight c_t.
__global__ void k_commit(DevState* st, int d, int force_flip, int recycle) {
  if (threadIdx.x != 0) return;
  const bool flip = force_flip || (st->flag && !st->err);
  if (recycle && !st->err) {
    const double lc = st->logc;
    const double M = fmax(st->rc_max, lc);
    const double sc = (st->rc_max == -INFINITY) ? 0.0 : exp(st->rc_max - M);
    const double e = exp(lc - M);
    st->rc_den = st->rc_den * sc + e;
    for (int c = 0; c < d; ++c) st->rc_num[c] = st->rc_num[c] * sc + e * st->mean[c];
    st->rc_max = M;
    if (st->fhat_out)
      for (int c = 0; c < d; ++c) st->fhat_out[c] = st->rc_num[c] / st->rc_den;
  }
  if (st->flag && !st->err) {
    st->last.survivors = (int64_t)st->survivors;
    if (st->trace) {
      const int64_t idx = st->t - st->trace_t0 - 1;
      if (idx >= 0) st->trace[idx].survivors = (int64_t)st->survivors;
    }
  }
  if (flip) st->cur ^= 1;
  st->lse_prev = flip ? 0.0 : st->lse;
}

// Zeroes the covariance output named by the running smc_step.
__global__ void k_zero_cov(DevState* st, int d) {
  double* c = st->cov_out;
  if (!c) return;
  for (int i = threadIdx.x; i < d * d; i += blockDim.x) c[i] = 0.0;
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
static cudaError_t launch_particles_t(int op, const ParticleArgs& a, int grid, cudaStream_t s) {
  switch (op) {
    case OP_INIT: k_init<T, DMAX><<<grid, kPThreads, 0, s>>>(a); break;
    case OP_MOVE: k_move_reweight<T, DMAX, true, false><<<grid, kPThreads, 0, s>>>(a); break;
    case OP_REWEIGHT: k_move_reweight<T, DMAX, false, true><<<grid, kPThreads, 0, s>>>(a); break;
    case OP_MOVE_REWEIGHT: k_move_reweight<T, DMAX, true, true><<<grid, kPThreads, 0, s>>>(a); break;
    default: return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

template <typename T>
static cudaError_t launch_particles_d(int op, const ParticleArgs& a, int grid, cudaStream_t s) {
  if (a.d <= 1) return launch_particles_t<T, 1>(op, a, grid, s);
  if (a.d <= 2) return launch_particles_t<T, 2>(op, a, grid, s);
  if (a.d <= 4) return launch_particles_t<T, 4>(op, a, grid, s);
  if (a.d <= 8) return launch_particles_t<T, 8>(op, a, grid, s);
  if (a.d <= 16) return launch_particles_t<T, 16>(op, a, grid, s);
  return launch_particles_t<T, 32>(op, a, grid, s);
}

cudaError_t launch_particles(int op, const ParticleArgs& a, int grid, cudaStream_t s) {
  return a.dtype == SMC_F64 ? launch_particles_d<double>(op, a, grid, s) : launch_particles_d<float>(op, a, grid, s);
}

cudaError_t launch_target_setup(TargetDev* tg, int kind, double nu, const double* mu, const double* sigma, int d,
                                DevState* st, cudaStream_t s) {
  k_target_setup<<<1, 32, 0, s>>>(tg, kind, nu, mu, sigma, d, st);
  return cudaGetLastError();
}

cudaError_t launch_est_finalize(const double* part, int nb, int d, DevState* st, int write_mean_out,
                                cudaStream_t s) {
  k_est_finalize<<<1, kFinThreads, 0, s>>>(part, nb, d, st, write_mean_out);
  return cudaGetLastError();
}

cudaError_t launch_cov(const ParticleArgs& a, double* cov, int grid, cudaStream_t s) {
  if (a.dtype == SMC_F64)
    k_cov<double><<<grid, kPThreads, 0, s>>>(a, cov);
  else
    k_cov<float><<<grid, kPThreads, 0, s>>>(a, cov);
  return cudaGetLastError();
}

cudaError_t launch_zero_cov(DevState* st, int d, cudaStream_t s) {
  k_zero_cov<<<1, 256, 0, s>>>(st, d);
  return cudaGetLastError();
}

cudaError_t launch_begin(DevState* st, cudaStream_t s) {
  k_begin<<<1, 32, 0, s>>>(st);
  return cudaGetLastError();
}

cudaError_t launch_commit(DevState* st, int d, int force_flip, int recycle, cudaStream_t s) {
  k_commit<<<1, 32, 0, s>>>(st, d, force_flip, recycle);
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
