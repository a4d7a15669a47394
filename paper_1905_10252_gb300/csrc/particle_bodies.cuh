// particle_bodies.cuh -- device bodies shared by the particle kernels
// (k_particles.cu) and the fused small-sampler iteration (k_resample.cu): the
// log targets, row I/O, the per-block maximum of log w, the generic move +
// reweight (one thread per particle) and the single-block maximum finaliser.
#pragma once

#include <cfloat>
#include <cmath>

#include "smc_internal.cuh"
#include "smc_kernels.h"

namespace smc {

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

// Bayesian logistic regression, one particle against all M data rows, in the
// order of the definition: z_m = sum_c X_mc b_c, then s += y_m z_m - softplus(z_m) over
// m, minus |b|^2 / (2 prior_var).  FP64: explicitly rounded operations;
// FP32: FP32 z and softplus, FP64 accumulation over the rows.
__device__ __forceinline__ double softplus64(double z) { return z > 0.0 ? z + log1p(exp(-z)) : log1p(exp(z)); }
__device__ __forceinline__ float softplus32(float z) { return z > 0.0f ? z + log1pf(expf(-z)) : log1pf(expf(z)); }

template <int DMAX>
__device__ double logpi_logistic(const double (&x)[DMAX], int d, const TargetDev* __restrict__ tg) {
  const float* __restrict__ X = tg->X;
  const float* __restrict__ y = tg->y;
  double s = 0.0;
  for (int m = 0; m < tg->m; ++m) {
    double z = 0.0;
#pragma unroll
    for (int c = 0; c < DMAX; ++c)
      if (c < d) z = __dadd_rn(z, __dmul_rn(double(X[int64_t(m) * d + c]), x[c]));
    s = __dadd_rn(s, __dsub_rn(__dmul_rn(double(y[m]), z), softplus64(z)));
  }
  double b2 = 0.0;
#pragma unroll
  for (int c = 0; c < DMAX; ++c)
    if (c < d) b2 = __dadd_rn(b2, __dmul_rn(x[c], x[c]));
  return __dsub_rn(s, __ddiv_rn(b2, __dmul_rn(2.0, tg->prior_var)));
}

template <int DMAX>
__device__ float logpi_logistic(const float (&x)[DMAX], int d, const TargetDev* __restrict__ tg) {
  const float* __restrict__ X = tg->X;
  const float* __restrict__ y = tg->y;
  double s = 0.0;
  for (int m = 0; m < tg->m; ++m) {
    float z = 0.0f;
#pragma unroll
    for (int c = 0; c < DMAX; ++c)
      if (c < d) z = fmaf(X[int64_t(m) * d + c], x[c], z);
    s += double(y[m]) * double(z) - double(softplus32(z));
  }
  float b2 = 0.0f;
#pragma unroll
  for (int c = 0; c < DMAX; ++c)
    if (c < d) b2 = fmaf(x[c], x[c], b2);
  return float(s - double(b2) / (2.0 * tg->prior_var));
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

// One record per block: rec[0] = max log w of the block, rec[1] = 1.
__device__ __forceinline__ void block_write_max(const MaxTracker& mt, double* __restrict__ rec, DevState* st) {
  __shared__ long long shm[kPThreads / 32];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
  if (mt.nan) record_error(st, SMC_ENONFINITE);
  const long long wm = warp_max_ll(mt.best);
  if (lane == 0) shm[wid] = wm;
  __syncthreads();
  if (threadIdx.x == 0) {
    long long v = shm[0];
    for (int w = 1; w < nw; ++w) v = shm[w] > v ? shm[w] : v;
    rec[0] = from_ordered_key(v);
    rec[1] = 1.0;
  }
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
__device__ __forceinline__ T eval_logpi(const T (&x)[DMAX], int d, int kind, const TargetSmem<T>& ts, T nu,
                                        const TargetDev* __restrict__ tg) {
  if (kind == SMC_STUDENT_T) return logpi_student(x[0], ts.mu[0], nu);
  if (kind == SMC_LOGISTIC) return logpi_logistic<DMAX>(x, d, tg);
  return logpi_gauss<DMAX>(x, d, ts.F, ts.mu);
}

// ---------------------------------------------------------------- move + reweight
// MOVE:     x_t = x_{t-1} + eps z, z from the MOVE stream at iteration t.
// REWEIGHT: log w_t = log w_{t-1} + (log pi(x_t) - log pi(x_{t-1})); the
//           forward-kernel L/q factor of eq. (5) is exactly one.
// Works in place on the current buffers.
// Block blk of nblk: the block's first nthr threads own particles
// blk nthr + threadIdx.x, then every nblk nthr-th; the iteration index is
// st->t + t_ahead (1 in the fused small-sampler iteration, whose increment of
// t follows its move).
template <typename T, int DMAX, bool MOVE, bool REWEIGHT>
__device__ __forceinline__ void move_reweight_generic_body(const ParticleArgs& a, TargetSmem<T>& ts, int blk,
                                                           int nblk, int nthr, int t_ahead) {
  if (REWEIGHT) load_target<T>(a.tg, a.d, ts);
  MaxTracker mt;
  mt.init();
  const int cur = a.st->cur;
  const uint64_t t = uint64_t(a.st->t + t_ahead);
  T* __restrict__ x = static_cast<T*>(cur ? a.x[1] : a.x[0]);
  T* __restrict__ lp = static_cast<T*>(cur ? a.logpi[1] : a.logpi[0]);
  const T nu = T(a.tg->nu);
  for (int64_t i = blk * int64_t(nthr) + threadIdx.x; int(threadIdx.x) < nthr && i < a.n; i += int64_t(nblk) * nthr) {
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
      const T lpi = eval_logpi<T, DMAX>(xr, a.d, a.kind, ts, nu, a.tg);
      const T lpp = lp[i];
      double lw;
      if constexpr (sizeof(T) == 8)
        lw = __dadd_rn(a.logw[i], __dsub_rn(lpi, lpp));
      else
        lw = a.logw[i] + double(lpi - lpp);
      lp[i] = lpi;
      a.logw[i] = lw;
      mt.add(lw);
    }
  }
  if (REWEIGHT) block_write_max(mt, a.part + 2 * blk, a.st);
}

// ---------------------------------------------------------------- finalise the maximum
// Single block: m = max over the blocks' maxima; a NaN seen by any block, or a
// maximum that is not finite (every log-weight -inf, or +inf), is an error.
__device__ __forceinline__ void max_finalize_body(const double* __restrict__ part, int nb, DevState* st) {
  __shared__ long long shm[32];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
  // (thread 0 loads the flags it updates now, overlapping the reduction)
  int wu = 0, pend = 0, cur = 0, rsw = 0;
  if (threadIdx.x == 0) {
    wu = st->w_uniform;
    pend = st->pending;
    cur = st->cur;
    rsw = st->rs_w;
  }
  long long m = ordered_key(-INFINITY);
  for (int b = threadIdx.x; b < nb; b += blockDim.x) {
    const long long k = ordered_key(part[2 * b]);
    m = k > m ? k : m;
  }
  m = warp_max_ll(m);
  if (lane == 0) shm[wid] = m;
  __syncthreads();
  if (threadIdx.x == 0) {
    long long v = shm[0];
    for (int w = 1; w < nw; ++w) v = shm[w] > v ? shm[w] : v;
    const double M = from_ordered_key(v);
    st->m = M;
    if (!(M > -INFINITY && M < INFINITY)) record_error(st, SMC_ENONFINITE);
    // the move kernel that just ran wrote eq. (7) records iff the weights it
    // started from were uniform; after its reweight they are not
    st->est_ready = wu;
    st->w_uniform = 0;
    // a move that gathered a deferred resampling's rows wrote them to the
    // other buffer, which is now current; the run starts it read stay set,
    // so the next scan writes the other array (which that move reset if it
    // was dirty) and this one is marked dirty
    if (pend) {
      st->cur = cur ^ 1;
      st->pending = 0;
      st->rs_w = rsw ^ 1;
      st->rs_dirty = 1;
    }
  }
}

}  // namespace smc
