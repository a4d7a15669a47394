/*
 * smc_oracle.c -- plain, slow, single-threaded FP64 CPU oracle for one SMC
 * sampler iteration (Varsi, Kekempanos, Thiyagalingam & Maskell, "A Single SMC
 * Sampler on MPI that Outperforms a Single MCMC Sampler", arXiv:1905.10252).
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product path may include, link,
 * import or run this file.  Only tests/, __graft_entry__.smoke() and bench.py's
 * cpu_baseline / reference leg use it, through oracle/oracle.py.  It shares no
 * code, header, table or constant generator with the CUDA path.
 *
 * Every function restates a passage of the paper, or a reading of a passage
 * the paper leaves open; the citation is given beside it.  No blocking, fusion
 * or reordering beyond what the definition states: loops run in index order.
 *
 * Build: gcc -O2 -std=c11 -ffp-contract=off -fno-fast-math -shared -fPIC
 * (contraction is off so that every a*b+c below is two roundings unless it is
 * written as fma(); the arithmetic is then a fixed sequence of IEEE-754 basic
 * operations and gives the same bits on any conforming machine).
 *
 * Parity status per function (pins live in tests/test_oracle_*.py):
 *   orc_philox4x32_10       pinned: cuRAND host generator PHILOX4_32_10 (independent library)
 *   orc_log, orc_sincos2pi  pinned: libm / mpmath within 2 ulp
 *   orc_normals             pinned: moments over 2^16 draws; Box-Muller identity
 *   orc_move                pinned: each coordinate the correctly rounded x + eps z (exact
 *                           rationals); increment std = eps (a variance reading fails)
 *   orc_expfx               pinned: Decimal exp within 2^-54 relative; tables vs exact roots
 *   orc_cholesky, logpi     pinned: numpy.linalg inverse quadratic form
 *   orc_lse_ess             pinned: closed forms (equal / one-hot weights)
 *   orc_systematic          pinned: sum == N, floor bounds, exhaustive-U mean
 *   orc_redistribute        pinned: brute-force stable repeat, all compositions
 *   orc_nearly_sort         pinned: hand-worked cases, Definition 1 (ascending Nearly-Sorted),
 *                           stable partition over every key vector of small N
 *   orc_run (Gaussian)      pinned: closed-form posterior moments within MC error
 *   logistic logpi          pinned: b = 0 closed form (-M log 2), scipy Bernoulli log-likelihood
 *                           + normal prior, closed-form gradient by central differences,
 *                           label-flip symmetry
 *   orc_run (logistic)      pinned: posterior mean and variance against grid quadrature of
 *                           the posterior density (D = 1, 2), within MC error
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

typedef unsigned __int128 u128;

/* ------------------------------------------------------------------------ */
/* Counter-based random numbers: Philox4x32-10 (Salmon, Moraes, Dror & Shaw,
 * "Parallel random numbers: as easy as 1, 2, 3", SC'11).  Ten rounds of two
 * 32x32->64 multiplies; the key is bumped by the Weyl constants between
 * rounds.  The paper fixes no generator; Philox lets both implementations draw
 * the same numbers from (seed, iteration, particle). */
#define PHILOX_M0 0xD2511F53u
#define PHILOX_M1 0xCD9E8D57u
#define PHILOX_W0 0x9E3779B9u
#define PHILOX_W1 0xBB67AE85u

void orc_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4]) {
  uint32_t c0 = ctr[0], c1 = ctr[1], c2 = ctr[2], c3 = ctr[3];
  uint32_t k0 = key[0], k1 = key[1];
  for (int r = 0; r < 10; ++r) {
    uint64_t p0 = (uint64_t)PHILOX_M0 * c0;
    uint64_t p1 = (uint64_t)PHILOX_M1 * c2;
    uint32_t n0 = (uint32_t)(p1 >> 32) ^ c1 ^ k0;
    uint32_t n1 = (uint32_t)p1;
    uint32_t n2 = (uint32_t)(p0 >> 32) ^ c3 ^ k1;
    uint32_t n3 = (uint32_t)p0;
    c0 = n0; c1 = n1; c2 = n2; c3 = n3;
    k0 += PHILOX_W0;
    k1 += PHILOX_W1;
  }
  out[0] = c0; out[1] = c1; out[2] = c2; out[3] = c3;
}

/* Purposes: the third counter word carries (purpose << 24) | block. */
enum { ORC_INIT = 1, ORC_MOVE = 2, ORC_RESAMPLE = 3 };

/* 32-bit word w of the random stream of particle i at iteration t:
 * counter (i, t, purpose << 24 | w / 4, 0), key (seed low, seed high). */
static uint32_t stream_word(uint64_t seed, uint64_t t, uint32_t purpose, uint64_t i, uint64_t w) {
  uint32_t ctr[4] = {(uint32_t)i, (uint32_t)t, (purpose << 24) | (uint32_t)(w >> 2), 0};
  uint32_t key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)};
  uint32_t out[4];
  orc_philox4x32_10(ctr, key, out);
  return out[w & 3];
}

/* 64-bit word: 32-bit words 2w (high half) and 2w+1 (low half). */
static uint64_t stream_word64(uint64_t seed, uint64_t t, uint32_t purpose, uint64_t i, uint64_t w) {
  return ((uint64_t)stream_word(seed, t, purpose, i, 2 * w) << 32) | stream_word(seed, t, purpose, i, 2 * w + 1);
}

/* ------------------------------------------------------------------------ */
/* Deterministic elementary functions built only from IEEE basic operations
 * and fma, so that both implementations produce identical bits.  Used for the
 * Box-Muller transform of the FP64 path and for the reset value -log N. */
static const double LN2_HI = 0x1.62e42fee00000p-1; /* ln 2 with 21 low bits cleared */
static const double LN2_LO = 0x1.a39ef35793c76p-33; /* ln 2 - LN2_HI, rounded       */
static const double SQRT2_D = 0x1.6a09e667f3bcdp+0;
static const double TWO_PI_D = 0x1.921fb54442d18p+2;

/* log(u) for a finite normal u > 0.  u = 2^e * m with m in [sqrt(1/2), sqrt(2));
 * log m = 2 atanh(s) = 2 s sum_k s^(2k)/(2k+1), s = (m-1)/(m+1), |s| < 0.172;
 * eleven terms leave a truncation error below 1e-17. */
double orc_log(double u) {
  uint64_t b;
  memcpy(&b, &u, 8);
  int e = (int)((b >> 52) & 0x7ff) - 1023;
  uint64_t mb = (b & 0x000FFFFFFFFFFFFFULL) | 0x3FF0000000000000ULL;
  double m;
  memcpy(&m, &mb, 8);
  if (m > SQRT2_D) { m = m * 0.5; e += 1; }
  double s = (m - 1.0) / (m + 1.0);
  double s2 = s * s;
  double p = 1.0 / 23.0;
  p = fma(p, s2, 1.0 / 21.0);
  p = fma(p, s2, 1.0 / 19.0);
  p = fma(p, s2, 1.0 / 17.0);
  p = fma(p, s2, 1.0 / 15.0);
  p = fma(p, s2, 1.0 / 13.0);
  p = fma(p, s2, 1.0 / 11.0);
  p = fma(p, s2, 1.0 / 9.0);
  p = fma(p, s2, 1.0 / 7.0);
  p = fma(p, s2, 1.0 / 5.0);
  p = fma(p, s2, 1.0 / 3.0);
  p = fma(p, s2, 1.0);
  double logm = (2.0 * s) * p;
  double de = (double)e;
  return fma(de, LN2_HI, fma(de, LN2_LO, logm));
}

/* sin and cos of 2*pi*a for a = v * 2^-53, 0 <= v < 2^53.  The quarter-turn
 * q = round(4a) is taken exactly on the integer v, leaving a reduced angle in
 * [-pi/4, pi/4] for Taylor series to degree 17 (sin) and 18 (cos). */
void orc_sincos2pi_u53(uint64_t v, double* s_out, double* c_out) {
  uint64_t q = (v + (1ULL << 50)) >> 51;                      /* 0..4 */
  int64_t vr = (int64_t)v - (int64_t)(q << 51);               /* [-2^50, 2^50] */
  double x = (double)vr * 0x1p-53;                            /* exact */
  double t = x * TWO_PI_D;
  double t2 = t * t;
  double ps = -1.0 / 121645100408832000.0;                    /* -1/19! */
  ps = fma(ps, t2, 1.0 / 355687428096000.0);                  /* 1/17! */
  ps = fma(ps, t2, -1.0 / 1307674368000.0);                   /* 1/15! */
  ps = fma(ps, t2, 1.0 / 6227020800.0);                       /* 1/13! */
  ps = fma(ps, t2, -1.0 / 39916800.0);                        /* 1/11! */
  ps = fma(ps, t2, 1.0 / 362880.0);                           /* 1/9!  */
  ps = fma(ps, t2, -1.0 / 5040.0);                            /* 1/7!  */
  ps = fma(ps, t2, 1.0 / 120.0);                              /* 1/5!  */
  ps = fma(ps, t2, -1.0 / 6.0);                               /* 1/3!  */
  ps = fma(ps, t2, 1.0);
  double sn = t * ps;
  double pc = 1.0 / 6402373705728000.0;                       /* 1/18! */
  pc = fma(pc, t2, -1.0 / 20922789888000.0);                  /* 1/16! */
  pc = fma(pc, t2, 1.0 / 87178291200.0);                      /* 1/14! */
  pc = fma(pc, t2, -1.0 / 479001600.0);                       /* 1/12! */
  pc = fma(pc, t2, 1.0 / 3628800.0);                          /* 1/10! */
  pc = fma(pc, t2, -1.0 / 40320.0);                           /* 1/8!  */
  pc = fma(pc, t2, 1.0 / 720.0);                              /* 1/6!  */
  pc = fma(pc, t2, -1.0 / 24.0);                              /* 1/4!  */
  pc = fma(pc, t2, 1.0 / 2.0);                                /* 1/2!  */
  double cs = fma(-pc, t2, 1.0);
  switch (q & 3) {
    case 0: *s_out = sn; *c_out = cs; break;
    case 1: *s_out = cs; *c_out = -sn; break;
    case 2: *s_out = -sn; *c_out = -cs; break;
    default: *s_out = -cs; *c_out = sn; break;
  }
}

/* D standard normals for particle i (Box-Muller on consecutive uniform
 * pairs).  ubits = 53: uniform k is the top 53 bits of 64-bit word k (32-bit
 * words 2k, 2k+1).  ubits = 24: uniform k is the top 24 bits of 32-bit word k,
 * the resolution the FP32 path draws at.  For a pair (a, b):
 * u1 = 1 - a in (0, 1], r = sqrt(-2 log u1), theta = 2 pi b,
 * z = (r cos theta, r sin theta). */
void orc_normals(uint64_t seed, uint64_t t, uint32_t purpose, uint64_t i, int D, int ubits,
                 double* z) {
  for (int p = 0; 2 * p < D; ++p) {
    uint64_t va, vb; /* 53-bit integers: a = va * 2^-53 */
    if (ubits == 53) {
      va = stream_word64(seed, t, purpose, i, 2 * p) >> 11;
      vb = stream_word64(seed, t, purpose, i, 2 * p + 1) >> 11;
    } else {
      va = (uint64_t)(stream_word(seed, t, purpose, i, 2 * p) >> 8) << 29;
      vb = (uint64_t)(stream_word(seed, t, purpose, i, 2 * p + 1) >> 8) << 29;
    }
    double u1 = (double)((1ULL << 53) - va) * 0x1p-53;
    double r = sqrt(-2.0 * orc_log(u1));
    double sn, cs;
    orc_sincos2pi_u53(vb, &sn, &cs);
    z[2 * p] = r * cs;
    if (2 * p + 1 < D) z[2 * p + 1] = r * sn;
  }
}

/* ------------------------------------------------------------------------ */
/* Fixed-point exponential used to quantise weights (reading: the paper gives
 * MVR only as "a variant of systematic resampling using a cumulative sum",
 * Sec. 3.3; making the CDF integer makes the copy counts exact).  For y <= 0:
 *   E(y) ~= 2^62 exp(y), an integer in [0, 2^62], E(0) = 2^62,
 * computed as exp(y) = 2^-z, z = -y log2(e) = k + f:
 *   A = floor(-y 2^57); Z = A * L2E (L2E = round(log2(e) 2^62)); k = Z >> 119;
 *   f = the 64 fraction bits below; j1 = top 6 bits of f, j2 = next 6 bits,
 *   g = the low 52 bits;  2^-f = T1[j1] T2[j2] exp(-g ln 2);
 *   h = g ln 2 (H = h 2^76); exp(-h) = C0 - h(C1 - h(C2 - h(C3 - h C4)))
 *   in 2^63 fixed point with C_k = floor(2^63 / k!);
 *   E = ((T1[j1] T2[j2] >> 63) P) >> (64 + k).
 * T1[j] ~= 2^63 2^(-j/64) and T2[j] ~= 2^63 2^(-j/4096) are products of
 * c_b ~= 2^63 2^(-2^-b) over the set bits of j (b = 1..6 for T1, 7..12 for
 * T2), c_0 = 2^62, c_b = isqrt(c_{b-1} 2^63) -- every step an exact integer
 * operation, so any correct implementation gives the same tables. */
#define L2E_62 0x5C551D94AE0BF85EULL  /* round(log2(e) * 2^62) */
#define LN2_64 0xB17217F7D1CF79ACULL  /* round(ln(2) * 2^64)   */

/* floor(sqrt(n)) by the bitwise restoring method. */
static uint64_t isqrt_u128(u128 n) {
  u128 res = 0;
  u128 bit = (u128)1 << 126;
  while (bit > n) bit >>= 2;
  while (bit != 0) {
    if (n >= res + bit) {
      n -= res + bit;
      res = (res >> 1) + bit;
    } else {
      res >>= 1;
    }
    bit >>= 2;
  }
  return (uint64_t)res;
}

static uint64_t g_T[128]; /* T1 = g_T[0..63], T2 = g_T[64..127] */
static uint64_t g_C[5];
static int g_T_ready = 0;

static void build_T(void) {
  uint64_t c[13];
  c[0] = 1ULL << 62;
  for (int b = 1; b <= 12; ++b) c[b] = isqrt_u128((u128)c[b - 1] << 63);
  for (int t = 0; t < 2; ++t)
    for (int j = 0; j < 64; ++j) {
      uint64_t acc = 1ULL << 63;
      for (int b = 1; b <= 6; ++b)
        if (j & (1 << (6 - b))) acc = (uint64_t)(((u128)acc * c[6 * t + b]) >> 63);
      g_T[64 * t + j] = acc;
    }
  uint64_t fact = 1;
  for (int k = 0; k <= 4; ++k) {
    if (k > 0) fact *= (uint64_t)k;
    g_C[k] = (1ULL << 63) / fact;
  }
  g_T_ready = 1;
}

void orc_expfx_table(uint64_t* out128) {
  if (!g_T_ready) build_T();
  memcpy(out128, g_T, sizeof g_T);
}

uint64_t orc_expfx(double y) {
  if (!g_T_ready) build_T();
  double a = -y;
  if (!(a < 44.0)) return 0; /* exp(-44) 2^62 < 1 */
  uint64_t bits;
  memcpy(&bits, &a, 8);
  int e = (int)((bits >> 52) & 0x7ff);
  uint64_t A;
  if (e == 0) {
    A = 0; /* zero or subnormal */
  } else {
    uint64_t mant = (bits & 0x000FFFFFFFFFFFFFULL) | (1ULL << 52);
    int sh = e - 1018; /* a = mant 2^(e-1075); A = floor(a 2^57) */
    if (sh >= 0) A = mant << sh;
    else if (sh > -64) A = mant >> (-sh);
    else A = 0;
  }
  u128 Z = (u128)A * L2E_62;
  unsigned k = (unsigned)(Z >> 119);
  uint64_t f = (uint64_t)(Z >> 55);
  unsigned j1 = (unsigned)(f >> 58);
  unsigned j2 = (unsigned)((f >> 52) & 63);
  uint64_t g = f & ((1ULL << 52) - 1);
  uint64_t H = (uint64_t)(((u128)(g << 12) * LN2_64) >> 64); /* h = H 2^-76 */
  uint64_t P = g_C[4];
  for (int kk = 3; kk >= 0; --kk) P = g_C[kk] - (uint64_t)(((u128)H * P) >> 76);
  uint64_t T = (uint64_t)(((u128)g_T[j1] * g_T[64 + j2]) >> 63);
  return (uint64_t)(((u128)T * P) >> (64 + k));
}

/* Fixed-point scale F of the weights: F = min(62, 63 - ceil(log2 N)), so that
 * S = sum W <= 2^63, N C_i + U < 2^95, 2 S^2 < 2^128 and N sum W^2 < 2^127. */
int orc_quant_shift(int64_t N) {
  int c = 0;
  while (((int64_t)1 << c) < N) ++c;
  int F = 63 - c;
  return F > 62 ? 62 : F;
}

/* ------------------------------------------------------------------------ */
/* Targets pi(x), normalising constants dropped (they cancel in the
 * normalised weights, eq. (2)).  Gaussian: log pi = -1/2 (x-mu)^T Sigma^-1
 * (x-mu) via the Cholesky factor L (Sigma = L L^T) and forward substitution
 * z = L^-1 (x - mu).  Logistic regression (the batched/tensor-core workload):
 * log pi(beta) = sum_m [y_m z_m - softplus(z_m)] - |beta|^2/(2 prior_var),
 * z = X beta.  Student-t (Sec. 5.2.3, eq. (14), one dimension):
 * log pi = -(nu+1)/2 log(1 + (x-mu)^2/nu). */
enum { ORC_GAUSS = 1, ORC_LOGISTIC = 2, ORC_STUDENT_T = 3 };

typedef struct {
  int kind;
  int D;
  double* mu;
  double* L;     /* D x D lower triangular, row-major */
  int M;
  double* X;     /* M x D row-major */
  double* y;     /* M */
  double prior_var;
  double nu;
} orc_target;

/* Cholesky-Banachiewicz, row by row; returns nonzero if Sigma is not positive
 * definite. */
int orc_cholesky(int D, const double* S, double* L) {
  memset(L, 0, sizeof(double) * (size_t)D * D);
  for (int i = 0; i < D; ++i) {
    for (int j = 0; j <= i; ++j) {
      double s = 0.0;
      for (int k = 0; k < j; ++k) s = fma(L[i * D + k], L[j * D + k], s);
      if (i == j) {
        double d = S[i * D + i] - s;
        if (!(d > 0.0)) return 1;
        L[i * D + i] = sqrt(d);
      } else {
        L[i * D + j] = (S[i * D + j] - s) / L[j * D + j];
      }
    }
  }
  return 0;
}

void* orc_target_gauss(int D, const double* mu, const double* Sigma) {
  orc_target* t = calloc(1, sizeof *t);
  t->kind = ORC_GAUSS;
  t->D = D;
  t->mu = malloc(sizeof(double) * D);
  t->L = malloc(sizeof(double) * D * D);
  memcpy(t->mu, mu, sizeof(double) * D);
  if (orc_cholesky(D, Sigma, t->L)) { free(t->mu); free(t->L); free(t); return NULL; }
  return t;
}

void* orc_target_logistic(int D, int M, const double* X, const double* y, double prior_var) {
  orc_target* t = calloc(1, sizeof *t);
  t->kind = ORC_LOGISTIC;
  t->D = D;
  t->M = M;
  t->X = malloc(sizeof(double) * (size_t)M * D);
  t->y = malloc(sizeof(double) * M);
  memcpy(t->X, X, sizeof(double) * (size_t)M * D);
  memcpy(t->y, y, sizeof(double) * M);
  t->prior_var = prior_var;
  return t;
}

void* orc_target_student_t(double mu, double nu) {
  orc_target* t = calloc(1, sizeof *t);
  t->kind = ORC_STUDENT_T;
  t->D = 1;
  t->mu = malloc(sizeof(double));
  t->mu[0] = mu;
  t->nu = nu;
  return t;
}

void orc_target_free(void* h) {
  orc_target* t = h;
  if (!t) return;
  free(t->mu); free(t->L); free(t->X); free(t->y); free(t);
}

void orc_target_chol(const void* h, double* L) {
  const orc_target* t = h;
  memcpy(L, t->L, sizeof(double) * t->D * t->D);
}

static double softplus(double z) { return z > 0.0 ? z + log1p(exp(-z)) : log1p(exp(z)); }

double orc_logpi(const void* h, const double* x) {
  const orc_target* t = h;
  const int D = t->D;
  if (t->kind == ORC_GAUSS) {
    double z[64];
    double q = 0.0;
    for (int r = 0; r < D; ++r) {
      double acc = x[r] - t->mu[r];
      for (int c = 0; c < r; ++c) acc = fma(-t->L[r * D + c], z[c], acc);
      z[r] = acc / t->L[r * D + r];
      q = fma(z[r], z[r], q);
    }
    return -0.5 * q;
  }
  if (t->kind == ORC_LOGISTIC) {
    double s = 0.0;
    for (int m = 0; m < t->M; ++m) {
      double zm = 0.0;
      for (int c = 0; c < D; ++c) zm += t->X[(size_t)m * D + c] * x[c];
      s += t->y[m] * zm - softplus(zm);
    }
    double b2 = 0.0;
    for (int c = 0; c < D; ++c) b2 += x[c] * x[c];
    return s - b2 / (2.0 * t->prior_var);
  }
  /* Student-t */
  double d = x[0] - t->mu[0];
  return -0.5 * (t->nu + 1.0) * log1p(d * d / t->nu);
}

/* log q0(x) for q0 = N(0, s^2 I), constants dropped. */
static double logq0(int D, double s, const double* x) {
  double q = 0.0;
  for (int c = 0; c < D; ++c) q = fma(x[c], x[c], q);
  return (-0.5 * q) / (s * s);
}

/* ------------------------------------------------------------------------ */
/* Algorithm 2, line 1: x0 ~ q0 = N(0, s^2 I), w0 = pi(x0)/q0(x0). */
void orc_init(const void* tgt, int64_t N, int D, uint64_t seed, double init_scale, int ubits,
              double* x, double* logw, double* logpi) {
  double z[64];
  for (int64_t i = 0; i < N; ++i) {
    orc_normals(seed, 0, ORC_INIT, (uint64_t)i, D, ubits, z);
    for (int c = 0; c < D; ++c) x[i * D + c] = init_scale * z[c];
    logpi[i] = orc_logpi(tgt, &x[i * D]);
    logw[i] = logpi[i] - logq0(D, init_scale, &x[i * D]);
  }
}

/* Algorithm 2, line 4 (proposal): x_t = x_{t-1} + eps z, z ~ N(0, I) -- the
 * random-walk proposal of Sec. 5.2.3 with eps read as a standard deviation. */
void orc_move(int64_t N, int D, uint64_t seed, uint64_t t, double step, int ubits,
              const double* x_in, double* x_out) {
  double z[64];
  for (int64_t i = 0; i < N; ++i) {
    orc_normals(seed, t, ORC_MOVE, (uint64_t)i, D, ubits, z);
    for (int c = 0; c < D; ++c) x_out[i * D + c] = fma(step, z[c], x_in[i * D + c]);
  }
}

/* Eq. (5): w_t = w_{t-1} pi(x_t)/pi(x_{t-1}) L(x_{t-1}|x_t)/q(x_t|x_{t-1}).
 * With the forward-proposal L-kernel of Sec. 5.2.3, L = q and the last
 * factor is 1; it is evaluated anyway so that other kernels can plug in:
 * log L - log q = -|x_{t-1}-x_t|^2/(2 eps^2) + |x_t-x_{t-1}|^2/(2 eps^2). */
void orc_reweight(const void* tgt, int64_t N, int D, double step, const double* x_prev,
                  const double* x, const double* logpi_prev, double* logw, double* logpi) {
  for (int64_t i = 0; i < N; ++i) {
    double lp = orc_logpi(tgt, &x[i * D]);
    double lL = 0.0, lq = 0.0;
    if (x_prev) {
      for (int c = 0; c < D; ++c) {
        double a = x_prev[i * D + c] - x[i * D + c];
        double b = x[i * D + c] - x_prev[i * D + c];
        lL += a * a;
        lq += b * b;
      }
      lL = -lL / (2.0 * step * step);
      lq = -lq / (2.0 * step * step);
    }
    logw[i] = logw[i] + (lp - logpi_prev[i]) + (lL - lq);
    logpi[i] = lp;
  }
}

/* Eqs. (1), (2): normalised weights and N_eff, in log space for range:
 * m = max logw, LSE = m + log sum exp(logw - m), N_eff = (sum e)^2 / sum e^2.
 * Returns nonzero if any logw is NaN or every logw is -inf. */
int orc_lse_ess(int64_t N, const double* logw, double* m_out, double* lse_out, double* ess_out) {
  double m = -INFINITY;
  for (int64_t i = 0; i < N; ++i) {
    if (isnan(logw[i])) return 1;
    if (logw[i] > m) m = logw[i];
  }
  if (!isfinite(m)) return 1;
  double s1 = 0.0, s2 = 0.0;
  for (int64_t i = 0; i < N; ++i) {
    double e = exp(logw[i] - m);
    s1 += e;
    s2 += e * e;
  }
  *m_out = m;
  *lse_out = m + log(s1);
  *ess_out = s1 * s1 / s2;
  return 0;
}

/* Eq. (7): f_t = sum_i x_i w~_i, plus the weighted covariance. */
void orc_estimate(int64_t N, int D, const double* x, const double* logw, double lse,
                  double* mean, double* cov) {
  for (int c = 0; c < D; ++c) mean[c] = 0.0;
  for (int64_t i = 0; i < N; ++i) {
    double w = exp(logw[i] - lse);
    for (int c = 0; c < D; ++c) mean[c] += w * x[i * D + c];
  }
  if (!cov) return;
  for (int a = 0; a < D * D; ++a) cov[a] = 0.0;
  for (int64_t i = 0; i < N; ++i) {
    double w = exp(logw[i] - lse);
    for (int a = 0; a < D; ++a)
      for (int b = 0; b < D; ++b)
        cov[a * D + b] += w * (x[i * D + a] - mean[a]) * (x[i * D + b] - mean[b]);
  }
}

/* Quantised weights W_i = E(logw_i - m) >> (62 - F) and their exact sums.
 * sums = {S, sumW2_lo, sumW2_hi, sumE_lo, sumE_hi}. */
void orc_quantise(int64_t N, const double* logw, double m, uint64_t* W, uint64_t* sums) {
  int F = orc_quant_shift(N);
  u128 s = 0, s2 = 0, se = 0;
  for (int64_t i = 0; i < N; ++i) {
    uint64_t E = orc_expfx(logw[i] - m);
    uint64_t w = E >> (62 - F);
    W[i] = w;
    s += w;
    s2 += (u128)w * w;
    se += E;
  }
  sums[0] = (uint64_t)s;
  sums[1] = (uint64_t)s2;
  sums[2] = (uint64_t)(s2 >> 64);
  sums[3] = (uint64_t)se;
  sums[4] = (uint64_t)(se >> 64);
}

/* Resampling decision of Algorithm 2 (line 7: resample iff N_eff < N*), with
 * N_eff from eq. (1) on the quantised weights, N_eff = S^2 / sum W^2, taken
 * exactly in integers: N_eff < N*  <=>  S^2 < N* sum W^2.  nstar = 0 selects
 * the paper's N* = N/2 (Sec. 3.1) as 2 S^2 < N sum W^2, exact for odd N too.
 * mode 0: that rule; 1: always (the worst case of Sec. 5.2); 2: never. */
int orc_decide_nstar(int64_t N, int64_t nstar, uint64_t S, uint64_t sw2_lo, uint64_t sw2_hi, int mode) {
  if (mode == 1) return 1;
  if (mode == 2) return 0;
  u128 sw2 = ((u128)sw2_hi << 64) | sw2_lo;
  if (nstar == 0) return (u128)S * S * 2 < (u128)N * sw2;
  return (u128)S * S < (u128)nstar * sw2;
}

int orc_decide(int64_t N, uint64_t S, uint64_t sw2_lo, uint64_t sw2_hi, int mode) {
  return orc_decide_nstar(N, 0, S, sw2_lo, sw2_hi, mode);
}

/* The systematic offset U in [0, S): U = floor(r S / 2^64), r the first 64-bit
 * word of the resampling stream of iteration t (particle index 2^32 - 1). */
uint64_t orc_resample_u(uint64_t seed, uint64_t t, uint64_t S) {
  uint64_t r = stream_word64(seed, t, ORC_RESAMPLE, 0xFFFFFFFFu, 0);
  return (uint64_t)(((u128)r * S) >> 64);
}

/* MVR as systematic resampling on the integer CDF C_i = sum_{j<=i} W_j
 * (Algorithm 4, line 1; eq. (9)):
 *   ncopies_i = floor((N C_i + U)/S) - floor((N C_{i-1} + U)/S),
 * off_i = floor((N C_{i-1} + U)/S) is the exclusive cumulative sum of ncopies. */
void orc_systematic(int64_t N, const uint64_t* W, uint64_t S, uint64_t U, int32_t* ncopies,
                    uint32_t* off) {
  u128 C = 0;
  uint64_t prev = (uint64_t)((u128)U / S);
  for (int64_t i = 0; i < N; ++i) {
    C += W[i];
    uint64_t cur = (uint64_t)(((u128)N * C + U) / S);
    if (off) off[i] = (uint32_t)prev;
    ncopies[i] = (int32_t)(cur - prev);
    prev = cur;
  }
}

/* Algorithm 5 (S-R): for each j, copy row j ncopies_j times, in order.  The
 * printed line x_new^i <- x^i is read as x_new^i <- x^j (the only reading
 * under which the routine duplicates particles). */
void orc_redistribute(int64_t N, int64_t row_bytes, const int32_t* ncopies, const void* x,
                      void* x_new) {
  const char* src = x;
  char* dst = x_new;
  int64_t i = 0;
  for (int64_t j = 0; j < N; ++j)
    for (int32_t k = 0; k < ncopies[j]; ++k) {
      memcpy(dst + i * row_bytes, src + j * row_bytes, (size_t)row_bytes);
      ++i;
    }
}

/* Algorithm 8 (S-NS, Sec. 4.2): a single pass in index order with two
 * cursors; an element whose copy count is positive takes the next free slot
 * from the right end of the output, any other element the next free slot
 * from the left end.  The keys come out as an ascending Nearly-Sorted
 * sequence (Definition 1: zeros first, then the positive counts); each
 * particle row travels with its key. */
void orc_nearly_sort(int64_t N, int64_t row_bytes, const int32_t* ncopies, const void* x,
                     int32_t* ncopies_new, void* x_new) {
  const char* src = x;
  char* dst = x_new;
  int64_t l = 0, r = N - 1;
  for (int64_t i = 0; i < N; ++i) {
    int64_t k;
    if (ncopies[i] > 0) {
      k = r;
      --r;
    } else {
      k = l;
      ++l;
    }
    ncopies_new[k] = ncopies[i];
    memcpy(dst + k * row_bytes, src + i * row_bytes, (size_t)row_bytes);
  }
}

/* Algorithm 4, line 3: all weights reset to 1/N. */
double orc_reset_logw(int64_t N) { return -orc_log((double)N); }

/* Whole resampling step of Algorithm 4 on logw (for stage tests): returns
 * nonzero on non-finite weights.  out_stats = {m, did, S, U, sw2_lo, sw2_hi,
 * se_lo, se_hi} as raw 64-bit words (m as the bits of a double). */
int orc_resample(int64_t N, const double* logw, uint64_t seed, uint64_t t, int mode,
                 int32_t* ncopies, uint32_t* off, uint64_t* W, uint64_t* out_stats) {
  double m = -INFINITY;
  for (int64_t i = 0; i < N; ++i) {
    if (isnan(logw[i])) return 1;
    if (logw[i] > m) m = logw[i];
  }
  if (!isfinite(m)) return 1;
  uint64_t sums[5];
  orc_quantise(N, logw, m, W, sums);
  int did = orc_decide(N, sums[0], sums[1], sums[2], mode);
  uint64_t U = orc_resample_u(seed, t, sums[0]);
  if (did) orc_systematic(N, W, sums[0], U, ncopies, off);
  memcpy(&out_stats[0], &m, 8);
  out_stats[1] = (uint64_t)did;
  out_stats[2] = sums[0];
  out_stats[3] = U;
  out_stats[4] = sums[1];
  out_stats[5] = sums[2];
  out_stats[6] = sums[3];
  out_stats[7] = sums[4];
  return 0;
}

/* ------------------------------------------------------------------------ */
/* Algorithm 2: the SMC sampler with recycling, K iterations.
 * trace[t*6 + {0..5}] = {LSE_t, log c_t, N_eff, m, resampled, distinct survivors}
 * for t = 1..K (row t-1); means[(t-1)*D + c] = f_t (eq. (7)); cov = final
 * weighted covariance; fhat = recycled estimate (eq. (6)) with weights c_t
 * (eq. (8)).  ncopies_trace (K x N, may be NULL) records each iteration's copy
 * counts (zeros where no resampling happened).  ubits selects the uniform
 * resolution (53 for the FP64 state, 24 for the FP32 state).  Returns nonzero on
 * failure. */
int orc_run(const void* tgt, int64_t N, int D, uint64_t seed, double init_scale, double step,
            int mode, int64_t nstar, int ubits, int K, double* x, double* logw, double* logpi, double* trace,
            double* means, double* cov, double* fhat, int32_t* ncopies_trace) {
  size_t nd = (size_t)N * D;
  double* xp = malloc(sizeof(double) * nd);
  double* xn = malloc(sizeof(double) * nd);
  double* lpp = malloc(sizeof(double) * N);
  uint64_t* W = malloc(sizeof(uint64_t) * N);
  int32_t* nc = malloc(sizeof(int32_t) * N);
  double* lpn = malloc(sizeof(double) * N);
  int rc = 0;
  orc_init(tgt, N, D, seed, init_scale, ubits, x, logw, logpi);
  double lse_prev;
  {
    double m0, ess0;
    if (orc_lse_ess(N, logw, &m0, &lse_prev, &ess0)) { rc = 1; goto done; }
  }
  double logc_max = -INFINITY;
  double* logcs = malloc(sizeof(double) * (K > 0 ? K : 1));
  for (int t = 1; t <= K; ++t) {
    /* line 4: importance sampling (move, then eq. (5)) */
    memcpy(xp, x, sizeof(double) * nd);
    orc_move(N, D, seed, (uint64_t)t, step, ubits, xp, x);
    orc_reweight(tgt, N, D, step, xp, x, logpi, logw, logpi);
    /* line 5: normalise; line 3 (read after IS): c_t, eq. (8) */
    double m, lse, ess;
    if (orc_lse_ess(N, logw, &m, &lse, &ess)) { rc = 1; free(logcs); goto done; }
    double logc = lse - lse_prev;
    /* line 6: estimate, eq. (7) */
    orc_estimate(N, D, x, logw, lse, &means[(size_t)(t - 1) * D], t == K ? cov : NULL);
    /* lines 7-9: N_eff and resampling */
    uint64_t sums[5];
    orc_quantise(N, logw, m, W, sums);
    int did = orc_decide_nstar(N, nstar, sums[0], sums[1], sums[2], mode);
    int64_t distinct = 0;
    if (did) {
      uint64_t U = orc_resample_u(seed, (uint64_t)t, sums[0]);
      orc_systematic(N, W, sums[0], U, nc, NULL);
      orc_redistribute(N, (int64_t)sizeof(double) * D, nc, x, xn);
      memcpy(x, xn, sizeof(double) * nd);
      orc_redistribute(N, (int64_t)sizeof(double), nc, logpi, lpn);
      memcpy(logpi, lpn, sizeof(double) * N);
      double r = orc_reset_logw(N);
      for (int64_t i = 0; i < N; ++i) logw[i] = r;
      lse_prev = 0.0; /* sum of N weights 1/N */
      for (int64_t i = 0; i < N; ++i) distinct += nc[i] > 0;
      if (ncopies_trace) memcpy(&ncopies_trace[(size_t)(t - 1) * N], nc, sizeof(int32_t) * N);
    } else {
      lse_prev = lse;
      if (ncopies_trace) memset(&ncopies_trace[(size_t)(t - 1) * N], 0, sizeof(int32_t) * N);
    }
    double* tr = &trace[(size_t)(t - 1) * 6];
    tr[0] = lse; tr[1] = logc; tr[2] = ess; tr[3] = m; tr[4] = did; tr[5] = (double)distinct;
    logcs[t - 1] = logc;
    if (logc > logc_max) logc_max = logc;
  }
  /* line 11: recycling, eq. (6), weights c_t scaled by their maximum */
  if (fhat && K > 0) {
    double den = 0.0;
    for (int c = 0; c < D; ++c) fhat[c] = 0.0;
    for (int t = 0; t < K; ++t) {
      double ct = exp(logcs[t] - logc_max);
      den += ct;
      for (int c = 0; c < D; ++c) fhat[c] += ct * means[(size_t)t * D + c];
    }
    for (int c = 0; c < D; ++c) fhat[c] /= den;
  }
  free(logcs);
done:
  free(xp); free(xn); free(lpp); free(W); free(nc); free(lpn);
  return rc;
}
