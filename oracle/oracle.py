"""ctypes binding of the FP64 CPU oracle (smc_oracle.c).

TEST INFRASTRUCTURE ONLY: imported by tests/, by ``__graft_entry__.smoke()`` and by
the ``cpu_baseline`` / ``--impl reference`` legs of ``bench.py``, and by nothing in
the product package.  The oracle shares no code with the CUDA path; the two meet
only through the seeded inputs of ``paper_1905_10252_gb300.inputs``.

Every wrapper takes and returns numpy arrays; sizes are read from the arrays.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
from pathlib import Path

import numpy as np

_HERE = Path(__file__).resolve().parent
_SRC = _HERE / "smc_oracle.c"
_LIB = _HERE / "liboracle.so"
_CFLAGS = ["-O2", "-std=c11", "-ffp-contract=off", "-fno-fast-math", "-Wall", "-shared", "-fPIC"]

ORC_INIT, ORC_MOVE, ORC_RESAMPLE = 1, 2, 3
RESAMPLE_ESS, RESAMPLE_ALWAYS, RESAMPLE_NEVER = 0, 1, 2


def build(force: bool = False) -> Path:
    """Compile liboracle.so with gcc (contraction off) if missing or stale."""
    if force or not _LIB.exists() or _LIB.stat().st_mtime < _SRC.stat().st_mtime:
        tmp = _LIB.with_suffix(f".{os.getpid()}.tmp.so")
        subprocess.run(["gcc", *_CFLAGS, "-o", str(tmp), str(_SRC), "-lm"], check=True)
        os.replace(tmp, _LIB)
    return _LIB


_lib = None


def lib() -> C.CDLL:
    global _lib
    if _lib is None:
        _lib = C.CDLL(str(build()))
        _declare(_lib)
    return _lib


_u64p = C.POINTER(C.c_uint64)
_dp = C.POINTER(C.c_double)
_i32p = C.POINTER(C.c_int32)
_u32p = C.POINTER(C.c_uint32)


def _declare(L: C.CDLL) -> None:
    L.orc_philox4x32_10.argtypes = [_u32p, _u32p, _u32p]
    L.orc_log.argtypes = [C.c_double]
    L.orc_log.restype = C.c_double
    L.orc_sincos2pi_u53.argtypes = [C.c_uint64, _dp, _dp]
    L.orc_normals.argtypes = [C.c_uint64, C.c_uint64, C.c_uint32, C.c_uint64, C.c_int, C.c_int, _dp]
    L.orc_expfx.argtypes = [C.c_double]
    L.orc_expfx.restype = C.c_uint64
    L.orc_expfx_table.argtypes = [_u64p]
    L.orc_quant_shift.argtypes = [C.c_int64]
    L.orc_quant_shift.restype = C.c_int
    L.orc_cholesky.argtypes = [C.c_int, _dp, _dp]
    L.orc_cholesky.restype = C.c_int
    L.orc_target_gauss.argtypes = [C.c_int, _dp, _dp]
    L.orc_target_gauss.restype = C.c_void_p
    L.orc_target_logistic.argtypes = [C.c_int, C.c_int, _dp, _dp, C.c_double]
    L.orc_target_logistic.restype = C.c_void_p
    L.orc_target_student_t.argtypes = [C.c_double, C.c_double]
    L.orc_target_student_t.restype = C.c_void_p
    L.orc_target_free.argtypes = [C.c_void_p]
    L.orc_target_chol.argtypes = [C.c_void_p, _dp]
    L.orc_logpi.argtypes = [C.c_void_p, _dp]
    L.orc_logpi.restype = C.c_double
    L.orc_init.argtypes = [C.c_void_p, C.c_int64, C.c_int, C.c_uint64, C.c_double, C.c_int, _dp, _dp, _dp]
    L.orc_move.argtypes = [C.c_int64, C.c_int, C.c_uint64, C.c_uint64, C.c_double, C.c_int, _dp, _dp]
    L.orc_reweight.argtypes = [C.c_void_p, C.c_int64, C.c_int, C.c_double, _dp, _dp, _dp, _dp, _dp]
    L.orc_lse_ess.argtypes = [C.c_int64, _dp, _dp, _dp, _dp]
    L.orc_lse_ess.restype = C.c_int
    L.orc_estimate.argtypes = [C.c_int64, C.c_int, _dp, _dp, C.c_double, _dp, _dp]
    L.orc_quantise.argtypes = [C.c_int64, _dp, C.c_double, _u64p, _u64p]
    L.orc_decide.argtypes = [C.c_int64, C.c_uint64, C.c_uint64, C.c_uint64, C.c_int]
    L.orc_decide.restype = C.c_int
    L.orc_decide_nstar.argtypes = [C.c_int64, C.c_int64, C.c_uint64, C.c_uint64, C.c_uint64, C.c_int]
    L.orc_decide_nstar.restype = C.c_int
    L.orc_resample_u.argtypes = [C.c_uint64, C.c_uint64, C.c_uint64]
    L.orc_resample_u.restype = C.c_uint64
    L.orc_systematic.argtypes = [C.c_int64, _u64p, C.c_uint64, C.c_uint64, _i32p, _u32p]
    L.orc_redistribute.argtypes = [C.c_int64, C.c_int64, _i32p, C.c_void_p, C.c_void_p]
    L.orc_nearly_sort.argtypes = [C.c_int64, C.c_int64, _i32p, C.c_void_p, _i32p, C.c_void_p]
    L.orc_reset_logw.argtypes = [C.c_int64]
    L.orc_reset_logw.restype = C.c_double
    L.orc_resample.argtypes = [C.c_int64, _dp, C.c_uint64, C.c_uint64, C.c_int, _i32p, _u32p, _u64p, _u64p]
    L.orc_resample.restype = C.c_int
    L.orc_run.argtypes = [C.c_void_p, C.c_int64, C.c_int, C.c_uint64, C.c_double, C.c_double, C.c_int,
                          C.c_int64, C.c_int, C.c_int, _dp, _dp, _dp, _dp, _dp, _dp, _dp, _i32p]
    L.orc_run.restype = C.c_int


def _p(a: np.ndarray, ctype):
    return a.ctypes.data_as(C.POINTER(ctype))


def _f64(a) -> np.ndarray:
    return np.ascontiguousarray(a, dtype=np.float64)


# ---------------------------------------------------------------------------- RNG
def philox4x32_10(ctr, key) -> np.ndarray:
    c = np.ascontiguousarray(ctr, dtype=np.uint32)
    k = np.ascontiguousarray(key, dtype=np.uint32)
    out = np.zeros(4, dtype=np.uint32)
    lib().orc_philox4x32_10(_p(c, C.c_uint32), _p(k, C.c_uint32), _p(out, C.c_uint32))
    return out


def det_log(u: float) -> float:
    return lib().orc_log(float(u))


def det_sincos2pi_u53(v: int) -> tuple[float, float]:
    s, c = C.c_double(), C.c_double()
    lib().orc_sincos2pi_u53(int(v), C.byref(s), C.byref(c))
    return s.value, c.value


def normals(seed: int, t: int, purpose: int, i: int, D: int, ubits: int = 53) -> np.ndarray:
    z = np.zeros(D, dtype=np.float64)
    lib().orc_normals(seed, t, purpose, i, D, ubits, _p(z, C.c_double))
    return z


# ----------------------------------------------------------------- quantisation
def expfx(y: float) -> int:
    return int(lib().orc_expfx(float(y)))


def expfx_table() -> np.ndarray:
    """T1 (entries 0..63, ~2^63 2^(-j/64)) and T2 (64..127, ~2^63 2^(-j/4096))."""
    out = np.zeros(128, dtype=np.uint64)
    lib().orc_expfx_table(_p(out, C.c_uint64))
    return out


def quant_shift(N: int) -> int:
    return int(lib().orc_quant_shift(N))


def quantise(logw, m: float):
    """Returns (W, S, sumW2, sumE) with the sums as Python ints (exact)."""
    lw = _f64(logw)
    W = np.zeros(lw.size, dtype=np.uint64)
    sums = np.zeros(5, dtype=np.uint64)
    lib().orc_quantise(lw.size, _p(lw, C.c_double), float(m), _p(W, C.c_uint64), _p(sums, C.c_uint64))
    s = [int(v) for v in sums]
    return W, s[0], s[1] | (s[2] << 64), s[3] | (s[4] << 64)


def decide(N: int, S: int, sumW2: int, mode: int = RESAMPLE_ESS, nstar: int = 0) -> bool:
    """Algorithm 2, line 7: resample iff N_eff = S^2 / sum W^2 < N* (nstar = 0:
    the paper's N* = N/2)."""
    return bool(lib().orc_decide_nstar(N, nstar, S, sumW2 & ((1 << 64) - 1), sumW2 >> 64, mode))


def resample_u(seed: int, t: int, S: int) -> int:
    return int(lib().orc_resample_u(seed, t, S))


def systematic(W, S: int, U: int):
    Wa = np.ascontiguousarray(W, dtype=np.uint64)
    nc = np.zeros(Wa.size, dtype=np.int32)
    off = np.zeros(Wa.size, dtype=np.uint32)
    lib().orc_systematic(Wa.size, _p(Wa, C.c_uint64), S, U, _p(nc, C.c_int32), _p(off, C.c_uint32))
    return nc, off


def resample(logw, seed: int, t: int, mode: int = RESAMPLE_ESS):
    """Algorithm 4, line 1 on logw.  Returns dict(ncopies, off, W, m, did, S, U, sumW2, sumE)."""
    lw = _f64(logw)
    N = lw.size
    nc = np.zeros(N, dtype=np.int32)
    off = np.zeros(N, dtype=np.uint32)
    W = np.zeros(N, dtype=np.uint64)
    st = np.zeros(8, dtype=np.uint64)
    rc = lib().orc_resample(N, _p(lw, C.c_double), seed, t, mode, _p(nc, C.c_int32), _p(off, C.c_uint32),
                            _p(W, C.c_uint64), _p(st, C.c_uint64))
    if rc:
        raise FloatingPointError("non-finite log-weights")
    s = [int(v) for v in st]
    m = np.array([s[0]], dtype=np.uint64).view(np.float64)[0]
    return dict(ncopies=nc, off=off, W=W, m=float(m), did=bool(s[1]), S=s[2], U=s[3],
                sumW2=s[4] | (s[5] << 64), sumE=s[6] | (s[7] << 64))


def redistribute(ncopies, x: np.ndarray) -> np.ndarray:
    """Algorithm 5 on the rows of x (any dtype; rows are copied as bytes)."""
    nc = np.ascontiguousarray(ncopies, dtype=np.int32)
    xa = np.ascontiguousarray(x)
    out = np.empty_like(xa)
    N = nc.size
    row_bytes = xa.nbytes // N if N else 0
    lib().orc_redistribute(N, row_bytes, _p(nc, C.c_int32), xa.ctypes.data_as(C.c_void_p),
                           out.ctypes.data_as(C.c_void_p))
    return out


def nearly_sort(ncopies, x: np.ndarray):
    """Algorithm 8 (S-NS) on the keys ncopies and the rows of x: returns
    (ncopies_new, x_new)."""
    nc = np.ascontiguousarray(ncopies, dtype=np.int32)
    xa = np.ascontiguousarray(x)
    nc_new = np.empty_like(nc)
    out = np.empty_like(xa)
    N = nc.size
    row_bytes = xa.nbytes // N if N else 0
    lib().orc_nearly_sort(N, row_bytes, _p(nc, C.c_int32), xa.ctypes.data_as(C.c_void_p), _p(nc_new, C.c_int32),
                          out.ctypes.data_as(C.c_void_p))
    return nc_new, out


def reset_logw(N: int) -> float:
    return float(lib().orc_reset_logw(N))


# ---------------------------------------------------------------------- targets
class Target:
    """Owns an oracle target handle."""

    def __init__(self, handle, D: int):
        if not handle:
            raise ValueError("target construction failed (Sigma not positive definite?)")
        self.h = C.c_void_p(handle)
        self.D = D

    def __del__(self):
        try:
            lib().orc_target_free(self.h)
        except Exception:
            pass

    @classmethod
    def gauss(cls, mu, Sigma):
        mu, S = _f64(mu), _f64(Sigma)
        D = mu.size
        return cls(lib().orc_target_gauss(D, _p(mu, C.c_double), _p(S, C.c_double)), D)

    @classmethod
    def logistic(cls, X, y, prior_var: float):
        X, y = _f64(X), _f64(y)
        M, D = X.shape
        return cls(lib().orc_target_logistic(D, M, _p(X, C.c_double), _p(y, C.c_double), prior_var), D)

    @classmethod
    def student_t(cls, mu: float, nu: float):
        return cls(lib().orc_target_student_t(mu, nu), 1)

    def chol(self) -> np.ndarray:
        L = np.zeros((self.D, self.D))
        lib().orc_target_chol(self.h, _p(L, C.c_double))
        return L

    def logpi(self, x) -> np.ndarray:
        xa = _f64(x).reshape(-1, self.D)
        return np.array([lib().orc_logpi(self.h, _p(np.ascontiguousarray(r), C.c_double)) for r in xa])


def cholesky(Sigma) -> np.ndarray:
    S = _f64(Sigma)
    D = S.shape[0]
    L = np.zeros((D, D))
    if lib().orc_cholesky(D, _p(S, C.c_double), _p(L, C.c_double)):
        raise ValueError("not positive definite")
    return L


# ----------------------------------------------------------------------- stages
def init(tgt: Target, N: int, seed: int, init_scale: float, ubits: int = 53):
    D = tgt.D
    x = np.zeros((N, D))
    lw = np.zeros(N)
    lp = np.zeros(N)
    lib().orc_init(tgt.h, N, D, seed, init_scale, ubits, _p(x, C.c_double), _p(lw, C.c_double),
                   _p(lp, C.c_double))
    return x, lw, lp


def move(x, seed: int, t: int, step: float, ubits: int = 53) -> np.ndarray:
    xa = _f64(x)
    N, D = xa.shape
    out = np.zeros_like(xa)
    lib().orc_move(N, D, seed, t, step, ubits, _p(xa, C.c_double), _p(out, C.c_double))
    return out


def reweight(tgt: Target, x_prev, x, logpi_prev, logw, step: float):
    """Eq. (5).  Returns (logw_new, logpi_new); inputs are not modified."""
    xa = _f64(x)
    N, D = xa.shape
    xp = _f64(x_prev) if x_prev is not None else None
    lpp = _f64(logpi_prev).copy()
    lw = _f64(logw).copy()
    lp = np.zeros(N)
    lib().orc_reweight(tgt.h, N, D, step, _p(xp, C.c_double) if xp is not None else None,
                       _p(xa, C.c_double), _p(lpp, C.c_double), _p(lw, C.c_double), _p(lp, C.c_double))
    return lw, lp


def lse_ess(logw):
    lw = _f64(logw)
    m, lse, ess = C.c_double(), C.c_double(), C.c_double()
    if lib().orc_lse_ess(lw.size, _p(lw, C.c_double), C.byref(m), C.byref(lse), C.byref(ess)):
        raise FloatingPointError("non-finite log-weights")
    return m.value, lse.value, ess.value


def estimate(x, logw, lse: float, with_cov: bool = True):
    xa = _f64(x)
    N, D = xa.shape
    lw = _f64(logw)
    mean = np.zeros(D)
    cov = np.zeros((D, D)) if with_cov else None
    lib().orc_estimate(N, D, _p(xa, C.c_double), _p(lw, C.c_double), lse, _p(mean, C.c_double),
                       _p(cov, C.c_double) if cov is not None else None)
    return mean, cov


def run(tgt: Target, N: int, seed: int, K: int, init_scale: float = 2.0, step: float = 0.5,
        mode: int = RESAMPLE_ESS, ubits: int = 53, ncopies_trace: bool = False, nstar: int = 0):
    """Algorithm 2 for K iterations; returns a dict of final state and traces."""
    D = tgt.D
    x = np.zeros((N, D))
    lw = np.zeros(N)
    lp = np.zeros(N)
    trace = np.zeros((max(K, 1), 6))
    means = np.zeros((max(K, 1), D))
    cov = np.zeros((D, D))
    fhat = np.zeros(D)
    nct = np.zeros((K, N), dtype=np.int32) if ncopies_trace else None
    rc = lib().orc_run(tgt.h, N, D, seed, init_scale, step, mode, nstar, ubits, K, _p(x, C.c_double),
                       _p(lw, C.c_double), _p(lp, C.c_double), _p(trace, C.c_double), _p(means, C.c_double),
                       _p(cov, C.c_double), _p(fhat, C.c_double),
                       _p(nct, C.c_int32) if nct is not None else None)
    if rc:
        raise FloatingPointError("oracle run failed (non-finite weights)")
    return dict(x=x, logw=lw, logpi=lp, trace=trace[:K], means=means[:K], cov=cov, fhat=fhat,
                ncopies=nct)
