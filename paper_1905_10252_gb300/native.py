"""Thin ctypes binding of libsmc.so (include/smc.h), same names as the C-ABI.

Only argument marshalling lives here: torch tensors supply device memory and
streams, every step of the sampler runs in the library's CUDA kernels.  There
is no CPU fallback: ``lib()`` raises when libsmc.so has not been built or no
CUDA device is present.
"""
from __future__ import annotations

import ctypes as C
from pathlib import Path

import torch

_LIB_PATH = Path(__file__).resolve().with_name("libsmc.so")

SMC_OK, SMC_EINVAL, SMC_ENOMEM, SMC_ECUDA, SMC_ETIMEOUT, SMC_ENONFINITE = range(6)
SMC_F32, SMC_F64 = 1, 2
SMC_GAUSS, SMC_LOGISTIC, SMC_STUDENT_T = 1, 2, 3
RESAMPLE_ESS, RESAMPLE_ALWAYS, RESAMPLE_NEVER = 0, 1, 2
FLAG_LOGISTIC_CUDA_CORES = 1  # SMC_FLAG_LOGISTIC_CUDA_CORES
FLAG_TEST_STALL_LIKELIHOOD = 2  # SMC_FLAG_TEST_STALL_LIKELIHOOD
FLAG_DEFER_REDISTRIBUTE = 4  # SMC_FLAG_DEFER_REDISTRIBUTE
FLAG_TEST_STALL_BARRIER = 8  # SMC_FLAG_TEST_STALL_BARRIER

EXPORTED = [
    "smc_workspace_bytes", "smc_init", "smc_move", "smc_reweight", "smc_estimate", "smc_resample",
    "smc_redistribute", "smc_step", "smc_step_profile", "smc_sync", "smc_read_stats", "smc_current", "smc_materialize",
    "smc_destroy",
    "smc_last_error", "smc_redistribute_ws_bytes", "smc_redistribute_raw", "smc_resample_raw", "smc_ws_status",
    "smc_redistribute_raw_noalloc", "smc_batch_ws_bytes", "smc_batch_create", "smc_batch_step",
    "smc_batch_step_profile", "smc_batch_set_variant", "smc_batch_tune", "smc_batch_sync", "smc_batch_destroy", "smc_batch_last_error",
    "smc_checkpoint_bytes", "smc_checkpoint_save", "smc_checkpoint_load",
    "smc_nearly_sort_ws_bytes", "smc_nearly_sort_raw", "smc_redistribute_raw_profile",
    "smc_slots_ws_bytes", "smc_slots_create", "smc_slots_attach", "smc_slots_detach", "smc_slots_step",
    "smc_slots_sync", "smc_slots_destroy", "smc_slots_last_error",
]
LAST_ERROR = ("smc_last_error", "smc_batch_last_error", "smc_slots_last_error")

BATCH_MOVE_VARIANTS, BATCH_COPY_VARIANTS = 5, 3  # SMC_BATCH_MOVE_VARIANTS, SMC_BATCH_COPY_VARIANTS

NOALLOC_MAX_N = 1 << 20  # SMC_NOALLOC_MAX_N


class SmcError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"smc error {code}: {msg}")
        self.code = code


class smc_config(C.Structure):
    _fields_ = [
        ("n", C.c_int64), ("d", C.c_int32), ("dtype", C.c_int32), ("seed", C.c_uint64),
        ("target", C.c_int32), ("resample_mode", C.c_int32), ("step", C.c_double), ("init_scale", C.c_double),
        ("mu_dev", C.c_void_p), ("sigma_dev", C.c_void_p), ("X_dev", C.c_void_p), ("y_dev", C.c_void_p),
        ("m", C.c_int32), ("flags", C.c_int32), ("prior_var", C.c_double), ("nu", C.c_double),
        ("nstar", C.c_int64),
    ]


class smc_iter_stats(C.Structure):
    _fields_ = [("lse", C.c_double), ("logc", C.c_double), ("ess", C.c_double), ("max_logw", C.c_double),
                ("resampled", C.c_int64), ("t", C.c_int64), ("survivors", C.c_int64)]

    def as_dict(self) -> dict:
        return {k: getattr(self, k) for k, _ in self._fields_}


STATS_FIELDS = [k for k, _ in smc_iter_stats._fields_]
STATS_WORDS = len(STATS_FIELDS)

_lib = None


def lib_path() -> Path:
    return _LIB_PATH


def load_library() -> C.CDLL:
    """Loads libsmc.so without touching the GPU (used to check the exports)."""
    global _lib
    if _lib is None:
        if not _LIB_PATH.exists():
            raise RuntimeError(f"{_LIB_PATH} is missing: build it with paper_1905_10252_gb300/build.py "
                               "(there is no CPU fallback)")
        L = C.CDLL(str(_LIB_PATH))
        _declare(L)
        _lib = L
    return _lib


def lib() -> C.CDLL:
    if not torch.cuda.is_available():
        raise RuntimeError("libsmc needs a CUDA device; there is no CPU fallback")
    return load_library()


def _declare(L: C.CDLL) -> None:
    vp, i32, i64, u64, dbl, sz = C.c_void_p, C.c_int32, C.c_int64, C.c_uint64, C.c_double, C.c_size_t
    L.smc_workspace_bytes.argtypes = [C.POINTER(smc_config), C.POINTER(sz)]
    L.smc_init.argtypes = [C.POINTER(vp), C.POINTER(smc_config), vp, vp, vp, vp, vp, vp, sz, vp]
    for name in ("smc_move", "smc_reweight", "smc_sync", "smc_materialize", "smc_destroy"):
        getattr(L, name).argtypes = [vp]
    L.smc_estimate.argtypes = [vp, vp, vp]
    L.smc_resample.argtypes = [vp, vp, vp]
    L.smc_redistribute.argtypes = [vp, vp]
    L.smc_step.argtypes = [vp, i32, vp, vp, vp, vp]
    L.smc_step_profile.argtypes = [vp, vp, C.POINTER(vp), i32]
    L.smc_read_stats.argtypes = [vp, C.POINTER(smc_iter_stats)]
    L.smc_current.argtypes = [vp, C.POINTER(i32)]
    L.smc_last_error.argtypes = [vp]
    L.smc_last_error.restype = C.c_char_p
    L.smc_redistribute_ws_bytes.argtypes = [i64, C.POINTER(sz)]
    L.smc_redistribute_raw.argtypes = [i64, i32, vp, vp, vp, vp, vp]
    L.smc_resample_raw.argtypes = [i64, vp, u64, u64, i32, vp, vp, vp, vp]
    L.smc_ws_status.argtypes = [vp, vp]
    L.smc_redistribute_raw_noalloc.argtypes = [i64, i32, vp, vp, vp, vp, vp]
    L.smc_batch_ws_bytes.argtypes = [C.POINTER(vp), i32, C.POINTER(sz)]
    L.smc_batch_create.argtypes = [C.POINTER(vp), C.POINTER(vp), i32, vp, sz, vp]
    L.smc_batch_step.argtypes = [vp, i32, C.POINTER(vp), C.POINTER(vp), C.POINTER(vp)]
    L.smc_batch_step_profile.argtypes = [vp, C.POINTER(vp), i32]
    L.smc_batch_set_variant.argtypes = [vp, i32, i32]
    L.smc_batch_tune.argtypes = [vp, i32, C.POINTER(i32)]
    L.smc_batch_sync.argtypes = [vp, C.POINTER(i32)]
    L.smc_batch_destroy.argtypes = [vp]
    L.smc_batch_last_error.argtypes = [vp]
    L.smc_batch_last_error.restype = C.c_char_p
    L.smc_redistribute_raw_profile.argtypes = [i64, i32, vp, vp, vp, vp, vp, C.POINTER(vp), i32]
    L.smc_nearly_sort_ws_bytes.argtypes = [i64, C.POINTER(sz)]
    L.smc_nearly_sort_raw.argtypes = [i64, i32, vp, vp, vp, vp, vp, vp]
    L.smc_checkpoint_bytes.argtypes = [vp, C.POINTER(sz)]
    L.smc_checkpoint_save.argtypes = [vp, vp, sz]
    L.smc_checkpoint_load.argtypes = [vp, vp, sz]
    L.smc_slots_ws_bytes.argtypes = [C.POINTER(i64), i32, C.POINTER(sz)]
    L.smc_slots_create.argtypes = [C.POINTER(vp), C.POINTER(i64), i32, vp, sz, vp]
    L.smc_slots_attach.argtypes = [vp, i32, vp, vp, vp, vp]
    L.smc_slots_detach.argtypes = [vp, i32]
    L.smc_slots_step.argtypes = [vp, C.POINTER(i32)]
    L.smc_slots_sync.argtypes = [vp, C.POINTER(i32)]
    L.smc_slots_destroy.argtypes = [vp]
    L.smc_slots_last_error.argtypes = [vp]
    L.smc_slots_last_error.restype = C.c_char_p
    for name in EXPORTED:
        if name not in LAST_ERROR:
            getattr(L, name).restype = C.c_int


def _check(rc: int, handle=None) -> None:
    if rc != SMC_OK:
        msg = lib().smc_last_error(handle).decode(errors="replace")
        raise SmcError(rc, msg)


def _ptr(t) -> int | None:
    if t is None:
        return None
    if not t.is_cuda:
        raise ValueError("expected a CUDA tensor")
    if not t.is_contiguous():
        raise ValueError("expected a contiguous tensor")
    return t.data_ptr()


def _stream_ptr(stream) -> int | None:
    if stream is None:
        stream = torch.cuda.current_stream()
    return stream.cuda_stream or None


def _event_handle(e: torch.cuda.Event) -> int:
    """The cudaEvent_t of a torch event (torch creates it at its first record)."""
    if not e.cuda_event:
        e.record(torch.cuda.current_stream())
    return e.cuda_event


def _alloc_ws(nbytes: int, device) -> torch.Tensor:
    return torch.empty(max(int(nbytes), 256), dtype=torch.uint8, device=device)


# ----------------------------------------------------------------- stateless
def smc_redistribute_ws_bytes(n: int) -> int:
    out = C.c_size_t()
    _check(lib().smc_redistribute_ws_bytes(int(n), C.byref(out)))
    return out.value


def smc_redistribute_raw(ncopies: torch.Tensor, x_in: torch.Tensor, x_out: torch.Tensor | None = None,
                         ws: torch.Tensor | None = None, stream=None) -> torch.Tensor:
    """Algorithm 5 on the rows of x_in (any dtype); returns x_out."""
    n = ncopies.numel()
    if x_in.shape[0] != n:
        raise ValueError("x_in must have one row per ncopies entry")
    if x_out is None:
        x_out = torch.empty_like(x_in)
    if ws is None:
        ws = _alloc_ws(smc_redistribute_ws_bytes(n), x_in.device)
    row_bytes = x_in[0].numel() * x_in.element_size() if n else 0
    _check(lib().smc_redistribute_raw(n, row_bytes, _ptr(ncopies), _ptr(x_in), _ptr(x_out), _ptr(ws),
                                      _stream_ptr(stream)))
    return x_out


def smc_nearly_sort_ws_bytes(n: int) -> int:
    out = C.c_size_t()
    _check(lib().smc_nearly_sort_ws_bytes(int(n), C.byref(out)))
    return out.value


def smc_nearly_sort_raw(ncopies: torch.Tensor, x_in: torch.Tensor, ncopies_out: torch.Tensor | None = None,
                        x_out: torch.Tensor | None = None, ws: torch.Tensor | None = None, stream=None):
    """Algorithm 8 (S-NS) on the keys ncopies (int32) and the rows of x_in;
    returns (ncopies_out, x_out)."""
    n = ncopies.numel()
    if x_in.shape[0] != n:
        raise ValueError("x_in must have one row per ncopies entry")
    if ncopies.dtype != torch.int32:
        raise ValueError("ncopies must be int32")
    if ncopies_out is None:
        ncopies_out = torch.empty_like(ncopies)
    if x_out is None:
        x_out = torch.empty_like(x_in)
    if ws is None:
        ws = _alloc_ws(smc_nearly_sort_ws_bytes(n), x_in.device)
    row_bytes = x_in[0].numel() * x_in.element_size() if n else 0
    _check(lib().smc_nearly_sort_raw(n, row_bytes, _ptr(ncopies), _ptr(x_in), _ptr(ncopies_out), _ptr(x_out),
                                     _ptr(ws), _stream_ptr(stream)))
    return ncopies_out, x_out


def smc_redistribute_raw_profile(ncopies: torch.Tensor, x_in: torch.Tensor, x_out: torch.Tensor, ws: torch.Tensor,
                                 events, stream=None) -> torch.Tensor:
    """smc_redistribute_raw with three caller events: before, after the
    ncopies scan, after the row copy."""
    n = ncopies.numel()
    row_bytes = x_in[0].numel() * x_in.element_size() if n else 0
    arr = (C.c_void_p * 3)(*[_event_handle(e) for e in events])
    _check(lib().smc_redistribute_raw_profile(n, row_bytes, _ptr(ncopies), _ptr(x_in), _ptr(x_out), _ptr(ws),
                                              _stream_ptr(stream), arr, 3))
    return x_out


def smc_resample_raw(logw: torch.Tensor, seed: int, t: int, mode: int = RESAMPLE_ESS,
                     ncopies: torch.Tensor | None = None, ws: torch.Tensor | None = None, stream=None,
                     stats: torch.Tensor | None = None):
    """Algorithm 4, line 1 on logw (float64).  Returns (ncopies int32, stats tensor of 6 x 8 bytes)."""
    n = logw.numel()
    if logw.dtype != torch.float64:
        raise ValueError("logw must be float64")
    if ncopies is None:
        ncopies = torch.empty(n, dtype=torch.int32, device=logw.device)
    if ws is None:
        ws = _alloc_ws(smc_redistribute_ws_bytes(n), logw.device)
    if stats is None:
        stats = torch.zeros(STATS_WORDS, dtype=torch.float64, device=logw.device)
    _check(lib().smc_resample_raw(n, _ptr(logw), int(seed), int(t), int(mode), _ptr(ncopies), _ptr(stats),
                                  _ptr(ws), _stream_ptr(stream)))
    return ncopies, stats


def decode_stats(stats: torch.Tensor) -> dict:
    """One smc_iter_stats record (6 x 8 bytes) as a dict."""
    raw = stats.detach().cpu().contiguous()
    b = raw.numpy().tobytes()[: C.sizeof(smc_iter_stats)]
    return smc_iter_stats.from_buffer_copy(b).as_dict()


def smc_redistribute_raw_noalloc(ncopies: torch.Tensor, x_in: torch.Tensor, x_out: torch.Tensor,
                                 status: torch.Tensor | None = None, stream=None) -> torch.Tensor:
    """Algorithm 5 on the rows of x_in into the caller's x_out, using the
    library's fixed internal scratch instead of a workspace (n <= 2^20).  The
    library allocates nothing; status (device int32[1], optional) receives
    SMC_OK or SMC_EINVAL for an invalid ncopies vector."""
    n = ncopies.numel()
    if x_in.shape[0] != n or x_out.shape != x_in.shape:
        raise ValueError("x_in and x_out must have one row per ncopies entry")
    row_bytes = x_in[0].numel() * x_in.element_size() if n else 0
    _check(lib().smc_redistribute_raw_noalloc(n, row_bytes, _ptr(ncopies), _ptr(x_in), _ptr(x_out),
                                              _ptr(status), _stream_ptr(stream)))
    return x_out


def smc_ws_status(ws: torch.Tensor, stream=None) -> int:
    return int(lib().smc_ws_status(_ptr(ws), _stream_ptr(stream)))


# ----------------------------------------------------------------- sampler
class Sampler:
    """Owns the device buffers of one sampler and a libsmc handle.

    target='gauss' needs mu [D] and sigma [D, D]; target='student_t' needs mu
    (scalar) and nu; target='logistic' needs X [M, D], y [M] and prior_var.
    dtype is torch.float32 or torch.float64 (particle state).  nstar is the
    resampling threshold N* of Algorithm 2 (0: N/2).
    """

    def __init__(self, n: int, d: int, *, dtype=torch.float32, seed: int = 0, target: str = "gauss",
                 mu=None, sigma=None, nu: float = 0.0, step: float = 0.5, init_scale: float = 2.0,
                 resample_mode: int = RESAMPLE_ESS, device="cuda", stream: torch.cuda.Stream | None = None,
                 X=None, y=None, prior_var: float = 4.0, flags: int = 0, nstar: int = 0):
        L = lib()
        self.n, self.d, self.dtype = int(n), int(d), dtype
        self.device = torch.device(device)
        self.stream = stream if stream is not None else torch.cuda.Stream(device=self.device)
        cur = torch.cuda.current_stream(self.device)
        kind = {"gauss": SMC_GAUSS, "student_t": SMC_STUDENT_T, "logistic": SMC_LOGISTIC}[target]
        cfg = smc_config()
        cfg.n, cfg.d = self.n, self.d
        cfg.dtype = SMC_F64 if dtype == torch.float64 else SMC_F32
        cfg.seed, cfg.target, cfg.resample_mode = int(seed), kind, int(resample_mode)
        cfg.step, cfg.init_scale, cfg.nu = float(step), float(init_scale), float(nu)
        cfg.flags = int(flags)
        cfg.nstar = int(nstar)  # resampling threshold N* (0: N/2)
        self.mu = self.sigma = self.X = self.y = None
        if target == "logistic":
            self.X = torch.as_tensor(X, dtype=torch.float32).reshape(-1, d).contiguous().to(self.device)
            self.y = torch.as_tensor(y, dtype=torch.float32).reshape(-1).contiguous().to(self.device)
            cfg.X_dev, cfg.y_dev = self.X.data_ptr(), self.y.data_ptr()
            cfg.m, cfg.prior_var = int(self.X.shape[0]), float(prior_var)
        else:
            self.mu = torch.as_tensor(mu, dtype=torch.float64).reshape(-1).to(self.device)
            self.sigma = (torch.as_tensor(sigma, dtype=torch.float64).reshape(d, d).contiguous().to(self.device)
                          if sigma is not None else None)
            cfg.mu_dev = self.mu.data_ptr()
            cfg.sigma_dev = self.sigma.data_ptr() if self.sigma is not None else None
        self.cfg = cfg
        nbytes = C.c_size_t()
        _check(L.smc_workspace_bytes(C.byref(cfg), C.byref(nbytes)))
        dev = self.device
        self.x = torch.empty(self.n, self.d, dtype=dtype, device=dev)
        self.x_alt = torch.empty_like(self.x)
        self.logw = torch.empty(self.n, dtype=torch.float64, device=dev)
        self.logpi = torch.empty(self.n, dtype=dtype, device=dev)
        self.logpi_alt = torch.empty_like(self.logpi)
        self.ws = _alloc_ws(nbytes.value, dev)
        self.stream.wait_stream(cur)
        h = C.c_void_p()
        rc = L.smc_init(C.byref(h), C.byref(cfg), _ptr(self.x), _ptr(self.x_alt), _ptr(self.logw),
                        _ptr(self.logpi), _ptr(self.logpi_alt), _ptr(self.ws), nbytes.value,
                        self.stream.cuda_stream or None)
        _check(rc, None)
        self.h = h
        self._done()

    # every call: our stream waits for the caller's, the caller's waits for ours
    def _enter(self):
        self.stream.wait_stream(torch.cuda.current_stream(self.device))

    def _done(self):
        torch.cuda.current_stream(self.device).wait_stream(self.stream)

    def _call(self, fn, *args):
        self._enter()
        _check(fn(self.h, *args), self.h)
        self._done()

    def move(self):
        self._call(lib().smc_move)

    def reweight(self):
        self._call(lib().smc_reweight)

    def estimate(self, cov: bool = False):
        mean = torch.empty(self.d, dtype=torch.float64, device=self.device)
        c = torch.empty(self.d, self.d, dtype=torch.float64, device=self.device) if cov else None
        self._call(lib().smc_estimate, _ptr(mean), _ptr(c))
        return mean, c

    def resample(self):
        nc = torch.empty(self.n, dtype=torch.int32, device=self.device)
        did = torch.zeros(1, dtype=torch.int32, device=self.device)
        self._call(lib().smc_resample, _ptr(nc), _ptr(did))
        return nc, did

    def redistribute(self, ncopies: torch.Tensor):
        self._call(lib().smc_redistribute, _ptr(ncopies))

    def step(self, k: int, cov: bool = False, trace: bool = False, fhat: bool = False):
        mean = torch.empty(self.d, dtype=torch.float64, device=self.device)
        c = torch.empty(self.d, self.d, dtype=torch.float64, device=self.device) if cov else None
        tr = torch.zeros(max(k, 1), STATS_WORDS, dtype=torch.float64, device=self.device) if trace else None
        fh = torch.empty(self.d, dtype=torch.float64, device=self.device) if fhat else None
        self._call(lib().smc_step, int(k), _ptr(mean), _ptr(c), _ptr(tr), _ptr(fh))
        return dict(mean=mean, cov=c, trace=tr, fhat=fh)

    def step_profile(self, events=None, mean: torch.Tensor | None = None):
        """One iteration with 8 caller-created CUDA events recorded around its stages."""
        if events is not None:
            arr = (C.c_void_p * 8)(*[_event_handle(e) for e in events])
            n = 8
        else:
            arr, n = None, 0
        self._call(lib().smc_step_profile, _ptr(mean), arr, n)

    def sync(self) -> None:
        _check(lib().smc_sync(self.h), self.h)

    def materialize(self) -> None:
        """Completes a redistribution deferred by FLAG_DEFER_REDISTRIBUTE (the
        rows, log pi and log w in self's buffers are then the state)."""
        self._call(lib().smc_materialize)

    def stats(self) -> dict:
        s = smc_iter_stats()
        _check(lib().smc_read_stats(self.h, C.byref(s)), self.h)
        return s.as_dict()

    def current(self):
        """(x, logpi) tensors holding the current particles (synchronises)."""
        w = C.c_int32()
        _check(lib().smc_current(self.h, C.byref(w)), self.h)
        return (self.x, self.logpi) if w.value == 0 else (self.x_alt, self.logpi_alt)

    def checkpoint(self) -> bytes:
        """The sampler's state between iterations as bytes (smc_checkpoint_save)."""
        L = lib()
        nb = C.c_size_t()
        _check(L.smc_checkpoint_bytes(self.h, C.byref(nb)), self.h)
        buf = C.create_string_buffer(nb.value)
        self._enter()
        _check(L.smc_checkpoint_save(self.h, buf, nb.value), self.h)
        return buf.raw

    def restore(self, blob: bytes) -> None:
        """Continues from a checkpoint of a sampler with this configuration."""
        buf = C.create_string_buffer(bytes(blob), len(blob))
        self._call(lib().smc_checkpoint_load, buf, len(blob))

    def close(self):
        if getattr(self, "h", None):
            lib().smc_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def _check_batch(rc: int, handle=None) -> None:
    if rc != SMC_OK:
        msg = lib().smc_batch_last_error(handle).decode(errors="replace")
        raise SmcError(rc, msg)


def _ptr_array(tensors):
    if tensors is None:
        return None
    return (C.c_void_p * len(tensors))(*[_ptr(t) for t in tensors])


class Batch:
    """Many FP32 Gaussian samplers stepped with one launch per stage.

    Members keep their own buffers; the batch owns its workspace (kernel
    arguments and block maps) and a stream.  Results per member equal those of
    ``Sampler.step`` on that member alone.  Call ``sync()`` before using a
    member's own methods.
    """

    def __init__(self, members: list[Sampler], stream: torch.cuda.Stream | None = None):
        L = lib()
        self.members = list(members)
        self.device = self.members[0].device
        self.stream = stream if stream is not None else torch.cuda.Stream(device=self.device)
        handles = (C.c_void_p * len(self.members))(*[m.h for m in self.members])
        nbytes = C.c_size_t()
        _check_batch(L.smc_batch_ws_bytes(handles, len(self.members), C.byref(nbytes)))
        self.ws = _alloc_ws(nbytes.value, self.device)
        self.stream.wait_stream(torch.cuda.current_stream(self.device))
        h = C.c_void_p()
        _check_batch(L.smc_batch_create(C.byref(h), handles, len(self.members), _ptr(self.ws), nbytes.value,
                                        self.stream.cuda_stream or None))
        self.h = h

    def _enter(self):
        self.stream.wait_stream(torch.cuda.current_stream(self.device))

    def _done(self):
        torch.cuda.current_stream(self.device).wait_stream(self.stream)

    def step(self, k: int, mean: bool = True, trace: bool = False, fhat: bool = False):
        dev, n = self.device, len(self.members)
        means = [torch.empty(m.d, dtype=torch.float64, device=dev) for m in self.members] if mean else None
        trs = ([torch.zeros(max(k, 1), STATS_WORDS, dtype=torch.float64, device=dev) for _ in range(n)]
               if trace else None)
        fhs = [torch.empty(m.d, dtype=torch.float64, device=dev) for m in self.members] if fhat else None
        self._enter()
        _check_batch(lib().smc_batch_step(self.h, int(k), _ptr_array(means), _ptr_array(trs), _ptr_array(fhs)),
                     self.h)
        self._done()
        return dict(mean=means, trace=trs, fhat=fhs)

    def step_raw(self, k: int, means=None, traces=None, fhats=None):
        """k iterations with caller-provided output tensors (lists or None)."""
        self._enter()
        _check_batch(lib().smc_batch_step(self.h, int(k), _ptr_array(means), _ptr_array(traces),
                                          _ptr_array(fhats)), self.h)
        self._done()

    def step_profile(self, events=None):
        """One batched iteration with 8 caller-created CUDA events around its stages."""
        if events is not None:
            arr, n = (C.c_void_p * 8)(*[_event_handle(e) for e in events]), 8
        else:
            arr, n = None, 0
        self._enter()
        _check_batch(lib().smc_batch_step_profile(self.h, arr, n), self.h)
        self._done()

    def set_variant(self, move_variant: int, copy_variant: int) -> None:
        _check_batch(lib().smc_batch_set_variant(self.h, int(move_variant), int(copy_variant)), self.h)

    def tune(self, reps: int = 5) -> tuple[int, int]:
        self._enter()
        out = (C.c_int32 * 2)()
        _check_batch(lib().smc_batch_tune(self.h, int(reps), out), self.h)
        return int(out[0]), int(out[1])

    def sync(self) -> None:
        which = C.c_int32(-1)
        _check_batch(lib().smc_batch_sync(self.h, C.byref(which)), self.h)

    def close(self):
        if getattr(self, "h", None):
            lib().smc_batch_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def _check_slots(rc: int, handle=None) -> None:
    if rc != SMC_OK:
        msg = lib().smc_slots_last_error(handle).decode(errors="replace")
        raise SmcError(rc, msg)


class Slots:
    """A standing batch of slots of fixed capacity (cap[s] particles): FP32
    Gaussian samplers are attached to and detached from slots between steps
    without rebuilding the launch layout, and each step runs a per-slot
    number of iterations in one launch per stage.  Results per sampler equal
    those of ``Sampler.step`` alone."""

    def __init__(self, caps, stream: torch.cuda.Stream | None = None, device="cuda"):
        L = lib()
        self.caps = [int(c) for c in caps]
        self.count = len(self.caps)
        self.device = torch.device(device)
        self.stream = stream if stream is not None else torch.cuda.Stream(device=self.device)
        arr = (C.c_int64 * self.count)(*self.caps)
        nbytes = C.c_size_t()
        _check_slots(L.smc_slots_ws_bytes(arr, self.count, C.byref(nbytes)))
        self.ws = _alloc_ws(nbytes.value, self.device)
        self.stream.wait_stream(torch.cuda.current_stream(self.device))
        h = C.c_void_p()
        _check_slots(L.smc_slots_create(C.byref(h), arr, self.count, _ptr(self.ws), nbytes.value,
                                        self.stream.cuda_stream))
        self.h = h
        self.members: list = [None] * self.count

    def attach(self, slot: int, sampler: Sampler, mean: torch.Tensor | None = None,
               trace: torch.Tensor | None = None, fhat: torch.Tensor | None = None) -> None:
        _check_slots(lib().smc_slots_attach(self.h, int(slot), sampler.h, _ptr(mean), _ptr(trace), _ptr(fhat)),
                     self.h)
        self.members[slot] = sampler

    def detach(self, slot: int) -> None:
        _check_slots(lib().smc_slots_detach(self.h, int(slot)), self.h)
        self.members[slot] = None

    def step(self, iters) -> None:
        """iters: per-slot iteration counts (0 for idle and empty slots)."""
        arr = (C.c_int32 * self.count)(*[int(v) for v in iters])
        self.stream.wait_stream(torch.cuda.current_stream(self.device))
        _check_slots(lib().smc_slots_step(self.h, arr), self.h)

    def sync(self) -> None:
        which = C.c_int32(-1)
        _check_slots(lib().smc_slots_sync(self.h, C.byref(which)), self.h)

    def close(self):
        if getattr(self, "h", None):
            lib().smc_slots_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def trace_dicts(tr: torch.Tensor) -> list[dict]:
    """Decodes a [K, 7] smc_iter_stats trace (the last three fields are int64)."""
    raw = tr.detach().cpu().contiguous()
    ints = raw.view(torch.int64)
    out = []
    for k in range(raw.shape[0]):
        out.append(dict(lse=float(raw[k, 0]), logc=float(raw[k, 1]), ess=float(raw[k, 2]),
                        max_logw=float(raw[k, 3]), resampled=int(ints[k, 4]), t=int(ints[k, 5]),
                        survivors=int(ints[k, 6])))
    return out
