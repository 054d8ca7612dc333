"""ctypes binding of libhikf.so: argument marshalling only.

Every step of the filter runs in the CUDA library; this module converts numpy
arrays and torch device tensors into plain pointers and sizes, calls the C ABI
of ``include/hikf.h`` and turns status codes into exceptions. If the library
is missing it raises: there is no CPU fallback.
"""
from __future__ import annotations

import ctypes as C
import os
from pathlib import Path
from typing import Optional

import numpy as np

LIB_PATH = Path(__file__).resolve().parent / "_lib" / "libhikf.so"

HIKF_OK, HIKF_EINVAL, HIKF_ENOMEM, HIKF_ECUDA, HIKF_ENOTPD, HIKF_ETIMEOUT, HIKF_ESTATE = range(7)
STATUS_NAMES = {0: "HIKF_OK", 1: "HIKF_EINVAL", 2: "HIKF_ENOMEM", 3: "HIKF_ECUDA", 4: "HIKF_ENOTPD",
                5: "HIKF_ETIMEOUT", 6: "HIKF_ESTATE"}
KERNEL_WHITE, KERNEL_EXP, KERNEL_GAUSS, KERNEL_GCF, KERNEL_LOG = 0, 1, 2, 3, 4
PREC_FP32, PREC_MIXED, PREC_FP64 = 0, 1, 2
PRECISIONS = {"fp32": PREC_FP32, "mixed": PREC_MIXED, "fp64": PREC_FP64}
CHAIN_AUTO, CHAIN_FACTOR, CHAIN_SPECTRAL = 0, 1, 2
CHAINS = {"auto": CHAIN_AUTO, "factor": CHAIN_FACTOR, "spectral": CHAIN_SPECTRAL}
FORM_CROSS, FORM_EIGEN, FORM_NSPACE, FORM_AUTO = 0, 1, 2, 3
FORMS = {"cross": FORM_CROSS, "eigen": FORM_EIGEN, "nspace": FORM_NSPACE, "auto": FORM_AUTO}
M2L_AUTO, M2L_TENSOR, M2L_SIMT = 0, 1, 2
M2LS = {"auto": M2L_AUTO, "tensor": M2L_TENSOR, "simt": M2L_SIMT}

# every symbol include/hikf.h declares
EXPORTED = ["hikf_options_default", "hikf_create", "hikf_create_dense_r", "hikf_create_with_cq", "hikf_assimilate",
            "hikf_assimilate_device", "hikf_sync", "hikf_get_mean", "hikf_get_variance",
            "hikf_get_mean_device", "hikf_get_variance_device", "hikf_get_cq", "hikf_get_cross",
            "hikf_get_perm", "hikf_info", "hikf_step", "hikf_stream", "hikf_last_error", "hikf_destroy", "hikf_h2_qht",
            "hikf_profile_enable", "hikf_profile_read", "hikf_spd_inverse", "hikf_spd_inverse_noalloc",
            "hikf_test_set_wait_limit", "hikf_create_shard", "hikf_shard_rows", "hikf_shard_caller_index",
            "hikf_shard_step_begin", "hikf_shard_step_end", "hikf_shard_get_mean", "hikf_shard_get_variance",
            "hikf_assimilate_batch", "hikf_release_cached_memory"]

# hikf_allreduce_fn: int (*)(double* d_buf, int64_t count, void* ctx)
ALLREDUCE_FN = C.CFUNCTYPE(C.c_int, C.c_void_p, C.c_int64, C.c_void_p)


class HikfError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"{STATUS_NAMES.get(code, code)}: {msg}")
        self.code = code


class Kernel(C.Structure):
    _fields_ = [("pow", C.c_int), ("theta", C.c_double), ("length", C.c_double), ("shape", C.c_double)]


class Options(C.Structure):
    _fields_ = [("cheb_order", C.c_int), ("leaf_size", C.c_int), ("max_depth", C.c_int),
                ("precision", C.c_int), ("cuda_stream", C.c_void_p), ("chain", C.c_int), ("form", C.c_int),
                ("graph", C.c_int), ("m2l", C.c_int), ("sweep_products", C.c_int)]


class Shard(C.Structure):
    _fields_ = [("rank", C.c_int), ("nranks", C.c_int), ("allreduce", ALLREDUCE_FN), ("ctx", C.c_void_p)]


class Info(C.Structure):
    _fields_ = [("m", C.c_int64), ("n", C.c_int), ("dim", C.c_int), ("depth", C.c_int),
                ("cheb_order", C.c_int), ("precision", C.c_int), ("step", C.c_int64),
                ("device_bytes", C.c_int64), ("create_ms", C.c_double), ("sweep_launches", C.c_int),
                ("chain", C.c_int), ("form", C.c_int), ("eig_sweeps", C.c_int), ("cond_s", C.c_double),
                ("sweep_products", C.c_int)]


_lib = None


def load(path: Optional[os.PathLike] = None) -> C.CDLL:
    """Load libhikf.so (raises if it was not built)."""
    global _lib
    if _lib is not None and path is None:
        return _lib
    p = Path(path) if path else LIB_PATH
    if not p.exists():
        raise FileNotFoundError(f"{p} not found: build it with `python -m paper_1404_3816_gb300.build`")
    lib = C.CDLL(str(p))
    dp, ip, vp = C.POINTER(C.c_double), C.POINTER(C.c_int64), C.c_void_p
    H = C.c_void_p
    lib.hikf_options_default.argtypes = [C.POINTER(Options)]
    lib.hikf_create.argtypes = [C.POINTER(H), C.c_int, C.c_int64, dp, Kernel, C.c_int, ip, ip, dp, dp, dp,
                                Kernel, C.POINTER(Options)]
    lib.hikf_create_dense_r.argtypes = [C.POINTER(H), C.c_int, C.c_int64, dp, Kernel, C.c_int, ip, ip, dp, dp, dp,
                                        Kernel, C.POINTER(Options)]
    lib.hikf_create_with_cq.argtypes = [C.POINTER(H), C.c_int, C.c_int64, dp, Kernel, C.c_int, ip, ip, dp, dp,
                                        dp, Kernel, dp, dp, C.POINTER(Options)]
    lib.hikf_assimilate.argtypes = [H, dp]
    lib.hikf_assimilate_device.argtypes = [H, vp]
    lib.hikf_assimilate_batch.argtypes = [C.POINTER(H), C.POINTER(vp), C.c_int]
    lib.hikf_sync.argtypes = [H]
    for nm in ("hikf_get_mean", "hikf_get_variance", "hikf_get_cq", "hikf_get_cross"):
        getattr(lib, nm).argtypes = [H, dp]
    lib.hikf_get_mean_device.argtypes = [H, vp]
    lib.hikf_get_variance_device.argtypes = [H, vp]
    lib.hikf_get_perm.argtypes = [H, ip]
    lib.hikf_info.argtypes = [H, C.POINTER(Info)]
    lib.hikf_stream.argtypes = [H]
    lib.hikf_stream.restype = C.c_void_p
    lib.hikf_last_error.argtypes = [H]
    lib.hikf_last_error.restype = C.c_char_p
    lib.hikf_destroy.argtypes = [H]
    lib.hikf_destroy.restype = None
    lib.hikf_profile_enable.argtypes = [H, C.c_int]
    lib.hikf_profile_read.argtypes = [H, dp, ip]
    lib.hikf_spd_inverse.argtypes = [vp, C.c_int, vp, vp]
    lib.hikf_spd_inverse_noalloc.argtypes = [vp, C.c_int, vp, vp]
    lib.hikf_h2_qht.argtypes = [C.c_int, C.c_int64, dp, Kernel, C.c_int, ip, ip, dp, C.POINTER(Options), dp]
    lib.hikf_test_set_wait_limit.argtypes = [C.c_uint64]
    lib.hikf_release_cached_memory.argtypes = []
    lib.hikf_create_shard.argtypes = [C.POINTER(H), C.POINTER(Shard), C.c_int, C.c_int64, dp, Kernel, C.c_int, ip, ip,
                                      dp, dp, dp, Kernel, C.POINTER(Options)]
    lib.hikf_shard_rows.argtypes = [H, ip, ip]
    lib.hikf_shard_caller_index.argtypes = [H, ip]
    lib.hikf_shard_step_begin.argtypes = [H, vp, vp]
    lib.hikf_shard_step_end.argtypes = [H, vp]
    lib.hikf_shard_get_mean.argtypes = [H, dp]
    lib.hikf_shard_get_variance.argtypes = [H, dp]
    lib.hikf_step.argtypes = [H]
    lib.hikf_step.restype = C.c_int64
    for nm in EXPORTED:
        if nm not in ("hikf_stream", "hikf_last_error", "hikf_destroy", "hikf_step"):
            getattr(lib, nm).restype = C.c_int
    if path is None:
        _lib = lib
    return lib


def _dp(a: Optional[np.ndarray]):
    if a is None:
        return None
    return a.ctypes.data_as(C.POINTER(C.c_double))


def _ip(a: np.ndarray):
    return a.ctypes.data_as(C.POINTER(C.c_int64))


def _f64(a) -> np.ndarray:
    return np.ascontiguousarray(np.asarray(a, dtype=np.float64))


def _i64(a) -> np.ndarray:
    return np.ascontiguousarray(np.asarray(a, dtype=np.int64))


def kernel_struct(spec) -> Kernel:
    """From an object with .pow/.theta/.length[/.shape] or a (pow, theta, length[, shape]) tuple."""
    if isinstance(spec, tuple):
        return Kernel(int(spec[0]), float(spec[1]), float(spec[2]), float(spec[3]) if len(spec) > 3 else 1.0)
    return Kernel(int(spec.pow), float(spec.theta), float(spec.length), float(getattr(spec, "shape", 1.0)))


def options(cheb_order: int = 8, leaf_size: int = 64, max_depth: int = -1, precision="fp32",
            stream=None, chain="auto", form="auto", graph=True, m2l="auto", sweep_products=0) -> Options:
    o = Options()
    load().hikf_options_default(C.byref(o))
    o.cheb_order = int(cheb_order)
    o.leaf_size = int(leaf_size)
    o.max_depth = int(max_depth)
    o.precision = PRECISIONS[precision] if isinstance(precision, str) else int(precision)
    o.chain = CHAINS[chain] if isinstance(chain, str) else int(chain)
    o.form = FORMS[form] if isinstance(form, str) else int(form)
    o.graph = 1 if graph else 0
    o.m2l = M2LS[m2l] if isinstance(m2l, str) else int(m2l)
    o.sweep_products = int(sweep_products)
    if stream is not None:
        o.cuda_stream = C.c_void_p(int(getattr(stream, "cuda_stream", stream)))
    return o


def _device_f64(t, shape, what: str, device=None) -> int:
    """Pointer of a CUDA float64 tensor after checking it, before anything is launched.

    The kernels behind a device pointer read or write exactly prod(shape) contiguous
    float64 values on the handle's device; anything else (another dtype, a host or
    strided tensor, a short buffer, another device) would make them read or write
    outside it, so it is refused here with HIKF_EINVAL.
    """
    import torch
    if not (hasattr(t, "data_ptr") and hasattr(t, "is_cuda") and hasattr(t, "is_contiguous")):
        raise HikfError(HIKF_EINVAL, f"{what}: expected a torch CUDA tensor, got {type(t).__name__}")
    if not t.is_cuda:
        raise HikfError(HIKF_EINVAL, f"{what}: tensor is not on a CUDA device ({t.device})")
    if t.dtype != torch.float64:
        raise HikfError(HIKF_EINVAL, f"{what}: dtype {t.dtype}, expected torch.float64")
    if tuple(t.shape) != tuple(shape):
        raise HikfError(HIKF_EINVAL, f"{what}: shape {tuple(t.shape)}, expected {tuple(shape)}")
    if not t.is_contiguous():
        raise HikfError(HIKF_EINVAL, f"{what}: tensor is not contiguous")
    if device is not None and t.device.index != device:
        raise HikfError(HIKF_EINVAL, f"{what}: tensor on cuda:{t.device.index}, the handle on cuda:{device}")
    return int(t.data_ptr())


def _host_f64(a, count: int, what: str) -> int:
    """Address of a host float64 buffer of exactly `count` contiguous values (numpy or a CPU tensor)."""
    if hasattr(a, "data_ptr"):
        import torch
        if a.is_cuda or a.dtype != torch.float64 or not a.is_contiguous() or a.numel() != count:
            raise HikfError(HIKF_EINVAL, f"{what}: expected a contiguous host float64 tensor of {count} values")
        return int(a.data_ptr())
    if not isinstance(a, np.ndarray) or a.dtype != np.float64 or not a.flags.c_contiguous or a.size != count:
        raise HikfError(HIKF_EINVAL, f"{what}: expected a contiguous float64 array of {count} values")
    return int(a.ctypes.data)


def _current_device():
    """The CUDA device current at handle creation (None when torch has not set one up)."""
    import sys
    torch = sys.modules.get("torch")
    try:
        if torch is not None and torch.cuda.is_available() and torch.cuda.is_initialized():
            return int(torch.cuda.current_device())
    except Exception:
        pass
    return None


def _check(code: int, h=None):
    if code != HIKF_OK:
        msg = load().hikf_last_error(h)
        raise HikfError(code, msg.decode() if msg else "")


class Filter:
    """One HiKF filter (a handle of the C ABI)."""

    def __init__(self, points, q, h_rowptr, h_col, h_val, r_diag, x0=None, p0=None, cq=None, c0=None,
                 r_full=None, **opts):
        """r_diag: the diagonal of R (n); or r_full: the full n x n R (hikf_create_dense_r)."""
        lib = load()
        self._keep = []
        pts = _f64(points)
        m, dim = pts.shape
        rowptr, col, val = _i64(h_rowptr), _i64(h_col), _f64(h_val)
        rd = None if r_diag is None else _f64(r_diag)
        n = rowptr.shape[0] - 1
        x0a = None if x0 is None else _f64(x0)
        p0k = kernel_struct(p0) if p0 is not None else Kernel(int(getattr(q, "pow", 1)), 0.0, 1.0,
                                                              float(getattr(q, "shape", 1.0)))
        o = options(**opts)
        self.h = C.c_void_p()
        if r_full is not None:
            rf = _f64(r_full)
            if rf.shape != (n, n):
                raise HikfError(HIKF_EINVAL, f"r_full: shape {rf.shape}, expected ({n}, {n})")
            code = lib.hikf_create_dense_r(C.byref(self.h), dim, m, _dp(pts), kernel_struct(q), n, _ip(rowptr),
                                           _ip(col), _dp(val), _dp(rf), _dp(x0a), p0k, C.byref(o))
        elif cq is None:
            code = lib.hikf_create(C.byref(self.h), dim, m, _dp(pts), kernel_struct(q), n, _ip(rowptr), _ip(col),
                                   _dp(val), _dp(rd), _dp(x0a), p0k, C.byref(o))
        else:
            cqa, c0a = _f64(cq), _f64(c0)
            code = lib.hikf_create_with_cq(C.byref(self.h), dim, m, _dp(pts), kernel_struct(q), n, _ip(rowptr),
                                           _ip(col), _dp(val), _dp(rd), _dp(x0a), p0k, _dp(cqa), _dp(c0a),
                                           C.byref(o))
        if code != HIKF_OK:
            self.h = None
            _check(code, None)
        self.m, self.n, self.dim = m, n, dim
        self.device = _current_device()

    @classmethod
    def from_workload(cls, w, **opts):
        """Build from a ``workload.Workload`` (points, kernels, CSR H, R, x0)."""
        opts.setdefault("cheb_order", w.cheb_order)
        opts.setdefault("leaf_size", w.leaf_size)
        return cls(w.points, w.q, w.h_rowptr, w.h_col, w.h_val, w.r_diag, w.x0, w.p0, **opts)

    def close(self):
        if getattr(self, "h", None):
            load().hikf_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    # --- measurement update -------------------------------------------------
    def assimilate(self, y):
        ya = _f64(y)
        if ya.shape != (self.n,):
            raise HikfError(HIKF_EINVAL, f"y: shape {ya.shape}, expected ({self.n},)")
        _check(load().hikf_assimilate(self.h, _dp(ya)), self.h)

    def assimilate_device(self, d_y):
        """y as a CUDA tensor of n float64 (contiguous, on the handle's device); asynchronous."""
        ptr = _device_f64(d_y, (self.n,), "y", self.device)
        _check(load().hikf_assimilate_device(self.h, C.c_void_p(ptr)), self.h)

    def sync(self):
        _check(load().hikf_sync(self.h), self.h)

    # --- outputs --------------------------------------------------------------
    def mean(self) -> np.ndarray:
        out = np.empty(self.m)
        _check(load().hikf_get_mean(self.h, _dp(out)), self.h)
        return out

    def variance(self) -> np.ndarray:
        out = np.empty(self.m)
        _check(load().hikf_get_variance(self.h, _dp(out)), self.h)
        return out

    def mean_into(self, out) -> None:
        """Host (numpy or CPU tensor, possibly pinned) or device (torch CUDA tensor) m-vector of float64."""
        self._vec_into(out, "hikf_get_mean", "hikf_get_mean_device", "mean out")

    def variance_into(self, out) -> None:
        self._vec_into(out, "hikf_get_variance", "hikf_get_variance_device", "variance out")

    def _vec_into(self, out, host_fn: str, dev_fn: str, what: str) -> None:
        if getattr(out, "is_cuda", False):
            ptr = _device_f64(out, (self.m,), what, self.device)
            _check(getattr(load(), dev_fn)(self.h, C.c_void_p(ptr)), self.h)
        else:
            ptr = _host_f64(out, self.m, what)
            _check(getattr(load(), host_fn)(self.h, C.cast(C.c_void_p(ptr), C.POINTER(C.c_double))), self.h)

    def cq(self) -> np.ndarray:
        out = np.empty((self.m, self.n))
        _check(load().hikf_get_cq(self.h, _dp(out)), self.h)
        return out

    def cross(self) -> np.ndarray:
        out = np.empty((self.m, self.n))
        _check(load().hikf_get_cross(self.h, _dp(out)), self.h)
        return out

    def perm(self) -> np.ndarray:
        out = np.empty(self.m, dtype=np.int64)
        _check(load().hikf_get_perm(self.h, _ip(out)), self.h)
        return out

    def step(self) -> int:
        """Measurement updates applied so far."""
        return int(load().hikf_step(self.h))

    def info(self) -> dict:
        i = Info()
        _check(load().hikf_info(self.h, C.byref(i)), self.h)
        return {k: getattr(i, k) for k, _ in Info._fields_}

    def profile(self, enable: bool = True):
        _check(load().hikf_profile_enable(self.h, int(enable)), self.h)

    def profile_read(self):
        """(total sweep ms, number of recorded sweep launches)."""
        ms = C.c_double()
        cnt = C.c_int64()
        _check(load().hikf_profile_read(self.h, C.byref(ms), C.byref(cnt)), self.h)
        return ms.value, cnt.value

    @property
    def stream(self) -> int:
        return int(load().hikf_stream(self.h) or 0)


def assimilate_batch(filters, d_ys) -> None:
    """One step of each filter (filters[i] takes d_ys[i]: a CUDA tensor of its n float64),
    asynchronous: the MIXED tensor-core sweeps of all of them in one launch per MMA width
    (hikf_assimilate_batch); each filter's result is that of filters[i].assimilate_device."""
    k = len(filters)
    if len(d_ys) != k:
        raise HikfError(HIKF_EINVAL, f"{k} filters, {len(d_ys)} measurement vectors")
    hs = (C.c_void_p * max(k, 1))(*[f.h for f in filters])
    ys = (C.c_void_p * max(k, 1))(*[_device_f64(y, (f.n,), "y", f.device) for f, y in zip(filters, d_ys)])
    _check(load().hikf_assimilate_batch(hs, ys, k), None)  # the message: hikf_last_error(NULL)


def h2_qht(points, kernel, h_rowptr, h_col, h_val, **opts) -> np.ndarray:
    """The H^2 product Q H^T alone (m x n, caller order)."""
    lib = load()
    pts = _f64(points)
    m, dim = pts.shape
    rowptr, col, val = _i64(h_rowptr), _i64(h_col), _f64(h_val)
    n = rowptr.shape[0] - 1
    out = np.empty((m, n))
    o = options(**opts)
    _check(lib.hikf_h2_qht(dim, m, _dp(pts), kernel_struct(kernel), n, _ip(rowptr), _ip(col), _dp(val),
                           C.byref(o), _dp(out)), None)
    return out


def _spd_args(d_S, d_M):
    n = int(d_S.shape[0]) if hasattr(d_S, "shape") and len(d_S.shape) == 2 else -1
    if n < 1:
        raise HikfError(HIKF_EINVAL, "S: expected an n x n CUDA float64 tensor")
    dev = d_S.device.index if getattr(d_S, "is_cuda", False) else None
    ps = _device_f64(d_S, (n, n), "S")
    pm = _device_f64(d_M, (n, n), "M", dev)
    return n, ps, pm


def _stream_ptr(stream):
    return None if stream is None else C.c_void_p(int(getattr(stream, "cuda_stream", stream)))


def release_cached_memory() -> None:
    """Return the device memory cached in the library's pool (freed state and create scratch)."""
    _check(load().hikf_release_cached_memory(), None)


def spd_inverse(d_S, d_M, stream=None):
    """M = S^{-1} for device tensors (n x n float64) through hikf_spd_inverse."""
    n, ps, pm = _spd_args(d_S, d_M)
    _check(load().hikf_spd_inverse(C.c_void_p(ps), n, C.c_void_p(pm), _stream_ptr(stream)), None)


def spd_inverse_noalloc(d_S, d_M, stream=None):
    """hikf_spd_inverse_noalloc: the same inverse with the library's static device scratch."""
    n, ps, pm = _spd_args(d_S, d_M)
    _check(load().hikf_spd_inverse_noalloc(C.c_void_p(ps), n, C.c_void_p(pm), _stream_ptr(stream)), None)


def set_wait_limit(ns: int) -> None:
    """Test hook hikf_test_set_wait_limit: limit (ns) of the sweep's abortable waits; 0 = default."""
    _check(load().hikf_test_set_wait_limit(int(ns)), None)
