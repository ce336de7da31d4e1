"""Thin Python binding of libkatz.so (include/katz.h).

Argument marshalling only: every step of the ranking runs in the CUDA
kernels behind the C ABI.  Arrays may be numpy arrays (host) or torch
tensors (host or CUDA); the binding passes their raw pointers.  The library
must have been built (``build.build()``); importing fails loudly otherwise,
there is no CPU fallback.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

from . import build as _build

__all__ = [
    "KatzError", "katz_opts", "katz_info", "katz_default_opts", "katz_create_csr", "katz_destroy",
    "katz_rank_static", "katz_rank", "katz_checkpoint", "katz_restore", "KATZ_CRIT_TOPK", "KATZ_CRIT_RANKING", "KATZ_CRIT_SCORE", "KATZ_CRIT_PAIR",
    "katz_get_ranking", "katz_get_bounds", "katz_get_walk", "katz_get_trace",
    "katz_apply_update_batch", "katz_certify_topk_noalloc", "katz_convert_f64_f32", "katz_server_opts", "katz_request_result",
    "katz_server_default_opts", "Server", "katz_last_error", "katz_status_string", "KATZ_FP64", "KATZ_FP32_CERT", "KATZ_FP32_CERT_AUTO",
    "KATZ_MAX_K", "library_path",
]

KATZ_FP64, KATZ_FP32_CERT, KATZ_FP32_CERT_AUTO = 0, 1, 2
KATZ_CRIT_TOPK, KATZ_CRIT_RANKING, KATZ_CRIT_SCORE, KATZ_CRIT_PAIR = 0, 1, 2, 3
KATZ_MAX_K = 8192
STATUS = ["KATZ_OK", "KATZ_EINVAL", "KATZ_EALPHA", "KATZ_ENOMEM", "KATZ_ECUDA", "KATZ_ENOTCONV",
          "KATZ_EPRECISION", "KATZ_ETIMEOUT", "KATZ_EBUSY", "KATZ_ESTATE"]


class katz_opts(ctypes.Structure):
    _fields_ = [("precision", ctypes.c_int32), ("undirected", ctypes.c_int32), ("keep_history", ctypes.c_int32),
                ("r_max", ctypes.c_int32), ("deg_bound", ctypes.c_int64), ("frontier_abort_frac", ctypes.c_double),
                ("cuda_stream", ctypes.c_void_p), ("use_graph", ctypes.c_int32), ("inbound", ctypes.c_int32),
                ("profile", ctypes.c_int32), ("fp32_from", ctypes.c_int32),
                ("offsets64", ctypes.c_int32), ("l2_fetch_bytes", ctypes.c_int32),
                ("locality", ctypes.c_int32), ("reserved", ctypes.c_int32)]


class katz_info(ctypes.Structure):
    _fields_ = [("r", ctypes.c_int32), ("converged", ctypes.c_int32), ("active", ctypes.c_int64),
                ("k", ctypes.c_int64), ("alpha", ctypes.c_double), ("gamma", ctypes.c_double),
                ("time_ms", ctypes.c_double), ("nnz", ctypes.c_int64), ("fp32_levels", ctypes.c_int32),
                ("full_levels", ctypes.c_int32), ("affected", ctypes.c_int64), ("spmv_ms", ctypes.c_double),
                ("launches", ctypes.c_int64), ("spmv_launches", ctypes.c_int32), ("escalated", ctypes.c_int32)]

    def as_dict(self) -> dict:
        return {f: getattr(self, f) for f, _ in self._fields_ if f != "reserved"}


class katz_server_opts(ctypes.Structure):
    _fields_ = [("workers", ctypes.c_int32), ("slots", ctypes.c_int32), ("slot_updates", ctypes.c_int64),
                ("admit_updates", ctypes.c_int64), ("admit_bytes", ctypes.c_int64),
                ("pair_batches", ctypes.c_int32), ("reserved", ctypes.c_int32)]


class katz_request_result(ctypes.Structure):
    _fields_ = [("status", ctypes.c_int32), ("paired", ctypes.c_int32), ("k", ctypes.c_int64),
                ("info", katz_info), ("queue_ms", ctypes.c_double), ("wait_ms", ctypes.c_double),
                ("service_ms", ctypes.c_double), ("latency_ms", ctypes.c_double)]


class KatzError(RuntimeError):
    def __init__(self, status: int, what: str, detail: str = ""):
        name = STATUS[status] if 0 <= status < len(STATUS) else str(status)
        super().__init__(f"{what}: {name}" + (f" ({detail})" if detail else ""))
        self.status = status
        self.name = name


_lib = None


def library_path() -> str:
    return _build.LIB


def _load():
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(_build.LIB):
        raise ImportError(f"{_build.LIB} is missing: build it with paper_1807_03847_gb300.build.build()")
    lib = ctypes.CDLL(_build.LIB)
    P, i64, i32, dbl = ctypes.c_void_p, ctypes.c_int64, ctypes.c_int32, ctypes.c_double
    sig = {
        "katz_default_opts": (None, [ctypes.POINTER(katz_opts)]),
        "katz_status_string": (ctypes.c_char_p, [ctypes.c_int]),
        "katz_create_csr": (ctypes.c_int, [ctypes.POINTER(P), i64, i64, P, P, ctypes.POINTER(katz_opts)]),
        "katz_destroy": (None, [P]),
        "katz_last_error": (ctypes.c_char_p, [P]),
        "katz_rank_static": (ctypes.c_int, [P, dbl, i64, dbl, ctypes.POINTER(katz_info)]),
        "katz_rank": (ctypes.c_int, [P, dbl, i32, i64, P, dbl, ctypes.POINTER(katz_info)]),
        "katz_checkpoint_size": (ctypes.c_int, [P, ctypes.POINTER(ctypes.c_uint64)]),
        "katz_checkpoint": (ctypes.c_int, [P, P, ctypes.c_uint64]),
        "katz_restore": (ctypes.c_int, [ctypes.POINTER(P), P, ctypes.c_uint64, ctypes.POINTER(katz_opts)]),
        "katz_get_ranking": (ctypes.c_int, [P, P, i64]),
        "katz_get_bounds": (ctypes.c_int, [P, P, P, P]),
        "katz_get_walk": (ctypes.c_int, [P, i32, P]),
        "katz_get_trace": (ctypes.c_int, [P, P, i32]),
        "katz_apply_update_batch": (ctypes.c_int, [P, P, P, P, i64, ctypes.POINTER(katz_info)]),
        "katz_submit_update_batch": (ctypes.c_int, [P, P, P, P, i64, ctypes.POINTER(ctypes.c_uint64)]),
        "katz_poll": (ctypes.c_int, [P, ctypes.c_uint64, ctypes.POINTER(katz_info)]),
        "katz_certify_topk_noalloc": (ctypes.c_int, [P, P, i64, i64, dbl, P, P, P]),
        "katz_convert_f64_f32": (ctypes.c_int, [P, i64, P, P]),
        "katz_server_default_opts": (None, [ctypes.POINTER(katz_server_opts)]),
        "katz_server_create": (ctypes.c_int, [ctypes.POINTER(P), ctypes.POINTER(katz_server_opts)]),
        "katz_server_attach": (ctypes.c_int, [P, P, i64]),
        "katz_server_submit": (ctypes.c_int, [P, P, P, P, P, i64, ctypes.POINTER(ctypes.c_uint64)]),
        "katz_server_wait": (ctypes.c_int, [P, ctypes.c_uint64, i64, P, ctypes.POINTER(katz_request_result)]),
        "katz_server_destroy": (None, [P]),
    }
    for name, (res, args) in sig.items():
        f = getattr(lib, name)
        f.restype = res
        f.argtypes = args
    _lib = lib
    return lib


def _ptr(a):
    """Raw address of a numpy array or torch tensor (None passes NULL)."""
    if a is None:
        return None
    if isinstance(a, np.ndarray):
        if not a.flags["C_CONTIGUOUS"]:
            raise ValueError("array must be C-contiguous")
        return a.ctypes.data
    if hasattr(a, "data_ptr"):
        if not a.is_contiguous():
            raise ValueError("tensor must be contiguous")
        return a.data_ptr()
    raise TypeError(f"expected numpy array or torch tensor, got {type(a)}")


def _check(h, status, what):
    if status != 0:
        detail = _load().katz_last_error(h).decode() if h else ""
        raise KatzError(status, what, detail)


def katz_status_string(status: int) -> str:
    return _load().katz_status_string(status).decode()


def katz_default_opts(**kw) -> katz_opts:
    o = katz_opts()
    _load().katz_default_opts(ctypes.byref(o))
    for k, v in kw.items():
        if not hasattr(o, k):
            raise AttributeError(k)
        setattr(o, k, v)
    return o


def katz_create_csr(n: int, nnz: int, rowptr, col, opts: katz_opts | None = None) -> int:
    """Create a handle (copies the CSR to library-owned device memory)."""
    lib = _load()
    h = ctypes.c_void_p()
    st = lib.katz_create_csr(ctypes.byref(h), int(n), int(nnz), _ptr(rowptr), _ptr(col),
                             ctypes.byref(opts) if opts is not None else None)
    if st != 0:
        raise KatzError(st, "katz_create_csr")
    return h.value


def katz_destroy(h) -> None:
    if h:
        _load().katz_destroy(h)


def katz_last_error(h) -> str:
    return _load().katz_last_error(h).decode()


def katz_rank_static(h, alpha: float, k: int, eps: float, check: bool = True) -> katz_info:
    info = katz_info()
    st = _load().katz_rank_static(h, float(alpha), int(k), float(eps), ctypes.byref(info))
    if check:
        _check(h, st, "katz_rank_static")
    info.status = st
    return info


def katz_rank(h, alpha: float, criterion: int, eps: float, k: int = 0, pair=None, check: bool = True) -> katz_info:
    """Algorithm 1 with a stopping criterion of Sec. 3.1 (KATZ_CRIT_*)."""
    info = katz_info()
    pa = np.ascontiguousarray(pair, np.int32) if pair is not None else None
    st = _load().katz_rank(h, float(alpha), int(criterion), int(k), _ptr(pa), float(eps), ctypes.byref(info))
    if check:
        _check(h, st, "katz_rank")
    info.status = st
    return info


def katz_checkpoint(h) -> np.ndarray:
    """The handle's state as a byte array (see katz_restore)."""
    lib = _load()
    size = ctypes.c_uint64()
    _check(h, lib.katz_checkpoint_size(h, ctypes.byref(size)), "katz_checkpoint_size")
    buf = np.empty(size.value, np.uint8)
    _check(h, lib.katz_checkpoint(h, _ptr(buf), size.value), "katz_checkpoint")
    return buf


def katz_restore(image, opts: katz_opts | None = None) -> int:
    """A new handle from a checkpoint image (byte array)."""
    image = np.ascontiguousarray(image, np.uint8)
    h = ctypes.c_void_p()
    st = _load().katz_restore(ctypes.byref(h), _ptr(image), image.nbytes, ctypes.byref(opts) if opts else None)
    if st != 0:
        raise KatzError(st, "katz_restore")
    return h.value


def katz_get_ranking(h, k: int, out=None):
    if out is None:
        out = np.empty(int(k), np.int32)
    _check(h, _load().katz_get_ranking(h, _ptr(out), int(k)), "katz_get_ranking")
    return out


def katz_get_bounds(h, n: int | None = None, lower=None, upper=None, err=None):
    if lower is None and upper is None and err is None:
        lower, upper, err = (np.empty(int(n), np.float64) for _ in range(3))
    _check(h, _load().katz_get_bounds(h, _ptr(lower), _ptr(upper), _ptr(err)), "katz_get_bounds")
    return lower, upper, err


def katz_get_walk(h, i: int, n: int | None = None, out=None):
    if out is None:
        out = np.empty(int(n), np.float64)
    _check(h, _load().katz_get_walk(h, int(i), _ptr(out)), "katz_get_walk")
    return out


def katz_get_trace(h, cap: int = 1024) -> np.ndarray:
    out = np.zeros(cap, np.int64)
    _check(h, _load().katz_get_trace(h, _ptr(out), int(cap)), "katz_get_trace")
    return out


def katz_apply_update_batch(h, src, dst, is_insert, m: int | None = None, check: bool = True) -> katz_info:
    info = katz_info()
    if m is None:
        m = len(src)
    st = _load().katz_apply_update_batch(h, _ptr(src), _ptr(dst), _ptr(is_insert), int(m), ctypes.byref(info))
    if check:
        _check(h, st, "katz_apply_update_batch")
    info.status = st
    return info


def katz_submit_update_batch(h, src, dst, is_insert) -> int:
    """Queue a batch (host arrays) for asynchronous application; the ticket."""
    src = np.ascontiguousarray(src, np.int32)
    dst = np.ascontiguousarray(dst, np.int32)
    ins = np.ascontiguousarray(is_insert, np.uint8)
    t = ctypes.c_uint64()
    st = _load().katz_submit_update_batch(h, _ptr(src), _ptr(dst), _ptr(ins), len(src), ctypes.byref(t))
    if st != 0:
        raise KatzError(st, "katz_submit_update_batch")
    return t.value


def katz_poll(h, ticket: int) -> katz_info | None:
    """None while the batch is queued or running; else its katz_info, with
    the batch's own outcome in .status."""
    info = katz_info()
    st = _load().katz_poll(h, int(ticket), ctypes.byref(info))
    if st == 8:  # KATZ_EBUSY
        return None
    if st == 9:  # KATZ_ESTATE: unknown or collected ticket
        raise KatzError(st, "katz_poll")
    info.status = st
    return info


def katz_convert_f64_f32(x):
    """The FP32-certified levels' rounding of the non-negative float64 device
    tensor x to float32 and the exact widening back (katz_convert_f64_f32)."""
    import torch
    assert x.is_cuda and x.dtype == torch.float64 and x.is_contiguous()
    out = torch.empty(x.shape, dtype=torch.float32, device=x.device)
    back = torch.empty(x.shape, dtype=torch.float64, device=x.device)
    st = _load().katz_convert_f64_f32(x.data_ptr(), x.numel(), out.data_ptr(), back.data_ptr())
    if st != 0:
        raise KatzError(st, "katz_convert_f64_f32")
    return out, back


def _require_device_tensor(name, t, dtype_name, min_numel, exact=False):
    """The library's kernels read and write this buffer directly: it must be a
    contiguous CUDA tensor of the given dtype on the current device, with at
    least (or, exact, exactly) min_numel elements."""
    if not (hasattr(t, "is_cuda") and hasattr(t, "dtype")) or not t.is_cuda:
        raise ValueError(f"{name}: expected a CUDA tensor")
    import torch

    if t.dtype != getattr(torch, dtype_name):
        raise ValueError(f"{name}: expected dtype {dtype_name}, got {t.dtype}")
    if t.device.index != torch.cuda.current_device():
        raise ValueError(f"{name}: on cuda:{t.device.index}, the current device is cuda:{torch.cuda.current_device()}")
    if not t.is_contiguous():
        raise ValueError(f"{name}: tensor must be contiguous")
    if (t.numel() != min_numel) if exact else (t.numel() < min_numel):
        raise ValueError(f"{name}: {t.numel()} elements, {'expected' if exact else 'need at least'} {min_numel}")


def katz_certify_topk_noalloc(lower, upper, k: int, eps: float, ids_out, certified_out, stream=None) -> None:
    """Top-k ids and the separation verdict from device bounds, with no
    allocation by the library; lower/upper (float64, n each), ids_out (int32,
    >= k) and certified_out (int32, >= 1) are CUDA tensors on the current
    device that the caller owns; stream: a torch.cuda.Stream or raw handle.
    Anything else raises ValueError before the library is called."""
    _require_device_tensor("lower", lower, "float64", 1)
    n = lower.numel()
    _require_device_tensor("upper", upper, "float64", n, exact=True)
    _require_device_tensor("ids_out", ids_out, "int32", max(int(k), 1))
    _require_device_tensor("certified_out", certified_out, "int32", 1)
    handle = getattr(stream, "cuda_stream", stream)
    st = _load().katz_certify_topk_noalloc(_ptr(lower), _ptr(upper), int(n), int(k), float(eps), _ptr(ids_out),
                                           _ptr(certified_out), handle)
    _check(None, st, "katz_certify_topk_noalloc")


def katz_server_default_opts(**kw) -> katz_server_opts:
    o = katz_server_opts()
    _load().katz_server_default_opts(ctypes.byref(o))
    for k, v in kw.items():
        if not hasattr(o, k):
            raise AttributeError(k)
        setattr(o, k, v)
    return o


class Server:
    """Owning wrapper around a katz_server (destroyed with the object)."""

    def __init__(self, opts: katz_server_opts | None = None, **kw):
        if opts is None:
            opts = katz_server_default_opts(**kw)
        self.opts = opts
        h = ctypes.c_void_p()
        st = _load().katz_server_create(ctypes.byref(h), ctypes.byref(opts))
        if st != 0:
            raise KatzError(st, "katz_server_create")
        self.s = h.value
        self.k = {}

    def attach(self, katz, k: int) -> None:
        hh = katz.h if isinstance(katz, Katz) else katz
        _check(hh, _load().katz_server_attach(self.s, hh, int(k)), "katz_server_attach")
        self.k[hh] = int(k)

    def submit(self, katz, src, dst, is_insert) -> int:
        hh = katz.h if isinstance(katz, Katz) else katz
        src = np.ascontiguousarray(src, np.int32)
        dst = np.ascontiguousarray(dst, np.int32)
        ins = np.ascontiguousarray(is_insert, np.uint8)
        t = ctypes.c_uint64()
        st = _load().katz_server_submit(self.s, hh, _ptr(src), _ptr(dst), _ptr(ins), len(src), ctypes.byref(t))
        if st != 0:
            raise KatzError(st, "katz_server_submit")
        return t.value

    def wait(self, ticket: int, timeout_ms: int = 60000):
        """(status, ids, result) of a finished request; raises KatzError
        (KATZ_ETIMEOUT) if it does not finish in time."""
        ids = np.empty(KATZ_MAX_K, np.int32)
        res = katz_request_result()
        st = _load().katz_server_wait(self.s, int(ticket), int(timeout_ms), _ptr(ids), ctypes.byref(res))
        if st != 0:
            raise KatzError(st, "katz_server_wait")
        return res.status, ids[: res.k].copy(), res

    def close(self):
        if getattr(self, "s", None):
            _load().katz_server_destroy(self.s)
            self.s = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Katz:
    """Owning wrapper around a handle (destroyed with the object)."""

    @classmethod
    def restore(cls, image, opts: katz_opts | None = None) -> "Katz":
        """A handle from a checkpoint image (katz_restore)."""
        obj = cls.__new__(cls)
        obj.h = katz_restore(image, opts)
        # n follows the image header's magic, version, layout word and options
        off = 16 + ctypes.sizeof(katz_opts)
        obj.n = int(np.frombuffer(np.ascontiguousarray(image[off:off + 8], np.uint8).tobytes(), np.int64)[0])
        return obj

    def checkpoint(self) -> np.ndarray:
        return katz_checkpoint(self.h)

    def __init__(self, rowptr, col, opts: katz_opts | None = None):
        rowptr_np = rowptr
        n = (rowptr.shape[0] if hasattr(rowptr, "shape") else len(rowptr)) - 1
        nnz = col.shape[0] if hasattr(col, "shape") else len(col)
        self.n = int(n)
        self.h = katz_create_csr(self.n, int(nnz), rowptr_np, col, opts)

    def close(self):
        if self.h:
            katz_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def rank(self, alpha=0.0, k=100, eps=1e-9, check=True) -> katz_info:
        return katz_rank_static(self.h, alpha, k, eps, check)

    def rank_by(self, criterion, alpha=0.0, eps=1e-9, k=0, pair=None, check=True) -> katz_info:
        return katz_rank(self.h, alpha, criterion, eps, k, pair, check)

    def ranking(self, k):
        return katz_get_ranking(self.h, k)

    def bounds(self):
        return katz_get_bounds(self.h, self.n)

    def walk(self, i):
        return katz_get_walk(self.h, i, self.n)

    def trace(self, cap=1024):
        return katz_get_trace(self.h, cap)

    def update(self, src, dst, is_insert, check=True) -> katz_info:
        return katz_apply_update_batch(self.h, src, dst, is_insert, check=check)

    def submit(self, src, dst, is_insert) -> int:
        return katz_submit_update_batch(self.h, src, dst, is_insert)

    def poll(self, ticket: int) -> katz_info | None:
        return katz_poll(self.h, ticket)


_load()
