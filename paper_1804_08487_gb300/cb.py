"""Thin ctypes binding of ``lib/libcb.so`` (the C ABI in ``include/cb.h``).

Functions keep the C names; they only marshal arguments (numpy arrays are
passed as host memory, CUDA torch tensors as device memory) and turn negative
return codes into :class:`CbError`.  Every step of the super step runs in the
CUDA library; there is no CPU fallback: if the library is missing this module
raises instead of computing anything.
"""
import ctypes as C
import re
from pathlib import Path

import numpy as np

from .build import INCLUDE, LIBDIR

CB_OK = 0
CB_EINVAL = -1
CB_ENOMEM = -2
CB_ECUDA = -3
CB_ECHECK = -5
CB_ESIZE = -6
CB_ERANGE = -7
CB_HOST = 0
CB_DEVICE = 1

LIB_PATH = LIBDIR / "libcb.so"
_lib = None


class CbError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"{msg} (code {code})")
        self.code = code


def declared_functions():
    """Names of the functions declared in include/cb.h."""
    text = (Path(INCLUDE) / "cb.h").read_text()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(cb_[a-z_0-9]+)\s*\(", text)))


def load():
    """Load libcb.so (raises if it has not been built)."""
    global _lib
    if _lib is not None:
        return _lib
    if not LIB_PATH.exists():
        raise RuntimeError(f"{LIB_PATH} is missing: build it with __graft_entry__.build()")
    lib = C.CDLL(str(LIB_PATH))
    vp, i64, u64, u32, i32 = C.c_void_p, C.c_int64, C.c_uint64, C.c_uint32, C.c_int
    lib.cb_create.restype = i32
    lib.cb_create.argtypes = [i64, vp, vp, u64, u64, i32, vp, C.POINTER(vp)]
    lib.cb_global_trades.restype = i32
    lib.cb_global_trades.argtypes = [vp, u32]
    lib.cb_export_edges.restype = i32
    lib.cb_export_edges.argtypes = [vp, vp, i64, C.POINTER(i64), i32]
    lib.cb_destroy.restype = None
    lib.cb_destroy.argtypes = [vp]
    lib.cb_step.restype = i32
    lib.cb_step.argtypes = [vp, C.POINTER(u64)]
    lib.cb_sync.restype = i32
    lib.cb_sync.argtypes = [vp]
    lib.cb_last_error.restype = C.c_char_p
    lib.cb_last_error.argtypes = [vp]
    lib.cb_info.restype = i32
    lib.cb_info.argtypes = [vp, C.POINTER(i64), C.POINTER(i64)]
    lib.cb_permutation.restype = i32
    lib.cb_permutation.argtypes = [vp, u64, vp, i32]
    lib.cb_stats.restype = i32
    lib.cb_stats.argtypes = [vp, C.POINTER(i64), i32]
    lib.cb_permutation_static.restype = i32
    lib.cb_permutation_static.argtypes = [i64, u64, u64, vp, vp]
    lib.cb_timings.restype = i32
    lib.cb_timings.argtypes = [vp, C.POINTER(C.c_double), i32]
    lib.cb_set_option.restype = i32
    lib.cb_set_option.argtypes = [vp, C.c_char_p, i64]
    _lib = lib
    return lib


def _ptr(x):
    """(pointer, mem_kind, keepalive) for a numpy array or a torch tensor."""
    if x is None:
        return None, CB_HOST, None
    if isinstance(x, np.ndarray):
        a = np.ascontiguousarray(x)
        return (a.ctypes.data if a.size else None), CB_HOST, a
    # torch tensor
    if not x.is_contiguous():
        raise ValueError("tensor must be contiguous")
    return x.data_ptr(), (CB_DEVICE if x.is_cuda else CB_HOST), x


def _check(rc: int, h=None):
    if rc < 0:
        msg = load().cb_last_error(h).decode(errors="replace")
        raise CbError(rc, msg)
    return rc


def cb_create(n, row_ptr, col, seed, first_step=0, stream=None):
    """Handle for the graph (row_ptr int64[n+1], col int32[row_ptr[n]])."""
    lib = load()
    if isinstance(row_ptr, np.ndarray):
        row_ptr = np.ascontiguousarray(row_ptr, dtype=np.int64)
        col = np.ascontiguousarray(col, dtype=np.int32)
    rp, kind_rp, keep_rp = _ptr(row_ptr)
    cp, kind_c, keep_c = _ptr(col)
    if cp is not None and kind_rp != kind_c:
        raise ValueError("row_ptr and col must live in the same memory")
    h = C.c_void_p()
    s = None if stream is None else C.c_void_p(stream if isinstance(stream, int) else stream.cuda_stream)
    _check(lib.cb_create(n, rp, cp, C.c_uint64(seed & (2**64 - 1)), C.c_uint64(first_step), kind_rp, s,
                         C.byref(h)))
    return h


def cb_global_trades(h, supersteps: int):
    return _check(load().cb_global_trades(h, supersteps), h)


def cb_export_edges(h, out=None):
    """Canonical edge list: numpy int32 (m, 2) on the host, or into `out`
    (an int32 CUDA tensor with at least 2m entries)."""
    lib = load()
    m = C.c_int64(0)
    _check(lib.cb_export_edges(h, None, 0, C.byref(m), CB_HOST), h)
    if out is None:
        arr = np.zeros((m.value, 2), dtype=np.int32)
        if m.value:
            _check(lib.cb_export_edges(h, arr.ctypes.data, m.value, C.byref(m), CB_HOST), h)
        return arr
    p, kind, _ = _ptr(out)
    _check(lib.cb_export_edges(h, p, out.numel() // 2, C.byref(m), kind), h)
    return out


def cb_destroy(h):
    load().cb_destroy(h)


def cb_step(h) -> int:
    g = C.c_uint64(0)
    _check(load().cb_step(h, C.byref(g)), h)
    return g.value


def cb_sync(h):
    return _check(load().cb_sync(h), h)


def cb_last_error(h=None) -> str:
    return load().cb_last_error(h).decode(errors="replace")


def cb_info(h):
    n, m = C.c_int64(0), C.c_int64(0)
    _check(load().cb_info(h, C.byref(n), C.byref(m)), h)
    return n.value, m.value


def cb_permutation(h, g: int):
    n, _ = cb_info(h)
    out = np.zeros(n, dtype=np.int32)
    if n:
        _check(load().cb_permutation(h, g, out.ctypes.data, CB_HOST), h)
    return out


def cb_permutation_static(n: int, seed: int, g: int, order_out, stream=None):
    """Permutation of super step g into `order_out` (an int32 CUDA tensor of n
    entries) without any allocation; runs on `stream` (None: default stream)."""
    p, kind, _ = _ptr(order_out)
    if kind != CB_DEVICE:
        raise ValueError("order_out must be device memory")
    s = None if stream is None else C.c_void_p(stream if isinstance(stream, int) else stream.cuda_stream)
    return _check(load().cb_permutation_static(n, C.c_uint64(seed & (2**64 - 1)), C.c_uint64(g), p, s))


def cb_stats(h):
    out = (C.c_int64 * 8)()
    k = _check(load().cb_stats(h, out, 8), h)
    names = ["passes", "deferred", "tile_trades", "block_trades", "global_ws_trades", "launches"]
    return {names[i]: out[i] for i in range(k)}


def cb_timings(h):
    out = (C.c_double * 4)()
    k = _check(load().cb_timings(h, out, 4), h)
    names = ["permutation_ms", "threshold_ms", "rebuild_ms", "step_ms"]
    return {names[i]: out[i] for i in range(k)}


def cb_set_option(h, key: str, value: int):
    return _check(load().cb_set_option(h, key.encode(), value), h)


class Curveball:
    """Owning wrapper around a cb handle."""

    def __init__(self, row_ptr, col, seed, first_step=0, stream=None):
        n = len(row_ptr) - 1
        self.h = cb_create(n, row_ptr, col, seed, first_step, stream)

    def global_trades(self, supersteps: int = 1):
        cb_global_trades(self.h, supersteps)

    def edges(self, out=None):
        return cb_export_edges(self.h, out)

    @property
    def step(self) -> int:
        return cb_step(self.h)

    def permutation(self, g: int):
        return cb_permutation(self.h, g)

    def stats(self):
        return cb_stats(self.h)

    def timings(self):
        return cb_timings(self.h)

    def set_option(self, key, value):
        cb_set_option(self.h, key, value)

    def sync(self):
        cb_sync(self.h)

    def close(self):
        if getattr(self, "h", None):
            cb_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
