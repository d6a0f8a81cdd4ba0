"""Thin ctypes binding of ``lib/libcb.so`` (the C ABI in ``include/cb.h``).

Functions keep the C names; they only marshal arguments (numpy arrays are
passed as host memory, CUDA torch tensors as device memory) and turn negative
return codes into :class:`CbError`.  Every step of the super step runs in the
CUDA library; there is no CPU fallback: if the library is missing this module
raises instead of computing anything.
"""
import ctypes as C
import os
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
CB_ETIMEOUT = -8
CB_EIO = -9
CB_HOST = 0
CB_DEVICE = 1

LIB_PATH = LIBDIR / "libcb.so"
_lib = None


class CbError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"{msg} (code {code})")
        self.code = code


def declared_functions():
    """Names of the functions declared in include/*.h."""
    names = set()
    for hdr in sorted(Path(INCLUDE).glob("*.h")):
        text = re.sub(r"/\*.*?\*/", "", hdr.read_text(), flags=re.S)
        names |= set(re.findall(r"\b(cb_[a-z_0-9]+)\s*\(", text))
    return sorted(names)


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
    lib.cb_create_batch.restype = i32
    lib.cb_create_batch.argtypes = [i32, vp, vp, vp, vp, u64, i32, vp, C.POINTER(vp)]
    lib.cb_graph_count.restype = i32
    lib.cb_graph_count.argtypes = [vp]
    lib.cb_graph_info.restype = i32
    lib.cb_graph_info.argtypes = [vp, i32, C.POINTER(i64), C.POINTER(i64)]
    lib.cb_export_graph.restype = i32
    lib.cb_export_graph.argtypes = [vp, i32, vp, i64, C.POINTER(i64), i32]
    lib.cb_autotune.restype = i32
    lib.cb_autotune.argtypes = [vp, u32, C.POINTER(i64), i32]
    for f in ("cb_autotune_cached", "cb_tune_key", "cb_tune_cache_lookup", "cb_tune_cache_store"):
        getattr(lib, f).restype = i32
    lib.cb_autotune_cached.argtypes = [vp, u32, C.c_char_p, C.POINTER(i64), i32]
    lib.cb_tune_key.argtypes = [vp, C.c_char_p, i32]
    lib.cb_tune_cache_lookup.argtypes = [C.c_char_p, C.c_char_p, C.POINTER(i64), i32]
    lib.cb_tune_cache_store.argtypes = [C.c_char_p, C.c_char_p, C.POINTER(i64), i32]
    lib.cb_device_bytes.restype = i32
    lib.cb_device_bytes.argtypes = [vp, C.POINTER(i64), C.POINTER(i64)]
    lib.cb_estimate_bytes.restype = i64
    lib.cb_estimate_bytes.argtypes = [i64, i64, i64]
    lib.cb_server_create.restype = i32
    lib.cb_server_create.argtypes = [i64, i32, i32, C.POINTER(vp)]
    lib.cb_server_submit.restype = i32
    lib.cb_server_submit.argtypes = [vp, i64, vp, vp, u64, u32, C.POINTER(i64)]
    lib.cb_server_poll.restype = i32
    lib.cb_server_poll.argtypes = [vp, C.POINTER(i64), i32, i32]
    lib.cb_server_result.restype = i32
    lib.cb_server_result.argtypes = [vp, i64, vp, i64, C.POINTER(i64), C.POINTER(C.c_double)]
    lib.cb_server_stats.restype = i32
    lib.cb_server_stats.argtypes = [vp, C.POINTER(i64), i32]
    lib.cb_server_destroy.restype = None
    lib.cb_server_destroy.argtypes = [vp]
    lib.cb_swap_counts.restype = i32
    lib.cb_swap_counts.argtypes = [vp, C.POINTER(i64), C.POINTER(i64)]
    lib.cb_uniform_trades.restype = i32
    lib.cb_uniform_trades.argtypes = [vp, u64]
    lib.cb_uniform_next.restype = i32
    lib.cb_uniform_next.argtypes = [vp, C.POINTER(u64)]
    lib.cb_uniform_pairs.restype = i32
    lib.cb_uniform_pairs.argtypes = [u64, i64, u64, i64, vp, vp]
    lib.cb_generate_pld.restype = i32
    lib.cb_generate_pld.argtypes = [i64, i32, i32, C.c_double, u64, vp, C.POINTER(i64), vp]
    lib.cb_generate_hh.restype = i32
    lib.cb_generate_hh.argtypes = [i64, vp, vp, vp, C.POINTER(i64), vp]
    lib.cb_autocorr.restype = i32
    lib.cb_autocorr.argtypes = [vp, i32, i32, C.POINTER(i64), C.POINTER(i64), C.POINTER(i64), C.POINTER(i64)]
    lib.cb_successors.restype = i32
    lib.cb_successors.argtypes = [i64, vp, i64, vp, vp, vp]
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


def _numel(x) -> int:
    """Element count of a numpy array or a torch tensor."""
    return int(x.size) if isinstance(x, np.ndarray) else int(x.numel())


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


def cb_create_batch(ns, row_ptr, col, seeds, first_step=0, stream=None):
    """Handle for an ensemble: ns[i] nodes per graph, row_ptr = every graph's
    n_i+1 offsets one after another, col = every graph's entries (local ids)
    one after another, seeds[i] per graph."""
    lib = load()
    ns = np.ascontiguousarray(ns, dtype=np.int64)
    seeds = np.ascontiguousarray(np.asarray(seeds, dtype=np.uint64))
    if isinstance(row_ptr, np.ndarray):
        row_ptr = np.ascontiguousarray(row_ptr, dtype=np.int64)
        col = np.ascontiguousarray(col, dtype=np.int32)
    rp, kind_rp, keep_rp = _ptr(row_ptr)
    cp, kind_c, keep_c = _ptr(col)
    if cp is not None and kind_rp != kind_c:
        raise ValueError("row_ptr and col must live in the same memory")
    h = C.c_void_p()
    s = None if stream is None else C.c_void_p(stream if isinstance(stream, int) else stream.cuda_stream)
    _check(lib.cb_create_batch(len(ns), ns.ctypes.data, rp, cp, seeds.ctypes.data, C.c_uint64(first_step),
                               kind_rp, s, C.byref(h)))
    return h


def cb_graph_count(h) -> int:
    return _check(load().cb_graph_count(h), h)


def cb_graph_info(h, index: int):
    n, m = C.c_int64(0), C.c_int64(0)
    _check(load().cb_graph_info(h, index, C.byref(n), C.byref(m)), h)
    return n.value, m.value


def cb_export_graph(h, index: int, out=None):
    """Canonical edge list of graph `index` (local ids), as cb_export_edges."""
    lib = load()
    m = C.c_int64(0)
    _check(lib.cb_export_graph(h, index, None, 0, C.byref(m), CB_HOST), h)
    if out is None:
        arr = np.zeros((m.value, 2), dtype=np.int32)
        if m.value:
            _check(lib.cb_export_graph(h, index, arr.ctypes.data, m.value, C.byref(m), CB_HOST), h)
        return arr
    p, kind, _ = _ptr(out)
    _check(lib.cb_export_graph(h, index, p, _numel(out) // 2, C.byref(m), kind), h)
    return out


def cb_autotune(h, max_steps: int):
    out = (C.c_int64 * 6)()
    k = _check(load().cb_autotune(h, max_steps, out, 6), h)
    names = ["tile_max", "block_max", "smem_max", "inorder_threads", "steps", "retry_passes"]
    return {names[i]: out[i] for i in range(k)}


_TUNE_NAMES = ["tile_max", "block_max", "smem_max", "inorder_threads", "retry_passes"]


def cb_autotune_cached(h, max_steps: int, cache_path: str):
    out = (C.c_int64 * 6)()
    k = _check(load().cb_autotune_cached(h, max_steps, os.fsencode(cache_path), out, 6), h)
    names = ["tile_max", "block_max", "smem_max", "inorder_threads", "steps", "retry_passes"]
    return {names[i]: out[i] for i in range(k)}


def cb_tune_key(h) -> str:
    buf = C.create_string_buffer(512)
    _check(load().cb_tune_key(h, buf, len(buf)), h)
    return buf.value.decode()


def cb_tune_cache_lookup(path: str, key: str):
    """The settings stored under key (a dict), or None."""
    out = (C.c_int64 * 5)()
    k = _check(load().cb_tune_cache_lookup(os.fsencode(path), key.encode(), out, 5))
    return {_TUNE_NAMES[i]: out[i] for i in range(k)} if k else None


def cb_tune_cache_store(path: str, key: str, settings: dict):
    vals = (C.c_int64 * 5)(*[int(settings[nm]) for nm in _TUNE_NAMES])
    return _check(load().cb_tune_cache_store(os.fsencode(path), key.encode(), vals, 5))


def cb_global_trades(h, supersteps: int):
    return _check(load().cb_global_trades(h, supersteps), h)


def cb_export_edges(h, out=None):
    """Canonical edge list: numpy int32 (m, 2) on the host, or into `out`
    (a numpy array or a torch tensor, int32, with at least 2m entries)."""
    lib = load()
    m = C.c_int64(0)
    _check(lib.cb_export_edges(h, None, 0, C.byref(m), CB_HOST), h)
    if out is None:
        arr = np.zeros((m.value, 2), dtype=np.int32)
        if m.value:
            _check(lib.cb_export_edges(h, arr.ctypes.data, m.value, C.byref(m), CB_HOST), h)
        return arr
    p, kind, _ = _ptr(out)
    _check(lib.cb_export_edges(h, p, _numel(out) // 2, C.byref(m), kind), h)
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


def _stream(stream):
    return None if stream is None else C.c_void_p(stream if isinstance(stream, int) else stream.cuda_stream)


def cb_swap_counts(h):
    """(performed, possible) neighbourhood swaps since "swap_stats" was set."""
    a, b = C.c_int64(0), C.c_int64(0)
    _check(load().cb_swap_counts(h, C.byref(a), C.byref(b)), h)
    return a.value, b.value


def cb_uniform_trades(h, count: int):
    """Apply the handle's next `count` uniform single trades (Section 3.2)."""
    return _check(load().cb_uniform_trades(h, C.c_uint64(count)), h)


def cb_uniform_next(h) -> int:
    v = C.c_uint64(0)
    _check(load().cb_uniform_next(h, C.byref(v)), h)
    return v.value


def cb_uniform_pairs(seed: int, n: int, first: int, count: int, pairs_out, stream=None):
    """Node pairs of uniform trades first..first+count-1 into `pairs_out` (an
    int32 CUDA tensor of 2*count entries)."""
    p, kind, _ = _ptr(pairs_out)
    if kind != CB_DEVICE:
        raise ValueError("pairs_out must be device memory")
    return _check(load().cb_uniform_pairs(C.c_uint64(seed & (2**64 - 1)), n, C.c_uint64(first), count, p,
                                          _stream(stream)))


def cb_successors(n: int, pairs, suc_begin_out, suc_out, stream=None):
    """Successor lists (Section 4.1) of the trade sequence in `pairs` (int32
    CUDA tensor, 2 per trade) into suc_begin_out (int64, n+1) and suc_out
    (int32, 2 per trade), all device memory."""
    pp, k1, _ = _ptr(pairs)
    pb, k2, _ = _ptr(suc_begin_out)
    ps, k3, _ = _ptr(suc_out)
    if CB_HOST in (k2,) or (pp is not None and k1 != CB_DEVICE) or (ps is not None and k3 != CB_DEVICE):
        raise ValueError("cb_successors takes device memory")
    count = pairs.numel() // 2
    return _check(load().cb_successors(n, pp, count, pb, ps, _stream(stream)))


def cb_generate_pld(n: int, a: int, b: int, gamma: float, seed: int, deg_out, stream=None) -> int:
    """PLD([a,b), gamma) degrees into `deg_out` (an int32 CUDA tensor of n
    entries); returns their sum."""
    p, kind, _ = _ptr(deg_out)
    if n and kind != CB_DEVICE:
        raise ValueError("deg_out must be device memory")
    total = C.c_int64(0)
    _check(load().cb_generate_pld(n, a, b, float(gamma), C.c_uint64(seed & (2**64 - 1)), p, C.byref(total),
                                  _stream(stream)))
    return total.value


def cb_generate_hh(n: int, deg, row_ptr_out, col_out, stream=None) -> int:
    """Havel-Hakimi realisation of `deg` (int32 CUDA tensor) into row_ptr_out
    (int64, n+1) and col_out (int32, sum of degrees), CUDA tensors; returns m."""
    ptrs = [_ptr(x) for x in (deg, row_ptr_out, col_out)]
    if n and any(k != CB_DEVICE for p, k, _ in ptrs if p is not None):
        raise ValueError("cb_generate_hh takes device memory")
    m = C.c_int64(0)
    _check(load().cb_generate_hh(n, ptrs[0][0], ptrs[1][0], ptrs[2][0], C.byref(m), _stream(stream)))
    return m.value


def generate_powerlaw(n: int, a: int, b: int, gamma: float, seed: int, max_redraws: int = 64, stream=None):
    """(row_ptr, col, degree_seed) as CUDA tensors: PLD([a,b), gamma) degrees
    realised by Havel-Hakimi on the device, a non-graphical draw redrawn with
    seed+1 (the host generator's policy)."""
    import torch
    deg = torch.empty(max(n, 1), dtype=torch.int32, device="cuda")
    rp = torch.empty(n + 1, dtype=torch.int64, device="cuda")
    for k in range(max_redraws):
        total = cb_generate_pld(n, a, b, gamma, seed + k, deg, stream)
        col = torch.empty(max(total, 1), dtype=torch.int32, device="cuda")
        try:
            cb_generate_hh(n, deg, rp, col, stream)
        except CbError as e:
            if e.code == CB_EINVAL:
                continue
            raise
        return rp, col[:total], seed + k
    raise CbError(CB_EINVAL, f"no graphical draw in {max_redraws} tries")


def cb_autocorr(h, graph: int, kmax: int):
    """Edge autocorrelation of the presence record: (correlated counts for
    k = 1..kmax, near-tie counts, occurring edges, recorded states)."""
    corr = (C.c_int64 * kmax)()
    near = (C.c_int64 * kmax)()
    occ, st = C.c_int64(0), C.c_int64(0)
    _check(load().cb_autocorr(h, graph, kmax, corr, near, C.byref(occ), C.byref(st)), h)
    return list(corr), list(near), occ.value, st.value


TRADE_CLASSES = 9   # size classes of the threshold phase

# cb_stats: out[0..7), then trades and directed entries per size class of the
# first threshold pass
_STAT_NAMES = (["passes", "deferred", "tile_trades", "block_trades", "global_ws_trades", "launches",
                "inorder_trades"] + [f"class{k}_trades" for k in range(TRADE_CLASSES)]
               + [f"class{k}_entries" for k in range(TRADE_CLASSES)])
_TIMING_NAMES = (["permutation_ms", "threshold_ms", "rebuild_ms", "step_ms"]
                 + [f"class{k}_ms" for k in range(TRADE_CLASSES)] + ["retry_ms", "inorder_ms"])


def cb_stats(h):
    out = (C.c_int64 * len(_STAT_NAMES))()
    k = _check(load().cb_stats(h, out, len(_STAT_NAMES)), h)
    return {_STAT_NAMES[i]: out[i] for i in range(k)}


def cb_timings(h):
    out = (C.c_double * len(_TIMING_NAMES))()
    k = _check(load().cb_timings(h, out, len(_TIMING_NAMES)), h)
    return {_TIMING_NAMES[i]: out[i] for i in range(k)}


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

    def autotune(self, max_steps: int, cache_path=None):
        if cache_path is not None:
            return cb_autotune_cached(self.h, max_steps, cache_path)
        return cb_autotune(self.h, max_steps)

    def tune_key(self) -> str:
        return cb_tune_key(self.h)

    def uniform_trades(self, count: int = 1):
        cb_uniform_trades(self.h, count)

    def swap_counts(self):
        return cb_swap_counts(self.h)

    @property
    def uniform_next(self) -> int:
        return cb_uniform_next(self.h)

    def sync(self):
        cb_sync(self.h)

    def autocorr(self, kmax: int, graph: int = -1):
        return cb_autocorr(self.h, graph, kmax)

    def close(self):
        if getattr(self, "h", None):
            cb_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Ensemble(Curveball):
    """Owning wrapper around a handle of many independent graphs.

    `graphs` is a list of (row_ptr int64[n_i+1], col int32[...]) numpy pairs
    and `seeds` one seed per graph; they are passed to the library one after
    another (cb_create_batch)."""

    def __init__(self, graphs, seeds, first_step=0, stream=None):
        ns = [len(rp) - 1 for rp, _ in graphs]
        row_ptr = np.concatenate([np.asarray(rp, dtype=np.int64) for rp, _ in graphs])
        col = np.concatenate([np.asarray(c, dtype=np.int32) for _, c in graphs] + [np.zeros(0, np.int32)])
        self.h = cb_create_batch(ns, row_ptr, col, seeds, first_step, stream)

    def __len__(self):
        return cb_graph_count(self.h)

    def info(self, index: int):
        return cb_graph_info(self.h, index)

    def graph_edges(self, index: int, out=None):
        return cb_export_graph(self.h, index, out)


def cb_device_bytes(h):
    now, peak = C.c_int64(0), C.c_int64(0)
    _check(load().cb_device_bytes(h, C.byref(now), C.byref(peak)), h)
    return now.value, peak.value


def cb_estimate_bytes(n: int, nnz: int, max_degree: int) -> int:
    return _check(load().cb_estimate_bytes(n, nnz, max_degree))


def cb_server_create(hbm_budget_bytes: int, max_active: int = 64, depth: int = 2):
    s = C.c_void_p()
    _check(load().cb_server_create(int(hbm_budget_bytes), max_active, depth, C.byref(s)))
    return s


def cb_server_submit(s, row_ptr, col, seed: int, supersteps: int) -> int:
    rp = np.ascontiguousarray(row_ptr, dtype=np.int64)
    cl = np.ascontiguousarray(col, dtype=np.int32)
    rid = C.c_int64(0)
    _check(load().cb_server_submit(s, len(rp) - 1, rp.ctypes.data, cl.ctypes.data if cl.size else None,
                                   C.c_uint64(seed & (2**64 - 1)), supersteps, C.byref(rid)))
    return rid.value


def cb_server_poll(s, timeout_ms: int = 0, capacity: int = 1024):
    buf = (C.c_int64 * capacity)()
    k = _check(load().cb_server_poll(s, buf, capacity, timeout_ms))
    return [buf[i] for i in range(k)]


def cb_server_result(s, rid: int):
    """(edges int32 (m, 2), times [submitted, admitted, resident, finished]);
    raises CbError if the request failed.  Releases the request."""
    lib = load()
    m = C.c_int64(0)
    t = (C.c_double * 4)()
    _check(lib.cb_server_result(s, rid, None, 0, C.byref(m), t))
    arr = np.zeros((max(m.value, 1), 2), dtype=np.int32)
    _check(lib.cb_server_result(s, rid, arr.ctypes.data, m.value, C.byref(m), t))
    return arr[:m.value], [t[i] for i in range(4)]


def cb_server_stats(s):
    out = (C.c_int64 * 8)()
    k = _check(load().cb_server_stats(s, out, 8))
    names = ["submitted", "queued", "resident", "finished", "reserved_bytes", "reserved_peak_bytes",
             "steps_issued", "failed"]
    return {names[i]: out[i] for i in range(k)}


def cb_server_destroy(s):
    load().cb_server_destroy(s)


class Server:
    """Owning wrapper around the serving loop (include/cb_serve.h)."""

    def __init__(self, hbm_budget_bytes: int, max_active: int = 64, depth: int = 2):
        self.s = cb_server_create(hbm_budget_bytes, max_active, depth)

    def submit(self, row_ptr, col, seed: int, supersteps: int) -> int:
        return cb_server_submit(self.s, row_ptr, col, seed, supersteps)

    def poll(self, timeout_ms: int = 0, capacity: int = 1024):
        return cb_server_poll(self.s, timeout_ms, capacity)

    def result(self, rid: int):
        return cb_server_result(self.s, rid)

    def stats(self):
        return cb_server_stats(self.s)

    def close(self):
        if getattr(self, "s", None):
            cb_server_destroy(self.s)
            self.s = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
