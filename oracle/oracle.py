"""ctypes wrapper around the sequential C oracle (oracle/cb_oracle.c).

Test infrastructure: see the package docstring for who may use it.
"""
import ctypes as C

import numpy as np

from .build import build_oracle

_lib = None


def _load():
    global _lib
    if _lib is None:
        lib = C.CDLL(str(build_oracle()))
        vp, i64, u64, u32, ip = C.c_void_p, C.c_int64, C.c_uint64, C.c_uint32, C.POINTER(C.c_int)
        lib.or_create.restype = vp
        lib.or_create.argtypes = [i64, vp, vp, u64, u64, ip]
        lib.or_destroy.argtypes = [vp]
        lib.or_superstep.restype = C.c_int
        lib.or_superstep.argtypes = [vp, u32]
        lib.or_step.restype = u64
        lib.or_step.argtypes = [vp]
        lib.or_num_edges.restype = i64
        lib.or_num_edges.argtypes = [vp]
        lib.or_num_nodes.restype = i64
        lib.or_num_nodes.argtypes = [vp]
        lib.or_export.restype = i64
        lib.or_export.argtypes = [vp, vp, i64]
        lib.or_trade_explicit.restype = C.c_int
        lib.or_trade_explicit.argtypes = [vp, i64, i64, vp, i64]
        lib.or_disjoint.restype = i64
        lib.or_disjoint.argtypes = [vp, i64, i64, vp, i64, C.POINTER(C.c_int64)]
        lib.or_permutation.restype = C.c_int
        lib.or_permutation.argtypes = [vp, u64, vp]
        lib.or_clone.restype = vp
        lib.or_clone.argtypes = [vp, ip]
        lib.or_philox4x32_10.argtypes = [vp, u64, vp]
        lib.or_set_relaxed.argtypes = [vp, C.c_int]
        lib.or_uniform_pair.argtypes = [u64, i64, u64, C.POINTER(C.c_int64), C.POINTER(C.c_int64)]
        lib.or_uniform_trades.restype = C.c_int
        lib.or_uniform_trades.argtypes = [vp, u64]
        lib.or_uniform_next.restype = u64
        lib.or_uniform_next.argtypes = [vp]
        lib.or_set_uniform_next.argtypes = [vp, u64]
        lib.or_swap_counts.argtypes = [vp, C.POINTER(i64), C.POINTER(i64), C.c_int]
        lib.or_successors.restype = C.c_int
        lib.or_successors.argtypes = [i64, vp, i64, vp, vp]
        lib.or_lcg_params.argtypes = [vp, u64, C.POINTER(C.c_uint64), C.POINTER(C.c_uint64), C.POINTER(C.c_uint64)]
        _lib = lib
    return _lib


def philox4x32_10(ctr, seed: int) -> np.ndarray:
    """Philox4x32-10 of a 4-word counter under a 64-bit seed (the oracle's copy)."""
    lib = _load()
    c = np.ascontiguousarray(np.asarray(ctr, dtype=np.uint32).reshape(4))
    out = np.zeros(4, dtype=np.uint32)
    lib.or_philox4x32_10(c.ctypes.data, C.c_uint64(seed & (2**64 - 1)), out.ctypes.data)
    return out


def uniform_pair(seed: int, n: int, i: int):
    """Node pair (u, v) of uniform trade i on n >= 2 nodes (the oracle's draw)."""
    u, v = C.c_int64(0), C.c_int64(0)
    _load().or_uniform_pair(C.c_uint64(seed & (2**64 - 1)), n, C.c_uint64(i), C.byref(u), C.byref(v))
    return u.value, v.value


def successors(n: int, pairs):
    """Successor lists of a trade sequence (Section 4.1): (begin, suc) with
    node x's increasing trade indices in suc[begin[x]:begin[x+1]]."""
    p = np.ascontiguousarray(np.asarray(pairs, dtype=np.int32).reshape(-1, 2))
    begin = np.zeros(n + 1, dtype=np.int64)
    suc = np.zeros(max(2 * len(p), 1), dtype=np.int32)
    rc = _load().or_successors(n, p.ctypes.data, len(p), begin.ctypes.data, suc.ctypes.data)
    if rc:
        raise ValueError(f"oracle rejected the trade sequence (code {rc})")
    return begin, suc[:2 * len(p)]


class Oracle:
    """Sequential global Curveball on one simple undirected graph."""

    def __init__(self, row_ptr, col, seed: int, first_step: int = 0, _handle=None):
        lib = _load()
        if _handle is not None:
            self._h = _handle
            return
        self._rp = np.ascontiguousarray(row_ptr, dtype=np.int64)
        self._col = np.ascontiguousarray(col, dtype=np.int32)
        n = len(self._rp) - 1
        rc = C.c_int(0)
        h = lib.or_create(n, self._rp.ctypes.data, self._col.ctypes.data if self._col.size else None,
                          C.c_uint64(seed & (2**64 - 1)), C.c_uint64(first_step), C.byref(rc))
        if not h:
            raise ValueError(f"oracle rejected the graph (code {rc.value})")
        self._h = h
        del self._rp, self._col

    def close(self):
        if getattr(self, "_h", None):
            _load().or_destroy(self._h)
            self._h = None

    def __del__(self):
        self.close()

    @property
    def step(self) -> int:
        return int(_load().or_step(self._h))

    @property
    def m(self) -> int:
        return int(_load().or_num_edges(self._h))

    def superstep(self, count: int = 1):
        rc = _load().or_superstep(self._h, count)
        if rc:
            raise RuntimeError(f"oracle super step failed ({rc})")

    def edges(self) -> np.ndarray:
        """Canonical edge list: int32 (m, 2), a < b, sorted lexicographically."""
        m = self.m
        out = np.zeros((m, 2), dtype=np.int32)
        got = _load().or_export(self._h, out.ctypes.data, m)
        assert got == m
        return out

    def permutation(self, g: int) -> np.ndarray:
        """order[p] = node at position p in super step g."""
        n = self.n
        out = np.zeros(n, dtype=np.int64)
        rc = _load().or_permutation(self._h, g, out.ctypes.data)
        if rc:
            raise RuntimeError(rc)
        return out

    @property
    def n(self) -> int:
        return int(_load().or_num_nodes(self._h))

    def trade_explicit(self, u: int, v: int, sigma) -> None:
        """Trade u and v with sigma(D) given explicitly (node ids)."""
        s = np.ascontiguousarray(sigma, dtype=np.int32)
        rc = _load().or_trade_explicit(self._h, u, v, s.ctypes.data if s.size else None, len(s))
        if rc:
            raise ValueError(f"sigma is not a permutation of D ({rc})")

    def disjoint(self, u: int, v: int):
        """(D ascending by node id, |A_{u-v}|) for the current graph."""
        cap = 1 << 20
        out = np.zeros(cap, dtype=np.int32)
        a = C.c_int64(0)
        nd = _load().or_disjoint(self._h, u, v, out.ctypes.data, cap, C.byref(a))
        if nd < 0:
            raise ValueError(nd)
        return out[:nd].copy(), int(a.value)

    def set_relaxed(self, on: bool = True) -> None:
        """Permutations from linear congruential maps (Def. "Relaxed global trade")."""
        _load().or_set_relaxed(self._h, 1 if on else 0)

    def lcg_params(self, g: int):
        """(p, a, b) of super step g's map h(x) = (a x + b) mod p."""
        p, a, b = C.c_uint64(0), C.c_uint64(0), C.c_uint64(0)
        _load().or_lcg_params(self._h, g, C.byref(p), C.byref(a), C.byref(b))
        return p.value, a.value, b.value

    def uniform_trades(self, count: int = 1, first=None) -> None:
        """Apply the next `count` uniform single trades (Section 3.2); with
        `first`, the sequence continues from trade index `first`."""
        if first is not None:
            _load().or_set_uniform_next(self._h, C.c_uint64(first))
        rc = _load().or_uniform_trades(self._h, C.c_uint64(count))
        if rc:
            raise RuntimeError(f"oracle uniform trades failed (code {rc})")

    def swap_counts(self, reset: bool = False):
        """(performed, possible) neighbourhood swaps since creation or the last
        reset: edge ends that changed node, and deg(u) + deg(v) per trade."""
        a, b = C.c_int64(0), C.c_int64(0)
        _load().or_swap_counts(self._h, C.byref(a), C.byref(b), 1 if reset else 0)
        return a.value, b.value

    @property
    def uniform_next(self) -> int:
        return int(_load().or_uniform_next(self._h))

    def clone(self) -> "Oracle":
        rc = C.c_int(0)
        h = _load().or_clone(self._h, C.byref(rc))
        if not h:
            raise RuntimeError(rc.value)
        return Oracle(None, None, 0, _handle=h)
