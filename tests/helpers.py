"""Small test utilities shared by the CPU and GPU tests (no method arithmetic)."""
import hashlib

import numpy as np


def edge_hash(edges: np.ndarray) -> str:
    """sha256 of a canonical edge list (int32 pairs a<b, lexicographic), little endian."""
    e = np.ascontiguousarray(edges, dtype="<i4")
    return hashlib.sha256(memoryview(e).cast("B")).hexdigest()


def graph_hash(row_ptr: np.ndarray, col: np.ndarray) -> str:
    """sha256 of a CSR: row_ptr as int64 then col as int32, little endian."""
    h = hashlib.sha256()
    h.update(memoryview(np.ascontiguousarray(row_ptr, dtype="<i8")).cast("B"))
    h.update(memoryview(np.ascontiguousarray(col, dtype="<i4")).cast("B"))
    return h.hexdigest()


def csr_from_edges(edges: np.ndarray, n: int):
    """Symmetric CSR (rows ascending) from a canonical edge list."""
    e = np.asarray(edges, dtype=np.int64)
    src = np.concatenate([e[:, 0], e[:, 1]])
    dst = np.concatenate([e[:, 1], e[:, 0]])
    order = np.lexsort((dst, src))
    src, dst = src[order], dst[order]
    rp = np.zeros(n + 1, dtype=np.int64)
    np.add.at(rp, src + 1, 1)
    return np.cumsum(rp), dst.astype(np.int32)


def canonical_from_csr(row_ptr, col) -> np.ndarray:
    n = len(row_ptr) - 1
    src = np.repeat(np.arange(n, dtype=np.int64), np.diff(row_ptr))
    dst = np.asarray(col, dtype=np.int64)
    keep = src < dst
    pairs = np.stack([src[keep], dst[keep]], axis=1)
    order = np.lexsort((pairs[:, 1], pairs[:, 0]))
    return pairs[order].astype(np.int32)


def check_simple_canonical(edges: np.ndarray, n: int):
    e = np.asarray(edges, dtype=np.int64)
    assert (e[:, 0] < e[:, 1]).all(), "not canonical / self loop"
    assert (e >= 0).all() and (e < n).all()
    key = e[:, 0] * n + e[:, 1]
    assert (np.diff(key) > 0).all(), "not sorted or multi-edge"


def degrees(edges: np.ndarray, n: int) -> np.ndarray:
    return np.bincount(np.asarray(edges).ravel(), minlength=n)
