"""Seeded synthetic input graphs: PLD([a,b), gamma) degree sequences (Section 2)
realised as simple graphs by Havel-Hakimi (Section 5.2).

This module holds none of the Curveball method's arithmetic; the CUDA path and
the CPU oracle both take their inputs from it.
"""
import ctypes as C
from dataclasses import dataclass

import numpy as np

from .build import build_synth

_lib = None


def _load():
    global _lib
    if _lib is None:
        lib = C.CDLL(str(build_synth()))
        lib.cb_synth_pld.restype = C.c_int64
        lib.cb_synth_pld.argtypes = [C.c_int64, C.c_int32, C.c_int32, C.c_double, C.c_uint64, C.c_void_p]
        lib.cb_synth_hh.restype = C.c_int64
        lib.cb_synth_hh.argtypes = [C.c_int64, C.c_void_p, C.c_void_p, C.c_void_p]
        lib.cb_synth_uniform.restype = C.c_double
        lib.cb_synth_uniform.argtypes = [C.c_uint64, C.c_uint64, C.c_uint64]
        lib.cb_synth_exp2.restype = C.c_double
        lib.cb_synth_exp2.argtypes = [C.c_double]
        _lib = lib
    return _lib


class NotGraphical(ValueError):
    pass


def uniform(seed: int, stream: int, i: int) -> float:
    """Portable uniform draw in [0,1) (SplitMix64 stream)."""
    return float(_load().cb_synth_uniform(seed & (2**64 - 1), stream, i))


def pld_degrees(n: int, a: int, b: int, gamma: float, seed: int) -> np.ndarray:
    """n i.i.d. degrees from PLD([a,b), gamma); odd sum fixed by +1 on the last."""
    deg = np.zeros(n, dtype=np.int32)
    s = _load().cb_synth_pld(n, a, b, float(gamma), seed & (2**64 - 1), deg.ctypes.data)
    if s < 0:
        raise ValueError("bad PLD arguments")
    return deg


def havel_hakimi(deg: np.ndarray):
    """CSR (row_ptr int64[n+1], col int32[sum deg], rows ascending) or NotGraphical."""
    deg = np.ascontiguousarray(deg, dtype=np.int32)
    n = len(deg)
    total = int(deg.sum(dtype=np.int64))
    row_ptr = np.zeros(n + 1, dtype=np.int64)
    col = np.zeros(max(total, 1), dtype=np.int32)
    m = _load().cb_synth_hh(n, deg.ctypes.data, row_ptr.ctypes.data, col.ctypes.data)
    if m == -1:
        raise NotGraphical("degree sequence is not graphical")
    if m < 0:
        raise RuntimeError(f"havel_hakimi failed ({m})")
    return row_ptr, col[:total]


@dataclass
class Graph:
    row_ptr: np.ndarray
    col: np.ndarray
    degree_seed: int          # seed the degree sequence was finally drawn with

    @property
    def n(self) -> int:
        return len(self.row_ptr) - 1

    @property
    def m(self) -> int:
        return int(self.row_ptr[-1]) // 2


def powerlaw_graph(n: int, a: int, b: int, gamma: float, seed: int, max_redraws: int = 64) -> Graph:
    """PLD degrees realised by Havel-Hakimi; a non-graphical draw is redrawn with seed+1."""
    for k in range(max_redraws):
        deg = pld_degrees(n, a, b, gamma, seed + k)
        try:
            rp, col = havel_hakimi(deg)
            return Graph(rp, col, seed + k)
        except NotGraphical:
            continue
    raise NotGraphical(f"no graphical draw in {max_redraws} tries")


@dataclass(frozen=True)
class Workload:
    """One plain global-Curveball workload: graph recipe, chain seed, super steps."""
    name: str
    n: int
    a: int
    b: int
    gamma: float
    degree_seed: int
    chain_seed: int
    supersteps: int

    def graph(self) -> Graph:
        return powerlaw_graph(self.n, self.a, self.b, self.gamma, self.degree_seed)


# The plain workloads: n=4096 PLD([10,100),2) (degree seed 1, chain seed 42,
# 10 super steps); n=2^20 PLD([10,1000),2) (seed 7, 20 super steps); n=2^25
# PLD([10,10000),2) (seed 3, 10 super steps).  One seed drives degrees and
# chain where a single seed is given.
PLAIN = {
    "n4096": Workload("plain n=4096 PLD([10,100),2)", 4096, 10, 100, 2.0, 1, 42, 10),
    "n2^20": Workload("plain n=2^20 PLD([10,1000),2)", 1 << 20, 10, 1000, 2.0, 7, 7, 20),
    "n2^25": Workload("plain n=2^25 PLD([10,10000),2)", 1 << 25, 10, 10000, 2.0, 3, 3, 10),
    # the n=2^25 degree law at a size whose kernels can be profiled in full
    "n2^21": Workload("plain n=2^21 PLD([10,10000),2)", 1 << 21, 10, 10000, 2.0, 3, 3, 10),
}


SERVING_RATE = 200.0        # mean arrivals per second (Poisson)
SERVING_MASTER_SEED = 2018   # drives the inter-arrival times only


def serving_request(i: int):
    """Request i of the serving workload: n log-uniform in [2^12, 2^22], gamma
    uniform in [2,3], degrees on [4, n/16] (so b = n/16 + 1 exclusive), super
    steps uniform in [5, 50]; the request index seeds the graph and the chain
    (stream 3 draws n, gamma and the step count)."""
    n = int(_load().cb_synth_exp2(12.0 + 10.0 * uniform(i, 3, 0)))
    n = min(max(n, 1 << 12), 1 << 22)
    gamma = 2.0 + uniform(i, 3, 1)
    steps = 5 + min(int(46.0 * uniform(i, 3, 2)), 45)
    return Workload(f"request[{i}]", n, 4, n // 16 + 1, gamma, i, i, steps)


def serving_arrivals(count: int, rate: float = SERVING_RATE, seed: int = SERVING_MASTER_SEED) -> np.ndarray:
    """Arrival times (seconds from the first) of a Poisson process: exponential
    inter-arrival gaps -ln(1-U)/rate from stream 4 of the master seed."""
    gaps = [-np.log1p(-uniform(seed, 4, i)) / rate for i in range(count)]
    t = np.cumsum([0.0] + gaps[1:])
    return np.asarray(t, dtype=np.float64)


def ensemble_member(i: int):
    """Member i of the 256-graph ensemble: n log-uniform in [2^10, 2^16], gamma
    uniform in [2,3], degrees on [4, n/16), seed 1000+i (stream 3 draws n and gamma)."""
    seed = 1000 + i
    n = int(_load().cb_synth_exp2(10.0 + 6.0 * uniform(seed, 3, 0)))
    n = min(max(n, 1 << 10), 1 << 16)
    gamma = 2.0 + uniform(seed, 3, 1)
    return Workload(f"ensemble[{i}]", n, 4, max(n // 16, 5), gamma, seed, seed, 50)
