"""Parity of the device uniform single trades (Simple Undirected Curveball,
Section 3.2) and successor lists (Section 4.1) with the CPU oracle.

Both are integer work on a fixed random stream, so agreement is bit-exact:
the drawn pairs and the Suc lists element by element, the graph after every
call edge for edge.  The device runs the trade sequence as a dataflow over
Suc (Sections 4.1-4.2); the oracle applies the trades one after the other.
"""
import json
import os

import numpy as np
import pytest
import torch

from oracle import Oracle, successors, uniform_pair
from paper_1804_08487_gb300 import synth
from paper_1804_08487_gb300.cb import (CB_EINVAL, CbError, Curveball, Ensemble, cb_successors,
                                       cb_uniform_pairs)
from tests import exact
from tests.helpers import edge_hash

pytestmark = pytest.mark.gpu
GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


@pytest.mark.parametrize("n,first,count", [(2, 0, 100), (7, 5, 1000), (1000, (1 << 32) - 300, 600),
                                           (1 << 20, 12345, 5000), ((1 << 31) - 1, 9, 300)])
def test_pairs_match_oracle(n, first, count):
    out = torch.empty(2 * count, dtype=torch.int32, device="cuda")
    cb_uniform_pairs(77, n, first, count, out)
    torch.cuda.synchronize()
    got = out.cpu().numpy().reshape(-1, 2)
    want = np.array([uniform_pair(77, n, first + k) for k in range(count)], dtype=np.int64)
    assert np.array_equal(got, want)


def test_pairs_need_two_nodes():
    out = torch.empty(8, dtype=torch.int32, device="cuda")
    with pytest.raises(CbError) as e:
        cb_uniform_pairs(1, 1, 0, 4, out)
    assert e.value.code == CB_EINVAL


def _device_successors(n, pairs):
    p = torch.tensor(np.asarray(pairs, dtype=np.int32).reshape(-1), device="cuda")
    begin = torch.empty(n + 1, dtype=torch.int64, device="cuda")
    suc = torch.empty(max(p.numel(), 1), dtype=torch.int32, device="cuda")
    cb_successors(n, p, begin, suc)
    return begin.cpu().numpy(), suc.cpu().numpy()[:p.numel()]


def test_successors_worked_example():
    with open(os.path.join(GOLDEN, "suc_example.json")) as f:
        ex = json.load(f)
    pairs = [(a - 1, b - 1) for a, b in ex["trades"]]
    begin, suc = _device_successors(ex["n"], pairs)
    for x in range(ex["n"]):
        assert [int(i) + 1 for i in suc[begin[x]:begin[x + 1]]] == ex["suc"][str(x + 1)][:-1]


@pytest.mark.parametrize("n,count,seed", [(5000, 20000, 1), (3, 1000, 2), (1 << 16, 1 << 15, 3), (10, 0, 4)])
def test_successors_match_oracle(n, count, seed):
    pairs = np.array([uniform_pair(seed, n, k) for k in range(count)], dtype=np.int32).reshape(-1, 2)
    got_b, got_s = _device_successors(n, pairs)
    want_b, want_s = successors(n, pairs)
    assert np.array_equal(got_b, want_b)
    assert np.array_equal(got_s, want_s)


@pytest.mark.parametrize("pairs", [[(0, 3)], [(1, 1)], [(0, 1), (-1, 2)]])
def test_successors_reject_bad_pairs(pairs):
    with pytest.raises(CbError) as e:
        _device_successors(3, pairs)
    assert e.value.code == CB_EINVAL


def _run_pair(rp, col, seed, calls, steps_between=0, options=None):
    c = Curveball(rp, col, seed)
    for k, v in (options or {}).items():
        c.set_option(k, v)
    o = Oracle(rp, col, seed)
    for i, k in enumerate(calls):
        c.uniform_trades(k)
        o.uniform_trades(k)
        assert c.uniform_next == o.uniform_next
        got, want = c.edges(), o.edges()
        assert np.array_equal(got, want), f"after call {i} ({k} trades)"
        if steps_between:
            c.global_trades(steps_between)
            o.superstep(steps_between)
            assert np.array_equal(c.edges(), o.edges()), f"after the super steps following call {i}"
    return c, o


@pytest.mark.parametrize("n,a,b,gamma,seed,calls", [
    (2000, 3, 200, 2.0, 1, [1, 7, 1000, 4000]),
    (5001, 2, 2500, 2.0, 2, [2500, 2500]),            # hubs: trades above the shared-memory sort size
    (40, 10, 30, 2.0, 3, [20, 500, 3000]),            # dense: many common neighbours
    (300, 20, 200, 2.0, 4, [150, 150]),
    (777, 1, 20, 2.5, 5, [70000]),                    # two chunks of the sequence
])
def test_uniform_trades_match_oracle(n, a, b, gamma, seed, calls):
    g = synth.powerlaw_graph(n, a, b, gamma, seed)
    _run_pair(g.row_ptr, g.col, seed * 7 + 1, calls)


@pytest.mark.parametrize("edges,n", [([], 0), ([], 1), ([(0, 1)], 2), ([(0, 1), (1, 2)], 3), ([], 5),
                                     ([(0, 1), (2, 3)], 4), ([(0, 1), (1, 2), (2, 3), (3, 0), (0, 2)], 4)])
def test_uniform_trades_tiny_graphs(edges, n):
    rp, col = exact.to_csr(frozenset(edges), n)
    _run_pair(rp, col, 11, [1, 5, 200])


def test_uniform_trades_with_hubs_above_the_shared_hash():
    """Two hubs of 14000 and 13000 neighbours in a sparse graph: trades whose
    u has more than 12288 neighbours hash them in global memory, and trades
    above 2048 entries keep them in a per-CTA global slice.  The seed puts a
    hub in u's place in trades 1164, 9949 and 15107."""
    n = 20000
    g = synth.powerlaw_graph(n, 2, 20, 2.0, 61)
    rows = np.repeat(np.arange(n, dtype=np.int64), np.diff(g.row_ptr))
    edges = {(int(a), int(b)) for a, b in zip(rows, g.col) if a < b}
    edges |= {(0, x) for x in range(2, 14002)} | {(1, x) for x in range(5000, 18000)}
    rp, col = exact.to_csr(frozenset(edges), n)
    assert np.diff(rp)[0] > 12288 and np.diff(rp)[1] > 12288
    hub_u = [k for k in range(n) if uniform_pair(1, n, k)[0] in (0, 1)]
    assert hub_u[:3] == [1164, 9949, 15107]
    _run_pair(rp, col, 1, [n // 2, n // 2])


@pytest.mark.parametrize("threads", [256, 512])
def test_uniform_trades_on_other_executor_ctas(threads):
    """The executor with 256 or 512 threads per CTA (1024 by default): the same sequence,
    hubs above every shared-memory size included."""
    g = synth.powerlaw_graph(5001, 2, 2500, 2.0, 2)
    _run_pair(g.row_ptr, g.col, 15, [2500, 2500], options={"uniform_threads": threads})
    g = synth.powerlaw_graph(40, 10, 30, 2.0, 3)
    _run_pair(g.row_ptr, g.col, 22, [20, 500, 3000], options={"uniform_threads": threads})


def test_uniform_and_global_steps_alternate():
    g = synth.powerlaw_graph(3000, 3, 300, 2.0, 8)
    _run_pair(g.row_ptr, g.col, 21, [500, 1500, 1], steps_between=2)
    # with the super step recorded as a CUDA graph, which the uniform trades invalidate
    _run_pair(g.row_ptr, g.col, 22, [700, 800], steps_between=1, options={"cuda_graph": 1})


def test_uniform_trades_in_relaxed_mode():
    g = synth.powerlaw_graph(2500, 3, 250, 2.0, 9)
    c = Curveball(g.row_ptr, g.col, 31)
    o = Oracle(g.row_ptr, g.col, 31)
    c.set_option("relaxed", 1)
    o.set_relaxed(True)
    for _ in range(2):
        c.global_trades(1)
        o.superstep(1)
        c.uniform_trades(1250)
        o.uniform_trades(1250)
        assert np.array_equal(c.edges(), o.edges())


def test_uniform_trades_refuse_batches():
    g1 = exact.to_csr(frozenset({(0, 1)}), 3)
    g2 = exact.to_csr(frozenset({(0, 1), (1, 2)}), 3)
    ens = Ensemble([g1, g2], [1, 2])
    with pytest.raises(CbError) as e:
        ens.uniform_trades(5)
    assert e.value.code == CB_EINVAL


def test_plain_n2p20_half_n_uniform_trades():
    """The n=2^20 workload graph, n/2 uniform trades (as many trades as one
    global trade), against the oracle run live."""
    w = synth.PLAIN["n2^20"]
    g = w.graph()
    c = Curveball(g.row_ptr, g.col, w.chain_seed)
    o = Oracle(g.row_ptr, g.col, w.chain_seed)
    c.uniform_trades(g.n // 2)
    o.uniform_trades(g.n // 2)
    got = c.edges()
    assert edge_hash(got) == edge_hash(o.edges())
    assert not np.array_equal(got, np.asarray(exact_edges(g)))


def exact_edges(g):
    rows = np.repeat(np.arange(g.n, dtype=np.int64), np.diff(g.row_ptr))
    keep = rows < g.col
    return np.stack([rows[keep], g.col[keep]], axis=1)


@pytest.mark.parametrize("n,a,b,seed", [(3001, 3, 300, 41), (2000, 10, 11, 42), (5001, 2, 2500, 43)])
def test_swap_counts_match_oracle(n, a, b, seed):
    """Swap counts (Appendix "Swaps performed by Curveball and Global
    Curveball") of global super steps and of uniform trades equal the
    oracle's exactly."""
    g = synth.powerlaw_graph(n, a, b, 2.0, seed)
    c = Curveball(g.row_ptr, g.col, seed)
    o = Oracle(g.row_ptr, g.col, seed)
    c.global_trades(1)
    o.superstep(1)
    c.set_option("swap_stats", 1)
    o.swap_counts(reset=True)
    c.global_trades(2)
    o.superstep(2)
    assert c.swap_counts() == o.swap_counts()
    c.uniform_trades(n)
    o.uniform_trades(n)
    assert c.swap_counts() == o.swap_counts()
    assert np.array_equal(c.edges(), o.edges())
    c.set_option("swap_stats", 1)   # from zero again
    c.global_trades(1)
    o.swap_counts(reset=True)
    o.superstep(1)
    performed, possible = c.swap_counts()
    assert (performed, possible) == o.swap_counts() and 0 < performed <= possible


def test_swap_counts_refuse_batches():
    g1 = exact.to_csr(frozenset({(0, 1)}), 3)
    ens = Ensemble([g1, g1], [1, 2])
    with pytest.raises(CbError) as e:
        ens.set_option("swap_stats", 1)
    assert e.value.code == CB_EINVAL
