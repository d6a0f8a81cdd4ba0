"""Pins of the oracle's uniform single trades (Simple Undirected Curveball,
Section 3.2) and of the successor lists Suc (Section 4.1) against what the
paper and the mathematics fix: the worked Suc example, the exact transition
matrix of a uniform trade on tiny state spaces, and an independent
restatement of the trade sequence in the manner of IM-CB (Section 4.2 and its
appendix algorithm), in which each edge waits in the buffer of the endpoint
traded next."""
import json
import os

import numpy as np
import pytest

from oracle import Oracle, philox4x32_10, successors, uniform_pair
from paper_1804_08487_gb300 import synth
from tests import exact

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def test_successor_lists_worked_example():
    with open(os.path.join(GOLDEN, "suc_example.json")) as f:
        ex = json.load(f)
    n = ex["n"]
    pairs = [(a - 1, b - 1) for a, b in ex["trades"]]
    begin, suc = successors(n, pairs)
    for x in range(n):
        want = ex["suc"][str(x + 1)]
        assert want[-1] == "inf"
        got = [int(i) + 1 for i in suc[begin[x]:begin[x + 1]]]
        assert got == want[:-1], f"Suc(v{x + 1})"


def test_successor_lists_reject_bad_pairs():
    with pytest.raises(ValueError):
        successors(3, [(0, 3)])
    with pytest.raises(ValueError):
        successors(3, [(1, 1)])


@pytest.mark.parametrize("n", [2, 5, 7])
def test_uniform_pairs_are_distinct_and_uniform(n):
    from scipy.stats import chisquare
    counts = np.zeros((n, n), dtype=np.int64)
    draws = 600 * n * (n - 1)
    for i in range(draws):
        u, v = uniform_pair(2024, n, i)
        assert 0 <= u < n and 0 <= v < n and u != v
        counts[u, v] += 1
    obs = counts[~np.eye(n, dtype=bool)]
    assert chisquare(obs).pvalue > 1e-4


def test_uniform_pairs_use_the_high_index_word():
    a = [uniform_pair(7, 1000, i) for i in range(50)]
    b = [uniform_pair(7, 1000, i + (1 << 32)) for i in range(50)]
    assert a != b


def _uniform_matrix(deg):
    states = exact.omega(deg)
    n = len(deg)
    idx = {s: i for i, s in enumerate(states)}
    P = np.zeros((len(states), len(states)), dtype=object)
    for s in states:
        for s2, p in exact.single_trades_row(s, n, 1).items():
            P[idx[s], idx[s2]] = p          # KeyError if a trade leaves Omega_G
    return states, P


@pytest.mark.parametrize("deg", [[1] * 4, [2, 2, 1, 1, 0], [2, 1, 2, 2, 1], [2] * 6])
def test_uniform_trade_chain_is_symmetric_irreducible_aperiodic(deg):
    """Section 3.2: the chain of uniform trades is irreducible, aperiodic and
    symmetric, hence uniform on Omega_G (exact enumeration, exact fractions)."""
    states, P = _uniform_matrix(deg)
    k = len(states)
    reach, frontier = {0}, [0]
    for i in range(k):
        assert sum(P[i, :]) == 1
        assert P[i, i] > 0
        for j in range(k):
            assert P[i, j] == P[j, i]
    while frontier:
        i = frontier.pop()
        for j in range(k):
            if P[i, j] > 0 and j not in reach:
                reach.add(j)
                frontier.append(j)
    assert len(reach) == k


@pytest.mark.parametrize("deg,seed", [([1] * 4, 31), ([2, 1, 2, 2, 1], 32), ([2] * 6, 33)])
def test_oracle_uniform_transitions_follow_exact_row(deg, seed):
    """Empirical one-trade transitions of the oracle (Philox pair and sigma)
    match the exact enumeration over uniform pairs and uniform sigma."""
    from scipy.stats import chi2 as chi2dist
    states, P = _uniform_matrix(deg)
    n = len(deg)
    idx = {s: i for i, s in enumerate(states)}
    rp, col = exact.to_csr(states[0], n)
    o = Oracle(rp, col, seed=seed)
    counts = np.zeros((len(states), len(states)), dtype=np.int64)
    cur = 0
    for _ in range(20000):
        o.uniform_trades(1)
        nxt = idx[frozenset(tuple(e) for e in o.edges().tolist())]
        counts[cur, nxt] += 1
        cur = nxt
    stat, dof = 0.0, 0
    for i in range(len(states)):
        tot = counts[i].sum()
        if tot < 50:
            continue
        for j in range(len(states)):
            p = float(P[i, j])
            if p == 0:
                assert counts[i, j] == 0
                continue
            e = tot * p
            stat += (counts[i, j] - e) ** 2 / e
            dof += 1
        dof -= 1
    assert dof > 0
    assert chi2dist.sf(stat, dof) > 1e-4, (stat, dof)


def _sigma_from_keys(seed):
    def sigma(i, u, v, d, a):
        def key(x):
            r = philox4x32_10([x, i & 0xFFFFFFFF, i >> 32, 6], seed)
            return ((int(r[0]) << 32) | int(r[1]), x)
        return sorted(d, key=key)
    return sigma


@pytest.mark.parametrize("n,a,b,seed,count,first", [
    (60, 2, 20, 1, 200, 0),
    (200, 3, 40, 2, 450, 17),
    (31, 8, 25, 3, 120, (1 << 32) - 40),   # dense: many common neighbours; index crosses 2^32
    (500, 2, 100, 4, 1000, 5),
])
def test_oracle_equals_imcb_restatement(n, a, b, seed, count, first):
    """The oracle applies trades one after the other on incidence lists; the
    IM-CB restatement routes every edge to its endpoint's next trade through
    Suc.  With the same pairs and keys they must end in the same graph."""
    g = synth.powerlaw_graph(n, a, b, 2.0, seed)
    o = Oracle(g.row_ptr, g.col, seed)
    edges0 = [tuple(e) for e in o.edges().tolist()]
    o.uniform_trades(count, first=first)
    assert o.uniform_next == first + count
    pairs = [uniform_pair(seed, n, first + k) for k in range(count)]
    # the restatement numbers trades 0..count-1; keys use the global index
    sig = _sigma_from_keys(seed)
    want = exact.imcb(n, edges0, pairs, lambda i, u, v, d, k: sig(first + i, u, v, d, k))
    got = [tuple(e) for e in o.edges().tolist()]
    assert got == want
    assert got != edges0


def test_uniform_trades_keep_degrees_and_simplicity():
    g = synth.powerlaw_graph(1000, 3, 200, 2.0, 9)
    o = Oracle(g.row_ptr, g.col, 99)
    o.uniform_trades(5000)
    e = o.edges()
    assert len(e) == g.m
    assert np.all(e[:, 0] < e[:, 1])
    assert len({tuple(x) for x in e.tolist()}) == g.m
    deg = np.bincount(e.ravel(), minlength=g.n)
    assert np.array_equal(deg, np.diff(g.row_ptr))


def test_uniform_resume_and_interleaving():
    g = synth.powerlaw_graph(300, 3, 60, 2.0, 12)
    a = Oracle(g.row_ptr, g.col, 5)
    b = Oracle(g.row_ptr, g.col, 5)
    a.uniform_trades(100)
    a.superstep(1)
    a.uniform_trades(50)
    b.uniform_trades(40)
    b.uniform_trades(60)
    b.superstep(1)
    b.uniform_trades(50)
    assert a.uniform_next == b.uniform_next == 150
    assert np.array_equal(a.edges(), b.edges())


@pytest.mark.parametrize("edges,n", [([], 0), ([], 1), ([(0, 1)], 2), ([(0, 1), (1, 2)], 3)])
def test_uniform_trades_on_tiny_graphs(edges, n):
    rp, col = exact.to_csr(frozenset(edges), n)
    o = Oracle(rp, col, 3)
    o.uniform_trades(25)
    assert o.uniform_next == 25
    # with at most one other node, D has at most one element per side and degrees pin the graph
    assert sorted(tuple(e) for e in o.edges().tolist()) == sorted(edges)


@pytest.mark.parametrize("n,a,b,seed,count", [(50, 2, 15, 1, 300), (30, 6, 25, 2, 200), (120, 1, 10, 3, 500),
                                              (6, 1, 5, 4, 100)])
def test_device_protocol_runs_every_trade_and_equals_oracle(n, a, b, seed, count):
    """The device's inbox protocol for uniform trades (per-endpoint inboxes
    sized by degree, each edge sent to the next trade of either endpoint, a
    trade runs once both inboxes are full), modelled sequentially with the
    runnable trades taken in random orders: it never deadlocks and always
    ends in the oracle's graph."""
    import random
    g = synth.powerlaw_graph(n, a, b, 2.0, seed)
    o = Oracle(g.row_ptr, g.col, seed)
    edges = [tuple(e) for e in o.edges().tolist()]
    o.uniform_trades(count)
    want = [tuple(e) for e in o.edges().tolist()]
    pairs = [uniform_pair(seed, n, k) for k in range(count)]
    sig = _sigma_from_keys(seed)
    rng = random.Random(seed)
    for _ in range(3):
        got, ran = exact.uniform_dataflow(n, edges, pairs, sig, rng)
        assert ran == count
        assert got == want

