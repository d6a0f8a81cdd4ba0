"""Pins of the oracle's swap counts (Appendix "Swaps performed by Curveball
and Global Curveball"): a trade performs as many neighbourhood swaps as edge
ends that change node, out of deg(u) + deg(v) possible.

Fixed by the paper: Fig. 2's sigma exchanges four edges; on regular graphs
the performed fraction tends to 1/2 as common neighbours vanish.  Fixed by
the mathematics: u keeps a uniform a-subset of D (a = |A_{u-v}|, b =
|A_{v-u}|), so a hypergeometric count of u's neighbours leaves, with mean
ab/(a+b); the edge ends that change node number twice that.
"""
import json
import os
from fractions import Fraction

import numpy as np
import pytest

from oracle import Oracle, uniform_pair
from paper_1804_08487_gb300 import synth
from tests import exact

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def test_fig2_sigma_exchanges_four_edges():
    with open(os.path.join(GOLDEN, "fig2_trade.json")) as f:
        g = json.load(f)
    ids = g["node_ids"]
    node = lambda x: ids[str(x)]  # noqa: E731
    edges = [(ids["i"], node(x)) for x in g["A_i"]] + [(ids["j"], node(x)) for x in g["A_j"]]
    rp, col = exact.to_csr(frozenset((min(a, b), max(a, b)) for a, b in edges), 8)
    o = Oracle(rp, col, seed=0)
    o.trade_explicit(ids["i"], ids["j"], [node(x) for x in g["sigma_image"]])
    performed, possible = o.swap_counts()
    assert performed == g["edges_exchanged"]
    assert possible == len(g["A_i"]) + len(g["A_j"])


def _changed_ends(s0, s1, u, v):
    """Edge ends at u or v whose node changed from state s0 to s1."""
    def nb(s, x):
        return {b if a == x else a for a, b in s if x in (a, b)}
    return len(nb(s0, u) - nb(s1, u)) + len(nb(s0, v) - nb(s1, v))


@pytest.mark.parametrize("a_list,b_list,common", [([1, 2], [3, 4, 5], [6]), ([1], [2, 3, 4, 5], []),
                                                  ([1, 2, 3], [4, 5, 6], [7, 8])])
def test_expected_swaps_of_one_trade_by_enumeration(a_list, b_list, common):
    """Exact enumeration of one uniform trade: E[changed edge ends] = 2ab/(a+b)."""
    u, v = 0, 9
    state = frozenset([(u, x) for x in a_list + common] + [(v, x) for x in b_list + common])
    mean = sum(p * _changed_ends(state, s2, u, v) for s2, p in exact.trade_outcomes(state, 10, u, v).items())
    a, b = len(a_list), len(b_list)
    assert mean == Fraction(2 * a * b, a + b)


def test_oracle_swap_counts_follow_the_hypergeometric_mean():
    """Over many uniform trades the oracle's performed count matches the sum of
    the exact conditional means 2ab/(a+b) within five standard deviations."""
    g = synth.powerlaw_graph(400, 3, 80, 2.0, 5)
    seed = 17
    o = Oracle(g.row_ptr, g.col, seed)
    mean = var = 0.0
    trades = 3000
    for i in range(trades):
        u, v = uniform_pair(seed, g.n, i)
        d, a = o.disjoint(u, v)
        b = len(d) - a
        if a and b:
            mean += 2.0 * a * b / (a + b)
            # X ~ Hypergeometric(a + b, a, b): u's neighbours that leave; changed ends = 2X
            var += 4.0 * a * b * a * b / ((a + b) ** 2 * (a + b - 1)) if a + b > 1 else 0.0
        o.uniform_trades(1)
    performed, possible = o.swap_counts()
    assert abs(performed - mean) < 5 * np.sqrt(var) + 1
    assert possible == sum(int(g.row_ptr[x + 1] - g.row_ptr[x]) + int(g.row_ptr[y + 1] - g.row_ptr[y])
                           for x, y in (uniform_pair(seed, g.n, i) for i in range(trades)))


@pytest.mark.parametrize("kind", ["global", "uniform"])
def test_regular_graphs_swap_about_half(kind):
    """Appendix experiment: on 10-regular graphs the performed fraction tends
    to 1/2 (common neighbours vanish as n grows); n/2 uniform trades and one
    global trade perform alike."""
    g = synth.powerlaw_graph(6000, 10, 11, 2.0, 3)
    assert np.all(np.diff(g.row_ptr) == 10)
    o = Oracle(g.row_ptr, g.col, 8)
    o.superstep(10)                  # away from the structured Havel-Hakimi start
    o.swap_counts(reset=True)
    if kind == "global":
        o.superstep(2)
    else:
        o.uniform_trades(g.n)
    performed, possible = o.swap_counts()
    assert possible == 2 * 10 * g.n
    assert 0.47 < performed / possible < 0.505   # mean <= 1/2; one standard deviation is about 0.0015
