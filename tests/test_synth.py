"""Seeded input generator: PLD([a,b), gamma) sampling (Section 2) and
Havel-Hakimi realisation (Section 5.2)."""
import itertools

import numpy as np
import pytest

from paper_1804_08487_gb300 import synth
from tests.helpers import canonical_from_csr, check_simple_canonical, degrees


def erdos_gallai(d):
    """Erdos-Gallai criterion (textbook): d (sorted desc) is graphical iff the sum
    is even and sum_{i<=k} d_i <= k(k-1) + sum_{i>k} min(d_i, k) for all k."""
    d = sorted(d, reverse=True)
    if sum(d) % 2:
        return False
    n = len(d)
    for k in range(1, n + 1):
        if sum(d[:k]) > k * (k - 1) + sum(min(x, k) for x in d[k:]):
            return False
    return True


def test_havel_hakimi_agrees_with_erdos_gallai():
    rng = np.random.default_rng(3)
    seen = {True: 0, False: 0}
    for _ in range(3000):
        n = int(rng.integers(1, 9))
        d = rng.integers(0, n, size=n).astype(np.int32)
        if d.sum() % 2:
            continue
        ok = erdos_gallai(d.tolist())
        try:
            rp, col = synth.havel_hakimi(d)
            got = True
        except synth.NotGraphical:
            got = False
        assert got == ok, d
        seen[ok] += 1
        if got:
            assert (np.diff(rp) == d).all()
            e = canonical_from_csr(rp, col)
            check_simple_canonical(e, n) if len(e) else None
    assert seen[True] > 100 and seen[False] > 100


def test_havel_hakimi_exhaustive_small():
    for n in range(1, 6):
        for d in itertools.product(range(n), repeat=n):
            if sum(d) % 2:
                continue
            try:
                synth.havel_hakimi(np.array(d, dtype=np.int32))
                got = True
            except synth.NotGraphical:
                got = False
            assert got == erdos_gallai(list(d)), d


def test_powerlaw_graph_is_simple_with_exact_degrees():
    g = synth.powerlaw_graph(3000, 10, 200, 2.0, 5)
    deg = synth.pld_degrees(3000, 10, 200, 2.0, g.degree_seed)
    assert (np.diff(g.row_ptr) == deg).all()
    e = canonical_from_csr(g.row_ptr, g.col)
    check_simple_canonical(e, 3000)
    assert (degrees(e, 3000) == deg).all()
    # rows sorted and symmetric
    for x in range(0, 3000, 97):
        row = g.col[g.row_ptr[x]:g.row_ptr[x + 1]]
        assert (np.diff(row) > 0).all()
        for y in row[:5]:
            assert x in g.col[g.row_ptr[y]:g.row_ptr[y + 1]]


@pytest.mark.parametrize("gamma", [2.0, 2.5, 3.0])
def test_pld_matches_pmf(gamma):
    """Sampled degrees follow P[X=k] proportional to k^-gamma on [a,b) (chi-square)."""
    from scipy.stats import chisquare
    a, b, n = 4, 40, 200000
    deg = synth.pld_degrees(n, a, b, gamma, 77)[:-1]     # the last one may carry the odd-sum fix
    obs = np.bincount(deg - a, minlength=b - a)[: b - a].astype(float)
    k = np.arange(a, b, dtype=float)
    p = k ** -gamma
    p /= p.sum()
    assert chisquare(obs, p * obs.sum()).pvalue > 1e-4


def test_odd_sum_fix_and_determinism():
    d1 = synth.pld_degrees(1001, 3, 30, 2.0, 9)
    d2 = synth.pld_degrees(1001, 3, 30, 2.0, 9)
    assert (d1 == d2).all() and d1.sum() % 2 == 0
    assert not (d1 == synth.pld_degrees(1001, 3, 30, 2.0, 10)).all()


def test_plain_small_workload_shape():
    w = synth.PLAIN["n4096"]
    g = w.graph()
    assert g.n == 4096 and w.chain_seed == 42 and w.supersteps == 10
    deg = np.diff(g.row_ptr)
    assert deg.min() >= 10 and deg.max() <= 100
