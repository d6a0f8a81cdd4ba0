"""Pins of the edge-autocorrelation classifier (Section 5.1; the BIC reading
is stated in oracle/autocorr.py).  Series whose answer is known: i.i.d.
coin flips (independent), sticky two-state chains (correlated), constant
series, a hand-computed G^2, and thinning."""
import math

import numpy as np
import pytest

from oracle import autocorr as ac


def test_transition_counts_and_thinning():
    x = [0, 1, 1, 0, 1, 1, 1, 0]
    # pairs (0,1) (1,1) (1,0) (0,1) (1,1) (1,1) (1,0)
    assert ac.transition_counts(x).tolist() == [[0, 2], [2, 3]]
    assert ac.thinned(x, 3).tolist() == [0, 0, 1]
    assert ac.thinned(x, 1).tolist() == x


def test_g2_by_hand():
    # counts [[a, b], [c, d]] = [[3, 1], [1, 3]]: N = 8, rows 4/4, columns 4/4
    n = [[3, 1], [1, 3]]
    l1 = 3 * math.log(3 / 4) + 1 * math.log(1 / 4) + 1 * math.log(1 / 4) + 3 * math.log(3 / 4)
    l0 = 4 * math.log(4 / 8) + 4 * math.log(4 / 8)
    assert ac.g2_statistic(n) == pytest.approx(2 * (l1 - l0), rel=1e-15)
    # independence in the counts (rows proportional): G^2 = 0
    assert ac.g2_statistic([[2, 6], [1, 3]]) == pytest.approx(0.0, abs=1e-12)


def test_constant_and_short_series_are_independent():
    assert not ac.correlated(np.ones(500, dtype=np.uint8), 1)
    assert not ac.correlated(np.zeros(500, dtype=np.uint8), 3)
    assert not ac.correlated([1, 0], 1)        # one transition: not classified
    assert not ac.correlated([1], 1)


def test_iid_series_are_mostly_independent():
    rng = np.random.default_rng(11)
    flags = [ac.correlated(rng.integers(0, 2, 600), 1) for _ in range(400)]
    # BIC's false-positive rate with 1 degree of freedom and N ~ 600 is about
    # P(chi2_1 > ln 600 = 6.4) ~ 1 %
    assert sum(flags) <= 16


def test_sticky_chains_are_correlated_and_thinning_decorrelates_them():
    rng = np.random.default_rng(12)

    def sticky(T, stay):
        x = np.zeros(T, dtype=np.uint8)
        x[0] = rng.integers(0, 2)
        for t in range(1, T):
            x[t] = x[t - 1] if rng.random() < stay else 1 - x[t - 1]
        return x

    chains = [sticky(6000, 0.95) for _ in range(100)]
    assert sum(ac.correlated(x, 1) for x in chains) >= 99
    # after k = 200 steps the correlation 0.9^200 is gone
    assert sum(ac.correlated(x, 200) for x in chains) <= 10


def test_fraction_correlated_on_a_toy_chain():
    # two pairs over 5 steps of a 3-node graph: {0,1} always, {1,2} alternating
    lists = [[(0, 1)] + ([(1, 2)] if t % 2 == 0 else []) for t in range(41)]
    counts, occurring, near = ac.fraction_correlated(lists, 3, 2)
    assert occurring == 2
    # k = 1: the alternating pair is perfectly predictable (correlated);
    # k = 2: it is constant after thinning (independent)
    assert counts.tolist() == [1, 0]
    assert near.tolist() == [0, 0]
