"""Edge autocorrelation of a Markov chain of graphs (Section 5.1, "Mixing of
Edge-Switching, Curveball and Global Curveball").

Test infrastructure: only tests/ and bench.py's CPU legs use it.

The paper's method, step by step:
  1. run the chain from G_0 for T super steps, giving G_0, ..., G_T;
  2. for every edge e occurring in some G_t, the boolean series
     Z_{e,t} = [e in G_t], t = 0..T;
  3. the k-thinned series keeps every k-th entry: Z_{e,0}, Z_{e,k}, Z_{e,2k}, ...;
  4. its empirical transition probabilities are fitted to an independent
     model and to a Markov model; the edge counts as independent when the
     independent model is the better fit.

The paper cites, but does not print, the criterion that decides "better fit".
Reading used here (stated as such): the Bayesian information criterion of
the two maximum-likelihood fits of the thinned series' N = floor(T/k)
transitions x_{s-1} -> x_s.  With transition counts n_ab:
  independent model (x_s ~ Bernoulli(p), one parameter):
      L0 = sum_b n_{+b} ln(n_{+b} / N)
  first-order Markov model (P(x_s | x_{s-1}), two parameters):
      L1 = sum_{a,b} n_ab ln(n_ab / n_{a+})
  BIC_i = -2 L_i + (parameters) ln N; the Markov model fits better iff
  BIC_1 < BIC_0, i.e. G^2 = 2 (L1 - L0) > ln N.
Terms with a zero count are zero (x ln x -> 0).  A constant series (edge
always or never present over the thinned steps) has G^2 = 0 and counts as
independent.  A series with N < 2 transitions is not classified (neither
fit is defined); it is counted as independent.
"""
import math

import numpy as np


def thinned(series, k: int) -> np.ndarray:
    """Every k-th entry of a 0/1 series (entries 0, k, 2k, ...)."""
    return np.asarray(series, dtype=np.uint8)[::k]


def transition_counts(x) -> np.ndarray:
    """2x2 counts n[a, b] of consecutive pairs (x_{s-1}, x_s) of a 0/1 series."""
    x = np.asarray(x, dtype=np.int64)
    n = np.zeros((2, 2), dtype=np.int64)
    if len(x) >= 2:
        np.add.at(n, (x[:-1], x[1:]), 1)
    return n


def _xlogy(a: float, b: float) -> float:
    return 0.0 if a == 0 else a * math.log(a / b)


def g2_statistic(n) -> float:
    """G^2 = 2 (L1 - L0) of the Markov fit against the independent fit."""
    n = np.asarray(n, dtype=np.float64)
    N = n.sum()
    row = n.sum(axis=1)
    col = n.sum(axis=0)
    l1 = sum(_xlogy(n[a, b], row[a]) for a in range(2) for b in range(2))
    l0 = sum(_xlogy(col[b], N) for b in range(2))
    return 2.0 * (l1 - l0)


def correlated(series, k: int) -> bool:
    """True when the Markov model fits the k-thinned series better (BIC)."""
    n = transition_counts(thinned(series, k))
    N = int(n.sum())
    if N < 2:
        return False
    return g2_statistic(n) > math.log(N)


def margin(series, k: int) -> float:
    """G^2 - ln N of the k-thinned series (the sign decides; tests use the size
    to spot decisions that rounding could flip)."""
    n = transition_counts(thinned(series, k))
    N = int(n.sum())
    return g2_statistic(n) - math.log(N) if N >= 2 else -math.inf


def presence_series(edge_lists, n: int):
    """{pair index: 0/1 series over the steps} for every pair occurring in a
    list of canonical edge lists (one per step, pairs a < b); the pair index
    of a < b is a n - a (a + 1) / 2 + (b - a - 1)."""
    T = len(edge_lists)
    seen = {}
    for t, e in enumerate(edge_lists):
        e = np.asarray(e, dtype=np.int64).reshape(-1, 2)
        idx = e[:, 0] * n - e[:, 0] * (e[:, 0] + 1) // 2 + (e[:, 1] - e[:, 0] - 1)
        for p in idx.tolist():
            s = seen.get(p)
            if s is None:
                s = seen[p] = np.zeros(T, dtype=np.uint8)
            s[t] = 1
    return seen


def fraction_correlated(edge_lists, n: int, kmax: int):
    """(correlated counts for k = 1..kmax, occurring edges, near-ties) of the
    chain whose step-t graph has canonical edge list edge_lists[t]; near-ties
    count the (edge, k) decisions with |G^2 - ln N| < 1e-9."""
    series = presence_series(edge_lists, n)
    counts = np.zeros(kmax, dtype=np.int64)
    near = np.zeros(kmax, dtype=np.int64)
    for s in series.values():
        for k in range(1, kmax + 1):
            m = margin(s, k)
            counts[k - 1] += m > 0
            near[k - 1] += abs(m) < 1e-9
    return counts, len(series), near
