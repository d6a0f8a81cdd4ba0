"""Pins of the CPU oracle against what the paper and mathematics fix.

Sources: Def. "Simple Undirected Trade" and Fig. 2 (Section 3.2); Def.
"Undirected Global Trade" and Thm "globaltrades" with its proof and footnote
(Section 3.3); Section 4's trading procedure; Philox4x32-10 (Salmon et al.,
SC'11) checked against an independent implementation (Triton's).
"""
import itertools
import json
import math
import os
import subprocess
import sys
from collections import Counter

import numpy as np
import pytest

from oracle import Oracle, philox4x32_10
from paper_1804_08487_gb300 import synth
from tests import exact
from tests.helpers import check_simple_canonical, degrees

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")

# ---------------------------------------------------------------- Philox pin

_TRITON_SCRIPT = r"""
import os, sys, json
os.environ["TRITON_INTERPRET"] = "1"
import torch, triton, triton.language as tl

@triton.jit
def k(out, c0, c1, c2, c3, seed, N: tl.constexpr):
    i = tl.arange(0, N)
    r0, r1, r2, r3 = tl.philox(seed, tl.load(c0 + i), tl.load(c1 + i), tl.load(c2 + i), tl.load(c3 + i), 10)
    tl.store(out + 4 * i, r0)
    tl.store(out + 4 * i + 1, r1)
    tl.store(out + 4 * i + 2, r2)
    tl.store(out + 4 * i + 3, r3)

data = json.loads(sys.stdin.read())
ctr = torch.tensor(data["ctr"], dtype=torch.int64).to(torch.uint32)
res = {}
for seed in data["seeds"]:
    N = ctr.shape[0]
    out = torch.zeros(4 * N, dtype=torch.uint32)
    cols = [ctr[:, j].contiguous() for j in range(4)]
    k[(1,)](out, cols[0], cols[1], cols[2], cols[3], seed, N)
    res[str(seed)] = out.to(torch.int64).tolist()
print(json.dumps(res))
"""


def _philox_cases():
    rng = np.random.default_rng(20180423)
    ctr = rng.integers(0, 2**32, size=(60, 4), dtype=np.uint64)
    special = np.array([[0, 0, 0, 0], [1, 0, 0, 0], [0, 0, 0, 1], [2**32 - 1] * 4], dtype=np.uint64)
    return np.concatenate([special, ctr]).astype(np.int64)


def test_philox_matches_independent_implementation():
    """Own Philox4x32-10 == Triton's tl.philox (key words = low/high seed halves)."""
    pytest.importorskip("triton")
    ctr = _philox_cases()
    seeds = [0, 42, 7, 0x123456789ABCDEF0, 2**63 - 1]
    proc = subprocess.run([sys.executable, "-c", _TRITON_SCRIPT],
                          input=json.dumps({"ctr": ctr.tolist(), "seeds": seeds}),
                          capture_output=True, text=True, timeout=600)
    if proc.returncode != 0:
        pytest.skip(f"triton interpreter unavailable: {proc.stderr[-300:]}")
    ref = json.loads(proc.stdout.strip().splitlines()[-1])
    for seed in seeds:
        want = np.array(ref[str(seed)], dtype=np.int64).reshape(-1, 4)
        for i, c in enumerate(ctr):
            got = philox4x32_10(c, seed).astype(np.int64)
            assert (got == want[i]).all(), (seed, c.tolist(), got, want[i])


def test_philox_words_are_uniform():
    """Chi-square of the top byte of every output word over 4096 counters."""
    counts = np.zeros(256, dtype=np.int64)
    for x in range(4096):
        r = philox4x32_10([x, 0, 3, 0], 99)
        for w in r:
            counts[int(w) >> 24] += 1
    exp = counts.sum() / 256
    chi2 = ((counts - exp) ** 2 / exp).sum()
    # 255 dof: p=1e-4 critical value is about 353
    assert chi2 < 353, chi2


# --------------------------------------------------------- trade primitive

def _graph(edges, n):
    return exact.to_csr(frozenset((min(a, b), max(a, b)) for a, b in edges), n)


def _fig2():
    with open(os.path.join(GOLDEN, "fig2_trade.json")) as f:
        g = json.load(f)
    ids = g["node_ids"]
    node = lambda x: ids[str(x)]  # noqa: E731
    edges = [(ids["i"], node(x)) for x in g["A_i"]] + [(ids["j"], node(x)) for x in g["A_j"]]
    return g, ids, node, sorted({(min(a, b), max(a, b)) for a, b in edges})


def test_fig2_worked_trade():
    g, ids, node, edges = _fig2()
    rp, col = _graph(edges, 8)
    o = Oracle(rp, col, seed=0)
    d, a = o.disjoint(ids["i"], ids["j"])
    assert d.tolist() == [node(x) for x in g["D"]] and a == g["a"]
    o.trade_explicit(ids["i"], ids["j"], [node(x) for x in g["sigma_image"]])
    got = {tuple(e) for e in o.edges().tolist()}
    want = {(min(ids["i"], node(x)), max(ids["i"], node(x))) for x in g["B_i"]} | \
           {(min(ids["j"], node(x)), max(ids["j"], node(x))) for x in g["B_j"]}
    assert got == want


def test_trade_rule_exact_enumeration():
    """Over all |D|! orderings sigma, u's new disjoint set is each a-subset of D
    exactly |D|!/C(|D|,a) times; common neighbours and {u,v} stay (Def. trade)."""
    g, ids, node, edges = _fig2()
    rp, col = _graph(edges, 8)
    base = Oracle(rp, col, seed=0)
    i, j = ids["i"], ids["j"]
    d, a = base.disjoint(i, j)
    counts = Counter()
    for perm in itertools.permutations(d.tolist()):
        o = base.clone()
        o.trade_explicit(i, j, list(perm))
        e = {tuple(x) for x in o.edges().tolist()}
        new_u = frozenset(x for x in d.tolist() if (min(i, x), max(i, x)) in e)
        assert len(new_u) == a
        assert (min(i, j), max(i, j)) in e                       # edge {i,j} kept
        assert (min(i, 6), max(i, 6)) in e and (min(j, 6), max(j, 6)) in e  # common kept
        assert (degrees(np.array(sorted(e)), 8) == degrees(base.edges(), 8)).all()
        counts[new_u] += 1
    assert len(counts) == math.comb(len(d), a)
    assert set(counts.values()) == {math.factorial(len(d)) // math.comb(len(d), a)}


def test_trade_rejects_non_permutation():
    g, ids, node, edges = _fig2()
    rp, col = _graph(edges, 8)
    o = Oracle(rp, col, seed=0)
    with pytest.raises(ValueError):
        o.trade_explicit(ids["i"], ids["j"], [1, 2, 3, 4])
    with pytest.raises(ValueError):
        o.trade_explicit(ids["i"], ids["j"], [1, 1, 3, 4, 5])
    with pytest.raises(ValueError):
        o.trade_explicit(ids["i"], ids["j"], [1, 2, 3, 4, 6])


def test_trade_keeps_common_neighbours_and_degrees():
    gr = synth.powerlaw_graph(60, 4, 30, 2.0, 11)
    o = Oracle(gr.row_ptr, gr.col, seed=5)
    rng = np.random.default_rng(1)
    for _ in range(200):
        u, v = rng.choice(60, 2, replace=False)
        e0 = o.edges()
        adj = exact.adjacency({tuple(x) for x in e0.tolist()}, 60)
        common, uv = adj[u] & adj[v], v in adj[u]
        d, a = o.disjoint(int(u), int(v))
        assert set(d.tolist()) == (adj[u] ^ adj[v]) - {u, v}
        o.trade_explicit(int(u), int(v), rng.permutation(d).tolist())
        e1 = o.edges()
        adj1 = exact.adjacency({tuple(x) for x in e1.tolist()}, 60)
        assert adj1[u] & adj1[v] == common and (v in adj1[u]) == uv
        assert len(adj1[u] - adj1[v] - {v}) == a
        assert (degrees(e1, 60) == degrees(e0, 60)).all()


# --------------------------------------------------------- permutation pi

def test_permutation_is_the_key_sort():
    """order = nodes sorted by (philox64(seed; x,0,g,0), x), via numpy's sort."""
    gr = synth.powerlaw_graph(301, 3, 40, 2.0, 2)
    o = Oracle(gr.row_ptr, gr.col, seed=123456789)
    for g in (0, 1, 17):
        keys = np.array([(int(r[0]) << 32) | int(r[1]) for r in
                         (philox4x32_10([x, 0, g, 0], 123456789) for x in range(301))], dtype=np.uint64)
        want = np.lexsort((np.arange(301), keys))
        assert (o.permutation(g) == want).all()


def test_permutation_is_uniform():
    """All 4! orders of 4 nodes equally likely over super steps g (chi-square)."""
    rp, col = _graph([(0, 1), (2, 3)], 4)
    o = Oracle(rp, col, seed=2024)
    cnt = Counter(tuple(o.permutation(g).tolist()) for g in range(24000))
    assert len(cnt) == 24
    obs = np.array(list(cnt.values()), dtype=float)
    chi2 = ((obs - 1000) ** 2 / 1000).sum()
    assert chi2 < 59.7, chi2          # 23 dof, p = 1e-4


# -------------------------------------------------- global trade invariants

@pytest.mark.parametrize("n,a,b,seed", [(200, 3, 40, 1), (201, 3, 40, 2), (33, 5, 20, 3), (2, 1, 2, 4)])
def test_super_step_invariants(n, a, b, seed):
    gr = synth.powerlaw_graph(n, a, b, 2.0, seed)
    o = Oracle(gr.row_ptr, gr.col, seed=seed)
    e0 = o.edges()
    d0 = degrees(e0, n)
    for _ in range(5):
        o.superstep(1)
        e = o.edges()
        check_simple_canonical(e, n)
        assert len(e) == len(e0)
        assert (degrees(e, n) == d0).all()


def test_odd_n_untraded_node_only_relabelled():
    """For odd n the node at the last position trades nothing: each of its
    neighbours either stays or is replaced by that neighbour's trade partner."""
    gr = synth.powerlaw_graph(101, 3, 30, 2.0, 9)
    o = Oracle(gr.row_ptr, gr.col, seed=77)
    for g in range(4):
        order = o.permutation(g)
        pos = np.empty(101, dtype=np.int64)
        pos[order] = np.arange(101)
        w = int(order[100])
        before = exact.adjacency({tuple(x) for x in o.edges().tolist()}, 101)[w]
        o.superstep(1)
        after = exact.adjacency({tuple(x) for x in o.edges().tolist()}, 101)[w]
        partner = {int(order[p]): int(order[p ^ 1]) for p in range(100)}
        assert len(after) == len(before)
        for y in after:
            assert y in before or partner[y] in before


def test_determinism_and_resume():
    """Same seed: same chain; 10 super steps == 5, export, recreate at step 5, 5."""
    gr = synth.PLAIN["n4096"].graph()
    a = Oracle(gr.row_ptr, gr.col, seed=42)
    a.superstep(10)
    b = Oracle(gr.row_ptr, gr.col, seed=42)
    b.superstep(5)
    from tests.helpers import csr_from_edges
    rp, col = csr_from_edges(b.edges(), gr.n)
    c = Oracle(rp, col, seed=42, first_step=5)
    c.superstep(5)
    assert (a.edges() == c.edges()).all()
    d = Oracle(gr.row_ptr, gr.col, seed=43)
    d.superstep(10)
    assert not np.array_equal(a.edges(), d.edges())


# ------------------------------------------------ the Markov chain (Thm)

_TINY = [
    ("two_regular_6", [2] * 6),
    ("three_regular_6", [3] * 6),
    ("one_regular_4", [1] * 4),
]


@pytest.mark.parametrize("name,deg", _TINY)
def test_omega_counts(name, deg):
    with open(os.path.join(GOLDEN, "omega_counts.json")) as f:
        want = json.load(f)[name]
    assert len(exact.omega(deg)) == want


def _matrix(deg):
    states = exact.omega(deg)
    n = len(deg)
    idx = {s: i for i, s in enumerate(states)}
    P = np.zeros((len(states), len(states)), dtype=object)
    for s in states:
        for s2, p in exact.global_trade_row(s, n).items():
            P[idx[s], idx[s2]] = p          # KeyError if the chain leaves Omega_G
    return states, P


@pytest.mark.parametrize("deg", [[1] * 4, [2, 2, 1, 1, 0], [2, 1, 2, 2, 1], [2] * 6, [3, 2, 2, 2, 1, 2]])
def test_global_trade_chain_is_symmetric_irreducible_aperiodic(deg):
    """Thm 'globaltrades' (Section 3.3): transition matrix on Omega_G is symmetric,
    every state has a self loop, and the chain is irreducible, so uniform is stationary."""
    states, P = _matrix(deg)
    k = len(states)
    for i in range(k):
        assert sum(P[i, :]) == 1
        assert P[i, i] > 0
        for j in range(k):
            assert P[i, j] == P[j, i]
    reach = {0}
    frontier = [0]
    while frontier:
        i = frontier.pop()
        for j in range(k):
            if P[i, j] > 0 and j not in reach:
                reach.add(j)
                frontier.append(j)
    assert len(reach) == k


def test_counterexample_global_trade_differs_from_single_trades():
    """Footnote to the proof: for V={1..4}, E={[1,2],[3,4]} a global trade is
    not distributed as n/2 = 2 uniform single trades."""
    start = frozenset({(0, 1), (2, 3)})
    g_row = exact.global_trade_row(start, 4)
    s_row = exact.single_trades_row(start, 4, 2)
    assert set(g_row) == set(s_row) and len(g_row) == 3
    assert any(g_row[s] != s_row[s] for s in g_row)


def _chain_transition_counts(deg, seed, steps):
    states = exact.omega(deg)
    n = len(deg)
    idx = {s: i for i, s in enumerate(states)}
    rp, col = exact.to_csr(states[0], n)
    o = Oracle(rp, col, seed=seed)
    counts = np.zeros((len(states), len(states)), dtype=np.int64)
    cur = idx[states[0]]
    for _ in range(steps):
        o.superstep(1)
        nxt = idx[frozenset(tuple(e) for e in o.edges().tolist())]
        counts[cur, nxt] += 1
        cur = nxt
    return states, counts


@pytest.mark.parametrize("deg,seed", [([1] * 4, 3), ([2, 2, 1, 1, 0], 4), ([2, 1, 2, 2, 1], 5), ([2] * 6, 6)])
def test_oracle_transitions_follow_exact_chain(deg, seed):
    """Empirical one-step transitions of the oracle (Philox pi and sigma) match
    the exact enumeration of uniform pi and uniform sigma (pooled chi-square)."""
    from scipy.stats import chi2 as chi2dist
    states, P = _matrix(deg)
    _, counts = _chain_transition_counts(deg, seed, 30000)
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


@pytest.mark.parametrize("deg,seed", [([2] * 6, 11), ([3] * 6, 12), ([1] * 4, 13), ([2, 1, 2, 2, 1], 14)])
def test_long_run_is_uniform_on_omega(deg, seed):
    """The chain's visits (every 3rd super step) are uniform on Omega_G."""
    from scipy.stats import chisquare
    states = exact.omega(deg)
    n = len(deg)
    idx = {s: i for i, s in enumerate(states)}
    rp, col = exact.to_csr(states[0], n)
    o = Oracle(rp, col, seed=seed + 1000)
    visits = np.zeros(len(states), dtype=np.int64)
    for t in range(3 * 14000):
        o.superstep(1)
        if t % 3 == 2:
            visits[idx[frozenset(tuple(e) for e in o.edges().tolist())]] += 1
    assert chisquare(visits).pvalue > 1e-4


# ------------------------------------------- relaxed global trade (LCG maps)
# Def. "Relaxed global trade" (Appendix EM-GCB) with linear congruential maps
# h(x) = (a x + b) mod p (Section 4.3, Appendix "Linear congruential maps").

def _is_prime(q):
    return q >= 2 and all(q % d for d in range(2, int(q ** 0.5) + 1))


@pytest.mark.parametrize("n", [0, 1, 2, 3, 4, 5, 6, 7, 8, 24, 97, 1000, 65536, 1 << 20])
def test_lcg_prime_and_parameters(n):
    o = Oracle(np.zeros(n + 1, dtype=np.int64), np.zeros(0, dtype=np.int32), 11)
    for g in range(3):
        p, a, b = o.lcg_params(g)
        assert _is_prime(p) and p >= max(n, 2)
        assert all(not _is_prime(q) for q in range(max(n, 2), p))   # the smallest such prime
        assert 1 <= a < p and 0 <= b < p


@pytest.mark.parametrize("p", [2, 3, 7, 11, 101])
def test_lcg_is_a_bijection_with_the_stated_inverse(p):
    """Prop. "congruentialbijective": h is a bijection of Z_p and
    h^{-1}(y) = a^{-1} (y - b) mod p."""
    rng = np.random.default_rng(p)
    for _ in range(10):
        a = int(rng.integers(1, p)) if p > 2 else 1
        b = int(rng.integers(0, p))
        image = [(a * x + b) % p for x in range(p)]
        assert sorted(image) == list(range(p))
        ainv = pow(a, p - 2, p)
        assert all((ainv * (image[x] - b)) % p == x for x in range(p))


@pytest.mark.parametrize("p", [5, 7, 11])
def test_lcg_family_is_pairwise_uniform(p):
    """Lemma "statrandom": over all maps of the family, every pair of distinct
    keys goes to every pair of distinct values exactly once (the maps are
    bijections, so equal values never occur)."""
    for x1 in range(p):
        for x2 in range(p):
            if x1 == x2:
                continue
            cnt = {}
            for a in range(1, p):
                for b in range(p):
                    key = ((a * x1 + b) % p, (a * x2 + b) % p)
                    cnt[key] = cnt.get(key, 0) + 1
            assert all(y1 != y2 for (y1, y2) in cnt)
            assert len(cnt) == p * (p - 1) and set(cnt.values()) == {1}


def _rank_bounds(pi, x, xp, y):
    return y - (pi[xp] - xp), y - (pi[x] - x)


def test_sorted_rank_map_worked_example():
    """The paper's example for Prop. "bounds": im(h) = {0,1,2,3,5,6} (n = 6,
    p = 7; here a = 1, b = 5), pi(0) = 0 and pi(5) = 6 bound the rank of 2 to
    {1, 2}; its rank is 2."""
    n, p, a, b = 6, 7, 1, 5
    pi = sorted((a * x + b) % p for x in range(n))
    assert pi == [0, 1, 2, 3, 5, 6]
    assert pi[0] == 0 and pi[5] == 6
    lo, hi = _rank_bounds(pi, 0, 5, 2)
    assert (lo, hi) == (1, 2) and lo <= pi.index(2) <= hi


def test_sorted_rank_map_bounds_hold():
    """Prop. "bounds": for ranks x <= x' with pi(x) <= y <= pi(x'), the rank of
    y lies in [y - (pi(x') - x'), y - (pi(x) - x)]."""
    rng = np.random.default_rng(3)
    for n in [5, 30, 200, 1000]:
        p = next((q for q in range(max(n, 2), 2 * n + 10) if _is_prime(q)))
        for _ in range(20):
            a, b = int(rng.integers(1, p)), int(rng.integers(0, p))
            pi = sorted((a * x + b) % p for x in range(n))
            for _ in range(20):
                x, xp = sorted(int(v) for v in rng.integers(0, n, size=2))
                r = int(rng.integers(x, xp + 1))
                lo, hi = _rank_bounds(pi, x, xp, pi[r])
                assert lo <= r <= hi


def test_relaxed_oracle_orders_nodes_by_the_map():
    g = synth.powerlaw_graph(3001, 3, 80, 2.0, 2)
    o = Oracle(g.row_ptr, g.col, 17)
    o.set_relaxed(True)
    for step in range(3):
        p, a, b = o.lcg_params(step)
        want = np.argsort([(a * x + b) % p for x in range(g.n)], kind="stable")
        assert np.array_equal(o.permutation(step), want)
    deg0 = np.diff(g.row_ptr)
    o.superstep(4)
    e = o.edges()
    check_simple_canonical(e, g.n)
    assert np.array_equal(degrees(e, g.n), deg0)


@pytest.mark.parametrize("deg", [[1] * 4, [2, 2, 1, 1, 0], [2] * 6])
def test_relaxed_chain_is_symmetric(deg):
    """Each global trade for a fixed order is a symmetric transition (Thm
    "globaltrades"), so the relaxed chain, which draws the order from the LCG
    family, has a symmetric stochastic matrix on Omega_G: uniform is
    stationary.  Checked exactly by enumerating every map of the family."""
    states = exact.omega(deg)
    n = len(deg)
    idx = {s: i for i, s in enumerate(states)}
    P = np.zeros((len(states), len(states)), dtype=object)
    for s in states:
        for s2, q in exact.relaxed_global_trade_row(s, n).items():
            P[idx[s], idx[s2]] = q
    for i in range(len(states)):
        assert sum(P[i, :]) == 1
        for j in range(len(states)):
            assert P[i, j] == P[j, i]


@pytest.mark.parametrize("n,a,b,seed", [(60, 2, 20, 1), (41, 3, 30, 2), (24, 5, 20, 3)])
def test_global_trade_is_order_independent(n, a, b, seed):
    """Applying one global trade's trades in any topological order of the
    'joined by an edge' relation gives the index-order result, which is the
    oracle's.  The GPU threshold pass rests on this: it runs all trades at
    once and orders only those joined by an edge."""
    import random
    from paper_1804_08487_gb300 import synth
    from oracle import philox4x32_10
    g = synth.powerlaw_graph(n, a, b, 2.0, seed)
    o = Oracle(g.row_ptr, g.col, seed)
    edges = [tuple(e) for e in o.edges().tolist()]
    order = [int(x) for x in o.permutation(0)]

    def edge_key(t, lo, hi):
        r = philox4x32_10([lo, hi, 0, 1], seed)
        w = (r[0], r[1]) if (lo >> 1) == t else (r[2], r[3])
        return (int(w[0]) << 32) | int(w[1])

    want_index = exact.global_trade_by_edge_keys(n, edges, order, edge_key)
    o.superstep(1)
    assert want_index == [tuple(e) for e in o.edges().tolist()]
    rng = random.Random(seed)
    differs = 0
    for _ in range(5):
        topo = exact.random_topological_trade_order(n, edges, order, rng)
        differs += topo != list(range(n // 2))
        assert exact.global_trade_by_edge_keys(n, edges, order, edge_key, topo) == want_index
    if a <= 3:   # sparse graphs leave room for other orders (the dense one may not)
        assert differs > 0
