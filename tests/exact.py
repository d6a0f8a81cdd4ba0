"""Exact, enumerative statement of the global Curveball Markov chain for tiny
graphs (test helper; pure Python, no Philox, no keys).

A state is a frozenset of edges (a, b) with a < b.  A single trade of u and v
(Def. "Simple Undirected Trade", Section 3.2) keeps the common neighbours and
the edge {u, v}, and gives u a uniformly random |A_{u-v}|-subset of the disjoint
set D (Section 4: "draw |A_u n D| nodes from D for u uniformly at random").  A
global trade (Def. "Undirected Global Trade", Section 3.3) draws a uniform
permutation pi and applies the floor(n/2) trades {pi(2i-1), pi(2i)} in order.
`imcb` restates a given trade sequence in the manner of IM-CB (Section 4.2),
with sigma supplied by the caller.
"""
from fractions import Fraction
from itertools import combinations, permutations
from math import comb


def adjacency(state, n):
    adj = [set() for _ in range(n)]
    for a, b in state:
        adj[a].add(b)
        adj[b].add(a)
    return adj


def trade_outcomes(state, n, u, v):
    """{next_state: probability} of one uniform trade of u and v."""
    adj = adjacency(state, n)
    auv = adj[u] - adj[v] - {v}
    avu = adj[v] - adj[u] - {u}
    d = sorted(auv | avu)
    a = len(auv)
    rest = {e for e in state if u not in e and v not in e}
    keep = {(min(u, x), max(u, x)) for x in adj[u] - auv} | {(min(v, x), max(v, x)) for x in adj[v] - avu}
    out = {}
    p = Fraction(1, comb(len(d), a))
    for su in combinations(d, a):
        su = set(su)
        new = set(rest) | keep
        new |= {(min(u, x), max(u, x)) for x in su}
        new |= {(min(v, x), max(v, x)) for x in d if x not in su}
        key = frozenset(new)
        out[key] = out.get(key, 0) + p
    return out


def global_trade_outcomes(state, n, order):
    """Distribution after the trades (order[2t], order[2t+1]), t = 0.. in sequence."""
    dist = {state: Fraction(1)}
    for t in range(n // 2):
        u, v = order[2 * t], order[2 * t + 1]
        nd = {}
        for s, p in dist.items():
            for s2, q in trade_outcomes(s, n, u, v).items():
                nd[s2] = nd.get(s2, 0) + p * q
        dist = nd
    return dist


def global_trade_row(state, n):
    """Exact transition probabilities of one global trade from `state`."""
    row = {}
    perms = list(permutations(range(n)))
    w = Fraction(1, len(perms))
    for order in perms:
        for s2, q in global_trade_outcomes(state, n, order).items():
            row[s2] = row.get(s2, 0) + w * q
    return row


def single_trades_row(state, n, k):
    """k successive single trades, each on a uniformly random unordered pair."""
    pairs = list(combinations(range(n), 2))
    dist = {state: Fraction(1)}
    for _ in range(k):
        nd = {}
        for s, p in dist.items():
            for (u, v) in pairs:
                for s2, q in trade_outcomes(s, n, u, v).items():
                    nd[s2] = nd.get(s2, 0) + p * q / len(pairs)
        dist = nd
    return dist


def omega(degrees):
    """All simple graphs on len(degrees) labelled nodes with this degree sequence."""
    n = len(degrees)
    cand = list(combinations(range(n), 2))
    out = []

    def rec(i, rem, chosen):
        if i == len(cand):
            if all(r == 0 for r in rem):
                out.append(frozenset(chosen))
            return
        a, b = cand[i]
        # prune: remaining capacity of a must be satisfiable by later pairs
        if rem[a] > 0 and rem[b] > 0:
            rem[a] -= 1; rem[b] -= 1
            chosen.append((a, b))
            rec(i + 1, rem, chosen)
            chosen.pop()
            rem[a] += 1; rem[b] += 1
        # skip the pair only if a can still reach its degree with later pairs
        later_a = sum(1 for (x, y) in cand[i + 1:] if a in (x, y))
        if rem[a] <= later_a:
            rec(i + 1, rem, chosen)

    rec(0, list(degrees), [])
    return out


def to_csr(state, n):
    import numpy as np
    adj = adjacency(state, n)
    rp = np.zeros(n + 1, dtype=np.int64)
    rp[1:] = np.cumsum([len(adj[x]) for x in range(n)])
    col = np.array([y for x in range(n) for y in sorted(adj[x])], dtype=np.int32)
    return rp, col


def next_prime(n):
    """Smallest prime p >= n (p = 2 for n <= 2), by trial division."""
    p = max(n, 2)
    while any(p % d == 0 for d in range(2, int(p ** 0.5) + 1)):
        p += 1
    return p


def lcg_orders(n):
    """Every order of [n] induced by a linear congruential map
    h(x) = (a x + b) mod p, 1 <= a < p, 0 <= b < p, p the smallest prime >= n
    (Def. "Relaxed global trade": nodes in order of their image), one per map."""
    p = next_prime(n)
    return [sorted(range(n), key=lambda x: (a * x + b) % p) for a in range(1, p) for b in range(p)]


def relaxed_global_trade_row(state, n):
    """Exact transition probabilities of one relaxed global trade: the map
    drawn uniformly from the family, then the trades of its order."""
    row = {}
    orders = lcg_orders(n)
    w = Fraction(1, len(orders))
    for order in orders:
        for s2, q in global_trade_outcomes(state, n, order).items():
            row[s2] = row.get(s2, 0) + w * q
    return row


def imcb(n, edges, pairs, sigma):
    """The trade sequence `pairs` applied in the manner of the paper's IM-CB
    (Section 4.2 and its appendix algorithm): successor lists Suc, every edge
    kept once, in the buffer of the endpoint whose next trade comes first; a
    trade gathers the buffers of its two nodes, reassigns the disjoint
    neighbours and pushes every resulting edge to the endpoint traded next.

    sigma(i, u, v, d, a) returns sigma(D) for trade i, given D sorted by node
    id and a = |A_{u-v}|; u receives its first a elements (Fig. 2)."""
    inf = len(pairs)
    suc = [[] for _ in range(n)]
    for i, (u, v) in enumerate(pairs):
        suc[u].append(i)
        suc[v].append(i)
    idx = [0] * n

    def tau(x):
        return suc[x][idx[x]] if idx[x] < len(suc[x]) else inf

    buf = [[] for _ in range(n)]

    def push(a, b):
        if tau(a) <= tau(b):
            buf[a].append(b)
        else:
            buf[b].append(a)

    for a, b in edges:
        push(a, b)
    for i, (u, v) in enumerate(pairs):
        assert tau(u) == i and tau(v) == i
        nu, nv = set(buf[u]), set(buf[v])
        # the edge {u, v}, if present, sits in exactly one of the two buffers
        if u in nv:
            nu.add(v)
        if v in nu:
            nv.add(u)
        buf[u], buf[v] = [], []
        idx[u] += 1
        idx[v] += 1
        auv = nu - nv - {v}
        avu = nv - nu - {u}
        d = sorted(auv | avu)
        order = sigma(i, u, v, d, len(auv))
        assert sorted(order) == d
        new_u = (nu - auv) | set(order[:len(auv)])
        new_v = (nv - avu) | set(order[len(auv):])
        for x in new_u:
            push(u, x)
        for x in new_v:
            if x != u:
                push(v, x)
    out = set()
    for a in range(n):
        for b in buf[a]:
            out.add((min(a, b), max(a, b)))
    assert sum(len(b) for b in buf) == len(out) == len(edges)
    return sorted(out)


def global_trade_by_edge_keys(n, edges, order, edge_key, trade_order=None):
    """One global trade (Def. "Undirected Global Trade", Section 3.3) with
    sigma drawn from edge keys, the trades applied in `trade_order` (index
    order by default).

    Every edge keeps, for the whole step, the identity (lo, hi) of its
    endpoints' positions at the step's start.  edge_key(t, lo, hi) is trade
    t's key of such an edge; sigma(D) sorts D by (key, lo, hi) and u
    receives the first |A_{u-v}| (Fig. 2)."""
    pos = {x: p for p, x in enumerate(order)}
    ends = [list(e) for e in edges]
    ident = [tuple(sorted((pos[a], pos[b]))) for a, b in edges]
    inc = [set() for _ in range(n)]
    for e, (a, b) in enumerate(edges):
        inc[a].add(e)
        inc[b].add(e)

    def other(e, x):
        a, b = ends[e]
        return b if a == x else a

    T = n // 2
    for t in (range(T) if trade_order is None else trade_order):
        u, v = order[2 * t], order[2 * t + 1]
        nu = {other(e, u): e for e in inc[u]}
        nv = {other(e, v): e for e in inc[v]}
        auv = [x for x in nu if x not in nv and x != v]
        avu = [x for x in nv if x not in nu and x != u]
        d = [(x, nu[x], 0) for x in auv] + [(x, nv[x], 1) for x in avu]
        d.sort(key=lambda r: (edge_key(t, *ident[r[1]]), ident[r[1]]))
        a = len(auv)
        for k, (x, e, side) in enumerate(d):
            to_u = k < a
            if to_u and side == 1:      # edge {v, x} becomes {u, x}
                ends[e] = [u if y == v else y for y in ends[e]]
                inc[v].discard(e)
                inc[u].add(e)
            elif not to_u and side == 0:  # edge {u, x} becomes {v, x}
                ends[e] = [v if y == u else y for y in ends[e]]
                inc[u].discard(e)
                inc[v].add(e)
    return sorted(tuple(sorted(e)) for e in ends)


def random_topological_trade_order(n, edges, order, rng):
    """An order of the trades of one global trade in which two trades joined
    by an edge keep their index order.  Trades touch only edges at their own
    nodes, and a trade moves an edge from one of its nodes to the other, so
    which trades are joined does not change during the step; trades that
    are not joined commute."""
    pos = {x: p for p, x in enumerate(order)}
    T = n // 2
    preds = [set() for _ in range(T)]
    for a, b in edges:
        s, t = pos[a] >> 1, pos[b] >> 1
        if s != t and s < T and t < T:
            preds[max(s, t)].add(min(s, t))
    done, out = set(), []
    ready = [t for t in range(T) if not preds[t]]
    while ready:
        t = ready.pop(rng.randrange(len(ready)))
        out.append(t)
        done.add(t)
        for w in range(T):
            if w not in done and w not in ready and w not in out and preds[w] <= done:
                ready.append(w)
    assert len(out) == T
    return out


def uniform_dataflow(n, edges, pairs, sigma, rng):
    """The device protocol for a uniform trade sequence, run sequentially in a
    random order of runnable trades:
      - trade i has one inbox per endpoint, full at that endpoint's degree;
      - every edge goes to min(next trade of a, next trade of b), into the
        inbox of each endpoint that trades there, carrying the other
        endpoint and its next trade; if neither endpoint trades again it is
        final;
      - a trade runs once both inboxes are full, and sends every resulting
        edge on the same way.
    Returns the final edges and the number of trades that ran (all of them
    unless the protocol deadlocks)."""
    L = len(pairs)
    inf = L
    deg = [0] * n
    for a, b in edges:
        deg[a] += 1
        deg[b] += 1
    suc = [[] for _ in range(n)]
    for i, (u, v) in enumerate(pairs):
        suc[u].append(i)
        suc[v].append(i)

    def nxt(x, i):   # next trade of x after trade i (i = -1: its first)
        for j in suc[x]:
            if j > i:
                return j
        return inf

    inbox = {(i, s): [] for i in range(L) for s in (0, 1)}
    out = set()
    ready = []

    def full(d):
        u, v = pairs[d]
        return len(inbox[(d, 0)]) == deg[u] and len(inbox[(d, 1)]) == deg[v]

    def route(a, ta, b, tb):
        d = min(ta, tb)
        if d == inf:
            out.add((min(a, b), max(a, b)))
            return
        u, v = pairs[d]
        if ta == d:
            inbox[(d, 0 if a == u else 1)].append((b, tb))
        if tb == d:
            inbox[(d, 0 if b == u else 1)].append((a, ta))
        if full(d):
            ready.append(d)

    for d in range(L):
        u, v = pairs[d]
        if deg[u] == 0 and deg[v] == 0:
            ready.append(d)
    for a, b in edges:
        route(a, nxt(a, -1), b, nxt(b, -1))
    ran = 0
    while ready:
        d = ready.pop(rng.randrange(len(ready)))
        ran += 1
        u, v = pairs[d]
        A = dict(inbox[(d, 0)])
        B = dict(inbox[(d, 1)])
        nu, nv = nxt(u, d), nxt(v, d)
        auv = sorted(x for x in A if x not in B and x != v)
        avu = sorted(x for x in B if x not in A and x != u)
        order = sigma(d, u, v, sorted(auv + avu), len(auv))
        to_u = set(order[:len(auv)])
        for x in A:
            if x in B:
                route(u, nu, x, A[x])
                route(v, nv, x, B[x])
        if v in A:
            route(u, nu, v, nv)
        for x in auv + avu:
            tau = A[x] if x in A else B[x]
            if x in to_u:
                route(u, nu, x, tau)
            else:
                route(v, nv, x, tau)
    return sorted(out), ran
