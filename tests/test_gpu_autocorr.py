"""Edge autocorrelation on the GPU (Section 5.1) against the oracle's chain
and classifier (oracle/autocorr.py): the presence record after every super
step and the per-k counts of correlated edges (equal up to decisions within
1e-9 of the BIC boundary, which rounding could flip)."""
import numpy as np
import pytest

from oracle import Oracle
from oracle import autocorr as ac
from paper_1804_08487_gb300 import synth
from paper_1804_08487_gb300.cb import CB_EINVAL, CbError, Curveball, Ensemble

pytestmark = pytest.mark.gpu


def _oracle_lists(g, seed, steps):
    o = Oracle(g.row_ptr, g.col, seed)
    lists = [o.edges()]
    for _ in range(steps):
        o.superstep(1)
        lists.append(o.edges())
    return lists


def _check(got, lists, n, kmax):
    corr, near, occ, states = got
    want, occ_w, near_w = ac.fraction_correlated(lists, n, kmax)
    assert states == len(lists)
    assert occ == occ_w
    for k in range(kmax):
        assert abs(corr[k] - want[k]) <= near_w[k], (k + 1, corr[k], want[k])


@pytest.mark.parametrize("n,a,b,seed", [(300, 5, 40, 3), (257, 3, 120, 4)])
def test_plain_chain_matches_oracle(n, a, b, seed):
    g = synth.powerlaw_graph(n, a, b, 2.0, seed)
    steps, kmax = 120, 24
    c = Curveball(g.row_ptr, g.col, seed + 10)
    c.set_option("presence", steps)
    c.global_trades(steps + 5)          # states past the record's end are not recorded
    _check(c.autocorr(kmax), _oracle_lists(g, seed + 10, steps), n, kmax)
    c.close()


def test_batch_chains_match_oracle_per_graph():
    specs = [(200, 4, 30, 21), (151, 3, 20, 22), (1, 0, 1, 23), (90, 5, 40, 24)]
    graphs, seeds = [], []
    for n, a, b, s in specs:
        if n == 1:
            from tests.helpers import csr_from_edges
            rp, col = csr_from_edges(np.zeros((0, 2), dtype=np.int32), 1)
            graphs.append((rp, col))
        else:
            gg = synth.powerlaw_graph(n, a, b, 2.0, s)
            graphs.append((gg.row_ptr, gg.col))
        seeds.append(s + 100)
    steps, kmax = 60, 12
    e = Ensemble(graphs, seeds)
    e.set_option("presence", steps)
    e.global_trades(steps)
    total_occ = 0
    for i, ((rp, col), s) in enumerate(zip(graphs, seeds)):
        n = len(rp) - 1
        o = Oracle(rp, col, s)
        lists = [o.edges()]
        for _ in range(steps):
            o.superstep(1)
            lists.append(o.edges())
        got = e.autocorr(kmax, graph=i)
        _check(got, lists, n, kmax)
        total_occ += got[2]
    assert e.autocorr(kmax)[2] == total_occ
    e.close()


def test_presence_restart_and_errors():
    g = synth.powerlaw_graph(120, 3, 20, 2.0, 8)
    c = Curveball(g.row_ptr, g.col, 5)
    with pytest.raises(CbError) as err:
        c.autocorr(4)                    # no record yet
    assert err.value.code == CB_EINVAL
    c.set_option("presence", 10)
    c.global_trades(3)
    assert c.autocorr(4)[3] == 4         # step 0 and three super steps
    c.set_option("presence", 30)         # a new record starts from the current state
    lists_start = c.edges()
    c.global_trades(30)
    got = c.autocorr(8)
    o = Oracle(g.row_ptr, g.col, 5)
    o.superstep(3)
    assert np.array_equal(o.edges(), lists_start)
    lists = [o.edges()]
    for _ in range(30):
        o.superstep(1)
        lists.append(o.edges())
    _check(got, lists, 120, 8)
    with pytest.raises(CbError):
        c.autocorr(65)
    c.set_option("presence", 0)
    with pytest.raises(CbError):
        c.autocorr(4)
    c.close()
