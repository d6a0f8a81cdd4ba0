"""Relaxed global trades (Def. "Relaxed global trade", Appendix EM-GCB): the
permutation of each super step comes from a linear congruential map
h(x) = (a x + b) mod p (Appendix "Linear congruential maps"); on the GPU it is
computed without sorting (positions skip the p - n gap values).  Every result
must equal the oracle's, edge list for edge list."""
import numpy as np
import pytest

from oracle import Oracle
from paper_1804_08487_gb300 import synth
from paper_1804_08487_gb300.cb import CB_EINVAL, CbError, Curveball, Ensemble
from tests import exact

pytestmark = pytest.mark.gpu


def _pair(rp, col, seed, first_step=0):
    c = Curveball(rp, col, seed, first_step)
    o = Oracle(rp, col, seed, first_step)
    c.set_option("relaxed", 1)
    o.set_relaxed(True)
    return c, o


@pytest.mark.parametrize("n,b,seed", [(2, 2, 1), (3, 2, 2), (101, 20, 3), (4096, 100, 4), (30001, 900, 5)])
def test_relaxed_permutation_matches_oracle(n, b, seed):
    if n <= 3:
        rp, col = exact.to_csr(frozenset({(0, 1)}), n)
    else:
        g = synth.powerlaw_graph(n, 3, b, 2.0, seed)
        rp, col = g.row_ptr, g.col
    c, o = _pair(rp, col, seed)
    for g in [0, 1, 7, 12345]:
        assert np.array_equal(c.permutation(g), o.permutation(g))


@pytest.mark.parametrize("n,b,seed,steps", [(1001, 60, 1, 5), (4096, 100, 2, 5), (20001, 2000, 3, 3)])
def test_relaxed_super_steps_match_oracle(n, b, seed, steps):
    g = synth.powerlaw_graph(n, 3, b, 2.0, seed)
    c, o = _pair(g.row_ptr, g.col, seed)
    for step in range(steps):
        c.global_trades(1)
        o.superstep(1)
        assert np.array_equal(c.edges(), o.edges()), f"step {step + 1}"


def test_switching_modes_mid_chain():
    g = synth.powerlaw_graph(5000, 3, 300, 2.0, 9)
    c = Curveball(g.row_ptr, g.col, 4)
    o = Oracle(g.row_ptr, g.col, 4)
    plan = [(False, 2), (True, 2), (False, 1), (True, 3)]
    for relaxed, k in plan:
        c.set_option("relaxed", int(relaxed))
        o.set_relaxed(relaxed)
        c.global_trades(k)
        o.superstep(k)
        assert np.array_equal(c.edges(), o.edges())


def test_relaxed_with_cuda_graph_and_options():
    g = synth.powerlaw_graph(6001, 3, 500, 2.0, 13)
    c, o = _pair(g.row_ptr, g.col, 21, first_step=5)
    c.set_option("cuda_graph", 1)
    c.global_trades(3)
    o.superstep(3)
    assert np.array_equal(c.edges(), o.edges())
    c.set_option("tile_max", 32)
    c.global_trades(2)
    o.superstep(2)
    assert np.array_equal(c.edges(), o.edges())


def test_relaxed_rejected_for_batches():
    rp, col = exact.to_csr(frozenset({(0, 1)}), 2)
    ens = Ensemble([(rp, col), (rp, col)], [1, 2])
    with pytest.raises(CbError) as e:
        ens.set_option("relaxed", 1)
    assert e.value.code == CB_EINVAL
