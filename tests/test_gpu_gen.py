"""Device input generation (include/cb_gen.h) against the host generator:
the same PLD degree draws and the same Havel-Hakimi graphs, byte for byte
(Section 2's PLD, Section 5.2's Havel-Hakimi realisation)."""
import json
import os

import numpy as np
import pytest

from paper_1804_08487_gb300 import cb, synth
from tests.helpers import graph_hash

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")
GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


@pytest.mark.parametrize("n,a,b,gamma,seed", [(0, 1, 5, 2.0, 1), (1, 1, 5, 2.0, 2), (1000, 10, 100, 2.0, 3),
                                              (100001, 10, 10000, 2.0, 4), (5000, 4, 300, 2.5, 5),
                                              (5000, 4, 300, 3.0, 6), (7777, 2, 50, 2.73, 7)])
def test_pld_degrees_equal_host(n, a, b, gamma, seed):
    want = synth.pld_degrees(n, a, b, gamma, seed)
    out = torch.zeros(max(n, 1), dtype=torch.int32, device="cuda")
    total = cb.cb_generate_pld(n, a, b, gamma, seed, out)
    assert np.array_equal(out.cpu().numpy()[:n], want)
    assert total == int(want.sum())


def _hh_device(deg):
    n = len(deg)
    d = torch.from_numpy(np.ascontiguousarray(deg, dtype=np.int32)).cuda() if n else torch.zeros(1, dtype=torch.int32,
                                                                                                 device="cuda")
    rp = torch.zeros(n + 1, dtype=torch.int64, device="cuda")
    col = torch.zeros(max(int(np.sum(deg)), 1), dtype=torch.int32, device="cuda")
    m = cb.cb_generate_hh(n, d, rp, col)
    return rp.cpu().numpy(), col.cpu().numpy()[:2 * m], m


@pytest.mark.parametrize("n,a,b,gamma,seed", [(64, 3, 20, 2.0, 5), (2001, 10, 300, 2.0, 9), (3000, 4, 1500, 2.0, 13),
                                              (20000, 1, 3, 2.0, 23), (5000, 5, 500, 2.5, 31)])
def test_havel_hakimi_equals_host(n, a, b, gamma, seed):
    g = synth.powerlaw_graph(n, a, b, gamma, seed)
    deg = np.diff(g.row_ptr).astype(np.int32)
    rp, col, m = _hh_device(deg)
    assert m == g.m
    assert np.array_equal(rp, g.row_ptr)
    assert np.array_equal(col, g.col)


def test_havel_hakimi_edge_cases_and_rejections():
    rp, col, m = _hh_device(np.array([1, 1], dtype=np.int32))
    assert m == 1 and rp.tolist() == [0, 1, 2] and col.tolist() == [1, 0]
    rp, col, m = _hh_device(np.zeros(5, dtype=np.int32))
    assert m == 0 and rp.tolist() == [0] * 6
    for bad in ([3, 3, 1, 1], [1, 1, 1], [2, 0], [4, 1, 1, 1]):   # not graphical, odd, degree >= n
        with pytest.raises(cb.CbError) as e:
            _hh_device(np.array(bad, dtype=np.int32))
        assert e.value.code == cb.CB_EINVAL
        with pytest.raises(synth.NotGraphical):
            synth.havel_hakimi(np.array(bad, dtype=np.int32))


@pytest.mark.parametrize("name", ["n4096", "n2^20"])
def test_workload_graphs_equal_host(name):
    w = synth.PLAIN[name]
    rp, col, dseed = cb.generate_powerlaw(w.n, w.a, w.b, w.gamma, w.degree_seed)
    g = w.graph()
    assert dseed == g.degree_seed
    assert graph_hash(rp.cpu().numpy(), col.cpu().numpy()) == graph_hash(g.row_ptr, g.col)
    path = os.path.join(GOLDEN, f"plain_{name.replace('^', 'p')}.json")
    with open(path) as f:
        gold = json.load(f)
    if "graph_sha256" in gold:
        assert graph_hash(rp.cpu().numpy(), col.cpu().numpy()) == gold["graph_sha256"]
