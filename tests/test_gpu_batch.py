"""Ensembles (many independent graphs in one handle), CUDA-graph replay and
the autotuner, against the CPU oracle run on each graph alone.

Every graph of a batch must evolve exactly as it would in its own handle
(Def. "Undirected Global Trade", Section 3.3, applied per graph; an odd graph
leaves the node at its last position untraded), and neither the CUDA-graph
replay nor any tuning option may change a result.
"""
import json
import os

import numpy as np
import pytest

from oracle import Oracle
from paper_1804_08487_gb300 import synth
from paper_1804_08487_gb300.cb import CB_EINVAL, CbError, Curveball, Ensemble
from tests import exact
from tests.helpers import edge_hash

pytestmark = pytest.mark.gpu


def _csr(edges, n):
    return exact.to_csr(frozenset((min(a, b), max(a, b)) for a, b in edges), n)


def _mixed_graphs():
    """Small graphs of every awkward kind: empty, one node, odd and even n,
    no edges, several CTAs' worth of trades."""
    graphs = [_csr([], 0), _csr([], 1), _csr([(0, 1)], 2), _csr([(0, 1), (1, 2)], 3), _csr([], 4)]
    for n, b, seed in [(57, 12, 1), (200, 30, 2), (513, 60, 3), (1000, 90, 4), (1025, 200, 5), (4099, 300, 6)]:
        g = synth.powerlaw_graph(n, 3, b, 2.0, seed)
        graphs.append((g.row_ptr, g.col))
    return graphs


def _check_batch(ens, oracles, step):
    for i, o in enumerate(oracles):
        got, want = ens.graph_edges(i), o.edges()
        assert got.shape == want.shape, f"graph {i}, step {step}"
        assert np.array_equal(got, want), f"graph {i} differs from its oracle after super step {step}"


@pytest.mark.parametrize("use_graph", [0, 1])
def test_batch_matches_each_graph_alone(use_graph):
    graphs = _mixed_graphs()
    seeds = [7 + 13 * i for i in range(len(graphs))]
    ens = Ensemble(graphs, seeds)
    ens.set_option("cuda_graph", use_graph)
    oracles = [Oracle(rp, c, s) for (rp, c), s in zip(graphs, seeds)]
    assert len(ens) == len(graphs)
    for i, (rp, _) in enumerate(graphs):
        assert ens.info(i) == (len(rp) - 1, int(rp[-1]) // 2)
    _check_batch(ens, oracles, 0)
    for step in range(1, 6):
        ens.global_trades(1)
        for o in oracles:
            o.superstep(1)
        _check_batch(ens, oracles, step)
    assert ens.step == 5


def test_batch_several_steps_per_call_and_export_all():
    graphs = _mixed_graphs()
    seeds = [100 + i for i in range(len(graphs))]
    ens = Ensemble(graphs, seeds, first_step=3)
    ens.set_option("cuda_graph", 1)
    ens.global_trades(4)
    oracles = [Oracle(rp, c, s, 3) for (rp, c), s in zip(graphs, seeds)]
    for o in oracles:
        o.superstep(4)
    _check_batch(ens, oracles, 7)
    every = ens.edges()
    want = np.concatenate([o.edges() for o in oracles] + [np.zeros((0, 2), np.int32)])
    assert np.array_equal(every, want)


def test_batch_permutation_is_each_graphs_own():
    graphs = _mixed_graphs()
    seeds = [3 * i + 1 for i in range(len(graphs))]
    ens = Ensemble(graphs, seeds)
    order = ens.permutation(5)
    off = 0
    for (rp, c), s in zip(graphs, seeds):
        n = len(rp) - 1
        span = n + (n & 1)
        mine = order[off:off + span] - off
        want = Oracle(rp, c, s).permutation(5)
        assert np.array_equal(mine[:n], want)
        if span > n:
            assert mine[n] == n   # the padding node sorts last
        off += span


def test_ensemble_members_match_oracle():
    """Members of the 256-graph ensemble workload (n log-uniform in
    [2^10, 2^16], degrees on [4, n/16), gamma in [2, 3], seed 1000+i)."""
    members = [synth.ensemble_member(i) for i in range(6)]
    graphs, seeds = [], []
    for w in members:
        g = w.graph()
        graphs.append((g.row_ptr, g.col))
        seeds.append(w.chain_seed)
    ens = Ensemble(graphs, seeds)
    ens.set_option("cuda_graph", 1)
    oracles = [Oracle(rp, c, s) for (rp, c), s in zip(graphs, seeds)]
    for step in range(1, 4):
        ens.global_trades(1)
        for o in oracles:
            o.superstep(1)
        _check_batch(ens, oracles, step)


def test_plain_handle_cuda_graph_matches_oracle():
    g = synth.powerlaw_graph(6001, 3, 400, 2.0, 11)
    c = Curveball(g.row_ptr, g.col, 77)
    c.set_option("cuda_graph", 1)
    o = Oracle(g.row_ptr, g.col, 77)
    for step in range(4):
        c.global_trades(1)
        o.superstep(1)
        assert np.array_equal(c.edges(), o.edges()), f"step {step + 1}"
    st = c.stats()
    assert st["launches"] > 0
    # an option change re-records the graph; the chain continues unchanged
    c.set_option("tile_max", 64)
    c.global_trades(2)
    o.superstep(2)
    assert np.array_equal(c.edges(), o.edges())


def test_autotune_does_not_change_the_chain():
    g = synth.powerlaw_graph(20000, 3, 2000, 2.0, 21)
    tuned = Curveball(g.row_ptr, g.col, 5)
    plain = Curveball(g.row_ptr, g.col, 5)
    got = tuned.autotune(9)
    assert got["steps"] == 9
    assert got["tile_max"] in (32, 64, 128)
    assert got["block_max"] in (512, 1024, 2048, 128) or got["block_max"] >= got["tile_max"]
    assert got["smem_max"] in (4096, 8192)
    assert got["inorder_threads"] in (256, 1024)
    assert got["retry_passes"] in (1, 2, 3)
    assert tuned.step == 9
    tuned.set_option("cuda_graph", 1)
    tuned.global_trades(3)
    plain.global_trades(12)
    assert np.array_equal(tuned.edges(), plain.edges())
    o = Oracle(g.row_ptr, g.col, 5)
    o.superstep(12)
    assert np.array_equal(plain.edges(), o.edges())


def test_autotune_cache_reuses_settings(tmp_path):
    """The first handle tunes and stores its choice under its key; a second
    handle of the same graph takes it from the file without running a super
    step, and its chain still equals the oracle's."""
    g = synth.powerlaw_graph(20000, 3, 2000, 2.0, 21)
    path = str(tmp_path / "tune.json")
    first = Curveball(g.row_ptr, g.col, 5)
    key = first.tune_key()
    assert key.split("|")[1].startswith("sm") and len(key.split("|")[-1].split(",")) == 33
    got = first.autotune(20, cache_path=path)
    assert 0 < got["steps"] <= 20 and first.step == got["steps"]
    with open(path) as f:
        doc = json.load(f)
    assert [e["key"] for e in doc["entries"]] == [key]
    second = Curveball(g.row_ptr, g.col, 7)
    assert second.tune_key() == key
    again = second.autotune(20, cache_path=path)
    assert again["steps"] == 0 and second.step == 0
    for name in ("tile_max", "block_max", "smem_max", "inorder_threads", "retry_passes"):
        assert again[name] == got[name], name
    o = Oracle(g.row_ptr, g.col, 7)
    second.global_trades(3)
    o.superstep(3)
    assert np.array_equal(second.edges(), o.edges())
    # a batch of the same graphs has its own key (graph count)
    ens = Ensemble([(g.row_ptr, g.col)] * 4, [1, 2, 3, 4])
    assert ens.tune_key() != key


def test_batch_rejects_out_of_range_local_ids():
    good = _csr([(0, 1), (1, 2)], 3)
    bad_rp = np.array([0, 1, 2], dtype=np.int64)
    bad_col = np.array([1, 2], dtype=np.int32)   # id 2 is outside a 2-node graph
    with pytest.raises(CbError) as e:
        Ensemble([good, (bad_rp, bad_col)], [1, 2])
    assert e.value.code == CB_EINVAL


def test_batch_rejects_asymmetric_graph():
    good = _csr([(0, 1)], 2)
    rp = np.array([0, 1, 2, 2], dtype=np.int64)   # 0 -> 1 and 1 -> 2, neither mirrored
    col = np.array([1, 2], dtype=np.int32)
    with pytest.raises(CbError) as e:
        Ensemble([good, (rp, col)], [1, 2])
    assert e.value.code == CB_EINVAL


ENSEMBLE_GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "ensemble_256.json")


@pytest.mark.skipif(not os.path.exists(ENSEMBLE_GOLDEN), reason="ensemble golden not generated")
def test_full_ensemble_matches_oracle_hashes():
    """The whole batched-ensemble workload (256 graphs, 50 super steps) in one
    handle, against the oracle's per-graph hashes after steps 1, 10 and 50.
    The autotuner runs in the middle of the chain (its steps are real)."""
    with open(ENSEMBLE_GOLDEN) as f:
        gold = json.load(f)["graphs"]
    graphs, seeds = [], []
    for i in range(256):
        w = synth.ensemble_member(i)
        g = w.graph()
        assert g.m == gold[i]["m"]
        graphs.append((g.row_ptr, g.col))
        seeds.append(w.chain_seed)
    ens = Ensemble(graphs, seeds)
    ens.set_option("cuda_graph", 1)

    def check(step):
        for i in range(256):
            assert edge_hash(ens.graph_edges(i)) == gold[i]["edge_sha256_after_step"][str(step)], \
                f"graph {i} after super step {step}"

    ens.global_trades(1)
    check(1)
    ens.global_trades(9)
    check(10)
    tuned = ens.autotune(12)
    assert 1 <= tuned["steps"] <= 12 and ens.step == 10 + tuned["steps"]
    ens.set_option("cuda_graph", 1)
    ens.global_trades(50 - ens.step)
    assert ens.step == 50
    check(50)
