"""The serving loop: requests admitted by a device-memory budget, resident on
their own streams, stepped together.  Each result must be bit-identical to
the same request run alone (the oracle, and a plain handle on the GPU):
the work is integer and the random streams depend only on (seed, step,
position), never on what else is resident."""
import time

import numpy as np
import pytest

from oracle import Oracle
from paper_1804_08487_gb300 import synth
from paper_1804_08487_gb300.cb import (CB_ENOMEM, CbError, Curveball, Server, cb_device_bytes,
                                       cb_estimate_bytes)
from tests import exact

pytestmark = pytest.mark.gpu


def _requests():
    """Mixed sizes and step counts, including odd n, no edges and one node."""
    reqs = []
    for i, (n, b, steps) in enumerate([(4096, 256, 5), (6001, 375, 9), (1 << 14, 1024, 3), (777, 48, 12),
                                       (12345, 700, 6), (3000, 187, 1), (9999, 600, 7), (5000, 300, 4)]):
        g = synth.powerlaw_graph(n, 4, b, 2.0 + 0.1 * i, 500 + i)
        reqs.append((g.row_ptr, g.col, 9000 + i, steps))
    reqs.append((*exact.to_csr(frozenset(), 5), 1, 3))
    reqs.append((*exact.to_csr(frozenset(), 1), 2, 2))
    reqs.append((*exact.to_csr(frozenset({(0, 1), (1, 2), (2, 3), (0, 3)}), 4), 3, 0))
    return reqs


def _drain(srv, ids, timeout_s=120):
    got = {}
    t_end = time.time() + timeout_s
    while len(got) < len(ids) and time.time() < t_end:
        for rid in srv.poll(timeout_ms=100):
            got[rid] = srv.result(rid)
    assert len(got) == len(ids), f"only {len(got)} of {len(ids)} requests finished"
    return got


def test_every_result_equals_the_request_alone():
    reqs = _requests()
    srv = Server(int(8e9), max_active=6, depth=2)
    ids = [srv.submit(rp, col, seed, steps) for rp, col, seed, steps in reqs]
    assert ids == list(range(len(reqs)))
    got = _drain(srv, ids)
    st = srv.stats()
    assert st["finished"] == len(reqs) and st["failed"] == 0
    assert st["steps_issued"] == sum(r[3] for r in reqs)
    assert st["reserved_bytes"] == 0 and st["resident"] == 0
    srv.close()
    for rid, (rp, col, seed, steps) in zip(ids, reqs):
        edges, times = got[rid]
        o = Oracle(rp, col, seed)
        o.superstep(steps)
        assert np.array_equal(edges, o.edges()), f"request {rid} differs from the oracle alone"
        assert times[0] <= times[1] <= times[2] <= times[3]
    # and from a plain handle on the GPU, alone
    rp, col, seed, steps = reqs[4]
    c = Curveball(rp, col, seed)
    c.global_trades(steps)
    assert np.array_equal(c.edges(), got[ids[4]][0])


def test_budget_limits_what_is_resident():
    reqs = _requests()[:6]
    one = max(cb_estimate_bytes(len(rp) - 1, int(rp[-1]), int(np.diff(rp).max(initial=0)))
              for rp, _, _, _ in reqs)
    budget = int(one * 1.5)   # never two of the largest at once
    srv = Server(budget, max_active=16, depth=2)
    ids = [srv.submit(rp, col, seed, steps) for rp, col, seed, steps in reqs]
    got = _drain(srv, ids)
    st = srv.stats()
    assert 0 < st["reserved_peak_bytes"] <= budget
    srv.close()
    for rid, (rp, col, seed, steps) in zip(ids, reqs):
        o = Oracle(rp, col, seed)
        o.superstep(steps)
        assert np.array_equal(got[rid][0], o.edges())


def test_request_above_the_budget_fails_alone():
    g = synth.powerlaw_graph(4096, 4, 256, 2.0, 1)
    srv = Server(1 << 20, max_active=4)   # 1 MiB: nothing fits
    rid = srv.submit(g.row_ptr, g.col, 1, 2)
    ids = []
    t_end = time.time() + 30
    while not ids and time.time() < t_end:
        ids = srv.poll(timeout_ms=100)
    assert ids == [rid]
    with pytest.raises(CbError) as e:
        srv.result(rid)
    assert e.value.code == CB_ENOMEM
    assert srv.stats()["failed"] == 1
    srv.close()


@pytest.mark.parametrize("n,b", [(4096, 256), (50001, 3000), (1 << 16, 20000)])
def test_estimate_covers_what_a_handle_takes(n, b):
    g = synth.powerlaw_graph(n, 4, b, 2.0, 3)
    est = cb_estimate_bytes(g.n, int(g.row_ptr[-1]), int(np.diff(g.row_ptr).max()))
    c = Curveball(g.row_ptr, g.col, 1)
    c.global_trades(2)
    c.edges()
    now, peak = cb_device_bytes(c.h)
    assert 0 < peak <= est, (peak, est)
    assert now <= peak
