"""Bounded device waits report CB_ETIMEOUT and leave the handle destroyable.

Every wait on the device is bounded in time (option "wait_ms"): a trade of
the in-order pass waiting for the trade it depends on, a bulk copy into
shared memory, the uniform-trade executor's run queue and inboxes.  Test
hooks make a wait run out without any fault: "hold_publish" stops trades from
publishing that their threshold is ready, "hold_trade" drops the messages to
one uniform trade so it never becomes runnable.  The kernels record the
error, give up every other wait and return; the call reports CB_ETIMEOUT.
"""
import time

import numpy as np
import pytest

from oracle import Oracle
from paper_1804_08487_gb300 import synth
from paper_1804_08487_gb300.cb import CB_ETIMEOUT, CbError, Curveball

pytestmark = pytest.mark.gpu


def _fresh_handle_still_works(g, seed):
    c = Curveball(g.row_ptr, g.col, seed)
    o = Oracle(g.row_ptr, g.col, seed)
    c.global_trades(2)
    o.superstep(2)
    assert np.array_equal(c.edges(), o.edges())
    c.close()


@pytest.mark.parametrize("opts", [{}, {"cta_paths": 0, "tile_paths": 0}, {"inorder_threads": 256}])
def test_dependency_wait_runs_out(opts):
    g = synth.powerlaw_graph(400, 60, 300, 2.0, 5)   # dense: many trades depend on earlier ones
    c = Curveball(g.row_ptr, g.col, 9)
    for k, v in opts.items():
        c.set_option(k, v)
    c.set_option("wait_ms", 20)
    c.set_option("hold_publish", 1)
    t0 = time.perf_counter()
    with pytest.raises(CbError) as e:
        c.global_trades(1)
        c.sync()
    assert e.value.code == CB_ETIMEOUT
    assert time.perf_counter() - t0 < 20.0
    with pytest.raises(CbError) as e2:          # the error stays latched on the handle
        c.global_trades(1)
    assert e2.value.code == CB_ETIMEOUT
    c.close()                                    # and the handle is released
    _fresh_handle_still_works(g, 9)


def test_uniform_executor_wait_runs_out():
    g = synth.powerlaw_graph(2000, 5, 100, 2.0, 3)
    c = Curveball(g.row_ptr, g.col, 4)
    c.set_option("wait_ms", 20)
    c.set_option("hold_trade", 0)
    t0 = time.perf_counter()
    with pytest.raises(CbError) as e:
        c.uniform_trades(1000)
        c.sync()
    assert e.value.code == CB_ETIMEOUT
    assert time.perf_counter() - t0 < 20.0
    c.close()
    _fresh_handle_still_works(g, 4)


def test_wait_option_range():
    g = synth.powerlaw_graph(100, 2, 10, 2.0, 1)
    c = Curveball(g.row_ptr, g.col, 1)
    for bad in (0, 600001):
        with pytest.raises(CbError):
            c.set_option("wait_ms", bad)
    c.set_option("wait_ms", 1000)
    c.global_trades(1)
    c.close()
