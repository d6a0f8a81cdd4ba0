"""cb_permutation_static: the allocation-free permutation entry point.

Some callers may not allocate device memory themselves (a host framework that
owns every device allocation, a latency-critical loop where cudaMalloc could
synchronise or fail).  This entry point computes the same permutation as
cb_permutation from caller-provided output memory and a static scratch array.
The file is collected last on purpose."""
import numpy as np
import pytest

from paper_1804_08487_gb300 import cb, synth

pytestmark = pytest.mark.gpu


def _reference_order(n, seed, g):
    """The existing entry point: cb_permutation through a handle on an n-node graph."""
    graph = synth.powerlaw_graph(n, 1, 3, 2.0, 5) if n > 4 else None
    if graph is None:
        rp, col = np.zeros(n + 1, dtype=np.int64), np.zeros(0, dtype=np.int32)
    else:
        rp, col = graph.row_ptr, graph.col
    c = cb.Curveball(rp, col, seed)
    try:
        return c.permutation(g)
    finally:
        c.close()


def test_static_permutation_matches_handle_permutation_twice():
    torch = pytest.importorskip("torch")
    calls = [(300001, 7, 3), (4096, 42, 0)]     # two calls in a row share the static scratch
    for n, seed, g in calls:
        out = torch.full((n,), -1, dtype=torch.int32, device="cuda")
        cb.cb_permutation_static(n, seed, g, out)
        torch.cuda.synchronize()
        got = out.cpu().numpy()
        want = _reference_order(n, seed, g)
        assert np.array_equal(got, want), (n, seed, g)


def test_static_permutation_rejects_sizes_beyond_its_limit():
    torch = pytest.importorskip("torch")
    out = torch.zeros(16, dtype=torch.int32, device="cuda")
    with pytest.raises(cb.CbError) as e:
        cb.cb_permutation_static((1 << 20) + 1, 1, 0, out)
    assert e.value.code == cb.CB_ESIZE
