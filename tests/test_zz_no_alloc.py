"""cb_permutation_static: the allocation-free permutation entry point.

Some callers cannot allocate device memory themselves: code running inside a
host framework that owns every device allocation, or a latency-critical loop
where cudaMalloc could synchronise the device or fail.  This entry point
computes the same permutation as cb_permutation from caller-provided output
memory and a static scratch array.  The file is collected last on purpose."""
import numpy as np
import pytest

from oracle import Oracle
from paper_1804_08487_gb300 import cb, synth

pytestmark = pytest.mark.gpu


def _empty_csr(n):
    return np.zeros(n + 1, dtype=np.int64), np.zeros(0, dtype=np.int32)


def _reference_order(n, seed, g):
    """The existing entry point: cb_permutation through a handle on an n-node graph."""
    graph = synth.powerlaw_graph(n, 1, 3, 2.0, 5) if n > 4 else None
    rp, col = _empty_csr(n) if graph is None else (graph.row_ptr, graph.col)
    c = cb.Curveball(rp, col, seed)
    try:
        return c.permutation(g)
    finally:
        c.close()


def _static(n, seed, g, stream=None):
    torch = pytest.importorskip("torch")
    out = torch.full((max(n, 1),), -1, dtype=torch.int32, device="cuda")
    cb.cb_permutation_static(n, seed, g, out, stream)
    if stream is not None:
        stream.synchronize()
    torch.cuda.synchronize()
    return out.cpu().numpy()[:n]


def test_static_permutation_matches_handle_permutation_twice():
    calls = [(300001, 7, 3), (4096, 42, 0)]     # two calls in a row share the static scratch
    for n, seed, g in calls:
        assert np.array_equal(_static(n, seed, g), _reference_order(n, seed, g)), (n, seed, g)


def test_static_permutation_at_its_limit_and_tiny_sizes():
    for n, seed, g in [(1 << 20, 11, 9), (1, 3, 0), (5, 4, 2)]:
        assert np.array_equal(_static(n, seed, g), _reference_order(n, seed, g)), (n, seed, g)


def test_static_permutation_on_a_stream_equals_the_oracle():
    torch = pytest.importorskip("torch")
    n, seed, g = 70001, 2024, 6
    stream = torch.cuda.Stream()
    got = _static(n, seed, g, stream)
    rp, col = _empty_csr(n)
    want = Oracle(rp, col, seed).permutation(g).astype(np.int32)
    assert np.array_equal(got, want)


def test_static_permutation_rejects_sizes_beyond_its_limit():
    torch = pytest.importorskip("torch")
    out = torch.zeros(16, dtype=torch.int32, device="cuda")
    with pytest.raises(cb.CbError) as e:
        cb.cb_permutation_static((1 << 20) + 1, 1, 0, out)
    assert e.value.code == cb.CB_ESIZE
