"""GPU k-NN graph (built on the all-kNN traversal) against the oracle's graph,
edge for edge: the edge list is integer output, so it must match exactly."""
from __future__ import annotations

import numpy as np
import pytest

import oracle
from paper_2207_01834_gb300 import synth

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def api():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2207_01834_gb300 import api as a
    return a


def _cuda(x):
    return torch.from_numpy(np.ascontiguousarray(x, dtype=np.float32)).cuda()


def _graph(api, pts, k, leaf=16):
    t = api.pg_tree_build(_cuda(pts), leaf_size=leaf)
    g = api.pg_knn_graph(t, k).cpu().numpy().astype(np.int64)
    t.free()
    return g


@pytest.mark.parametrize("n,d,k,kind", [(20000, 3, 10, "uniform"), (15000, 2, 5, "gmm"), (8000, 5, 8, "gmm"),
                                        (3000, 7, 16, "uniform")])
def test_graph_matches_oracle(api, n, d, k, kind):
    pts = synth.uniform(n, d, 61 + d) if kind == "uniform" else synth.gmm(n, d, 62 + d)
    got = _graph(api, pts, k)
    want = oracle.knn_graph(pts, k, nthreads=0)
    assert np.array_equal(got, want)


def test_graph_lattice_ties_exact(api):
    # integer lattice: float32 distances are exact, so ties break by index on both sides
    pts = synth.lattice((40, 30))
    for k in (1, 4, 6):
        assert np.array_equal(_graph(api, pts, k), oracle.knn_graph(pts, k))


def test_graph_duplicates_padding_and_tiny(api):
    dup = np.repeat(synth.uniform(50, 3, 71), 4, axis=0)            # every point four times
    assert np.array_equal(_graph(api, dup, 5), oracle.knn_graph(dup, 5))
    small = synth.uniform(6, 3, 72)                                 # k above n - 1: every pair
    assert np.array_equal(_graph(api, small, 10), oracle.knn_graph(small, 10))
    one = synth.uniform(1, 3, 73)
    assert _graph(api, one, 3).shape == (0, 2)


def test_graph_count_only_and_capacity(api):
    import ctypes as C
    from paper_2207_01834_gb300._lib import PG_EINVAL, PgError, call

    pts = synth.uniform(5000, 3, 74)
    t = api.pg_tree_build(_cuda(pts), leaf_size=16)
    cnt = C.c_int64()
    call("pg_knn_graph", t.handle, 6, 0, None, C.byref(cnt), None)
    want = oracle.knn_graph(pts, 6)
    assert cnt.value == len(want)
    out = torch.empty((len(want) - 1, 2), dtype=torch.int32, device="cuda")
    with pytest.raises(PgError) as e:
        call("pg_knn_graph", t.handle, 6, len(want) - 1, out.data_ptr(), C.byref(cnt), None)
    assert e.value.status == PG_EINVAL and cnt.value == len(want)
    t.free()
