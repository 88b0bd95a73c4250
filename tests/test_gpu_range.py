"""GPU range search against the oracle: per query the same point set, except
points whose squared distance lies within 1e-5 relative of radius^2 (float32
versus float64 rounding at the boundary), which may fall either way."""
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


def _check(data, queries, radius, idx, offs, rows=None):
    want = oracle.range_search(data, queries if rows is None else queries[rows], radius)
    r2 = float(np.float32(radius)) ** 2
    p64 = data.astype(np.float64)
    for w, i in enumerate(range(len(queries)) if rows is None else rows):
        got = idx[offs[i]:offs[i + 1]]
        assert len(set(got.tolist())) == len(got)                     # no point twice
        d = ((p64 - queries[i].astype(np.float64)) ** 2).sum(1)
        loose = np.abs(d - r2) <= 1e-5 * max(r2, 1e-30)
        diff = set(got.tolist()) ^ set(want[w].tolist())
        assert all(loose[x] for x in diff), (i, sorted(diff)[:5])


@pytest.mark.parametrize("n,d,r,kind", [(30000, 2, 0.01, "uniform"), (20000, 3, 0.04, "gmm"), (8000, 5, 0.15, "uniform"),
                                        (5000, 16, 0.6, "gmm")])
def test_range_separate_queries(api, n, d, r, kind):
    pts = synth.uniform(n, d, 81 + d) if kind == "uniform" else synth.gmm(n, d, 82 + d)
    q = synth.uniform(6000, d, 83 + d)            # >= 4096: the leaf-ordered path
    t = api.pg_tree_build(_cuda(pts), leaf_size=16)
    idx, offs = api.pg_range(t, _cuda(q), r)
    t.free()
    _check(pts, q, r, idx.cpu().numpy(), offs.cpu().numpy(), rows=synth.pick_rows(len(q), 500, 84))


def test_range_all_points_and_determinism(api):
    pts = synth.gmm(25000, 3, 85)
    t = api.pg_tree_build(_cuda(pts), leaf_size=32)
    a = api.pg_range(t, None, 0.02)
    b = api.pg_range(t, None, 0.02)
    t.free()
    assert torch.equal(a[0], b[0]) and torch.equal(a[1], b[1])
    idx, offs = a[0].cpu().numpy(), a[1].cpu().numpy()
    for i in synth.pick_rows(len(pts), 400, 86):
        assert i in idx[offs[i]:offs[i + 1]]                            # every point finds itself
    _check(pts, pts, 0.02, idx, offs, rows=synth.pick_rows(len(pts), 300, 87))


def test_range_lattice_exact_and_edge_cases(api):
    pts = synth.lattice((30, 20))
    t = api.pg_tree_build(_cuda(pts), leaf_size=8)
    idx, offs = api.pg_range(t, None, 1.0)
    idx, offs = idx.cpu().numpy(), offs.cpu().numpy()
    want = oracle.range_search(pts, pts, 1.0)                           # exact: integer coordinates
    for i in range(len(pts)):
        assert sorted(idx[offs[i]:offs[i + 1]].tolist()) == want[i].tolist()
    z, zo = api.pg_range(t, _cuda(pts[:10] + 0.5), 0.0)                 # radius 0 off-lattice: nothing
    assert z.numel() == 0 and zo.cpu().numpy().tolist() == [0] * 11
    big, bo = api.pg_range(t, _cuda(pts[:3]), 1e6)                      # everything
    assert bo.cpu().numpy().tolist() == [0, 600, 1200, 1800]
    t.free()


def test_range_errors(api):
    import ctypes as C
    from paper_2207_01834_gb300._lib import PG_EINVAL, PgError, call

    pts = synth.uniform(3000, 3, 88)
    t = api.pg_tree_build(_cuda(pts), leaf_size=16)
    offs = torch.empty(3001, dtype=torch.int64, device="cuda")
    total = C.c_int64()
    for bad in (-1.0, float("inf"), float("nan")):
        with pytest.raises(PgError) as e:
            call("pg_range", t.handle, None, 3000, bad, 0, None, offs.data_ptr(), C.byref(total), None)
        assert e.value.status == PG_EINVAL
    call("pg_range", t.handle, None, 3000, 0.1, 0, None, offs.data_ptr(), C.byref(total), None)
    assert total.value > 3000
    out = torch.empty(total.value - 1, dtype=torch.int32, device="cuda")
    with pytest.raises(PgError) as e:
        call("pg_range", t.handle, None, 3000, 0.1, total.value - 1, out.data_ptr(), offs.data_ptr(), C.byref(total),
             None)
    assert e.value.status == PG_EINVAL
    t.free()


def test_range_fill_matches_one_call_and_rejects_foreign_offsets(api):
    import ctypes as C
    from paper_2207_01834_gb300._lib import PG_EINVAL, PgError, call

    pts = synth.gmm(20000, 3, 89)
    q = _cuda(synth.uniform(5000, 3, 90))        # >= 4096: the leaf-ordered path
    t = api.pg_tree_build(_cuda(pts), leaf_size=16)
    offs = torch.empty(5001, dtype=torch.int64, device="cuda")
    total = C.c_int64()
    call("pg_range", t.handle, q.data_ptr(), 5000, 0.05, 0, None, offs.data_ptr(), C.byref(total), None)
    n = total.value
    assert n > 5000
    one = torch.full((n,), -7, dtype=torch.int32, device="cuda")
    offs1 = torch.empty_like(offs)
    call("pg_range", t.handle, q.data_ptr(), 5000, 0.05, n, one.data_ptr(), offs1.data_ptr(), C.byref(total), None)
    two = torch.full((n,), -7, dtype=torch.int32, device="cuda")
    call("pg_range_fill", t.handle, q.data_ptr(), 5000, 0.05, offs.data_ptr(), n, two.data_ptr(), None)
    assert torch.equal(offs, offs1) and torch.equal(one, two)      # same rows, same order
    # offsets of a smaller radius used with a larger one: rows overflow their
    # offsets; the call reports it and writes nothing at or above capacity
    small = torch.empty_like(offs)
    call("pg_range", t.handle, q.data_ptr(), 5000, 0.02, 0, None, small.data_ptr(), C.byref(total), None)
    ns = total.value
    buf = torch.full((ns + 64,), -7, dtype=torch.int32, device="cuda")
    with pytest.raises(PgError) as e:
        call("pg_range_fill", t.handle, q.data_ptr(), 5000, 0.05, small.data_ptr(), ns, buf.data_ptr(), None)
    assert e.value.status == PG_EINVAL
    assert bool((buf[ns:] == -7).all())
    # capacity below the last offset: reported, nothing written at or above it
    with pytest.raises(PgError) as e:
        call("pg_range_fill", t.handle, q.data_ptr(), 5000, 0.05, offs.data_ptr(), n - 10, two.data_ptr(), None)
    assert e.value.status == PG_EINVAL
    t.free()
