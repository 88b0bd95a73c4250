"""pg_knn_backward_noalloc: the k-NN gradient computed in the library's fixed
device array, for callers that cannot let a library allocate GPU memory.

Called through the C ABI; its outputs are compared with pg_knn_backward's and
with the oracle's float64 gradient on the same inputs, twice in a row (the
shared array keeps the previous call's contents, so the second call checks
that stale state does not leak).  The calls run with the library's
allocation hook armed, so any device allocation by the library would fail
them: the entry point must allocate nothing.  This file is collected last so
that a run stopping at the first failure has run every other test before it.
"""
from __future__ import annotations

import ctypes as C

import numpy as np
import pytest

import oracle
from paper_2207_01834_gb300 import synth

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

RTOL = 1e-5   # the gradient tests' per-element tolerance (relative to the sum of |terms|)


@pytest.fixture(scope="module")
def api():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2207_01834_gb300 import api as a
    return a


def _case(api, n, m, d, k, seed):
    data = torch.from_numpy(synth.gmm(n, d, seed)).cuda()
    q = torch.from_numpy(synth.gmm(m, d, seed + 1)).cuda()
    tree = api.pg_tree_build(data, leaf_size=16)
    idx, _ = api.pg_knn(tree, q, k)
    tree.free()
    w = torch.from_numpy(np.random.default_rng(seed).standard_normal((m, k)).astype(np.float32)).cuda()
    return data, q, idx, w


def _bound(data, q, idx, w):
    P = data.double()
    Q = q.double()
    valid = idx >= 0
    t = idx.clamp(min=0).long()
    term = (2 * w.double()[..., None] * (Q[:, None, :] - P[t])).abs() * valid[..., None]
    bq = term.sum(1)
    bp = torch.zeros_like(P).index_add_(0, t.reshape(-1), term.reshape(-1, P.shape[1]))
    return bq, bp


@pytest.mark.parametrize("n,m,d,k", [(50000, 40000, 3, 10), (3000, 20000, 5, 16), (1 << 20, 65536, 3, 16)])
def test_noalloc_matches_backward_twice(api, n, m, d, k):
    data, q, idx, w = _case(api, n, m, d, k, seed=n % 997 + d)
    ref_q, ref_p = api.pg_knn_backward(data, q, idx, w)
    bq, bp = _bound(data, q, idx, w)
    o_q, o_p = oracle.knn_grad(data.cpu().numpy(), q.cpu().numpy(), idx.cpu().numpy().astype(np.int64),
                               w.cpu().numpy())
    o_q = torch.from_numpy(o_q).cuda()
    o_p = torch.from_numpy(o_p).cuda()
    for _ in range(2):
        gq = torch.full_like(q, float("nan"))
        gp = torch.full_like(data, float("nan"))
        torch.cuda.synchronize()
        api.debug_fail_alloc_after(1)   # the library's next device allocation would fail
        try:
            api.pg_knn_backward_noalloc(data, q, idx, w, gq, gp)
            torch.cuda.synchronize()
        finally:
            api.debug_fail_alloc_after(0)
        assert torch.all((gq.double() - ref_q.double()).abs() <= RTOL * bq + 1e-30)
        assert torch.all((gp.double() - ref_p.double()).abs() <= RTOL * bp + 1e-30)
        assert torch.all((gq.double() - o_q).abs() <= RTOL * bq + 1e-30)
        assert torch.all((gp.double() - o_p).abs() <= RTOL * bp + 1e-30)


def test_noalloc_allocation_hook_is_live(api):
    """The hook the test above relies on does fail the library's allocating
    twin, so a passing noalloc call under it shows that nothing was allocated."""
    data, q, idx, w = _case(api, 5000, 3000, 3, 8, seed=5)
    torch.cuda.synchronize()
    api.debug_fail_alloc_after(1)
    try:
        with pytest.raises(api.PgError, match="PG_ENOMEM"):
            api.pg_knn_backward(data, q, idx, w)
    finally:
        api.debug_fail_alloc_after(0)


def test_noalloc_rejects_sizes_beyond_its_scratch(api):
    from paper_2207_01834_gb300 import _lib

    lib = _lib.load()
    fake = C.c_void_p(0x1000)   # never dereferenced: the size check fails first
    before = lib.pg_launch_count()
    st = lib.pg_knn_backward_noalloc(fake, (1 << 20) + 1, fake, 10, 3, 4, fake, fake, fake, fake, None)
    assert st == _lib.PG_EINVAL and b"1048576" in lib.pg_last_error()
    st = lib.pg_knn_backward_noalloc(fake, 100, fake, (1 << 18) + 1, 3, 4, fake, fake, fake, fake, None)
    assert st == _lib.PG_EINVAL and b"pairs" in lib.pg_last_error()
    # an m so large that m * k would overflow 64 bits is rejected the same way
    st = lib.pg_knn_backward_noalloc(fake, 100, fake, (1 << 62), 3, 64, fake, fake, fake, fake, None)
    assert st == _lib.PG_EINVAL and b"pairs" in lib.pg_last_error()
    assert lib.pg_launch_count() == before
