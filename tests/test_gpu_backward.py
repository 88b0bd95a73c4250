"""GPU k-NN gradient (pg_knn_backward and the autograd wrapper) against the
oracle's closed-form float64 gradient and float64 central differences."""
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


def _cuda(x, dtype=np.float32):
    return torch.from_numpy(np.ascontiguousarray(x, dtype=dtype)).cuda()


def _bound(data, q, idx, w):
    """Per-element sum of |terms| of each gradient entry (float64): the float32
    result may differ from the exact one by a few ulp of this magnitude."""
    P = data.astype(np.float64)
    Q = q.astype(np.float64)
    m, k = idx.shape
    bq = np.zeros_like(Q)
    bp = np.zeros_like(P)
    for j in range(k):
        t = idx[:, j]
        ok = t >= 0
        term = np.abs(2 * w[ok, j][:, None] * (Q[ok] - P[t[ok]]))
        bq[ok] += term
        np.add.at(bp, t[ok], term)
    return bq, bp


def _check(got, want, bound, rtol=1e-5):
    err = np.abs(got.astype(np.float64) - want)
    assert np.all(err <= rtol * bound + 1e-30), float((err / (bound + 1e-30)).max())
    return float(err.max() / max(np.abs(want).max(), 1e-30))


@pytest.mark.parametrize("d,k,n,m", [(3, 10, 20000, 5000), (2, 1, 5000, 5000), (5, 16, 3000, 7000),
                                     (7, 8, 4000, 1000), (1, 3, 100, 2000), (16, 4, 2000, 500)])
def test_backward_matches_oracle(api, d, k, n, m):
    data = synth.gmm(n, d, 10 + d)
    q = synth.gmm(m, d, 20 + d)
    tree = api.pg_tree_build(_cuda(data), leaf_size=16)
    idx, _ = api.pg_knn(tree, _cuda(q), k)
    w = np.random.default_rng(d).standard_normal((m, k)).astype(np.float32)
    gq, gp = api.pg_knn_backward(_cuda(data), _cuda(q), idx, _cuda(w))
    idx_np = idx.cpu().numpy().astype(np.int64)
    oq, op = oracle.knn_grad(data, q, idx_np, w)
    bq, bp = _bound(data, q, idx_np, w)
    eq = _check(gq.cpu().numpy(), oq, bq)
    ep = _check(gp.cpu().numpy(), op, bp)
    print(f"d={d} k={k}: max rel err queries {eq:.2e} data {ep:.2e}")


def test_backward_padding_and_hubs(api):
    """k larger than n gives padding slots (skipped); every query sees the same
    few data points, so each data point sums thousands of contributions."""
    data = synth.uniform(6, 3, 1)
    q = synth.uniform(5000, 3, 2)
    tree = api.pg_tree_build(_cuda(data), leaf_size=4)
    idx, _ = api.pg_knn(tree, _cuda(q), 9)
    assert torch.all(idx[:, 6:] == -1)
    w = np.random.default_rng(3).standard_normal((5000, 9)).astype(np.float32)
    gq, gp = api.pg_knn_backward(_cuda(data), _cuda(q), idx, _cuda(w))
    idx_np = idx.cpu().numpy().astype(np.int64)
    oq, op = oracle.knn_grad(data, q, idx_np, w)
    bq, bp = _bound(data, q, idx_np, w)
    _check(gq.cpu().numpy(), oq, bq)
    _check(gp.cpu().numpy(), op, bp)
    # bitwise deterministic across runs
    gq2, gp2 = api.pg_knn_backward(_cuda(data), _cuda(q), idx, _cuda(w))
    assert torch.equal(gq, gq2) and torch.equal(gp, gp2)


def test_backward_deterministic_all_knn(api):
    data = synth.gmm(200000, 3, 5)
    x = _cuda(data)
    tree = api.pg_tree_build(x, leaf_size=16)
    idx, _ = api.pg_knn(tree, None, 8)
    w = _cuda(np.random.default_rng(4).standard_normal((200000, 8)))
    a = api.pg_knn_backward(x, x, idx, w)
    b = api.pg_knn_backward(x, x, idx, w)
    assert torch.equal(a[0], b[0]) and torch.equal(a[1], b[1])


def test_autograd_vs_finite_differences(api):
    """Chamfer-style loss through the autograd wrapper; float64 central
    differences (h = 1e-4) of the loss with the selection frozen."""
    from paper_2207_01834_gb300 import autograd

    a_np = synth.cloud(300, 3, 11)
    b_np = synth.cloud(250, 3, 12)
    a = _cuda(a_np).requires_grad_(True)
    b = _cuda(b_np).requires_grad_(True)
    k = 3
    dab, iab = autograd.knn_squared_distance(a, b, k)
    dba, iba = autograd.knn_squared_distance(b, a, k)
    loss = dab.sum() + dba.sum()
    loss.backward()
    iab_np = iab.cpu().numpy().astype(np.int64)
    iba_np = iba.cpu().numpy().astype(np.int64)
    ones_ab = np.ones(iab_np.shape)
    ones_ba = np.ones(iba_np.shape)

    def L(A, B):
        return oracle.knn_loss(B, A, iab_np, ones_ab) + oracle.knn_loss(A, B, iba_np, ones_ba)

    A = a_np.astype(np.float64)
    B = b_np.astype(np.float64)
    h = 1e-4
    fd_a = np.zeros_like(A)
    fd_b = np.zeros_like(B)
    for arr, fd in ((A, fd_a), (B, fd_b)):
        for i in range(0, arr.shape[0], 7):
            for c in range(3):
                keep = arr[i, c]
                arr[i, c] = keep + h
                lp = L(A, B)
                arr[i, c] = keep - h
                lm = L(A, B)
                arr[i, c] = keep
                fd[i, c] = (lp - lm) / (2 * h)
    ga = a.grad.cpu().numpy().astype(np.float64)
    gb = b.grad.cpu().numpy().astype(np.float64)
    rows_a = np.arange(0, A.shape[0], 7)
    rows_b = np.arange(0, B.shape[0], 7)
    err = max(np.abs(ga[rows_a] - fd_a[rows_a]).max(), np.abs(gb[rows_b] - fd_b[rows_b]).max())
    scale = max(np.abs(fd_a).max(), np.abs(fd_b).max())
    print(f"max |GPU - FD| / max |FD| = {err / scale:.2e}")
    assert err / scale < 1e-5
