"""Pins of the CPU oracle against facts fixed by the paper and the mathematics.

The oracle is trusted only after these pass.  None of them re-uses the oracle's
own arithmetic: the k-NN answer is checked against exact rational enumeration,
a closed form on an integer lattice and an independent library (scipy's
cKDTree); the gradient against float64 finite differences and torch autograd.
"""
from __future__ import annotations

import itertools
from fractions import Fraction

import numpy as np
import pytest

import oracle
from knn_compare import compare_knn
from paper_2207_01834_gb300 import synth


def _exact_knn_by_subsets(data, q, k, ids=None):
    """The k-NN set as the unique k-subset whose every member precedes every
    non-member in (exact rational squared distance, id) order."""
    n = len(data)
    ids = list(range(n)) if ids is None else list(ids)
    key = []
    for t in range(n):
        d = sum((Fraction(float(q[c])) - Fraction(float(data[t][c]))) ** 2 for c in range(len(q)))
        key.append((d, ids[t]))
    kk = min(k, n)
    winners = []
    for S in itertools.combinations(range(n), kk):
        rest = [t for t in range(n) if t not in S]
        if not rest or max(key[t] for t in S) < min(key[t] for t in rest):
            winners.append(S)
    assert len(winners) == 1
    S = sorted(winners[0], key=lambda t: key[t])
    return [ids[t] for t in S] + [-1] * (k - kk), [float(key[t][0]) for t in S] + [np.inf] * (k - kk)


@pytest.mark.parametrize("seed", range(6))
def test_knn_matches_exact_subset_enumeration(seed):
    g = np.random.default_rng(seed)
    n = int(g.integers(1, 9))
    d = int(g.integers(1, 4))
    k = int(g.integers(1, n + 2))
    # small integers: many exact ties, exercising the id tie-break
    data = g.integers(0, 3, size=(n, d)).astype(np.float32)
    queries = g.integers(0, 3, size=(4, d)).astype(np.float32)
    idx, dist = oracle.knn(data, queries, k)
    for r in range(len(queries)):
        want_idx, want_d = _exact_knn_by_subsets(data, queries[r], k)
        assert list(idx[r]) == want_idx
        assert np.allclose(dist[r], want_d, rtol=0, atol=0)
    # random reals: exact rational order
    data = g.random((n, d)).astype(np.float32)
    queries = g.random((3, d)).astype(np.float32)
    idx, dist = oracle.knn(data, queries, k)
    for r in range(len(queries)):
        want_idx, want_d = _exact_knn_by_subsets(data, queries[r], k)
        assert list(idx[r]) == want_idx
        np.testing.assert_allclose(dist[r], want_d, rtol=1e-14)


def test_knn_lattice_closed_form():
    """2D integer grid, k = 5, all-kNN: self at 0, then the 4 axis neighbours at
    distance exactly 1 in increasing id order (ids are row-major grid order)."""
    nx, ny = 20, 30
    pts = synth.lattice((nx, ny))
    idx, dist = oracle.knn(pts, pts, 5)
    for x in range(1, nx - 1):
        for y in range(1, ny - 1):
            me = x * ny + y
            nb = sorted([(x - 1) * ny + y, x * ny + y - 1, x * ny + y + 1, (x + 1) * ny + y])
            assert list(idx[me]) == [me] + nb
            assert list(dist[me]) == [0.0, 1.0, 1.0, 1.0, 1.0]
    # corner (0,0): self, then (0,1) id 1 and (1,0) id ny at 1, then (1,1) at 2,
    # then (0,2) id 2 and (2,0) id 2*ny at 4
    assert list(idx[0]) == [0, 1, ny, ny + 1, 2]
    assert list(dist[0]) == [0.0, 1.0, 1.0, 2.0, 4.0]


@pytest.mark.parametrize("d,k", [(2, 5), (3, 10), (5, 16), (7, 16)])
def test_knn_vs_scipy_ckdtree(d, k):
    """An independent library routine: scipy's exact kd-tree query."""
    spatial = pytest.importorskip("scipy.spatial")
    data = synth.uniform(3000, d, seed=11 + d)
    queries = synth.gmm(400, d, seed=5 + d)
    idx, dist = oracle.knn(data, queries, k, nthreads=4)
    sd, si = spatial.cKDTree(data.astype(np.float64)).query(queries.astype(np.float64), k=k)
    compare_knn(si.reshape(-1, k), (sd ** 2).reshape(-1, k), idx, dist, data, queries)


def test_knn_self_match_and_duplicates():
    data = synth.uniform(500, 3, seed=3)
    data[100] = data[7]                         # a duplicate with a larger index
    idx, dist = oracle.knn(data, data, 1)
    assert np.all(dist[:, 0] == 0.0)
    want = np.arange(500)
    want[100] = 7                               # tie at 0 broken by the smaller id
    assert np.array_equal(idx[:, 0], want)


def test_knn_padding_and_empty():
    data = synth.uniform(3, 2, seed=1)
    q = synth.uniform(4, 2, seed=2)
    idx, dist = oracle.knn(data, q, 5)
    assert np.all(idx[:, 3:] == -1) and np.all(np.isinf(dist[:, 3:]))
    assert np.all(idx[:, :3] >= 0)
    idx, dist = oracle.knn(np.zeros((0, 2), np.float32), q, 2)
    assert np.all(idx == -1) and np.all(np.isinf(dist))
    idx, dist = oracle.knn(data, np.zeros((0, 2), np.float32), 2)
    assert idx.shape == (0, 2)


def test_knn_live_mask_and_ids():
    data = synth.uniform(200, 3, seed=4)
    q = synth.uniform(50, 3, seed=5)
    live = np.ones(200, bool)
    live[::3] = False
    ids = np.arange(200, dtype=np.int64) * 10 + 7
    idx, dist = oracle.knn(data, q, 6, live=live, ids=ids)
    ref_idx, ref_dist = oracle.knn(data[live], q, 6)
    assert np.array_equal(idx, ids[live][ref_idx])
    assert np.array_equal(dist, ref_dist)


def test_knn_thread_count_does_not_change_result():
    data = synth.gmm(2000, 5, seed=9)
    q = synth.gmm(300, 5, seed=10)
    a = oracle.knn(data, q, 8, nthreads=1)
    b = oracle.knn(data, q, 8, nthreads=4)
    assert np.array_equal(a[0], b[0]) and np.array_equal(a[1], b[1])


# ---------------------------------------------------------------- gradients
def _fixed_selection(seed, n=60, m=25, d=3, k=4):
    g = np.random.default_rng(seed)
    data = g.random((n, d)).astype(np.float32)
    q = g.random((m, d)).astype(np.float32)
    idx, _ = oracle.knn(data, q, k)
    w = g.standard_normal((m, k))
    return data, q, idx, w


def test_grad_matches_torch_autograd():
    torch = pytest.importorskip("torch")
    data, q, idx, w = _fixed_selection(1)
    gq, gp = oracle.knn_grad(data, q, idx, w)
    P = torch.tensor(data, dtype=torch.float64, requires_grad=True)
    Q = torch.tensor(q, dtype=torch.float64, requires_grad=True)
    I = torch.tensor(idx)
    W = torch.tensor(w)
    L = (W * ((Q[:, None, :] - P[I]) ** 2).sum(-1)).sum()
    L.backward()
    np.testing.assert_allclose(gq, Q.grad.numpy(), rtol=1e-12, atol=1e-12)
    np.testing.assert_allclose(gp, P.grad.numpy(), rtol=1e-12, atol=1e-12)
    assert abs(oracle.knn_loss(data, q, idx, w) - float(L.detach())) < 1e-10


def test_grad_matches_central_differences():
    """With the selection frozen, L is quadratic in the coordinates, so float64
    central differences with h = 1e-4 are exact up to rounding."""
    data, q, idx, w = _fixed_selection(2, n=20, m=8, d=2, k=3)
    gq, gp = oracle.knn_grad(data, q, idx, w)
    h = 1e-4
    P = data.astype(np.float64)
    Q = q.astype(np.float64)
    for arr, grad in ((Q, gq), (P, gp)):
        for i in range(arr.shape[0]):
            for c in range(arr.shape[1]):
                keep = arr[i, c]
                arr[i, c] = keep + h
                lp = oracle.knn_loss(P, Q, idx, w)
                arr[i, c] = keep - h
                lm = oracle.knn_loss(P, Q, idx, w)
                arr[i, c] = keep
                assert abs((lp - lm) / (2 * h) - grad[i, c]) < 1e-8


def test_grad_ignores_padding():
    data = synth.uniform(2, 2, seed=8)
    q = synth.uniform(3, 2, seed=9)
    idx, _ = oracle.knn(data, q, 4)
    w = np.ones(idx.shape)
    gq, gp = oracle.knn_grad(data, q, idx, w)
    idx2 = idx[:, :2]
    gq2, gp2 = oracle.knn_grad(data, q, idx2, w[:, :2])
    assert np.array_equal(gq, gq2) and np.array_equal(gp, gp2)


def test_chamfer_special_cases():
    a = synth.uniform(50, 3, seed=1)
    off = np.array([0, 50])
    loss, iab, iba, ga, gb = oracle.chamfer(a, off, a.copy(), off, 1)
    assert loss[0] == 0.0 and np.all(ga == 0) and np.all(gb == 0)
    assert np.array_equal(iab[:, 0], np.arange(50))
    x = np.array([[0.0, 0.0, 0.0]], np.float32)
    y = np.array([[1.0, 2.0, 2.0]], np.float32)
    loss, _, _, ga, gb = oracle.chamfer(x, [0, 1], y, [0, 1], 1)
    assert loss[0] == 18.0                      # 2 * 9
    np.testing.assert_array_equal(ga, [[-4.0, -8.0, -8.0]])
    np.testing.assert_array_equal(gb, [[4.0, 8.0, 8.0]])


def test_chamfer_grad_matches_torch_autograd():
    torch = pytest.importorskip("torch")
    a, a_off, b, b_off = synth.cloud_pairs(2, seed=3, lo=40, hi=90)
    k = 3
    loss, iab, iba, ga, gb = oracle.chamfer(a, a_off, b, b_off, k)
    A = torch.tensor(a, dtype=torch.float64, requires_grad=True)
    B = torch.tensor(b, dtype=torch.float64, requires_grad=True)
    total = 0
    for i in range(2):
        Ai = A[a_off[i]:a_off[i + 1]]
        Bi = B[b_off[i]:b_off[i + 1]]
        total = total + ((Ai[:, None, :] - Bi[torch.tensor(iab[a_off[i]:a_off[i + 1]])]) ** 2).sum()
        total = total + ((Bi[:, None, :] - Ai[torch.tensor(iba[b_off[i]:b_off[i + 1]])]) ** 2).sum()
    total.backward()
    assert abs(float(total.detach()) - loss.sum()) < 1e-9 * max(1.0, loss.sum())
    np.testing.assert_allclose(ga, A.grad.numpy(), rtol=1e-10, atol=1e-12)
    np.testing.assert_allclose(gb, B.grad.numpy(), rtol=1e-10, atol=1e-12)


# ---------------------------------------------------------------- k-NN graph
def _graph_by_matrix(p, k):
    """Independent restatement: full float64 distance matrix, per row the k
    smallest (distance, index) over other indices, union of (min, max)."""
    p = np.asarray(p, np.float64)
    n = len(p)
    d = ((p[:, None, :] - p[None, :, :]) ** 2).sum(-1)
    edges = set()
    for i in range(n):
        order = sorted((d[i, j], j) for j in range(n) if j != i)
        for _, j in order[:k]:
            edges.add((min(i, j), max(i, j)))
    return np.array(sorted(edges), np.int64).reshape(-1, 2)


def test_knn_graph_hand_example():
    p = np.array([[0, 0], [1, 0], [3, 0], [6, 0], [10, 0]], np.float32)
    assert oracle.knn_graph(p, 1).tolist() == [[0, 1], [1, 2], [2, 3], [3, 4]]


def test_knn_graph_line_closed_form():
    # equally spaced line, k = 2: the path plus (0, 2) and (n-3, n-1)
    for n in (4, 7, 30):
        p = np.stack([np.arange(n), np.zeros(n)], 1).astype(np.float32)
        g = oracle.knn_graph(p, 2)
        want = sorted({(i, i + 1) for i in range(n - 1)} | {(0, 2), (n - 3, n - 1)})
        assert g.tolist() == [list(e) for e in want]
        assert len(g) == n + 1


def test_knn_graph_duplicates_and_tiny():
    p = np.zeros((3, 3), np.float32)
    assert oracle.knn_graph(p, 1).tolist() == [[0, 1], [0, 2]]
    assert oracle.knn_graph(p[:1], 3).shape == (0, 2)
    assert oracle.knn_graph(p[:2], 5).tolist() == [[0, 1]]


def test_knn_graph_matches_distance_matrix():
    rng = np.random.default_rng(5)
    for n, d, k in ((60, 2, 3), (80, 3, 5), (50, 5, 4)):
        p = rng.random((n, d)).astype(np.float32)
        assert np.array_equal(oracle.knn_graph(p, k), _graph_by_matrix(p, k))
        q = np.round(p * 4).astype(np.float32)       # many exact ties
        assert np.array_equal(oracle.knn_graph(q, k), _graph_by_matrix(q, k))


# ---------------------------------------------------------------- range search
def test_range_search_hand_example():
    p = np.array([[0, 0], [1, 0], [0, 2], [3, 4]], np.float32)
    got = oracle.range_search(p, np.array([[0, 0], [3, 3]], np.float32), 2.0)
    assert [g.tolist() for g in got] == [[0, 1, 2], [3]]          # |(3,4)-(3,3)| = 1; (0,2) is at sqrt(10)


def test_range_search_lattice_closed_form():
    # radius 1 on the integer grid: the point itself and its axis neighbours
    p = synth.lattice((7, 5))
    got = oracle.range_search(p, p, 1.0)
    for i, g in enumerate(got):
        x, y = p[i]
        want = 1 + (x > 0) + (x < 6) + (y > 0) + (y < 4)
        assert len(g) == want


def test_range_search_matches_cKDTree():
    spatial = pytest.importorskip("scipy.spatial")
    rng = np.random.default_rng(9)
    for n, d, r in ((2000, 2, 0.03), (1500, 3, 0.1), (800, 5, 0.3)):
        p = rng.random((n, d)).astype(np.float32)
        q = rng.random((200, d)).astype(np.float32)
        got = oracle.range_search(p, q, r)
        ref = spatial.cKDTree(p.astype(np.float64)).query_ball_point(q.astype(np.float64), float(np.float32(r)))
        for i in range(len(q)):
            dd = ((p.astype(np.float64) - q[i].astype(np.float64)) ** 2).sum(1)
            near = np.abs(dd - float(np.float32(r)) ** 2) <= 1e-9     # boundary cases may round either way
            a, b = set(got[i].tolist()), set(ref[i])
            assert {x for x in a ^ b if not near[x]} == set()
