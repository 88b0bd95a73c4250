"""GPU parity of the static kd-tree path: build invariants and k-NN against the
CPU oracle, called through the C ABI (via the thin binding)."""
from __future__ import annotations

import numpy as np
import pytest

import oracle
from knn_compare import compare_knn
from oracle.kdtree_check import check_tree
from paper_2207_01834_gb300 import synth

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def api():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2207_01834_gb300 import api as a
    return a


@pytest.fixture(params=[1, 2, 3, 4, 5], ids=["thread", "packet", "postponed", "warp", "postponed-heap"])
def variant(api, request):
    """This thread's traversal override for the test's PG_KNN_AUTO calls."""
    api.pg_knn_set_variant(request.param)
    yield request.param
    api.pg_knn_set_variant(0)


def _cuda(x):
    return torch.from_numpy(np.ascontiguousarray(x)).cuda()


def _chain_1d(n):
    # x_i = 2^-i: every midpoint split peels one point off, so the tree hits the depth cap
    return (2.0 ** -np.arange(n, dtype=np.float64)).astype(np.float32)[:, None]


TREE_CASES = {
    "uniform2d": (lambda: synth.uniform(20000, 2, 1), 16),
    "uniform3d_leaf8": (lambda: synth.uniform(50000, 3, 2), 8),
    "gmm5d_leaf32": (lambda: synth.gmm(30000, 5, 3), 32),
    "gmm7d": (lambda: synth.gmm(30000, 7, 4), 16),
    "dim1": (lambda: synth.uniform(5000, 1, 5), 4),
    "dim10": (lambda: synth.uniform(8000, 10, 6), 16),
    "dim16": (lambda: synth.gmm(8000, 16, 7), 16),
    "all_equal": (lambda: np.full((1000, 3), 0.25, np.float32), 16),
    "collinear": (lambda: np.repeat(synth.uniform(3000, 1, 8), 3, axis=1), 16),
    "one_point": (lambda: synth.uniform(1, 3, 9), 16),
    "below_leaf": (lambda: synth.uniform(5, 3, 10), 16),
    "duplicates": (lambda: np.repeat(synth.uniform(500, 3, 11), 7, axis=0), 4),
    "lattice3d": (lambda: synth.lattice((20, 20, 20)), 16),
    "depth_cap_chain": (lambda: _chain_1d(120), 1),
    "leaf1": (lambda: synth.uniform(3000, 2, 12), 1),
    "negative_coords": (lambda: synth.uniform(4000, 3, 13) - 0.5, 16),
    # several hundred 2048-point partition tiles: the upper levels' segments
    # span many tiles, so the carry into a tile is found across look-back windows
    "uniform3d_600k_leaf48": (lambda: synth.uniform(600000, 3, 14), 48),
    "gmm3d_400k_leaf16": (lambda: synth.gmm(400000, 3, 15), 16),
}


@pytest.mark.parametrize("case", sorted(TREE_CASES))
def test_tree_invariants(api, case):
    make, leaf = TREE_CASES[case]
    pts = make()
    tree = api.pg_tree_build(_cuda(pts), leaf_size=leaf)
    exp = tree.export()
    st = check_tree(pts, exp, leaf_size=leaf, depth_cap=48)
    assert exp["depth"] == st["depth"]
    if case == "all_equal":
        assert st["leaves"] == 1
    if case == "depth_cap_chain":
        assert st["depth"] == 48
    tree.free()


OBJECT_CASES = ["uniform2d", "uniform3d_leaf8", "gmm5d_leaf32", "gmm7d", "dim1", "dim16", "all_equal",
                "collinear", "one_point", "below_leaf", "duplicates", "lattice3d", "depth_cap_chain", "leaf1"]


@pytest.mark.parametrize("case", OBJECT_CASES)
def test_object_median_tree_invariants(api, case):
    make, leaf = TREE_CASES[case]
    pts = make()
    tree = api.pg_tree_build_split(_cuda(pts), leaf_size=leaf, split_rule=api.SPLIT_OBJECT)
    exp = tree.export()
    st = check_tree(pts, exp, leaf_size=leaf, depth_cap=48, split="object")
    assert exp["depth"] == st["depth"]
    if len(pts) > 1 and case not in ("all_equal",):
        # balanced: depth at most ceil(log2(n / leaf)) + 1
        assert st["depth"] <= int(np.ceil(np.log2(max(len(pts) / leaf, 1)))) + 1
    tree.free()


@pytest.mark.parametrize("v", [1, 2, 3])
def test_object_median_knn_equals_spatial(api, v):
    """k-NN answers do not depend on the split rule: bit-identical outputs."""
    pts = synth.gmm(60000, 3, 44)
    q = synth.gmm(8000, 3, 45)
    ts = api.pg_tree_build(_cuda(pts), leaf_size=16)
    to = api.pg_tree_build_split(_cuda(pts), leaf_size=16, split_rule=api.SPLIT_OBJECT)
    api.pg_knn_set_variant(v)
    try:
        for a, b in zip(api.pg_knn(ts, _cuda(q), 9) + api.pg_knn(ts, None, 6),
                        api.pg_knn(to, _cuda(q), 9) + api.pg_knn(to, None, 6)):
            assert torch.equal(a, b)
    finally:
        api.pg_knn_set_variant(0)
    ts.free()
    to.free()


def test_empty_tree(api):
    tree = api.pg_tree_build(torch.zeros((0, 3), device="cuda"), leaf_size=16)
    q = _cuda(synth.uniform(10, 3, 1))
    idx, dist = api.pg_knn(tree, q, 4)
    assert torch.all(idx == -1) and torch.all(torch.isinf(dist))


def test_all_knn_2d_20k_k5_full(api, variant):
    """2D all-kNN: n = 20,000 uniform points, leaf 16, k = 5, self included;
    every row checked against the oracle."""
    pts = synth.uniform(20000, 2, synth.BASE_SEED)
    tree = api.pg_tree_build(_cuda(pts), leaf_size=16)
    idx, dist = api.pg_knn(tree, None, 5)
    # separate queries equal to the points take the leaf-ordered path
    qi, qd = api.pg_knn(tree, _cuda(pts), 5)
    assert torch.equal(qi, idx) and torch.equal(qd, dist)
    o_idx, o_dist = oracle.knn(pts, pts, 5, nthreads=0)
    compare_knn(idx.cpu().numpy(), dist.cpu().numpy(), o_idx, o_dist, pts, pts)
    # self first (no duplicates in this set)
    assert np.array_equal(idx[:, 0].cpu().numpy(), np.arange(20000))


QUERY_CASES = [
    (1, 3, "uniform"), (2, 1, "uniform"), (2, 7, "gmm"), (3, 10, "uniform"), (3, 16, "gmm"),
    (3, 64, "uniform"), (4, 2, "gmm"), (5, 16, "gmm"), (6, 5, "uniform"), (7, 16, "gmm"),
    (8, 33, "uniform"), (10, 9, "gmm"), (16, 12, "uniform"), (16, 64, "gmm"), (3, 4, "gmm"),
]


@pytest.mark.parametrize("d,k,dist_name", QUERY_CASES)
def test_knn_separate_queries(api, variant, d, k, dist_name):
    gen = synth.uniform if dist_name == "uniform" else synth.gmm
    pts = gen(12000, d, 100 + d)
    q = gen(1500, d, 200 + d)
    tree = api.pg_tree_build(_cuda(pts), leaf_size=16)
    idx, dist = api.pg_knn(tree, _cuda(q), k)
    o_idx, o_dist = oracle.knn(pts, q, k, nthreads=0)
    compare_knn(idx.cpu().numpy(), dist.cpu().numpy(), o_idx, o_dist, pts, q)


def test_knn_lattice_exact(api, variant):
    """Integer lattice: all distances are exact in float32, so the answer must
    equal the oracle's bit for bit, ties broken by the smaller index."""
    pts = synth.lattice((24, 20, 16))
    tree = api.pg_tree_build(_cuda(pts), leaf_size=8)
    idx, dist = api.pg_knn(tree, None, 11)
    o_idx, o_dist = oracle.knn(pts, pts, 11, nthreads=0)
    assert np.array_equal(idx.cpu().numpy(), o_idx)
    assert np.array_equal(dist.cpu().numpy().astype(np.float64), o_dist)


@pytest.mark.parametrize("copies", [6, 20])   # 20: a list of 32 slots (a heap for the heap traversal)
def test_knn_duplicates_prefer_small_ids(api, variant, copies):
    base = synth.uniform(300, 3, 21)
    pts = np.concatenate([base] * copies)         # copies, ids i, i+300, ...
    tree = api.pg_tree_build(_cuda(pts), leaf_size=4)
    idx, dist = api.pg_knn(tree, _cuda(base), copies)
    want = np.arange(300)[:, None] + 300 * np.arange(copies)[None, :]
    assert np.array_equal(idx.cpu().numpy(), want)
    assert torch.all(dist == 0)


@pytest.mark.parametrize("k", [10, 40])
def test_knn_padding(api, variant, k):
    pts = synth.uniform(3, 3, 22)
    tree = api.pg_tree_build(_cuda(pts), leaf_size=16)
    idx, dist = api.pg_knn(tree, _cuda(synth.uniform(5, 3, 23)), k)
    idx = idx.cpu().numpy()
    assert np.all(idx[:, 3:] == -1) and torch.all(torch.isinf(dist[:, 3:]))
    assert np.all(np.sort(idx[:, :3], axis=1) == np.arange(3))


def test_variants_agree_bitwise(api):
    """Every traversal variant returns the exact k smallest (float32 distance,
    id) pairs, so their outputs are identical."""
    pts = synth.gmm(60000, 3, 41)
    q = synth.gmm(20000, 3, 42)
    tree = api.pg_tree_build(_cuda(pts), leaf_size=16)
    outs = []
    for v in api.KNN_VARIANTS:
        api.pg_knn_set_variant(v)
        outs.append(api.pg_knn(tree, _cuda(q), 12) + api.pg_knn(tree, None, 7) + api.pg_knn(tree, None, 40))
    api.pg_knn_set_variant(0)
    for other in outs[1:]:
        for a, b in zip(outs[0], other):
            assert torch.equal(a, b)


def test_touch_counting_instance_same_answer(api):
    """The counting instance of the postponed-leaf traversal returns the same
    bits, and its counts are plausible: every query loads at least k bucket
    entries (its list must fill) and at most two loads per entry (test and
    insertion), and a read resets them."""
    pts = synth.gmm(40000, 3, 43)
    k = 10
    tree = api.pg_tree_build(_cuda(pts), leaf_size=32)
    api.pg_knn_set_variant(3)
    try:
        ref = api.pg_knn(tree, None, k)
        api.pg_knn_touch_read()
        api.pg_knn_touch_enable(True)
        got = api.pg_knn(tree, None, k)
        api.pg_knn_touch_enable(False)
        nrec, nent = api.pg_knn_touch_read()
        assert api.pg_knn_touch_read() == (0, 0)
    finally:
        api.pg_knn_touch_enable(False)
        api.pg_knn_set_variant(0)
    assert torch.equal(ref[0], got[0]) and torch.equal(ref[1], got[1])
    n = len(pts)
    assert n * k <= nent <= 2 * n * n
    assert n <= nrec <= n * tree.info().num_nodes


def test_knn_deterministic_and_stream(api):
    pts = synth.gmm(50000, 3, 31)
    s = torch.cuda.Stream()
    with torch.cuda.stream(s):
        t1 = api.pg_tree_build(_cuda(pts), leaf_size=16)
        a = api.pg_knn(t1, None, 10)
        t2 = api.pg_tree_build(_cuda(pts), leaf_size=16)
        b = api.pg_knn(t2, None, 10)
    s.synchronize()
    assert torch.equal(a[0], b[0]) and torch.equal(a[1], b[1])
    e1, e2 = t1.export(), t2.export()
    assert np.array_equal(e1["nodes"].view(np.uint32), e2["nodes"].view(np.uint32))
    assert np.array_equal(e1["bucket"].view(np.uint32), e2["bucket"].view(np.uint32))


def _sample_rows(m, count, seed):
    return np.sort(synth.pick_rows(m, min(count, m), seed))


def _check_all_knn_rows(idx, dist, n):
    """Properties every all-kNN row must have, checked on the device for all
    rows: ascending distances, the point itself first at distance 0 (uniform
    float32 points are distinct), indices in range and distinct."""
    assert torch.all(dist[:, 1:] >= dist[:, :-1])
    assert torch.all(dist[:, 0] == 0)
    assert torch.equal(idx[:, 0], torch.arange(n, dtype=torch.int32, device=idx.device))
    assert torch.all((idx >= 0) & (idx < n))
    srt = torch.sort(idx, dim=1).values
    assert torch.all(srt[:, 1:] != srt[:, :-1])


def test_all_knn_3d_10m_k10_sampled(api):
    """3D all-kNN at full size (n = 10,000,000, k = 10) for the leaf sizes the
    workload names ({8, 16, 32}, automatic traversal); sampled rows against
    the oracle, properties on all."""
    n = 10_000_000
    pts = synth.uniform(n, 3, synth.BASE_SEED + 2)
    x = _cuda(pts)
    for leaf in (8, 16, 32):
        tree = api.pg_tree_build(x, leaf_size=leaf)
        idx, dist = api.pg_knn(tree, None, 10)
        rows = _sample_rows(n, 400, leaf)
        o_idx, o_dist = oracle.knn(pts, pts[rows], 10, nthreads=0)
        compare_knn(idx[rows].cpu().numpy(), dist[rows].cpu().numpy(), o_idx, o_dist, pts, pts[rows])
        _check_all_knn_rows(idx, dist, n)
        tree.free()
        del idx, dist


@pytest.mark.parametrize("leaf,var", [(48, 3), (64, 3), (32, 1), (48, 2), (48, 4)],
                         ids=["leaf48-postponed", "leaf64-postponed", "leaf32-thread", "leaf48-packet",
                              "leaf48-warp"])
def test_all_knn_3d_10m_k10_bench_config(api, leaf, var):
    """The benchmark's own workload and launch configuration: 10,000,000
    uniform 3D points (the benchmark's seed), all-kNN with k = 10, the leaf
    size and traversal named per call as the benchmark runs them; 512 sampled
    rows against the oracle, properties on every row."""
    n = 10_000_000
    pts = synth.uniform(n, 3, synth.BASE_SEED + 2)
    x = _cuda(pts)
    tree = api.pg_tree_build(x, leaf_size=leaf)
    idx, dist = api.pg_knn(tree, None, 10, variant=var)
    rows = _sample_rows(n, 512, 1000 + leaf + var)
    o_idx, o_dist = oracle.knn(pts, pts[rows], 10, nthreads=0)
    compare_knn(idx[rows].cpu().numpy(), dist[rows].cpu().numpy(), o_idx, o_dist, pts, pts[rows])
    _check_all_knn_rows(idx, dist, n)
    tree.free()


def test_per_call_variants_and_tune_table(api):
    """The traversal is chosen per call, per thread override, or by the tune
    table; every choice gives the same bits.  The counting instance (which
    runs only for the postponed-leaf kernel) shows which kernel ran."""
    import threading

    pts = synth.gmm(40000, 3, 47)
    tree = api.pg_tree_build(_cuda(pts), leaf_size=24)
    ref = api.pg_knn(tree, None, 10, variant=api.KNN_THREAD)
    for v in api.KNN_VARIANTS:
        got = api.pg_knn(tree, None, 10, variant=v)
        assert torch.equal(got[0], ref[0]) and torch.equal(got[1], ref[1])

    def counted(**kw):
        api.pg_knn_touch_read()
        api.pg_knn_touch_enable(True)
        try:
            out = api.pg_knn(tree, None, 10, **kw)
        finally:
            api.pg_knn_touch_enable(False)
        return out, api.pg_knn_touch_read()[1]

    try:
        api.pg_knn_tune_set(3, 10, True, api.KNN_THREAD)
        assert api.pg_knn_tune_get(3, 9, True) == api.KNN_THREAD       # same k class (9-10)
        out, cnt = counted()
        assert cnt == 0 and torch.equal(out[0], ref[0])
        api.pg_knn_tune_set(3, 10, True, api.KNN_POSTPONED)
        out, cnt = counted()
        assert cnt > 0 and torch.equal(out[0], ref[0])
        api.pg_knn_set_variant(api.KNN_THREAD)                        # this thread's override wins
        assert api.pg_knn_tune_get(3, 10, True) == api.KNN_THREAD
        out, cnt = counted()
        assert cnt == 0
        out, cnt = counted(variant=api.KNN_POSTPONED)                 # an explicit variant wins
        assert cnt > 0
        # another thread does not see this thread's override
        seen = {}
        th = threading.Thread(target=lambda: seen.setdefault("v", api.pg_knn_tune_get(3, 10, True)))
        th.start()
        th.join()
        assert seen["v"] == api.KNN_POSTPONED
    finally:
        api.pg_knn_set_variant(0)
        api.pg_knn_tune_set(3, 10, True, api.KNN_AUTO)
    with pytest.raises(api.PgError, match="variant"):
        api.pg_knn(tree, None, 10, variant=99)
    tree.free()


@pytest.mark.parametrize("d", [5, 7])
def test_gmm_2m_1m_queries_k16_sampled(api, variant, d):
    mix = synth.gmm_mixture(d, synth.BASE_SEED + 3)
    pts = synth.gmm_sample(2_000_000, mix, synth.BASE_SEED + 30 + d)
    q = synth.gmm_sample(1_000_000, mix, synth.BASE_SEED + 40 + d)
    tree = api.pg_tree_build(_cuda(pts), leaf_size=16)
    idx, dist = api.pg_knn(tree, _cuda(q), 16)
    rows = _sample_rows(len(q), 300, d)
    o_idx, o_dist = oracle.knn(pts, q[rows], 16, nthreads=0)
    compare_knn(idx[rows].cpu().numpy(), dist[rows].cpu().numpy(), o_idx, o_dist, pts, q[rows])
    assert torch.all(dist[:, 1:] >= dist[:, :-1])
