"""GPU BDL-tree (log-structured forest) against the oracle's bookkeeping model
and brute-force k-NN over the live set."""
from __future__ import annotations

import os

import numpy as np
import pytest

import oracle
from knn_compare import compare_knn
from oracle.bdl import BDLModel
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


def _same_structure(forest, model: BDLModel):
    st = forest.structure()
    assert st["F"] == model.F, (bin(st["F"]), bin(model.F))
    sizes = model.slot_sizes()
    for i in range(64):
        assert st["slot_live"][i] == sizes.get(i, 0), (i, st["slot_live"][i], sizes.get(i, 0))
    assert st["buffer_live"] == len(model.buffer)
    assert st["next_id"] == model.next_id
    assert np.array_equal(forest.slot_of().astype(np.int64), model.slot_of())
    assert forest.size() == model.size()


def _knn_matches(forest, model: BDLModel, q, k):
    idx, dist = forest.knn(_cuda(q), k)
    pts, ids = model.live_arrays()
    o_idx, o_dist = oracle.knn(pts, q, k, ids=ids, nthreads=0)
    compare_knn(idx.cpu().numpy(), dist.cpu().numpy(), o_idx, o_dist, pts, q, ids=ids)


@pytest.mark.parametrize("X", [3, 4, 7])
def test_insert_worked_example(api, golden_dir, X):
    rows = []
    for line in open(os.path.join(golden_dir, "bdl_insert_worked_example.txt")):
        line = line.strip()
        if line and not line.startswith("#"):
            e, F, b = line.split("\t")
            rows.append((e, int(F), int(b)))
    f = api.BDL(2, X, leaf_size=2)
    model = BDLModel(2, X)
    for seed, (expr, F, buf) in enumerate(rows):
        pts = synth.uniform(eval(expr, {"X": X}), 2, seed)
        f.insert(_cuda(pts))
        model.insert(pts)
        st = f.structure()
        assert st["F"] == F and st["buffer_live"] == buf
        _same_structure(f, model)
    _knn_matches(f, model, synth.uniform(50, 2, 99), 3)


@pytest.mark.parametrize("dim,X,leaf", [(3, 64, 16), (2, 37, 4), (7, 50, 8)])
def test_random_history_matches_model(api, dim, X, leaf):
    g = np.random.default_rng(dim * 100 + X)
    f = api.BDL(dim, X, leaf_size=leaf)
    model = BDLModel(dim, X)
    q = synth.gmm(400, dim, 1234 + dim)
    for step in range(24):
        if step % 3 == 2 and model.size() > 0:
            live, ids = model.live_arrays()
            cnt = int(g.integers(1, max(2, int(len(ids) * 0.6))))
            sel = g.choice(len(ids), size=cnt, replace=False)
            er = live[sel]
            if step % 2:
                er = np.concatenate([er, synth.uniform(5, dim, step)])   # absent points are ignored
            f.erase(_cuda(er))
            model.erase(er)
        else:
            p = synth.gmm(int(g.integers(1, 5 * X)), dim, 10 * step + dim)
            ids = f.insert(_cuda(p), return_ids=True)
            want = model.insert(p)
            assert np.array_equal(ids.cpu().numpy(), want)
        _same_structure(f, model)
        model.check_invariants()
        _knn_matches(f, model, q, 10)


def test_erase_all_copies_and_everything(api):
    X = 16
    f = api.BDL(3, X, leaf_size=4)
    model = BDLModel(3, X)
    base = synth.uniform(100, 3, 5)
    pts = np.concatenate([base, base[:10]])          # ids 100..109 duplicate 0..9
    f.insert(_cuda(pts))
    model.insert(pts)
    f.erase(_cuda(base[:5]))
    model.erase(base[:5])
    _same_structure(f, model)
    assert f.size() == 100
    f.erase(_cuda(base))
    model.erase(base)
    _same_structure(f, model)
    assert f.size() == 0
    idx, dist = f.knn(_cuda(synth.uniform(7, 3, 6)), 4)
    assert torch.all(idx == -1) and torch.all(torch.isinf(dist))
    # the forest keeps working after being emptied
    more = synth.uniform(40, 3, 7)
    f.insert(_cuda(more))
    model.insert(more)
    _same_structure(f, model)
    _knn_matches(f, model, synth.uniform(30, 3, 8), 5)


def test_batch_dynamic_schedule_3d(api):
    """Batch-dynamic schedule at paper scale: 4,000,000 initial uniform 3D
    points, buffer 65,536, then [insert 1,000,000, insert 1,000,000,
    erase 500,000 uniformly chosen live points] x 5; after every batch
    1,000,000 uniform queries with k = 10 over the whole forest (sampled rows
    against brute force over the live set, properties on all rows)."""
    X = 65536
    f = api.BDL(3, X, leaf_size=16)
    g = np.random.default_rng(77)
    chunks = []
    live = np.zeros(0, bool)
    total = 0
    for b, (op, cnt) in enumerate(synth.bdl_schedule()):
        if op == "I":
            p = synth.uniform(cnt, 3, synth.BASE_SEED + 100 + b)
            f.insert(_cuda(p))
            chunks.append(p)
            live = np.concatenate([live, np.ones(cnt, bool)])
            total += cnt
        else:
            ids = np.nonzero(live)[0]
            sel = ids[g.choice(len(ids), size=cnt, replace=False)]
            allp = np.concatenate(chunks)
            f.erase(_cuda(allp[sel]))
            live[sel] = False
        st = f.structure()
        if b == 0:
            assert st["F"] == 0b111101 and st["buffer_live"] == 2304
        assert f.size() == int(live.sum())
        slot_of = f.slot_of()
        assert np.array_equal((slot_of != -1), live)
        counts = np.bincount(slot_of[slot_of >= 0].astype(np.int64), minlength=64)
        assert np.array_equal(counts, st["slot_live"])
        for i in range(64):
            if (st["F"] >> i) & 1:
                assert 2 * st["slot_live"][i] >= X << i
            else:
                assert st["slot_live"][i] == 0
        assert st["buffer_live"] < X
        q = synth.uniform(1_000_000, 3, synth.BASE_SEED + 500 + b)
        idx, dist = f.knn(_cuda(q), 10)
        assert torch.all(dist[:, 1:] >= dist[:, :-1])
        rows = np.sort(synth.pick_rows(len(q), 60, b))
        allp = np.concatenate(chunks)
        lid = np.nonzero(live)[0]
        o_idx, o_dist = oracle.knn(allp[lid], q[rows], 10, ids=lid, nthreads=0)
        compare_knn(idx[rows].cpu().numpy(), dist[rows].cpu().numpy(), o_idx, o_dist, allp[lid], q[rows], ids=lid)
        assert live[idx.cpu().numpy().ravel()].all()       # erased points are never returned


@pytest.mark.parametrize("m", [300, 20000])
def test_forest_variants_agree_bitwise(api, m):
    """kNN_L over a forest with erased points: every traversal variant returns
    the same bits (each is the exact k smallest pairs over the live set), and
    the answer matches brute force over the live set.  20,000 queries are
    processed in leaf order, 300 in input order."""
    X = 512
    f = api.BDL(3, X, leaf_size=16)
    model = BDLModel(3, X)
    for step in range(6):
        p = synth.gmm(3000 + 1500 * step, 3, 600 + step)
        f.insert(_cuda(p))
        model.insert(p)
        if step % 2:
            live, _ = model.live_arrays()
            er = live[np.random.default_rng(step).choice(len(live), size=len(live) // 5, replace=False)]
            f.erase(_cuda(er))
            model.erase(er)
    assert bin(f.structure()["F"]).count("1") >= 3
    q = synth.gmm(m, 3, 700)
    outs = [f.knn(_cuda(q), 10, variant=v) for v in api.KNN_VARIANTS]
    for got in outs[1:]:
        assert torch.equal(got[0], outs[0][0]) and torch.equal(got[1], outs[0][1])
    wide = [f.knn(_cuda(q), 24, variant=v) for v in api.KNN_VARIANTS]   # lists of 32 slots
    for got in wide[1:]:
        assert torch.equal(got[0], wide[0][0]) and torch.equal(got[1], wide[0][1])
    pts, ids = model.live_arrays()
    o_idx, o_dist = oracle.knn(pts, q, 10, ids=ids, nthreads=0)
    compare_knn(outs[-1][0].cpu().numpy(), outs[-1][1].cpu().numpy(), o_idx, o_dist, pts, q, ids=ids)


@pytest.mark.parametrize("d", [2, 7])
def test_k_sweep_forest_by_5pct_inserts(api, d):
    """The k-sweep workload: 10,000,000 points (2D clustered, 7D uniform)
    inserted in 20 batches of 5%, 1,000,000 of the points as queries; for
    k = 2..11 every answer is the prefix of the k = 11 answer, and sampled
    rows of k = 2 and k = 11 match brute force over all points."""
    pts = synth.ksweep_points(d)
    n = len(pts)
    x = _cuda(pts)
    f = api.BDL(d, 65536, 16)
    step = n // synth.KSWEEP_BATCHES
    for i in range(synth.KSWEEP_BATCHES):
        f.insert(x[i * step:(i + 1) * step] if i < synth.KSWEEP_BATCHES - 1 else x[i * step:])
    assert f.size() == n
    qrows = synth.ksweep_queries(n, d)
    q = x[torch.from_numpy(qrows.astype(np.int64)).cuda()]
    top_i, top_d = f.knn(q, 11)
    for k in synth.KSWEEP_KS:
        gi, gd = f.knn(q, k)
        assert torch.equal(gi, top_i[:, :k]) and torch.equal(gd, top_d[:, :k]), k
    rows = np.sort(synth.pick_rows(len(qrows), 48, 900 + d))
    ids = np.arange(n, dtype=np.int64)   # ids are assigned in insertion order
    for k in (2, 11):
        o_idx, o_dist = oracle.knn(pts, pts[qrows[rows]], k, nthreads=0)
        compare_knn(top_i[rows, :k].cpu().numpy(), top_d[rows, :k].cpu().numpy(), o_idx, o_dist, pts,
                    pts[qrows[rows]], ids=ids)
    f.free()
