"""BDL forest updates that fail part-way, on the GPU, without a GPU fault.

The failure is made on the host: pg_debug_fail_alloc_after(n) makes the
library's n-th device allocation from then on return PG_ENOMEM before any
CUDA call.  Sweeping n over every allocation an update makes hits each of
its steps once.  An insert is all or nothing (the forest is as before the
call, ids included, and the retried insert ends where a clean run does); an
erase either fails before it removes anything or stands with its under-full
trees kept, and queries stay exact in every case."""
from __future__ import annotations

import numpy as np
import pytest

from oracle.bdl import BDLModel
from paper_2207_01834_gb300 import synth

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

X = 4096
SIZES = (10000, 7000, 5000)


@pytest.fixture(scope="module")
def api():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2207_01834_gb300 import api as a
    return a


def _cuda(x):
    return torch.from_numpy(np.ascontiguousarray(x, dtype=np.float32)).cuda()


def _state(f, q):
    st = f.structure()
    return (st["F"], tuple(int(v) for v in st["slot_live"]), st["buffer_live"], st["next_id"], f.size(),
            f.slot_of().tobytes()), f.knn(q, 10)


def _same(a, b):
    return a[0] == b[0] and all(torch.equal(x, y) for x, y in zip(a[1], b[1]))


def _batches():
    return [synth.uniform(n, 3, 800 + i) for i, n in enumerate(SIZES)]


def _grow(api, model=None):
    f = api.BDL(3, X, 16)
    for p in _batches():
        f.insert(_cuda(p))
        if model is not None:
            model.insert(p)
    return f


def test_failed_insert_changes_nothing(api):
    q = _cuda(synth.uniform(3000, 3, 811))
    extra = synth.uniform(9000, 3, 810)     # two full trees and a remainder: the cascade runs
    model = BDLModel(3, X)
    f = _grow(api, model)
    before = _state(f, q)
    failures = 0
    for n in range(1, 1000):
        api.debug_fail_alloc_after(n)
        try:
            f.insert(_cuda(extra))
            ok = True
        except api.PgError as e:
            ok = False
            assert e.status == 2, e          # PG_ENOMEM
        finally:
            api.debug_fail_alloc_after(0)
        if ok:
            break
        failures += 1
        assert _same(_state(f, q), before), n
    assert failures >= 10                  # the sweep reached allocations deep inside the tree builds
    model.insert(extra)
    clean = _grow(api)
    clean.insert(_cuda(extra))
    assert _same(_state(f, q), _state(clean, q))
    st = f.structure()
    assert st["F"] == model.F and st["next_id"] == model.next_id and f.size() == model.size()
    f.free()
    clean.free()


def test_failed_erase_is_exact_either_way(api):
    """Erasing most of one tree makes it under-full: its live points are
    reinserted.  A failure leaves the forest before the erase or after it
    (possibly without the reinsertion); the retry ends with the same live set
    as a clean run, and the forest still takes inserts."""
    q = _cuda(synth.uniform(3000, 3, 821))
    f0 = _grow(api)
    slot = f0.slot_of().astype(np.int64)
    f0.free()
    pts = np.concatenate(_batches())
    big = int(np.bincount(slot[slot >= 0]).argmax())
    mine = pts[slot == big]
    gone = mine[: len(mine) * 3 // 4]
    clean = _grow(api)
    pre = clean.knn(q, 10)
    clean.erase(_cuda(gone))
    post = clean.knn(q, 10)
    failures = 0
    for n in range(1, 1000):
        f = _grow(api)
        api.debug_fail_alloc_after(n)
        try:
            f.erase(_cuda(gone))
            ok = True
        except api.PgError as e:
            ok = False
            assert e.status == 2, e
        finally:
            api.debug_fail_alloc_after(0)
        if ok:
            got = f.knn(q, 10)
            assert torch.equal(got[0], post[0]) and torch.equal(got[1], post[1])
            f.free()
            break
        failures += 1
        got = f.knn(q, 10)
        assert (torch.equal(got[0], pre[0]) and torch.equal(got[1], pre[1])) or \
               (torch.equal(got[0], post[0]) and torch.equal(got[1], post[1])), n
        f.erase(_cuda(gone))                 # the retry
        got = f.knn(q, 10)
        assert torch.equal(got[0], post[0]) and torch.equal(got[1], post[1]), n
        f.insert(_cuda(synth.uniform(5000, 3, 830)))
        f.free()
    assert failures >= 3
    clean.free()
