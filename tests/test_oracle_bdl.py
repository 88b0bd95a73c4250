"""Pins of the BDL-tree bookkeeping model (oracle/bdl.py).

Pinned by: the paper's worked example of Insert_L (golden file), the closed
form of a pure-insert history (F = floor(N / X), buffer = N mod X, because
every insertion adds floor(|P|/X) plus the buffer carry to F), and the
invariants that Insert_L and Erase_L keep.
"""
from __future__ import annotations

import os

import numpy as np
import pytest

import oracle
from oracle.bdl import BDLModel
from paper_2207_01834_gb300 import synth


def _read_worked_example(path):
    rows = []
    for line in open(path):
        line = line.strip()
        if not line or line.startswith("#"):
            continue
        expr, F, buf = line.split("\t")
        rows.append((expr, int(F), int(buf)))
    return rows


@pytest.mark.parametrize("X", [3, 4, 7, 64])
def test_insert_worked_example(golden_dir, X):
    rows = _read_worked_example(os.path.join(golden_dir, "bdl_insert_worked_example.txt"))
    assert len(rows) == 4
    m = BDLModel(2, X)
    seed = 0
    for expr, F, buf in rows:
        size = eval(expr, {"X": X})          # expressions like "X+1" from the paper
        m.insert(synth.uniform(size, 2, seed=seed))
        seed += 1
        assert m.F == F and len(m.buffer) == buf
        m.check_invariants()


def test_pure_insert_closed_form():
    g = np.random.default_rng(0)
    X = 16
    m = BDLModel(3, X)
    total = 0
    for step in range(60):
        size = int(g.integers(0, 5 * X))
        m.insert(synth.uniform(size, 3, seed=100 + step))
        total += size
        assert m.F == total // X
        assert len(m.buffer) == total % X
        assert m.slot_sizes() == {i: m.capacity(i) for i in range(m.F.bit_length()) if (m.F >> i) & 1}
        m.check_invariants()


def test_batch_dynamic_start_closed_form():
    """4,000,000 = 61 * 65,536 + 2,304: F = 0b111101 and 2,304 buffered points.
    Checked on counts only (no coordinates needed)."""
    m = BDLModel(3, 65536)
    ids = list(range(4_000_000))
    m.next_id = len(ids)
    m._insert_ids(ids)
    assert m.F == 0b111101 == 61
    assert len(m.buffer) == 2304
    assert m.slot_sizes() == {0: 65536, 2: 262144, 3: 524288, 4: 1048576, 5: 2097152}


def test_cascade_assignment_reading():
    """F = 0b1010, q = 3: slot 1 (2X points) is destroyed; slot 0 gets X batch
    points, slot 2 gets slot 1's points plus 2X batch points."""
    X = 4
    m = BDLModel(1, X)
    m.insert(np.arange(2 * X, dtype=np.float32)[:, None])      # F = 2
    m.insert(np.arange(8 * X, dtype=np.float32)[:, None] + 100)  # F = 2 + 8 = 10
    assert m.F == 0b1010
    old_slot1 = sorted(m.slots[1])
    new = m.insert(np.arange(3 * X, dtype=np.float32)[:, None] + 1000)
    assert m.F == 0b1101
    assert sorted(m.slots[0]) == list(new[:X])
    assert sorted(m.slots[2]) == sorted(old_slot1 + list(new[X:]))
    m.check_invariants()


def test_erase_semantics_and_invariants():
    X = 8
    m = BDLModel(2, X)
    pts = synth.uniform(300, 2, seed=1)
    pts[10] = pts[3]                                        # duplicate coordinates
    m.insert(pts)
    # erasing one copy's coordinates removes every live copy; absent points are ignored
    removed = m.erase(np.concatenate([pts[3:4], np.array([[5.0, 5.0]], np.float32)]))
    assert removed == 2
    live = set(m.live_ids())
    assert 3 not in live and 10 not in live and len(live) == 298
    m.check_invariants()


def test_random_history_invariants_and_knn():
    g = np.random.default_rng(5)
    X = 32
    m = BDLModel(3, X)
    all_pts = []
    for step in range(40):
        if step % 3 == 2 and m.size() > 0:
            live_pts, ids = m.live_arrays()
            sel = g.choice(len(ids), size=int(g.integers(1, max(2, len(ids) // 2))), replace=False)
            m.erase(live_pts[sel])
        else:
            p = synth.uniform(int(g.integers(1, 6 * X)), 3, seed=step)
            all_pts.append(p)
            m.insert(p)
        m.check_invariants()
        # every slot is at least half full, the buffer below X
        for i, ids in m.slots.items():
            assert 2 * len(ids) >= m.capacity(i)
    # the forest's live set answers k-NN like brute force over it (definition)
    live_pts, ids = m.live_arrays()
    everything = np.concatenate(all_pts)
    alive = np.zeros(len(everything), bool)
    alive[ids] = True
    q = synth.uniform(50, 3, seed=999)
    a = oracle.knn(live_pts, q, 5, ids=ids)
    b = oracle.knn(everything, q, 5, live=alive)
    assert np.array_equal(a[0], b[0]) and np.array_equal(a[1], b[1])


def test_half_full_tree_stays_fewer_than_half_is_rebuilt():
    """Erase_L gathers only trees left with FEWER than half their capacity
    (Appendix A.3): slot 1 (capacity 2X) keeps X live points and stays; one
    more erase leaves X - 1 and its points go back through Insert_L."""
    X = 4
    m = BDLModel(1, X)
    pts = np.arange(2 * X, dtype=np.float32)[:, None]
    m.insert(pts)
    assert m.F == 0b10 and m.slot_sizes() == {1: 2 * X}
    m.erase(pts[:X])
    assert m.F == 0b10 and m.slot_sizes() == {1: X} and m.buffer == []
    m.erase(pts[X:X + 1])
    assert m.F == 0 and m.slot_sizes() == {} and len(m.buffer) == X - 1
    m.check_invariants()


def test_erase_reaches_the_buffer_tree():
    X = 8
    m = BDLModel(2, X)
    pts = synth.uniform(3 * X + 3, 2, seed=7)           # 3 points end up in the buffer
    ids = m.insert(pts)
    assert sorted(m.buffer) == list(ids[-3:])
    m.erase(pts[-2:])
    assert sorted(m.buffer) == [ids[-3]]
    assert set(m.live_ids()) == set(ids[:-2].tolist())
    m.check_invariants()
