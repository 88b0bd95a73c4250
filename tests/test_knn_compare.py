"""The parity comparator itself (tests/knn_compare.py), on the CPU: it accepts
the oracle's own answer and a tie resolved the other way, and rejects a wrong
index, a distance beyond the tolerance, a padding mismatch, a duplicate index
and an index out of range, so that a GPU parity test cannot pass vacuously."""
from __future__ import annotations

import numpy as np
import pytest

import oracle
from knn_compare import RTOL, compare_knn


def _case():
    # 1D points; query 0 at 5.0 has neighbours 4 and 6 tied at distance 1
    data = np.array([[0.0], [4.0], [6.0], [9.0], [5.5]], np.float32)
    q = np.array([[5.0], [0.2]], np.float32)
    idx, dist = oracle.knn(data, q, 3)
    return data, q, idx, dist


def test_accepts_the_oracle_answer():
    data, q, idx, dist = _case()
    assert compare_knn(idx, dist, idx, dist, data, q) == 0


def test_accepts_a_tie_resolved_the_other_way():
    data = np.array([[0.0], [4.0], [6.0], [9.0]], np.float32)
    q = np.array([[5.0]], np.float32)
    idx, dist = oracle.knn(data, q, 1)                 # 4.0 (id 1) and 6.0 (id 2) tie; the oracle keeps id 1
    assert idx[0, 0] == 1
    assert compare_knn(np.array([[2]]), dist, idx, dist, data, q) == 1


def test_rejects_a_wrong_index():
    data, q, idx, dist = _case()
    bad = idx.copy()
    bad[0, -1] = 3                                     # 9.0 is not among the 3 nearest of 5.0
    with pytest.raises(AssertionError):
        compare_knn(bad, dist, idx, dist, data, q)


def test_rejects_a_distance_beyond_the_tolerance_and_accepts_within():
    data, q, idx, dist = _case()
    off = dist.copy()
    off[1, 1] *= 1 + 10 * RTOL
    with pytest.raises(AssertionError):
        compare_knn(idx, off, idx, dist, data, q)
    near = dist.copy()
    near[1, 1] *= 1 + 0.1 * RTOL
    compare_knn(idx, near, idx, dist, data, q)


def test_rejects_padding_mismatch_duplicates_and_out_of_range():
    data, q, idx, dist = _case()
    ora_i, ora_d = oracle.knn(data[:2], q, 3)          # 2 points: one padded slot per row
    got_i, got_d = ora_i.copy(), ora_d.copy()
    got_i[0, 2], got_d[0, 2] = 0, 25.0                 # a point where padding belongs
    with pytest.raises(AssertionError):
        compare_knn(got_i, got_d, ora_i, ora_d, data[:2], q)
    dup = idx.copy()
    dup[0, 2] = dup[0, 1]
    with pytest.raises(AssertionError):
        compare_knn(dup, dist, idx, dist, data, q)
    oor = idx.copy()
    oor[1, 2] = 99
    with pytest.raises(AssertionError):
        compare_knn(oor, dist, idx, dist, data, q)
