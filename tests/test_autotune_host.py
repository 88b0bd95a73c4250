"""The autotuner's host logic on the CPU, with the timing call replaced: it
picks the fastest (leaf size, traversal), records the traversal in the
library's tune table (never in a process-wide override), caches the choice per
(GPU, workload shape) and reuses it without timing again."""
from __future__ import annotations

import numpy as np
import pytest

torch = pytest.importorskip("torch")


@pytest.fixture
def tuner(monkeypatch, tmp_path):
    from paper_2207_01834_gb300 import autotune

    state = {"timed": [], "tuned": [], "override": []}
    monkeypatch.setattr(autotune, "CACHE", str(tmp_path / "autotune.json"))
    monkeypatch.setattr(autotune.torch.cuda, "get_device_name", lambda *a: "GB300-test")
    monkeypatch.setattr(autotune.api, "pg_knn_tune_set", lambda *a: state["tuned"].append(a))
    monkeypatch.setattr(autotune.api, "pg_knn_set_variant", lambda v: state["override"].append(v))

    def fake_time(x, queries, k, leaf, variant, reps=2):
        state["timed"].append((leaf, variant))
        return abs(leaf - 32) + (0.5 if variant != 3 else 0.0)   # fastest: leaf 32, variant 3

    monkeypatch.setattr(autotune, "_time_leaf", fake_time)
    return autotune, state


def test_picks_the_fastest_and_caches(tuner):
    autotune, state = tuner
    x = torch.from_numpy(np.zeros((5000, 3), np.float32))
    assert autotune.best_config(x, 10) == (32, 3)
    assert state["tuned"] == [(3, 10, True, 3)]
    # k <= 16: the shared-memory heap variant is the register-list kernel itself, not timed twice
    small_k = set(autotune.VARIANT_CANDIDATES) - {autotune.api.KNN_POSTPONED_HEAP}
    assert len(state["timed"]) == len(autotune.LEAF_CANDIDATES) * len(small_k)
    assert set(v for _, v in state["timed"]) == small_k
    state["timed"].clear()
    assert autotune.best_config(x, 10, queries=None) == (32, 3)          # from the cache
    assert state["timed"] == [] and state["tuned"][-1] == (3, 10, True, 3)
    assert state["override"] == []                                       # no process-wide side effect


def test_large_k_times_the_heap_variant(tuner):
    autotune, state = tuner
    x = torch.from_numpy(np.zeros((5000, 3), np.float32))
    autotune.best_config(x, 32)
    assert set(v for _, v in state["timed"]) == set(autotune.VARIANT_CANDIDATES)


def test_cache_key_separates_workloads(tuner):
    autotune, state = tuner
    x = torch.from_numpy(np.zeros((5000, 3), np.float32))
    autotune.best_config(x, 10)
    n_first = len(state["timed"])
    autotune.best_config(x, 16)                             # another k: timed again
    autotune.best_config(x, 10, queries=x)                  # separate queries: timed again
    assert state["tuned"][-1] == (3, 10, False, 3)
    autotune.best_config(torch.from_numpy(np.zeros((70000, 3), np.float32)), 10)   # another size class
    assert len(state["timed"]) == 4 * n_first
    assert autotune.best_leaf(x, 10) == 32                  # cached
    assert len(state["timed"]) == 4 * n_first


def test_batched_leaf_picks_fastest_and_caches(tuner, monkeypatch):
    autotune, state = tuner
    timed = []

    def fake_time(a, a_off, b, b_off, k, leaf, reps=2):
        timed.append(leaf)
        return abs(leaf - 12) + 1.0

    monkeypatch.setattr(autotune, "_time_batched", fake_time)
    a = torch.zeros((300, 3))
    off = np.array([0, 100, 300])
    assert autotune.best_batched_leaf(a, off, a, off, 8) == 12
    assert sorted(timed) == sorted(autotune.BATCHED_LEAF_CANDIDATES)
    timed.clear()
    assert autotune.best_batched_leaf(a, off, a, off, 8) == 12
    assert timed == []
