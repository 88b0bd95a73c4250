"""The autotuner's host logic on the CPU, with the timing call replaced: it
picks the fastest (leaf size, variant), leaves that variant set, caches the
choice per (GPU, workload shape) and reuses it without timing again."""
from __future__ import annotations

import numpy as np
import pytest

torch = pytest.importorskip("torch")


@pytest.fixture
def tuner(monkeypatch, tmp_path):
    from paper_2207_01834_gb300 import autotune

    state = {"variant": None, "timed": []}
    monkeypatch.setattr(autotune, "CACHE", str(tmp_path / "autotune.json"))
    monkeypatch.setattr(autotune.torch.cuda, "get_device_name", lambda *a: "GB300-test")
    monkeypatch.setattr(autotune.api, "pg_knn_set_variant", lambda v: state.__setitem__("variant", v))

    def fake_time(x, queries, k, leaf, reps=2):
        state["timed"].append((leaf, state["variant"]))
        return abs(leaf - 32) + (0.5 if state["variant"] != 3 else 0.0)   # fastest: leaf 32, variant 3

    monkeypatch.setattr(autotune, "_time_leaf", fake_time)
    return autotune, state


def test_picks_the_fastest_and_caches(tuner):
    autotune, state = tuner
    x = torch.from_numpy(np.zeros((5000, 3), np.float32))
    assert autotune.best_config(x, 10) == (32, 3)
    assert state["variant"] == 3
    assert len(state["timed"]) == len(autotune.LEAF_CANDIDATES) * len(autotune.VARIANT_CANDIDATES)
    state["timed"].clear()
    state["variant"] = None
    assert autotune.best_config(x, 10) == (32, 3)          # from the cache
    assert state["timed"] == [] and state["variant"] == 3


def test_cache_key_separates_workloads(tuner):
    autotune, state = tuner
    x = torch.from_numpy(np.zeros((5000, 3), np.float32))
    autotune.best_config(x, 10)
    n_first = len(state["timed"])
    autotune.best_config(x, 16)                             # another k: timed again
    autotune.best_config(x, 10, queries=x)                  # separate queries: timed again
    autotune.best_config(torch.from_numpy(np.zeros((70000, 3), np.float32)), 10)   # another size class
    assert len(state["timed"]) == 4 * n_first
    assert autotune.best_leaf(x, 10) == 32                  # cached
    assert len(state["timed"]) == 4 * n_first
