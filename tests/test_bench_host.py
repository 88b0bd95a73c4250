"""Host-side bookkeeping of the benchmark's other workloads, on CPU: every
section runs in order and reports its keys, with a stand-in for the library
and for the CUDA timing calls (no kernel runs here; the numbers are the
stand-in's).  Guards the benchmark script's structure, not any result."""
from __future__ import annotations

import types

import numpy as np
import pytest

import bench


class _Arr:
    def __init__(self, a):
        self.a = np.asarray(a)
        self.shape = self.a.shape

    def to(self, dev):
        return self

    def numel(self):
        return self.a.size

    def __getitem__(self, k):
        return _Arr(self.a[k.a if isinstance(k, _Arr) else k])

    def __len__(self):
        return len(self.a)


class _Event:
    def __init__(self, enable_timing=False):
        pass

    def record(self, stream=None):
        pass

    def elapsed_time(self, other):
        return 2.0


class _Tree:
    def free(self):
        pass


class _Forest:
    def __init__(self, *args):
        self.n = 0

    def insert(self, p):
        self.n += p.shape[0]

    def erase(self, p):
        self.n -= p.shape[0]

    def knn(self, q, k):
        m = len(q) if q is not None else 0
        return _Arr(np.zeros((m, k), np.int32)), _Arr(np.zeros((m, k), np.float32))

    def structure(self):
        return {"F": 0b101, "slot_live": [0] * 64, "buffer_live": 3}

    def size(self):
        return self.n

    def free(self):
        pass


def _standins(monkeypatch):
    from paper_2207_01834_gb300 import autotune

    cuda = types.SimpleNamespace(current_stream=lambda: None, Event=_Event, synchronize=lambda: None)
    torch = types.SimpleNamespace(from_numpy=_Arr, cuda=cuda, cat=lambda xs: _Arr(np.concatenate([x.a for x in xs])),
                                  equal=lambda a, b: np.array_equal(a.a, b.a))
    api = types.SimpleNamespace(
        pg_tree_build=lambda x, leaf: _Tree(), pg_tree_build_split=lambda x, leaf, rule: _Tree(), SPLIT_OBJECT=1,
        pg_knn=lambda t, q, k, **kw: (_Arr(np.zeros((4, k), np.int32)), _Arr(np.zeros((4, k), np.float32))),
        pg_knn_graph=lambda t, k: _Arr(np.zeros((5, 2))), pg_knn_tune_get=lambda dim, k, all_knn: 5,
        pg_range=lambda t, q, r: (_Arr(np.zeros(7)), _Arr(np.zeros(3))),
        BDL=_Forest, KNN_POSTPONED=3, KNN_WARP=4, KNN_POSTPONED_HEAP=5, pg_knn_touch_enable=lambda on: None, pg_knn_touch_read=lambda: (10, 100))
    monkeypatch.setattr(autotune, "best_config", lambda pts, k, queries=None: (32, 3))
    return api, torch


def test_other_workloads_all_sections(monkeypatch):
    api, torch = _standins(monkeypatch)
    out = bench.other_configs(api, torch, "dev")
    assert sorted(out) == sorted(["2d_20k_k5", "knn_graph_2d_10m_k10", "range_2d_10m_all_r_for_10",
                                  "object_median_3d_10m_k10", "5d_gmm_2m_1mq_k16", "7d_gmm_2m_1mq_k16",
                                  "bdl_3d_4m_schedule", "k_sweep_2d_gmm_10m_5pct_inserts",
                                  "k_sweep_7d_uniform_10m_5pct_inserts"] +
                                 [f"large_k_3d_uniform_2m_{kind}_k{k}" for kind in ("1mq", "all") for k in (32, 64)])
    assert all(out[f"large_k_3d_uniform_2m_all_k{k}"]["variants_agree_bitwise"] for k in (32, 64))
    for name in ("k_sweep_2d_gmm_10m_5pct_inserts", "k_sweep_7d_uniform_10m_5pct_inserts"):
        assert out[name]["k"] == list(range(2, 12)) and out[name]["prefix_consistent_with_k11"]
    for key in ("insert_roofline", "erase_roofline", "forest_knn_roofline"):
        assert out["bdl_3d_4m_schedule"][key]["frac"] > 0
    # the schedule inserts 4M, then [1M, 1M, erase 500k] x 5
    assert out["bdl_3d_4m_schedule"]["live_points_end"] == 4_000_000 + 5 * (2_000_000 - 500_000)
    assert out["range_2d_10m_all_r_for_10"]["results"] == 7


def test_other_workloads_subset(monkeypatch):
    api, torch = _standins(monkeypatch)
    out = bench.other_configs(api, torch, "dev", only=["graph_range"])
    assert sorted(out) == ["knn_graph_2d_10m_k10", "range_2d_10m_all_r_for_10"]


def test_extras_only_rejects_unknown_names():
    with pytest.raises(SystemExit):
        bench.extras_only("graph_range,nonsense")
