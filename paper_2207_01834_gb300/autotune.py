"""Autotuner for the k-NN path's launch parameters.

It times the candidates on the caller's own data (build + query through the C
ABI, CUDA events, after a warm-up) and caches the winner in a JSON file keyed
by (GPU name, dimension, k, n rounded to a power of two).  Only parameters
that do not change the result are tuned, so the k-NN answer is the same for
every choice.
"""
from __future__ import annotations

import json
import os
import threading

import torch

from . import api
from .build import OUT_DIR

CACHE = os.path.join(OUT_DIR, "autotune.json")
LEAF_CANDIDATES = (8, 16, 32)
_lock = threading.Lock()


def _key(dim: int, k: int, n: int, what: str) -> str:
    name = torch.cuda.get_device_name()
    return f"{name}|{what}|d{dim}|k{k}|n2^{max(0, int(n).bit_length() - 1)}"


def _load() -> dict:
    try:
        return json.load(open(CACHE))
    except Exception:
        return {}


def _store(d: dict) -> None:
    os.makedirs(OUT_DIR, exist_ok=True)
    tmp = CACHE + f".{os.getpid()}.tmp"
    json.dump(d, open(tmp, "w"), indent=1, sort_keys=True)
    os.replace(tmp, CACHE)


def _time_leaf(x: torch.Tensor, queries, k: int, leaf: int, reps: int = 2) -> float:
    stream = torch.cuda.current_stream()
    best = float("inf")
    for r in range(reps + 1):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        t = api.pg_tree_build(x, leaf_size=leaf)
        api.pg_knn(t, queries, k)
        e1.record(stream)
        torch.cuda.synchronize()
        t.free()
        if r > 0:
            best = min(best, e0.elapsed_time(e1))
    return best


def best_leaf(x: torch.Tensor, k: int, queries=None, candidates=LEAF_CANDIDATES) -> int:
    """Leaf size minimising build + query time for this data (cached)."""
    n, dim = x.shape
    key = _key(dim, k, n, "leaf" if queries is None else "leaf_q")
    with _lock:
        cache = _load()
        if key in cache:
            return int(cache[key]["leaf"])
    times = {leaf: _time_leaf(x, queries, k, leaf) for leaf in candidates}
    leaf = min(times, key=times.get)
    with _lock:
        cache = _load()
        cache[key] = {"leaf": leaf, "ms": times}
        _store(cache)
    return leaf
