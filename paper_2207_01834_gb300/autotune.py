"""Autotuner for the k-NN path's launch parameters (leaf size, traversal
variant: thread per query, warp packets or postponed leaves).

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
LEAF_CANDIDATES = (8, 16, 32, 48, 64)
VARIANT_CANDIDATES = (1, 2, 3)   # thread per query, warp packets, postponed leaves
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


def best_config(x: torch.Tensor, k: int, queries=None, leaves=LEAF_CANDIDATES,
                variants=VARIANT_CANDIDATES) -> tuple[int, int]:
    """(leaf size, traversal variant) minimising build + query time for this
    data (cached).  Leaves the chosen variant set process-wide."""
    n, dim = x.shape
    key = _key(dim, k, n, "all" if queries is None else "queries") + \
        f"|L{','.join(map(str, leaves))}|V{','.join(map(str, variants))}"
    with _lock:
        cache = _load()
        if key in cache:
            leaf, var = int(cache[key]["leaf"]), int(cache[key]["variant"])
            api.pg_knn_set_variant(var)
            return leaf, var
    times = {}
    for var in variants:
        api.pg_knn_set_variant(var)
        for leaf in leaves:
            times[(leaf, var)] = _time_leaf(x, queries, k, leaf)
    leaf, var = min(times, key=times.get)
    api.pg_knn_set_variant(var)
    with _lock:
        cache = _load()
        cache[key] = {"leaf": leaf, "variant": var, "ms": {f"{a}/{b}": t for (a, b), t in times.items()}}
        _store(cache)
    return leaf, var


def best_leaf(x: torch.Tensor, k: int, queries=None, candidates=LEAF_CANDIDATES) -> int:
    """Leaf size (and, as a side effect, traversal variant) for this data."""
    return best_config(x, k, queries, leaves=candidates)[0]
