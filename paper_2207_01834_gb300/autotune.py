"""Autotuner for the k-NN path's launch parameters: the tree's leaf size, the
traversal kernel (thread per query, warp packets, postponed leaves, warp per
query) and where the k-list lives (one thread's registers, a binary heap in
shared memory for lists of more than 16 pairs, or spread across a warp's
lanes with warp per query), and the leaf size of the batched Chamfer path.

It times the candidates on the caller's own data (build + query through the C
ABI, CUDA events, after a warm-up; the traversal is named per call, so no
process-wide state changes while it measures), caches the winner in a JSON
file keyed by (GPU name, workload kind, dimension, k, n rounded to a power of
two), and records the chosen traversal in the library's tune table
(pg_knn_tune_set), so that later PG_KNN_AUTO calls of the same dimension
class, k class and kind use it.  Only parameters that do not change the
result are tuned: the k-NN answer is the same for every choice.
"""
from __future__ import annotations

import json
import os
import threading

import torch

from . import api
from .build import OUT_DIR

CACHE = os.path.join(OUT_DIR, "autotune.json")
LEAF_CANDIDATES = (8, 16, 32, 48, 64, 128)
VARIANT_CANDIDATES = api.KNN_VARIANTS
BATCHED_LEAF_CANDIDATES = (8, 12, 16, 24, 32)
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


def _best_of(fn, reps: int = 2) -> float:
    """Best CUDA-event time of `fn` over `reps` runs after one warm-up run."""
    stream = torch.cuda.current_stream()
    best = float("inf")
    for r in range(reps + 1):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        fn()
        e1.record(stream)
        torch.cuda.synchronize()
        if r > 0:
            best = min(best, e0.elapsed_time(e1))
    return best


def _time_leaf(x: torch.Tensor, queries, k: int, leaf: int, variant: int, reps: int = 2) -> float:
    def run():
        t = api.pg_tree_build(x, leaf_size=leaf)
        api.pg_knn(t, queries, k, variant=variant)
        t.free()
    return _best_of(run, reps)


def _time_batched(a, a_off, b, b_off, k: int, leaf: int, reps: int = 2) -> float:
    g = torch.ones(len(a_off) - 1, device=a.device)

    def run():
        _, iab, iba, _, _ = api.pg_batched_chamfer(a, a_off, b, b_off, k, leaf_size=leaf)
        api.pg_batched_chamfer_backward(a, a_off, b, b_off, k, iab, iba, g)
    return _best_of(run, reps)


def best_config(x: torch.Tensor, k: int, queries=None, leaves=LEAF_CANDIDATES,
                variants=VARIANT_CANDIDATES) -> tuple[int, int]:
    """(leaf size, traversal variant) minimising build + query time for this
    data (cached).  The traversal is recorded in the library's tune table for
    PG_KNN_AUTO requests of this dimension class, k class and kind."""
    n, dim = x.shape
    all_knn = queries is None
    key = _key(dim, k, n, "all" if all_knn else "queries") + \
        f"|L{','.join(map(str, leaves))}|V{','.join(map(str, variants))}"
    with _lock:
        cache = _load()
    if key in cache:
        leaf, var = int(cache[key]["leaf"]), int(cache[key]["variant"])
    else:
        # up to k = 16 the shared-memory heap variant runs the register-list kernel itself
        variants = [v for v in variants if not (v == api.KNN_POSTPONED_HEAP and k <= 16)] or list(variants)
        times = {(leaf, var): _time_leaf(x, queries, k, leaf, var) for var in variants for leaf in leaves}
        leaf, var = min(times, key=times.get)
        with _lock:
            cache = _load()
            cache[key] = {"leaf": leaf, "variant": var, "ms": {f"{a}/{b}": t for (a, b), t in times.items()}}
            _store(cache)
    api.pg_knn_tune_set(dim, k, all_knn, var)
    return leaf, var


def best_leaf(x: torch.Tensor, k: int, queries=None, candidates=LEAF_CANDIDATES) -> int:
    """Leaf size for this data (the traversal is recorded as in best_config)."""
    return best_config(x, k, queries, leaves=candidates)[0]


def best_batched_leaf(a: torch.Tensor, a_off, b: torch.Tensor, b_off, k: int,
                      candidates=BATCHED_LEAF_CANDIDATES) -> int:
    """Leaf size minimising the batched Chamfer forward + backward time on
    these clouds (cached per cloud count, total size, dimension and k)."""
    npairs = len(a_off) - 1
    total = int(a_off[-1]) + int(b_off[-1])
    key = _key(a.shape[1], k, total, f"batched{npairs}") + f"|L{','.join(map(str, candidates))}"
    with _lock:
        cache = _load()
    if key in cache:
        return int(cache[key]["leaf"])
    times = {leaf: _time_batched(a, a_off, b, b_off, k, leaf) for leaf in candidates}
    leaf = min(times, key=times.get)
    with _lock:
        cache = _load()
        cache[key] = {"leaf": leaf, "ms": {str(c): t for c, t in times.items()}}
        _store(cache)
    return leaf
