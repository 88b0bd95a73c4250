"""CPU oracle for the kd-tree / BDL-tree k-NN hot path — TEST INFRASTRUCTURE.

Only `tests/`, `__graft_entry__.smoke()` and the benchmark's `cpu_baseline` /
reference leg may import this package.  The product path (the CUDA library and
its Python binding) shares no code with it and never calls it.

Contents
  knn            exact brute-force k-NN in float64 (C, `pargeo_oracle.c`):
                 the plain definition of what the paper's k-NN answers
                 (Section 5 "Data-Parallel k-NN"; Appendix A.1.3).
  knn_grad       closed-form gradient of L = sum_ij w_ij * D(q_i, p_idx(i,j)).
                 The paper has no gradients; this is the derivative of the
                 squared Euclidean distance, written out.
  chamfer        bidirectional k-NN loss over cloud pairs, built from knn and
                 knn_grad.
  bdl            model of the BDL-tree's forest bookkeeping (Insert_L and
                 Erase_L, Section 5 "Parallel Batch Insertion", Appendix A.2-A.3)
                 and its live point set.
  kdtree_check   checker of the kd-tree invariants (Section 5 intro).
  range_search   every data point within distance r of each query (Section 4:
                 the kd-tree's range search), from the definition in float64.
  knn_graph      the k-NN graph (Section 4, geometric graph generators: the
                 k-NN graph comes from the kd-tree's k-NN search): every point
                 joined to its k nearest other points, undirected edges listed
                 once as (u, v), u < v, sorted.  The paper does not say whether
                 edges are directed; this oracle takes the symmetrised reading.

Every float computation here is float64 on float32 inputs.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "pargeo_oracle.c")
_LIB_DIR = os.path.join(_HERE, "_build")
_LIB = os.path.join(_LIB_DIR, "liboracle.so")
_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile the C oracle with gcc (plain -O2, no vector intrinsics)."""
    os.makedirs(_LIB_DIR, exist_ok=True)
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".{os.getpid()}.tmp"
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-pthread",
                               "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = ctypes.CDLL(build())
            lib.oracle_knn_f64.restype = ctypes.c_int
            lib.oracle_knn_f64.argtypes = [
                ctypes.c_void_p, ctypes.c_int64, ctypes.c_void_p, ctypes.c_int64, ctypes.c_int,
                ctypes.c_int, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p,
                ctypes.c_int]
            lib.oracle_default_threads.restype = ctypes.c_int
            _lib = lib
    return _lib


def default_threads() -> int:
    return int(_load().oracle_default_threads())


def knn(data, queries, k: int, live=None, ids=None, nthreads: int = 1):
    """Exact k-NN by brute force in float64.

    data (n, d) and queries (m, d) are float32.  live: optional bool (n,) mask;
    ids: optional int64 (n,) point ids (default: row index).
    Returns (idx int64 (m, k), dist float64 (m, k)); padding is (-1, +inf).
    Order within a row: ascending (distance, id).
    """
    data = np.ascontiguousarray(data, dtype=np.float32)
    queries = np.ascontiguousarray(queries, dtype=np.float32)
    n, d = data.shape if data.ndim == 2 else (0, queries.shape[1])
    m = queries.shape[0]
    if data.size == 0:
        data = np.zeros((0, queries.shape[1]), np.float32)
        n, d = 0, queries.shape[1]
    assert queries.shape[1] == d
    out_idx = np.empty((m, k), np.int64)
    out_dist = np.empty((m, k), np.float64)
    live_arr = None if live is None else np.ascontiguousarray(live, dtype=np.uint8)
    ids_arr = None if ids is None else np.ascontiguousarray(ids, dtype=np.int64)
    rc = _load().oracle_knn_f64(
        data.ctypes.data, n, queries.ctypes.data, m, d, k,
        None if live_arr is None else live_arr.ctypes.data,
        None if ids_arr is None else ids_arr.ctypes.data,
        out_idx.ctypes.data, out_dist.ctypes.data, nthreads)
    if rc != 0:
        raise ValueError("oracle_knn_f64: invalid arguments")
    return out_idx, out_dist


def knn_grad(data, queries, idx, w):
    """Gradient of L = sum_{i,j} w_ij * D(q_i, p_{idx_ij}) for a fixed selection.

    D(q, p) = sum_c (q_c - p_c)^2, so
        dL/dq_i = sum_j 2 w_ij (q_i - p_{idx_ij})
        dL/dp_t = - sum_{(i,j): idx_ij = t} 2 w_ij (q_i - p_t)
    Entries with idx = -1 (padding) contribute nothing.  float64 throughout.
    Returns (grad_queries (m, d), grad_data (n, d)).
    """
    P = np.asarray(data, np.float64)
    Q = np.asarray(queries, np.float64)
    idx = np.asarray(idx, np.int64)
    W = np.asarray(w, np.float64)
    m, k = idx.shape
    gq = np.zeros_like(Q)
    gp = np.zeros_like(P)
    valid = idx >= 0
    rows = np.repeat(np.arange(m), k).reshape(m, k)[valid]
    cols = idx[valid]
    coef = 2.0 * W[valid]
    diff = Q[rows] - P[cols]                      # (pairs, d)
    contrib = coef[:, None] * diff
    np.add.at(gq, rows, contrib)
    np.add.at(gp, cols, -contrib)
    return gq, gp


def knn_loss(data, queries, idx, w) -> float:
    """L = sum_{i,j} w_ij * D(q_i, p_{idx_ij}) in float64 (padding skipped)."""
    P = np.asarray(data, np.float64)
    Q = np.asarray(queries, np.float64)
    idx = np.asarray(idx, np.int64)
    W = np.asarray(w, np.float64)
    total = 0.0
    m, k = idx.shape
    for i in range(m):
        for j in range(k):
            t = idx[i, j]
            if t >= 0:
                total += W[i, j] * float(np.sum((Q[i] - P[t]) ** 2))
    return total


def chamfer(a, a_off, b, b_off, k: int, nthreads: int = 1):
    """Bidirectional k-NN ("Chamfer-style") loss over cloud pairs.

    For pair i with clouds A_i = a[a_off[i]:a_off[i+1]], B_i likewise:
        loss_i = sum_{x in A_i} sum_{j<k} D(x, nn_j^{B_i}(x))
               + sum_{y in B_i} sum_{j<k} D(y, nn_j^{A_i}(y))
    Returns (loss (npairs,) float64, idx_ab (|a|, k) int64 local to B_i,
             idx_ba (|b|, k) int64 local to A_i, grad_a, grad_b) where the
    gradients are of sum_i loss_i with respect to a and b, float64.
    """
    a = np.asarray(a, np.float32)
    b = np.asarray(b, np.float32)
    npairs = len(a_off) - 1
    loss = np.zeros(npairs)
    idx_ab = np.empty((a.shape[0], k), np.int64)
    idx_ba = np.empty((b.shape[0], k), np.int64)
    ga = np.zeros(a.shape, np.float64)
    gb = np.zeros(b.shape, np.float64)
    for i in range(npairs):
        A = a[a_off[i]:a_off[i + 1]]
        B = b[b_off[i]:b_off[i + 1]]
        iab, dab = knn(B, A, k, nthreads=nthreads)
        iba, dba = knn(A, B, k, nthreads=nthreads)
        idx_ab[a_off[i]:a_off[i + 1]] = iab
        idx_ba[b_off[i]:b_off[i + 1]] = iba
        loss[i] = np.where(iab >= 0, dab, 0.0).sum() + np.where(iba >= 0, dba, 0.0).sum()
        gq, gp = knn_grad(B, A, iab, np.ones(iab.shape))
        ga[a_off[i]:a_off[i + 1]] += gq
        gb[b_off[i]:b_off[i + 1]] += gp
        gq, gp = knn_grad(A, B, iba, np.ones(iba.shape))
        gb[b_off[i]:b_off[i + 1]] += gq
        ga[a_off[i]:a_off[i + 1]] += gp
    return loss, idx_ab, idx_ba, ga, gb


def knn_graph(points, k: int, nthreads: int = 1) -> np.ndarray:
    """k-NN graph of `points` as an (E, 2) int64 array of edges (u, v), u < v,
    in ascending (u, v) order (Section 4, geometric graph generators).

    Step by step, from the definitions: the k nearest other points of i are
    the k smallest (distance, index) pairs over indices j != i; an undirected
    edge {i, j} exists when j is among i's k or i among j's k.
    """
    p = np.asarray(points, np.float32)
    n = len(p)
    if n < 2:
        return np.zeros((0, 2), np.int64)
    idx, _ = knn(p, p, min(k + 1, n), nthreads=nthreads)
    edges = set()
    for i in range(n):
        others = [int(t) for t in idx[i] if t >= 0 and t != i]
        if len(others) > k:          # i itself was not among its k + 1
            others = others[:k]
        for j in others[:k]:
            edges.add((min(i, j), max(i, j)))
    if not edges:
        return np.zeros((0, 2), np.int64)
    return np.array(sorted(edges), np.int64)


def range_search(data, queries, radius: float):
    """For each query, the sorted indices of the data points p with
    D(q, p) <= radius^2, in float64 on the float32 inputs (Section 4, range
    search on the kd-tree).  Returns a list of int64 arrays."""
    p = np.asarray(data, np.float32).astype(np.float64)
    q = np.asarray(queries, np.float32).astype(np.float64)
    r2 = float(np.float32(radius)) ** 2
    out = []
    for i in range(len(q)):
        d = ((p - q[i]) ** 2).sum(1)
        out.append(np.nonzero(d <= r2)[0].astype(np.int64))
    return out

