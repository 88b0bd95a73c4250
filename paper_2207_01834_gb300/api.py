"""Thin Python binding of the C ABI (argument marshalling only).

Every function here checks tensor devices/dtypes/shapes, passes raw pointers
and the current CUDA stream to the C library, and wraps handles.  All compute
runs in the sm_103a kernels of libpargeo_gpu.so; there is no CPU or PyTorch
fallback.  Names follow the C ABI (pg_tree_build, pg_knn, pg_bdl_*, ...).
"""
from __future__ import annotations

import ctypes as C

import numpy as np
import torch

from . import _lib
from ._lib import (KNN_AUTO, KNN_PACKET, KNN_POSTPONED, KNN_POSTPONED_HEAP, KNN_THREAD, KNN_VARIANTS, KNN_WARP, PgError,
                   TreeInfo, call)

__all__ = ["Tree", "BDL", "PgError", "pg_tree_build", "pg_tree_build_split", "pg_knn", "pg_tree_free", "pg_tree_info",
           "pg_tree_export", "pg_knn_graph", "pg_range", "pg_knn_set_variant", "pg_knn_tune_set", "pg_knn_tune_get", "KNN_AUTO", "KNN_THREAD", "KNN_PACKET",
           "KNN_POSTPONED", "KNN_WARP", "KNN_POSTPONED_HEAP", "KNN_VARIANTS", "pg_knn_touch_enable", "pg_knn_touch_read", "pg_bdl_create", "pg_bdl_insert", "pg_bdl_erase", "pg_bdl_knn", "pg_bdl_size",
           "pg_bdl_structure", "pg_bdl_slot_of", "pg_bdl_free", "pg_knn_backward", "pg_knn_backward_noalloc",
           "pg_batched_chamfer",
           "pg_batched_chamfer_backward", "launch_count", "profile_enable", "profile_read", "version",
           "debug_fail_alloc_after", "debug_batched_faults"]


def _stream(stream=None) -> int:
    if stream is None:
        stream = torch.cuda.current_stream()
    return int(stream.cuda_stream) if hasattr(stream, "cuda_stream") else int(stream)


def _dev(t: torch.Tensor, dtype, what: str, ndim: int | None = None) -> torch.Tensor:
    if not isinstance(t, torch.Tensor):
        raise TypeError(f"{what} must be a torch.Tensor")
    if not t.is_cuda:
        raise ValueError(f"{what} must be a CUDA tensor")
    if t.dtype != dtype:
        raise TypeError(f"{what} must be {dtype}, got {t.dtype}")
    if ndim is not None and t.dim() != ndim:
        raise ValueError(f"{what} must have {ndim} dimensions")
    return t.contiguous()


def _ptr(t) -> int | None:
    return None if t is None else t.data_ptr()


# ---------------------------------------------------------------- static tree
class Tree:
    """Owner of a pg_tree handle."""

    def __init__(self, handle: int, points_shape, device):
        self._h = C.c_void_p(handle)
        self.n, self.dim = points_shape
        self.device = device

    @property
    def handle(self):
        if not self._h:
            raise RuntimeError("tree already freed")
        return self._h

    def free(self) -> None:
        if self._h:
            call("pg_tree_free", self._h)
            self._h = C.c_void_p(None)

    def __del__(self):
        try:
            self.free()
        except Exception:
            pass

    def info(self) -> TreeInfo:
        return pg_tree_info(self)

    def export(self) -> dict:
        return pg_tree_export(self)


def pg_tree_build(points: torch.Tensor, leaf_size: int = 16, stream=None) -> Tree:
    pts = _dev(points, torch.float32, "points", 2)
    n, dim = pts.shape
    out = C.c_void_p()
    call("pg_tree_build", _ptr(pts) if n else None, n, dim, leaf_size, _stream(stream), C.byref(out))
    return Tree(out.value, (n, dim), pts.device)


SPLIT_SPATIAL, SPLIT_OBJECT = 0, 1


def pg_tree_build_split(points: torch.Tensor, leaf_size: int = 16, split_rule: int = SPLIT_SPATIAL,
                        stream=None) -> Tree:
    """kd-tree with the spatial-median (0) or object-median (1) split."""
    pts = _dev(points, torch.float32, "points", 2)
    n, dim = pts.shape
    out = C.c_void_p()
    call("pg_tree_build_split", _ptr(pts) if n else None, n, dim, leaf_size, split_rule, _stream(stream),
         C.byref(out))
    return Tree(out.value, (n, dim), pts.device)


def _out(t, shape, dtype, dev, what):
    if t is None:
        return torch.empty(shape, dtype=dtype, device=dev)
    if not isinstance(t, torch.Tensor) or not t.is_cuda or t.dtype != dtype or tuple(t.shape) != tuple(shape) \
            or not t.is_contiguous() or t.device != dev:
        raise ValueError(f"{what} must be a contiguous {dtype} CUDA tensor of shape {tuple(shape)} on {dev}")
    return t


def pg_knn(tree: Tree, queries: torch.Tensor | None, k: int, out_idx=None, out_dist=None, stream=None,
           variant: int = KNN_AUTO):
    """k-NN of `queries` (m, dim) or, with queries=None, all-kNN of the tree's points.
    variant: KNN_AUTO (the library's choice) or a KNN_* traversal for this call."""
    if queries is None:
        m = tree.n
        qp = None
    else:
        queries = _dev(queries, torch.float32, "queries", 2)
        if queries.shape[1] != tree.dim:
            raise ValueError("queries have the wrong dimension")
        m = queries.shape[0]
        qp = _ptr(queries)
    dev = tree.device
    if queries is not None and queries.device != dev:
        raise ValueError("queries must be on the tree's device")
    out_idx = _out(out_idx, (m, k), torch.int32, dev, "out_idx")
    out_dist = _out(out_dist, (m, k), torch.float32, dev, "out_dist")
    call("pg_knn_ex", tree.handle, qp, m, k, variant, _ptr(out_idx), _ptr(out_dist), _stream(stream))
    return out_idx, out_dist


def pg_tree_free(tree: Tree) -> None:
    tree.free()


def pg_tree_info(tree: Tree) -> TreeInfo:
    info = TreeInfo()
    call("pg_tree_info", tree.handle, C.byref(info))
    return info


def pg_tree_export(tree: Tree) -> dict:
    info = pg_tree_info(tree)
    nn, n = info.num_nodes, info.n
    nodes = np.zeros((nn, info.node_floats), np.float32)
    sdim = np.zeros(nn, np.int32)
    sval = np.zeros(nn, np.float32)
    bucket = np.zeros((n, info.point_floats), np.float32)
    call("pg_tree_export", tree.handle, nodes.ctypes.data if nn else None, sdim.ctypes.data if nn else None,
         sval.ctypes.data if nn else None, bucket.ctypes.data if n else None)
    return {"dim": info.dim, "dc": info.dim_class, "nodes": nodes, "split_dim": sdim, "split_val": sval,
            "bucket": bucket, "root_ref": info.root_ref, "root_cnt": info.root_cnt,
            "root_lo": np.array(info.root_lo[:info.dim], np.float32),
            "root_hi": np.array(info.root_hi[:info.dim], np.float32), "num_nodes": nn,
            "depth": info.depth, "leaf_size": info.leaf_size}


def pg_knn_graph(tree: Tree, k: int, stream=None) -> torch.Tensor:
    """Undirected k-NN graph of the tree's points: (E, 2) int32 device tensor of
    edges (u, v), u < v, sorted; point i is joined to its k nearest other points."""
    n = tree.n
    cap = max(1, n * k)
    out = torch.empty((cap, 2), dtype=torch.int32, device=tree.device)
    cnt = C.c_int64()
    call("pg_knn_graph", tree.handle, k, cap, _ptr(out), C.byref(cnt), _stream(stream))
    return out[:cnt.value]


def pg_range(tree: Tree, queries: torch.Tensor | None, radius: float, stream=None):
    """Points within `radius` of each query (queries=None: of each tree point).
    Returns (idx int32 (total,), offsets int64 (m + 1,)) on the device; query
    i's points are idx[offsets[i]:offsets[i+1]]."""
    if queries is None:
        m, qp = tree.n, None
    else:
        queries = _dev(queries, torch.float32, "queries", 2)
        if queries.shape[1] != tree.dim:
            raise ValueError("queries have the wrong dimension")
        m, qp = queries.shape[0], _ptr(queries)
    offsets = torch.empty(m + 1, dtype=torch.int64, device=tree.device)
    total = C.c_int64()
    call("pg_range", tree.handle, qp, m, float(radius), 0, None, _ptr(offsets), C.byref(total), _stream(stream))
    idx = torch.empty(max(total.value, 1), dtype=torch.int32, device=tree.device)
    call("pg_range_fill", tree.handle, qp, m, float(radius), _ptr(offsets), idx.numel(), _ptr(idx), _stream(stream))
    return idx[:total.value], offsets


def pg_knn_set_variant(variant: int) -> None:
    """This thread's traversal for KNN_AUTO requests (KNN_AUTO clears it)."""
    call("pg_knn_set_variant", variant)


def pg_knn_tune_set(dim: int, k: int, all_knn: bool, variant: int) -> None:
    """Record the traversal KNN_AUTO uses for (dim class, k class, kind), process-wide."""
    call("pg_knn_tune_set", dim, k, 1 if all_knn else 0, variant)


def pg_knn_tune_get(dim: int, k: int, all_knn: bool) -> int:
    """The traversal a KNN_AUTO request of this thread resolves to."""
    v = C.c_int()
    call("pg_knn_tune_get", dim, k, 1 if all_knn else 0, C.byref(v))
    return int(v.value)


def pg_knn_touch_enable(on: bool = True) -> None:
    """Count node records and bucket entries loaded by later postponed-leaf launches (variants 3 and 5)."""
    call("pg_knn_touch_enable", 1 if on else 0)


def pg_knn_touch_read() -> tuple[int, int]:
    """(node records, bucket entries) loaded since the last read; resets them."""
    a, b = C.c_int64(), C.c_int64()
    call("pg_knn_touch_read", C.byref(a), C.byref(b))
    return int(a.value), int(b.value)


# ---------------------------------------------------------------- BDL forest
class BDL:
    """Owner of a pg_bdl handle (a batch-dynamic forest of kd-trees)."""

    def __init__(self, dim: int, buffer_size: int, leaf_size: int = 16, stream=None):
        out = C.c_void_p()
        call("pg_bdl_create", dim, buffer_size, leaf_size, _stream(stream), C.byref(out))
        self._h = out
        self.dim = dim
        self.buffer_size = buffer_size

    @property
    def handle(self):
        if not self._h:
            raise RuntimeError("forest already freed")
        return self._h

    def free(self) -> None:
        if self._h:
            call("pg_bdl_free", self._h)
            self._h = C.c_void_p(None)

    def __del__(self):
        try:
            self.free()
        except Exception:
            pass

    def insert(self, points: torch.Tensor, return_ids: bool = False):
        return pg_bdl_insert(self, points, return_ids)

    def erase(self, points: torch.Tensor) -> None:
        pg_bdl_erase(self, points)

    def knn(self, queries: torch.Tensor, k: int, variant: int = KNN_AUTO):
        return pg_bdl_knn(self, queries, k, variant)

    def size(self) -> int:
        return pg_bdl_size(self)

    def structure(self) -> dict:
        return pg_bdl_structure(self)

    def slot_of(self) -> np.ndarray:
        return pg_bdl_slot_of(self)


def pg_bdl_create(dim: int, buffer_size: int, leaf_size: int = 16, stream=None) -> BDL:
    return BDL(dim, buffer_size, leaf_size, stream)


def pg_bdl_insert(bdl: BDL, points: torch.Tensor, return_ids: bool = False):
    pts = _dev(points, torch.float32, "points", 2)
    cnt = pts.shape[0]
    ids = torch.empty(cnt, dtype=torch.int32, device=pts.device) if return_ids else None
    call("pg_bdl_insert", bdl.handle, _ptr(pts) if cnt else None, cnt, _ptr(ids))
    return ids


def pg_bdl_erase(bdl: BDL, points: torch.Tensor) -> None:
    pts = _dev(points, torch.float32, "points", 2)
    call("pg_bdl_erase", bdl.handle, _ptr(pts) if pts.shape[0] else None, pts.shape[0])


def pg_bdl_knn(bdl: BDL, queries: torch.Tensor, k: int, variant: int = KNN_AUTO):
    q = _dev(queries, torch.float32, "queries", 2)
    if q.shape[1] != bdl.dim:
        raise ValueError("queries have the wrong dimension")
    m = q.shape[0]
    oi = torch.empty((m, k), dtype=torch.int32, device=q.device)
    od = torch.empty((m, k), dtype=torch.float32, device=q.device)
    call("pg_bdl_knn_ex", bdl.handle, _ptr(q) if m else None, m, k, variant, _ptr(oi), _ptr(od))
    return oi, od


def pg_bdl_size(bdl: BDL) -> int:
    v = C.c_int64()
    call("pg_bdl_size", bdl.handle, C.byref(v))
    return int(v.value)


def pg_bdl_structure(bdl: BDL) -> dict:
    F = C.c_uint64()
    slots = np.zeros(64, np.int64)
    buf = C.c_int64()
    nid = C.c_int64()
    call("pg_bdl_structure", bdl.handle, C.byref(F), slots.ctypes.data, C.byref(buf), C.byref(nid))
    return {"F": int(F.value), "slot_live": slots, "buffer_live": int(buf.value), "next_id": int(nid.value)}


def pg_bdl_slot_of(bdl: BDL) -> np.ndarray:
    nid = pg_bdl_structure(bdl)["next_id"]
    out = np.zeros(max(nid, 1), np.int8)
    call("pg_bdl_slot_of", bdl.handle, out.ctypes.data)
    return out[:nid]


def pg_bdl_free(bdl: BDL) -> None:
    bdl.free()


# ---------------------------------------------------------------- backward
def _backward_inputs(data, queries, idx, grad_dist):
    """Checked (data, queries, idx, grad_dist, n, m, dim, k): float32/int32 CUDA
    tensors on one device, queries (m, dim) matching data (n, dim), grad_dist
    of idx's shape (m, k).  Types and shapes are checked before devices, so a
    malformed call fails the same way on any machine, before any launch."""
    spec = ((data, torch.float32, "data"), (queries, torch.float32, "queries"), (idx, torch.int32, "idx"),
            (grad_dist, torch.float32, "grad_dist"))
    for t, dtype, what in spec:
        if not isinstance(t, torch.Tensor):
            raise TypeError(f"{what} must be a torch.Tensor")
        if t.dtype != dtype:
            raise TypeError(f"{what} must be {dtype}, got {t.dtype}")
        if t.dim() != 2:
            raise ValueError(f"{what} must have 2 dimensions")
    n, dim = data.shape
    m, k = idx.shape
    if tuple(queries.shape) != (m, dim):
        raise ValueError(f"queries must have shape ({m}, {dim}) to match idx and data, got {tuple(queries.shape)}")
    if tuple(grad_dist.shape) != (m, k):
        raise ValueError(f"grad_dist must have idx's shape ({m}, {k}), got {tuple(grad_dist.shape)}")
    data = _dev(data, torch.float32, "data", 2)
    for t, what in ((queries, "queries"), (idx, "idx"), (grad_dist, "grad_dist")):
        if not t.is_cuda or t.device != data.device:
            raise ValueError(f"{what} must be a CUDA tensor on data's device {data.device}")
    return data, queries.contiguous(), idx.contiguous(), grad_dist.contiguous(), n, m, dim, k


def _grad_out(t, shape, dev, what):
    """A caller-provided gradient output: None, or a contiguous float32 CUDA
    tensor of exactly `shape` on `dev` (never copied: the kernels write it)."""
    if t is None:
        return None
    if not isinstance(t, torch.Tensor):
        raise TypeError(f"{what} must be a torch.Tensor or None")
    if t.dtype != torch.float32:
        raise TypeError(f"{what} must be torch.float32, got {t.dtype}")
    if tuple(t.shape) != tuple(shape):
        raise ValueError(f"{what} must have shape {tuple(shape)}, got {tuple(t.shape)}")
    if not t.is_contiguous():
        raise ValueError(f"{what} must be contiguous")
    if not t.is_cuda or t.device != dev:
        raise ValueError(f"{what} must be a CUDA tensor on {dev}")
    return t


def pg_knn_backward(data: torch.Tensor, queries: torch.Tensor, idx: torch.Tensor, grad_dist: torch.Tensor,
                    need_queries: bool = True, need_data: bool = True, stream=None):
    data, queries, idx, grad_dist, n, m, dim, k = _backward_inputs(data, queries, idx, grad_dist)
    gq = torch.empty((m, dim), dtype=torch.float32, device=data.device) if need_queries else None
    gp = torch.empty((n, dim), dtype=torch.float32, device=data.device) if need_data else None
    call("pg_knn_backward", _ptr(data) if n else None, n, _ptr(queries) if m else None, m, dim, k,
         _ptr(idx) if m else None, _ptr(grad_dist) if m else None, _ptr(gq) if gq is not None and m else None,
         _ptr(gp) if gp is not None and n else None, _stream(stream))
    return gq, gp


def pg_knn_backward_noalloc(data: torch.Tensor, queries: torch.Tensor, idx: torch.Tensor,
                            grad_dist: torch.Tensor, grad_queries: torch.Tensor | None,
                            grad_data: torch.Tensor | None, stream=None):
    """pg_knn_backward into caller-provided outputs (grad_queries (m, dim),
    grad_data (n, dim), float32, contiguous, on data's device; either may be
    None), using only the library's fixed device scratch: the library
    allocates nothing."""
    data, queries, idx, grad_dist, n, m, dim, k = _backward_inputs(data, queries, idx, grad_dist)
    gq = _grad_out(grad_queries, (m, dim), data.device, "grad_queries")
    gp = _grad_out(grad_data, (n, dim), data.device, "grad_data")
    call("pg_knn_backward_noalloc", _ptr(data) if n else None, n, _ptr(queries) if m else None, m, dim, k,
         _ptr(idx) if m else None, _ptr(grad_dist) if m else None, _ptr(gq) if gq is not None and m else None,
         _ptr(gp) if gp is not None and n else None, _stream(stream))
    return grad_queries, grad_data


# ---------------------------------------------------------------- batched
def _offsets(off) -> np.ndarray:
    if isinstance(off, torch.Tensor):
        off = off.detach().cpu().numpy()
    return np.ascontiguousarray(off, dtype=np.int64)


def pg_batched_chamfer(a: torch.Tensor, a_off, b: torch.Tensor, b_off, k: int, leaf_size: int = 16,
                       want_dist: bool = False, stream=None):
    a = _dev(a, torch.float32, "a", 2)
    b = _dev(b, torch.float32, "b", 2)
    ao, bo = _offsets(a_off), _offsets(b_off)
    npairs = len(ao) - 1
    dim = a.shape[1]
    dev = a.device
    loss = torch.empty(npairs, dtype=torch.float32, device=dev)
    iab = torch.empty((a.shape[0], k), dtype=torch.int32, device=dev)
    iba = torch.empty((b.shape[0], k), dtype=torch.int32, device=dev)
    dab = torch.empty((a.shape[0], k), dtype=torch.float32, device=dev) if want_dist else None
    dba = torch.empty((b.shape[0], k), dtype=torch.float32, device=dev) if want_dist else None
    call("pg_batched_chamfer", _ptr(a), ao.ctypes.data, _ptr(b), bo.ctypes.data, npairs, dim, k, leaf_size,
         _ptr(loss), _ptr(iab), _ptr(iba), _ptr(dab), _ptr(dba), _stream(stream))
    return loss, iab, iba, dab, dba


def pg_batched_chamfer_backward(a, a_off, b, b_off, k, idx_ab, idx_ba, grad_loss, stream=None):
    a = _dev(a, torch.float32, "a", 2)
    b = _dev(b, torch.float32, "b", 2)
    ao, bo = _offsets(a_off), _offsets(b_off)
    idx_ab = _dev(idx_ab, torch.int32, "idx_ab", 2)
    idx_ba = _dev(idx_ba, torch.int32, "idx_ba", 2)
    grad_loss = _dev(grad_loss, torch.float32, "grad_loss", 1)
    ga = torch.empty_like(a)
    gb = torch.empty_like(b)
    call("pg_batched_chamfer_backward", _ptr(a), ao.ctypes.data, _ptr(b), bo.ctypes.data, len(ao) - 1,
         a.shape[1], k, _ptr(idx_ab), _ptr(idx_ba), _ptr(grad_loss), _ptr(ga), _ptr(gb), _stream(stream))
    return ga, gb


# ---------------------------------------------------------------- diagnostics
def launch_count() -> int:
    return int(_lib.load().pg_launch_count())


def version() -> str:
    return _lib.load().pg_version().decode()


def profile_enable(on: bool = True) -> None:
    call("pg_profile_enable", 1 if on else 0)


def profile_read(prefix: str):
    ms = C.c_double()
    cnt = C.c_int64()
    call("pg_profile_read", prefix.encode(), C.byref(ms), C.byref(cnt))
    return float(ms.value), int(cnt.value)


def debug_fail_alloc_after(n: int) -> None:
    call("pg_debug_fail_alloc_after", n)


def debug_batched_faults(skip_publish: bool, wait_limit: int = 0) -> None:
    call("pg_debug_batched_faults", 1 if skip_publish else 0, wait_limit)
