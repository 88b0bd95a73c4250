"""torch.autograd wrappers of the k-NN distance and its backward kernel.

Forward: kd-tree build + exact k-NN through the C ABI (squared distances).
Backward: pg_knn_backward, which keeps only the neighbour indices, recomputes
the distances and returns deterministic gradients for queries and data.
"""
from __future__ import annotations

import torch

from . import api


class KnnSquaredDistance(torch.autograd.Function):
    """dist[i, j] = |queries[i] - data[idx[i, j]]|^2 for the k nearest data points."""

    @staticmethod
    def forward(ctx, queries, data, k: int, leaf_size: int = 16):
        tree = api.pg_tree_build(data.detach(), leaf_size=leaf_size)
        idx, dist = api.pg_knn(tree, queries.detach(), k)
        tree.free()
        ctx.save_for_backward(queries, data, idx)
        ctx.mark_non_differentiable(idx)
        return dist, idx

    @staticmethod
    def backward(ctx, grad_dist, grad_idx):
        queries, data, idx = ctx.saved_tensors
        need_q, need_p = ctx.needs_input_grad[0], ctx.needs_input_grad[1]
        gq, gp = api.pg_knn_backward(data.detach(), queries.detach(), idx, grad_dist.contiguous(),
                                     need_queries=need_q, need_data=need_p)
        return gq, gp, None, None


def knn_squared_distance(queries: torch.Tensor, data: torch.Tensor, k: int, leaf_size: int = 16):
    """(dist, idx) of the k nearest `data` points of every query, differentiable in dist."""
    return KnnSquaredDistance.apply(queries, data, k, leaf_size)


def chamfer(a: torch.Tensor, b: torch.Tensor, k: int = 1, leaf_size: int = 16) -> torch.Tensor:
    """Sum of squared distances from every point of a to its k nearest in b and back."""
    dab, _ = knn_squared_distance(a, b, k, leaf_size)
    dba, _ = knn_squared_distance(b, a, k, leaf_size)
    return dab.sum() + dba.sum()
