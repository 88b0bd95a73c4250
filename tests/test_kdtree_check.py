"""The kd-tree invariant checker accepts a hand-built valid tree and rejects
planted defects (each a plausible builder mistake)."""
from __future__ import annotations

import copy

import numpy as np
import pytest

from oracle.kdtree_check import TreeInvariantError, check_tree


def _hand_tree():
    """Four 2D points: split x at 0.5*0+0.5*3 = 1.5 -> {0,1 | 2,3}, then each side
    is a leaf of two points (leaf_size 2)."""
    pts = np.array([[0, 0], [3, 1], [1, 2], [2, 0]], np.float32)
    dc = 2
    # bucket order: left (x < 1.5) = ids 0, 2 ; right = ids 1, 3
    order = [0, 2, 1, 3]
    bucket = np.zeros((4, 4), np.float32)
    bucket[:, :2] = pts[order]
    bucket[:, dc] = np.asarray(order, np.int32).view(np.float32)
    node = np.zeros((1, 4 * dc + 4), np.float32)
    node[0, 0:2] = [0, 0]      # lo0
    node[0, 2:4] = [1, 2]      # hi0
    node[0, 4:6] = [2, 0]      # lo1
    node[0, 6:8] = [3, 1]      # hi1
    node[0, 8:12] = np.asarray([0, 2, 2, 2], np.int32).view(np.float32)
    return pts, {
        "dim": 2, "dc": dc, "nodes": node, "split_dim": np.array([0], np.int32),
        "split_val": np.array([1.5], np.float32), "bucket": bucket,
        "root_ref": 0, "root_cnt": 0, "root_lo": np.array([0, 0], np.float32),
        "root_hi": np.array([3, 2], np.float32), "num_nodes": 1,
    }


def test_valid_tree_passes():
    pts, exp = _hand_tree()
    st = check_tree(pts, exp, leaf_size=2, depth_cap=10)
    assert st == {"leaves": 2, "depth": 1, "max_leaf": 2}


def _mutations():
    def wrong_box(e):
        e["nodes"][0, 2] = 1.5
    def wrong_split_value(e):
        e["split_val"][0] = np.float32(1.25)
    def wrong_split_dim(e):
        e["split_dim"][0] = 1
    def lost_point(e):
        e["bucket"][3, 2] = np.asarray([2], np.int32).view(np.float32)[0]
    def moved_coordinate(e):
        e["bucket"][1, 0] = 1.0000001
    def overlapping_leaves(e):
        w = e["nodes"][0].view(np.int32)
        w[10] = 1
    def leaf_too_big(e):
        pass  # checked with leaf_size=1 below
    return [wrong_box, wrong_split_value, wrong_split_dim, lost_point, moved_coordinate,
            overlapping_leaves]


@pytest.mark.parametrize("mutate", _mutations())
def test_planted_defects_fail(mutate):
    pts, exp = _hand_tree()
    exp = copy.deepcopy(exp)
    mutate(exp)
    with pytest.raises(TreeInvariantError):
        check_tree(pts, exp, leaf_size=2, depth_cap=10)


def test_leaf_size_enforced():
    pts, exp = _hand_tree()
    with pytest.raises(TreeInvariantError):
        check_tree(pts, exp, leaf_size=1, depth_cap=10)


def _one_split_tree(pts, left, right, sd, sv):
    """A root node splitting `pts` into two leaves (left ids, right ids) with tight boxes."""
    dc = pts.shape[1]
    order = list(left) + list(right)
    bucket = np.zeros((len(pts), 4), np.float32)
    bucket[:, :dc] = pts[order]
    bucket[:, dc] = np.asarray(order, np.int32).view(np.float32)
    node = np.zeros((1, 4 * dc + 4), np.float32)
    for c, ids in enumerate((left, right)):
        node[0, 2 * c * dc:2 * c * dc + dc] = pts[list(ids)].min(0)
        node[0, 2 * c * dc + dc:2 * c * dc + 2 * dc] = pts[list(ids)].max(0)
    node[0, 4 * dc:4 * dc + 4] = np.asarray([0, len(left), len(left), len(right)], np.int32).view(np.float32)
    return {"dim": dc, "dc": dc, "nodes": node, "split_dim": np.array([sd], np.int32),
            "split_val": np.array([sv], np.float32), "bucket": bucket, "root_ref": 0, "root_cnt": 0,
            "root_lo": pts.min(0), "root_hi": pts.max(0), "num_nodes": 1}


def test_object_median_rule():
    pts = np.array([[0, 0], [3, 1], [1, 2], [2, 0]], np.float32)
    good = _one_split_tree(pts, [0, 2], [3, 1], 0, 2.0)        # the two smallest x left, value = first right x
    check_tree(pts, good, leaf_size=2, depth_cap=10, split="object")
    with pytest.raises(TreeInvariantError):
        check_tree(pts, good, leaf_size=2, depth_cap=10)       # not the spatial median (1.5)
    bad_sizes = _one_split_tree(pts, [0], [2, 3, 1], 0, 1.0)   # left is not the lower half
    with pytest.raises(TreeInvariantError):
        check_tree(pts, bad_sizes, leaf_size=3, depth_cap=10, split="object")
    bad_value = _one_split_tree(pts, [0, 2], [3, 1], 0, 0.5)   # a left point lies above the value
    with pytest.raises(TreeInvariantError):
        check_tree(pts, bad_value, leaf_size=2, depth_cap=10, split="object")
    bad_dim = _one_split_tree(pts, [0, 3], [1, 2], 1, 1.0)     # y is not the widest extent
    with pytest.raises(TreeInvariantError):
        check_tree(pts, bad_dim, leaf_size=2, depth_cap=10, split="object")
    ties = np.array([[0, 0], [1, 0], [1, 1], [1, 2], [2, 0]], np.float32)
    tied = _one_split_tree(ties, [0, 1], [2, 3, 4], 0, 1.0)    # equal coordinates on both sides are allowed
    check_tree(ties, tied, leaf_size=3, depth_cap=10, split="object")
