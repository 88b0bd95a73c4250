"""Checker of kd-tree invariants — TEST INFRASTRUCTURE.

A kd-tree (paper, Section 5 intro, after Bentley) is a binary tree in which
every internal node splits its point set into two by an axis-aligned
hyperplane, recursively, until a node holds a small constant number of points
(a leaf).  The paper's k-NN search uses every node's bounding box to prune
(Appendix A.1.3).  The checker verifies, on a tree exported from the CUDA
library, that:

  1. the leaf buckets hold every input point exactly once (same float32 bits,
     with the id it was given);
  2. the leaves' bucket ranges partition [0, n), and every subtree's points
     form one contiguous bucket range;
  3. every internal node has two non-empty children and the split property
     holds: left points have x[dim] < value, right points x[dim] >= value;
  4. the split is a spatial median: the node's tight box is cut in half along
     its widest dimension (reading of "splitting the space along a dimension
     in half", Section 6 BDL experiments): widest = the lowest dimension with
     the largest float32 extent hi - lo, value = fl(0.5*lo + 0.5*hi) in that
     dimension, or hi when that rounds down to lo;
  5. every child box stored in its parent is the exact tight bounding box of
     the child's points;
  6. leaves hold at most leaf_size points unless their points are all equal or
     they sit at the depth cap.

With split="object" rules 3 and 4 become the object-median split (Section 4:
splits by spatial or by object median): the split dimension is still the
widest extent of the tight box, the left child holds floor(c/2) of the node's
c points, and left coordinates <= value <= right coordinates along it.

The exported layout (see the C header) is: per node, float32 words
lo0[DC], hi0[DC], lo1[DC], hi1[DC] followed by int32 words ref0, cnt0, ref1,
cnt1 (cnt > 0: leaf child holding buckets [ref, ref+cnt); cnt == 0: internal
child at node index ref).
"""
from __future__ import annotations

import numpy as np


class TreeInvariantError(AssertionError):
    pass


def _fail(msg):
    raise TreeInvariantError(msg)


def check_tree(points, exp, leaf_size: int, depth_cap: int, split: str = "spatial") -> dict:
    """Check an exported tree against its input points.

    points : (n, dim) float32 input
    exp    : dict with keys dim, dc, nodes (float32 (N, 4*dc+4)), split_dim
             (int32 (N,)), split_val (float32 (N,)), bucket (float32 (n, 4*W)),
             root_ref, root_cnt, root_lo, root_hi (float32 (dim,))
    Returns statistics (number of leaves, max depth, max leaf size).
    """
    pts = np.ascontiguousarray(points, np.float32)
    n, dim = pts.shape
    dc = exp["dc"]
    bucket = exp["bucket"]
    nodes = exp["nodes"]
    if n == 0:
        if exp["root_cnt"] != 0 or exp.get("num_nodes", 0) != 0:
            _fail("empty tree must have no nodes")
        return {"leaves": 0, "depth": 0, "max_leaf": 0}
    ids = bucket[:, dc].view(np.int32).astype(np.int64)
    # 1. permutation and bitwise coordinates
    if not np.array_equal(np.sort(ids), np.arange(n)):
        _fail("bucket ids are not a permutation of 0..n-1")
    if not np.array_equal(bucket[:, :dim].view(np.uint32), pts[ids].view(np.uint32)):
        _fail("bucket coordinates differ from the input rows")
    if dc > dim and np.any(bucket[:, dim:dc] != 0):
        _fail("padding coordinates are not zero")
    coords = bucket[:, :dim]
    words = nodes.view(np.int32)
    lo_off = [0, 2 * dc]
    hi_off = [dc, 3 * dc]

    leaves = []
    max_depth = 0
    max_leaf = 0
    # stack entries: (ref, cnt, lo, hi, depth) where lo/hi is the stored box
    stack = [(exp["root_ref"], exp["root_cnt"], np.asarray(exp["root_lo"], np.float32),
              np.asarray(exp["root_hi"], np.float32), 0)]
    ranges = {}
    order = []
    while stack:
        ref, cnt, lo, hi, depth = stack.pop()
        max_depth = max(max_depth, depth)
        if cnt > 0:
            seg = coords[ref:ref + cnt]
            _check_box(seg, lo, hi, f"leaf [{ref},{ref + cnt})")
            if cnt > leaf_size:
                same = np.all(seg.view(np.uint32) == seg[0:1].view(np.uint32))
                if not same and depth < depth_cap:
                    _fail(f"leaf of {cnt} > leaf_size {leaf_size} points at depth {depth}")
            leaves.append((ref, cnt))
            max_leaf = max(max_leaf, cnt)
            continue
        if cnt != 0:
            _fail(f"bad child count {cnt}")
        node = ref
        if not (0 <= node < nodes.shape[0]):
            _fail(f"node index {node} out of range")
        if depth >= depth_cap:
            _fail(f"internal node at depth {depth} >= cap {depth_cap}")
        order.append((node, lo, hi, depth))
        for c in (0, 1):
            cref = int(words[node, 4 * dc + 2 * c])
            ccnt = int(words[node, 4 * dc + 2 * c + 1])
            clo = nodes[node, lo_off[c]:lo_off[c] + dim]
            chi = nodes[node, hi_off[c]:hi_off[c] + dim]
            stack.append((cref, ccnt, clo, chi, depth + 1))
    # 2. leaves partition [0, n)
    leaves.sort()
    pos = 0
    for ref, cnt in leaves:
        if ref != pos:
            _fail(f"leaf ranges do not tile [0,n): expected start {pos}, got {ref}")
        pos += cnt
    if pos != n:
        _fail(f"leaf ranges cover {pos} of {n} points")
    # subtree ranges (post-order over the recorded internal nodes)
    span = {}

    def child_span(node, c):
        cref = int(words[node, 4 * dc + 2 * c])
        ccnt = int(words[node, 4 * dc + 2 * c + 1])
        return (cref, cref + ccnt) if ccnt > 0 else span[cref]

    for node, lo, hi, depth in reversed(order):
        l0, l1 = child_span(node, 0)
        r0, r1 = child_span(node, 1)
        if l1 != r0:
            _fail(f"node {node}: children ranges not adjacent ({l0},{l1}) ({r0},{r1})")
        if l1 <= l0 or r1 <= r0:
            _fail(f"node {node}: empty child")
        span[node] = (l0, r1)
        # 5. child boxes are tight
        for c, (a, b) in enumerate(((l0, l1), (r0, r1))):
            clo = nodes[node, lo_off[c]:lo_off[c] + dim]
            chi = nodes[node, hi_off[c]:hi_off[c] + dim]
            _check_box(coords[a:b], clo, chi, f"node {node} child {c}")
        # 3. split property and 4. spatial-median rule
        sd = int(exp["split_dim"][node])
        sv = np.float32(exp["split_val"][node])
        if not (0 <= sd < dim):
            _fail(f"node {node}: split dim {sd}")
        seg = coords[l0:r1]
        tlo = seg.min(axis=0)
        thi = seg.max(axis=0)
        ext = (thi - tlo).astype(np.float32)
        want_dim = int(np.argmax(ext))
        if ext[want_dim] <= 0:
            _fail(f"node {node}: split of a set of identical points")
        if split == "object":
            if sd != want_dim:
                _fail(f"node {node}: split dim {sd} is not the widest {want_dim}")
            if l1 - l0 != (r1 - l0) // 2:
                _fail(f"node {node}: left child holds {l1 - l0} of {r1 - l0} points, not the lower half")
            if not np.all(coords[l0:l1, sd] <= sv) or not np.all(coords[r0:r1, sd] >= sv):
                _fail(f"node {node}: object-median split property violated (dim {sd}, value {sv})")
            continue
        if not np.all(coords[l0:l1, sd] < sv) or not np.all(coords[r0:r1, sd] >= sv):
            _fail(f"node {node}: split property violated (dim {sd}, value {sv})")
        lo_s, hi_s = tlo[want_dim], thi[want_dim]
        mid = np.float32(np.float32(0.5) * lo_s) + np.float32(np.float32(0.5) * hi_s)
        mid = np.float32(mid)
        if not mid > lo_s:
            mid = hi_s
        if mid > hi_s:
            mid = hi_s
        if sd != want_dim or sv.view(np.uint32) != np.float32(mid).view(np.uint32):
            _fail(f"node {node}: split ({sd},{sv}) is not the spatial median ({want_dim},{mid})")
    if exp["root_cnt"] == 0:
        r = span[exp["root_ref"]]
        if r != (0, n):
            _fail("root does not span all points")
    _check_box(coords, np.asarray(exp["root_lo"], np.float32), np.asarray(exp["root_hi"], np.float32), "root")
    return {"leaves": len(leaves), "depth": max_depth, "max_leaf": max_leaf}


def _check_box(seg, lo, hi, what):
    lo = np.asarray(lo, np.float32)
    hi = np.asarray(hi, np.float32)
    tlo = seg.min(axis=0)
    thi = seg.max(axis=0)
    if not (np.array_equal(tlo, lo) and np.array_equal(thi, hi)):
        _fail(f"{what}: stored box {lo},{hi} is not the tight box {tlo},{thi}")
