"""Tie-tolerant comparison of a k-NN answer with the oracle's.

Rule: per query, the returned index set equals the oracle's except for ties:
an index that is in one set and not the other must have an exact (float64)
distance within RTOL relative of the oracle's k-th distance.  Returned
distances (ascending) agree with the oracle's within RTOL relative, with an
absolute floor ATOL for exact zeros.  Padding (fewer than k live points) is
index -1 with distance +inf on both sides.
"""
from __future__ import annotations

import numpy as np

RTOL = 1e-5
ATOL = 1e-12


def exact_dist(data, q, idx):
    P = np.asarray(data, np.float64)[idx]
    return ((P - np.asarray(q, np.float64)[None, :]) ** 2).sum(axis=1)


def compare_knn(got_idx, got_dist, ora_idx, ora_dist, data, queries, ids=None,
                rtol=RTOL, atol=ATOL, max_report=5):
    """Raise AssertionError describing the first mismatching rows, if any.

    data/queries: the float32 arrays; ids: optional id per data row (when the
    answers are ids rather than row numbers).  Returns the number of rows where
    a tie was resolved differently (for reporting).
    """
    got_idx = np.asarray(got_idx, np.int64)
    ora_idx = np.asarray(ora_idx, np.int64)
    got_dist = np.asarray(got_dist, np.float64)
    ora_dist = np.asarray(ora_dist, np.float64)
    assert got_idx.shape == ora_idx.shape, (got_idx.shape, ora_idx.shape)
    m, k = ora_idx.shape
    if m == 0:
        return 0
    row_of = None
    if ids is not None:
        ids = np.asarray(ids, np.int64)
        row_of = {int(v): r for r, v in enumerate(ids)}
    problems = []
    # distances, slot by slot
    pad_g = got_idx < 0
    pad_o = ora_idx < 0
    bad_pad = np.any(pad_g != pad_o, axis=1)
    finite = ~pad_o
    tol = rtol * np.abs(ora_dist) + atol
    with np.errstate(invalid="ignore"):
        dbad = np.any(finite & ~(np.abs(got_dist - ora_dist) <= tol), axis=1)
        pbad = np.any(pad_g & ~np.isinf(got_dist), axis=1)
    for r in np.nonzero(bad_pad | dbad | pbad)[0][:max_report]:
        problems.append(f"row {r}: dist/pad mismatch got {got_idx[r]} {got_dist[r]} "
                        f"want {ora_idx[r]} {ora_dist[r]}")
    # index sets
    gs = np.sort(got_idx, axis=1)
    os_ = np.sort(ora_idx, axis=1)
    dup = np.any((gs[:, 1:] == gs[:, :-1]) & (gs[:, 1:] >= 0), axis=1)
    for r in np.nonzero(dup)[0][:max_report]:
        problems.append(f"row {r}: duplicate index in {got_idx[r]}")
    diff_rows = np.nonzero(np.any(gs != os_, axis=1))[0]
    ties = 0
    for r in diff_rows:
        g = set(int(v) for v in got_idx[r] if v >= 0)
        o = set(int(v) for v in ora_idx[r] if v >= 0)
        sym = sorted(g ^ o)
        kth = ora_dist[r][~pad_o[r]].max() if np.any(~pad_o[r]) else np.inf
        rows = [row_of[t] if row_of is not None else t for t in sym]
        if row_of is None and any(t < 0 or t >= len(data) for t in sym):
            problems.append(f"row {r}: index out of range {sym}")
            continue
        dd = exact_dist(data, queries[r], rows)
        ok = np.abs(dd - kth) <= rtol * kth + atol
        if not np.all(ok):
            if len(problems) < max_report:
                problems.append(f"row {r}: index sets differ beyond ties: got {sorted(g)} "
                                f"want {sorted(o)}; extra dists {dd} kth {kth}")
        else:
            ties += 1
    if problems:
        raise AssertionError(f"{len(problems)}+ mismatching rows of {m}:\n" + "\n".join(problems))
    return ties
