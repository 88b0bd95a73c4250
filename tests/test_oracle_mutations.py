"""Planted mistakes in the oracle, on the CPU: every mutant must fail at least
one of the pins the oracle is trusted by, and the unmodified oracle must pass
all of them.

C k-NN oracle: a copy of oracle/pargeo_oracle.c with one textual change (a
reversed tie-break, a dropped term, a sign or index error, a wrong insertion
bound, broken padding, an ignored live mask or id list, another metric) is
compiled with gcc and loaded beside the real one.  Python oracle functions
(knn_grad, range_search, knn_graph): a copy of the function's source with one
change, executed in the oracle module's namespace.  The pins here restate the
ones of test_oracle.py in a form that takes the implementation as an argument:
exact rational (distance, id) order, the integer-lattice closed form, scipy's
cKDTree, padding, live mask and ids; torch autograd and central differences
for the gradient; hand examples, closed forms and a distance-matrix
restatement for range search and the k-NN graph.  The BDL bookkeeping model:
a copy of the class with one change, run through the pins of
test_oracle_bdl.py (the paper's worked example, the pure-insert closed form,
the 4M start, the cascade reading, erase semantics, the half-capacity rule,
invariants)."""
from __future__ import annotations

import ctypes
import inspect
import os
import subprocess
from fractions import Fraction

import numpy as np
import pytest

import oracle
from knn_compare import compare_knn
from paper_2207_01834_gb300 import synth

SRC = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "oracle", "pargeo_oracle.c")

# ---------------------------------------------------------------- C k-NN oracle
C_MUTANTS = {
    "tie_break_reversed": [("a.d == b.d && a.id < b.id", "a.d == b.d && a.id > b.id")],
    "last_term_dropped": [("for (int c = 0; c < dim; ++c) {", "for (int c = 0; c < dim - 1; ++c) {")],
    "sign_error": [("double diff = (double)q[c] - (double)data", "double diff = (double)q[c] + (double)data")],
    "coordinate_index_dropped": [("(double)data[t * (int64_t)dim + c]", "(double)data[t * (int64_t)dim]")],
    "l1_metric": [("D += diff * diff;", "D += fabs(diff);")],
    "insertion_stops_at_slot_1": [("while (j > 0 && cand_less", "while (j > 1 && cand_less")],
    "kth_test_inverted": [("} else if (cand_less(x, best[k - 1])) {", "} else if (cand_less(best[k - 1], x)) {")],
    "padding_id_zero": [("out_idx[j] = -1;", "out_idx[j] = 0;")],
    "padding_distance_zero": [("out_dist[j] = INFINITY;", "out_dist[j] = 0.0;")],
    "live_mask_ignored": [("if (live && !live[t]) continue;", "")],
    "ids_ignored": [("cand x = {D, ids ? ids[t] : t};", "cand x = {D, t};")],
    "query_row_shifted": [("j->queries + i * (int64_t)j->dim", "j->queries + (i > 0 ? i - 1 : 0) * (int64_t)j->dim")],
}


def _load_c(path):
    lib = ctypes.CDLL(path)
    lib.oracle_knn_f64.restype = ctypes.c_int
    lib.oracle_knn_f64.argtypes = [
        ctypes.c_void_p, ctypes.c_int64, ctypes.c_void_p, ctypes.c_int64, ctypes.c_int, ctypes.c_int,
        ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int]

    def knn(data, queries, k, live=None, ids=None):
        data = np.ascontiguousarray(data, np.float32)
        queries = np.ascontiguousarray(queries, np.float32)
        n, m, d = data.shape[0], queries.shape[0], queries.shape[1]
        oi = np.empty((m, k), np.int64)
        od = np.empty((m, k), np.float64)
        lv = None if live is None else np.ascontiguousarray(live, np.uint8)
        ii = None if ids is None else np.ascontiguousarray(ids, np.int64)
        rc = lib.oracle_knn_f64(data.ctypes.data, n, queries.ctypes.data, m, d, k,
                                None if lv is None else lv.ctypes.data, None if ii is None else ii.ctypes.data,
                                oi.ctypes.data, od.ctypes.data, 1)
        assert rc == 0
        return oi, od

    knn._lib = lib   # keep the library loaded
    return knn


def _compile(tmp_path, name, edits):
    src = open(SRC).read()
    for old, new in edits:
        assert old in src, f"mutation {name}: pattern not found"
        src = src.replace(old, new)
    c = tmp_path / f"{name}.c"
    so = tmp_path / f"lib{name}.so"
    c.write_text(src)
    subprocess.check_call(["gcc", "-O1", "-std=c11", "-fPIC", "-shared", "-pthread", "-o", str(so), str(c), "-lm"])
    return _load_c(str(so))


def _exact(data, q, k):
    key = [(sum((Fraction(float(q[c])) - Fraction(float(p[c]))) ** 2 for c in range(len(q))), t)
           for t, p in enumerate(data)]
    order = sorted(range(len(data)), key=lambda t: key[t])[:k]
    return [t for t in order] + [-1] * (k - len(order)), [float(key[t][0]) for t in order] + [np.inf] * (k - len(order))


def _pin_subsets(knn):
    for seed in range(6):
        g = np.random.default_rng(seed)
        n, d = int(g.integers(1, 9)), int(g.integers(1, 4))
        k = int(g.integers(1, n + 2))
        for data, qs in ((g.integers(0, 3, (n, d)).astype(np.float32), g.integers(0, 3, (4, d)).astype(np.float32)),
                         (g.random((n, d)).astype(np.float32), g.random((3, d)).astype(np.float32))):
            idx, dist = knn(data, qs, k)
            for r in range(len(qs)):
                wi, wd = _exact(data, qs[r], k)
                assert list(idx[r]) == wi
                np.testing.assert_allclose(dist[r], wd, rtol=1e-14)


def _pin_lattice(knn):
    nx, ny = 12, 9
    pts = synth.lattice((nx, ny))
    idx, dist = knn(pts, pts, 5)
    for x in range(1, nx - 1):
        for y in range(1, ny - 1):
            me = x * ny + y
            assert list(idx[me]) == [me] + sorted([(x - 1) * ny + y, me - 1, me + 1, (x + 1) * ny + y])
            assert list(dist[me]) == [0.0, 1.0, 1.0, 1.0, 1.0]


def _pin_ckdtree(knn):
    spatial = pytest.importorskip("scipy.spatial")
    data = synth.uniform(1000, 3, seed=21)
    qs = synth.gmm(100, 3, seed=22)
    idx, dist = knn(data, qs, 10)
    sd, si = spatial.cKDTree(data.astype(np.float64)).query(qs.astype(np.float64), k=10)
    compare_knn(si, sd ** 2, idx, dist, data, qs)


def _pin_padding(knn):
    data = synth.uniform(3, 2, seed=1)
    idx, dist = knn(data, synth.uniform(4, 2, seed=2), 5)
    assert np.all(idx[:, 3:] == -1) and np.all(np.isinf(dist[:, 3:])) and np.all(idx[:, :3] >= 0)


def _pin_live_ids(knn):
    data = synth.uniform(200, 3, seed=4)
    qs = synth.uniform(50, 3, seed=5)
    live = np.ones(200, bool)
    live[::3] = False
    ids = np.arange(200, dtype=np.int64) * 10 + 7
    idx, dist = knn(data, qs, 6, live=live, ids=ids)
    ri, rd = knn(data[live], qs, 6)
    assert np.array_equal(idx, ids[live][ri]) and np.array_equal(dist, rd)


KNN_PINS = [_pin_subsets, _pin_lattice, _pin_ckdtree, _pin_padding, _pin_live_ids]


def _failing_pins(pins, impl):
    """Names of the pins that reject `impl` (a failed check, or a crash)."""
    failed = []
    for pin in pins:
        try:
            pin(impl)
        except Exception:
            failed.append(getattr(pin, "__name__", repr(pin)))
    return failed


def test_unmodified_c_oracle_passes_every_pin(tmp_path):
    assert _failing_pins(KNN_PINS, _compile(tmp_path, "original", [])) == []


@pytest.mark.parametrize("name", sorted(C_MUTANTS))
def test_c_oracle_mutant_fails_a_pin(tmp_path, name):
    assert _failing_pins(KNN_PINS, _compile(tmp_path, name, C_MUTANTS[name])), f"mutant {name} passed every pin"


# ---------------------------------------------------------------- Python oracle functions
def _mutant(fn, edits):
    src = inspect.getsource(fn)
    for old, new in edits:
        assert old in src, f"pattern not found in {fn.__name__}: {old}"
        src = src.replace(old, new)
    ns = dict(vars(oracle))
    exec(compile(src, f"<mutant of {fn.__name__}>", "exec"), ns)
    return ns[fn.__name__]


def _selection(seed, n=40, m=15, d=3, k=4, pad=False):
    g = np.random.default_rng(seed)
    data = g.random((n, d)).astype(np.float32)
    q = g.random((m, d)).astype(np.float32)
    idx, _ = oracle.knn(data, q, k)
    if pad:
        idx[::3, -1] = -1
    return data, q, idx, g.standard_normal((m, k))


def _pin_grad_autograd(grad):
    torch = pytest.importorskip("torch")
    data, q, idx, w = _selection(1)
    gq, gp = grad(data, q, idx, w)
    P = torch.tensor(data, dtype=torch.float64, requires_grad=True)
    Q = torch.tensor(q, dtype=torch.float64, requires_grad=True)
    (torch.tensor(w) * ((Q[:, None, :] - P[torch.tensor(idx)]) ** 2).sum(-1)).sum().backward()
    np.testing.assert_allclose(gq, Q.grad.numpy(), rtol=1e-12, atol=1e-12)
    np.testing.assert_allclose(gp, P.grad.numpy(), rtol=1e-12, atol=1e-12)


def _pin_grad_fd_with_padding(grad):
    data, q, idx, w = _selection(2, n=12, m=6, d=2, k=3, pad=True)
    gq, gp = grad(data, q, idx, w)
    P, Q = data.astype(np.float64), q.astype(np.float64)

    def loss():
        return sum(w[i, j] * float(((Q[i] - P[idx[i, j]]) ** 2).sum())
                   for i in range(len(Q)) for j in range(idx.shape[1]) if idx[i, j] >= 0)

    h = 1e-4
    for arr, g in ((Q, gq), (P, gp)):
        for i in range(arr.shape[0]):
            for c in range(arr.shape[1]):
                keep = arr[i, c]
                arr[i, c] = keep + h
                lp = loss()
                arr[i, c] = keep - h
                lm = loss()
                arr[i, c] = keep
                assert abs((lp - lm) / (2 * h) - g[i, c]) < 1e-8


GRAD_MUTANTS = {
    "factor_2_dropped": [("coef = 2.0 * W[valid]", "coef = W[valid]")],
    "data_sign_flipped": [("np.add.at(gp, cols, -contrib)", "np.add.at(gp, cols, contrib)")],
    "operands_transposed": [("diff = Q[rows] - P[cols]", "diff = P[cols] - Q[rows]")],
    "padding_counted": [("valid = idx >= 0", "valid = idx >= -1")],
    "weights_ignored": [("coef = 2.0 * W[valid]", "coef = 2.0 * np.ones_like(W[valid])")],
}


def _pin_range_hand(rs):
    p = np.array([[0, 0], [1, 0], [0, 2], [3, 4]], np.float32)
    assert [g.tolist() for g in rs(p, np.array([[0, 0], [3, 3]], np.float32), 2.0)] == [[0, 1, 2], [3]]


def _pin_range_lattice(rs):
    p = synth.lattice((7, 5))
    for i, g in enumerate(rs(p, p, 1.0)):
        x, y = p[i]
        assert len(g) == 1 + (x > 0) + (x < 6) + (y > 0) + (y < 4)


def _pin_range_ckdtree(rs):
    spatial = pytest.importorskip("scipy.spatial")
    rng = np.random.default_rng(9)
    p = rng.random((1500, 3)).astype(np.float32)
    q = rng.random((100, 3)).astype(np.float32)
    r = 0.1
    got = rs(p, q, r)
    ref = spatial.cKDTree(p.astype(np.float64)).query_ball_point(q.astype(np.float64), float(np.float32(r)))
    for i in range(len(q)):
        dd = ((p.astype(np.float64) - q[i].astype(np.float64)) ** 2).sum(1)
        near = np.abs(dd - float(np.float32(r)) ** 2) <= 1e-9
        assert {x for x in set(got[i].tolist()) ^ set(ref[i]) if not near[x]} == set()


RANGE_MUTANTS = {
    "strict_boundary": [("np.nonzero(d <= r2)", "np.nonzero(d < r2)")],
    "radius_not_squared": [("r2 = float(np.float32(radius)) ** 2", "r2 = float(np.float32(radius))")],
    "term_dropped": [("d = ((p - q[i]) ** 2).sum(1)", "d = ((p - q[i])[:, :-1] ** 2).sum(1)")],
}


def _pin_graph_hand(kg):
    p = np.array([[0, 0], [1, 0], [3, 0], [6, 0], [10, 0]], np.float32)
    assert kg(p, 1).tolist() == [[0, 1], [1, 2], [2, 3], [3, 4]]


def _pin_graph_line(kg):
    for n in (4, 7, 30):
        p = np.stack([np.arange(n), np.zeros(n)], 1).astype(np.float32)
        want = sorted({(i, i + 1) for i in range(n - 1)} | {(0, 2), (n - 3, n - 1)})
        assert kg(p, 2).tolist() == [list(e) for e in want]


def _pin_graph_matrix(kg):
    rng = np.random.default_rng(5)
    for n, d, k in ((40, 2, 3), (50, 3, 5)):
        for p in (rng.random((n, d)).astype(np.float32), np.round(rng.random((n, d)) * 4).astype(np.float32)):
            p64 = p.astype(np.float64)
            dm = ((p64[:, None, :] - p64[None, :, :]) ** 2).sum(-1)
            edges = set()
            for i in range(n):
                for _, j in sorted((dm[i, j], j) for j in range(n) if j != i)[:k]:
                    edges.add((min(i, j), max(i, j)))
            assert kg(p, k).tolist() == [list(e) for e in sorted(edges)]


GRAPH_MUTANTS = {
    "one_neighbour_short": [("for j in others[:k]:", "for j in others[:k - 1]:")],
    "directed_edges": [("edges.add((min(i, j), max(i, j)))", "edges.add((i, j))")],
    "self_kept": [("others = [int(t) for t in idx[i] if t >= 0 and t != i]",
                   "others = [int(t) for t in idx[i] if t >= 0]")],
}

PY_CASES = {
    "knn_grad": (oracle.knn_grad, [_pin_grad_autograd, _pin_grad_fd_with_padding], GRAD_MUTANTS),
    "range_search": (oracle.range_search, [_pin_range_hand, _pin_range_lattice, _pin_range_ckdtree], RANGE_MUTANTS),
    "knn_graph": (oracle.knn_graph, [_pin_graph_hand, _pin_graph_line, _pin_graph_matrix], GRAPH_MUTANTS),
}


@pytest.mark.parametrize("fname", sorted(PY_CASES))
def test_unmodified_python_oracle_passes_every_pin(fname):
    fn, pins, _ = PY_CASES[fname]
    assert _failing_pins(pins, fn) == []


@pytest.mark.parametrize("fname,name", [(f, m) for f in sorted(PY_CASES) for m in sorted(PY_CASES[f][2])])
def test_python_oracle_mutant_fails_a_pin(fname, name):
    fn, pins, mutants = PY_CASES[fname]
    assert _failing_pins(pins, _mutant(fn, mutants[name])), f"mutant {fname}/{name} passed every pin"


# ---------------------------------------------------------------- BDL bookkeeping model
BDL_MUTANTS = {
    "overflow_needs_more_than_X": [("if len(merged) >= X:", "if len(merged) > X:")],
    "carry_not_counted": [("            q += 1\n", "            q += 0\n")],
    "half_rule_inclusive": [("if 2 * len(self.slots[slot]) < self.capacity(slot):",
                             "if 2 * len(self.slots[slot]) <= self.capacity(slot):")],
    "buffer_not_erased": [("self.buffer = [i for i in self.buffer if keep(i)]", "self.buffer = list(self.buffer)")],
    "F_or_instead_of_add": [("self.F = F_new", "self.F = self.F | F_new")],
    "consumed_trees_kept": [("        for i in consumed:\n            del self.slots[i]\n", "")],
    "cascade_from_higher_slots": [("if i < j and i not in taken:", "if i > j and i not in taken:")],
    "gathered_points_dropped": [("self._insert_ids(sorted(R))", "self._insert_ids([])")],
}


def _bdl_pins(monkeypatch):
    import test_oracle_bdl as tob

    golden = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")
    names = ["test_pure_insert_closed_form", "test_batch_dynamic_start_closed_form", "test_cascade_assignment_reading",
             "test_erase_semantics_and_invariants", "test_random_history_invariants_and_knn",
             "test_half_full_tree_stays_fewer_than_half_is_rebuilt", "test_erase_reaches_the_buffer_tree"]

    def with_model(fn, *args):
        def pin(cls):
            monkeypatch.setattr(tob, "BDLModel", cls)
            fn(*args)
        pin.__name__ = fn.__name__ + "".join(f"[{a}]" for a in args if isinstance(a, int))
        return pin

    pins = [with_model(tob.test_insert_worked_example, golden, X) for X in (3, 4, 7, 64)]
    return pins + [with_model(getattr(tob, n)) for n in names]


def _bdl_mutant(edits):
    import oracle.bdl as bdl

    src = inspect.getsource(bdl.BDLModel)
    for old, new in edits:
        assert old in src, f"pattern not found in BDLModel: {old}"
        src = src.replace(old, new)
    ns = dict(vars(bdl))
    exec(compile(src, "<mutant of BDLModel>", "exec"), ns)
    return ns["BDLModel"]


def test_unmodified_bdl_model_passes_every_pin(monkeypatch):
    from oracle.bdl import BDLModel

    assert _failing_pins(_bdl_pins(monkeypatch), BDLModel) == []


@pytest.mark.parametrize("name", sorted(BDL_MUTANTS))
def test_bdl_model_mutant_fails_a_pin(monkeypatch, name):
    assert _failing_pins(_bdl_pins(monkeypatch), _bdl_mutant(BDL_MUTANTS[name])), f"mutant {name} passed every pin"
