"""GPU batched multi-cloud path (the level kernels split every cloud's tree at
once, then one persistent launch finishes the segments and runs every query
chunk) against the per-cloud plain path (bit for bit) and the CPU oracle; its
backward twin against the oracle's gradient and float64 finite differences."""
from __future__ import annotations

import numpy as np
import pytest

import oracle
from knn_compare import compare_knn
from paper_2207_01834_gb300 import synth

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def api():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2207_01834_gb300 import api as a
    return a


def _cuda(x):
    return torch.from_numpy(np.ascontiguousarray(x, dtype=np.float32)).cuda()


def _plain(api, a, a_off, b, b_off, k, leaf=16):
    """One pg_tree_build + pg_knn per cloud and direction (the plain sequence)."""
    A, B = _cuda(a), _cuda(b)
    iab, dab, iba, dba = [], [], [], []
    for i in range(len(a_off) - 1):
        Ai = A[a_off[i]:a_off[i + 1]]
        Bi = B[b_off[i]:b_off[i + 1]]
        ta = api.pg_tree_build(Ai, leaf)
        tb = api.pg_tree_build(Bi, leaf)
        x = api.pg_knn(tb, Ai, k)
        y = api.pg_knn(ta, Bi, k)
        iab.append(x[0]); dab.append(x[1]); iba.append(y[0]); dba.append(y[1])
        ta.free(); tb.free()
    return torch.cat(iab), torch.cat(dab), torch.cat(iba), torch.cat(dba)


def _check_against_oracle(a, a_off, b, b_off, k, iab, dab, iba, dba, loss, rows_per_pair=None):
    total = 0.0
    for i in range(len(a_off) - 1):
        A = a[a_off[i]:a_off[i + 1]]
        B = b[b_off[i]:b_off[i + 1]]
        ra = np.arange(len(A)) if rows_per_pair is None else np.sort(synth.pick_rows(len(A), min(rows_per_pair, len(A)), i))
        rb = np.arange(len(B)) if rows_per_pair is None else np.sort(synth.pick_rows(len(B), min(rows_per_pair, len(B)), i + 7))
        oi, od = oracle.knn(B, A[ra], k, nthreads=0)
        compare_knn(iab[a_off[i]:a_off[i + 1]][ra], dab[a_off[i]:a_off[i + 1]][ra], oi, od, B, A[ra])
        oi, od = oracle.knn(A, B[rb], k, nthreads=0)
        compare_knn(iba[b_off[i]:b_off[i + 1]][rb], dba[b_off[i]:b_off[i + 1]][rb], oi, od, A, B[rb])
        if rows_per_pair is None:
            want = oracle.chamfer(A, [0, len(A)], B, [0, len(B)], k)[0][0]
            assert abs(float(loss[i]) - want) <= 1e-5 * max(want, 1e-30), (i, float(loss[i]), want)
            total += want
    return total


@pytest.mark.parametrize("dim,k,seed", [(3, 1, 1), (3, 8, 2), (2, 3, 3), (5, 16, 4), (7, 8, 5), (3, 10, 6)])
def test_batched_matches_plain_and_oracle(api, dim, k, seed):
    a, a_off, b, b_off = synth.cloud_pairs(5, seed=seed, d=dim, lo=30, hi=3000)
    loss, iab, iba, dab, dba = api.pg_batched_chamfer(_cuda(a), a_off, _cuda(b), b_off, k, want_dist=True)
    p_iab, p_dab, p_iba, p_dba = _plain(api, a, a_off, b, b_off, k)
    assert torch.equal(iab, p_iab) and torch.equal(dab, p_dab)
    assert torch.equal(iba, p_iba) and torch.equal(dba, p_dba)
    _check_against_oracle(a, a_off, b, b_off, k, iab.cpu().numpy(), dab.cpu().numpy(), iba.cpu().numpy(),
                          dba.cpu().numpy(), loss.cpu().numpy())
    # replaying the cached plan gives the same bits
    loss2, iab2, iba2, _, _ = api.pg_batched_chamfer(_cuda(a), a_off, _cuda(b), b_off, k)
    assert torch.equal(loss, loss2) and torch.equal(iab, iab2) and torch.equal(iba, iba2)


def test_batched_deep_cloud_takes_the_global_memory_finisher(api):
    """A dense cluster behind a geometric row of outliers: every spatial-median
    level peels off about one outlier, so after all the forest levels the
    cluster is still one segment far above the shared-memory capacity and is
    finished by the global-memory block builder (scratch from the pool)."""
    rng = np.random.default_rng(31)
    cluster = (0.3 + 1e-5 * rng.random((12000, 3))).astype(np.float32)
    row = np.zeros((40, 3), np.float32)
    row[:, 0] = (0.3 + 2.0 ** -np.arange(40)).astype(np.float32)
    row[:, 1:] = 0.3
    deep = np.concatenate([cluster, row])[rng.permutation(12040)]
    other = synth.cloud(3000, 3, 32)
    a = np.concatenate([deep, other]).astype(np.float32)
    b = np.concatenate([synth.cloud(2000, 3, 33), deep[::3]]).astype(np.float32)
    a_off = np.array([0, 12040, 15040])
    b_off = np.array([0, 2000, 2000 + len(deep[::3])])
    k = 8
    loss, iab, iba, dab, dba = api.pg_batched_chamfer(_cuda(a), a_off, _cuda(b), b_off, k, want_dist=True)
    p_iab, p_dab, p_iba, p_dba = _plain(api, a, a_off, b, b_off, k)
    assert torch.equal(iab, p_iab) and torch.equal(dab, p_dab)
    assert torch.equal(iba, p_iba) and torch.equal(dba, p_dba)
    _check_against_oracle(a, a_off, b, b_off, k, iab.cpu().numpy(), dab.cpu().numpy(), iba.cpu().numpy(),
                          dba.cpu().numpy(), loss.cpu().numpy(), rows_per_pair=600)


def test_batched_many_small_clouds_take_the_multi_kernel_level_path(api):
    """16,600 clouds: the forest's first level has more segment slots than one
    block handles (16,384), so it runs as classify + device-wide scans + link."""
    rng = np.random.default_rng(41)
    npairs, k = 8300, 4
    sa = rng.integers(1, 40, npairs)
    sb = rng.integers(1, 40, npairs)
    a = rng.random((int(sa.sum()), 3)).astype(np.float32)
    b = rng.random((int(sb.sum()), 3)).astype(np.float32)
    a_off = np.concatenate([[0], np.cumsum(sa)])
    b_off = np.concatenate([[0], np.cumsum(sb)])
    loss, iab, iba, dab, dba = api.pg_batched_chamfer(_cuda(a), a_off, _cuda(b), b_off, k, want_dist=True)
    iab, iba, dab, dba, loss = (t.cpu().numpy() for t in (iab, iba, dab, dba, loss))
    for i in np.sort(rng.choice(npairs, 300, replace=False)):
        A, B = a[a_off[i]:a_off[i + 1]], b[b_off[i]:b_off[i + 1]]
        oi, od = oracle.knn(B, A, k, nthreads=0)
        compare_knn(iab[a_off[i]:a_off[i + 1]], dab[a_off[i]:a_off[i + 1]], oi, od, B, A)
        oi, od = oracle.knn(A, B, k, nthreads=0)
        compare_knn(iba[b_off[i]:b_off[i + 1]], dba[b_off[i]:b_off[i + 1]], oi, od, A, B)
        want = oracle.chamfer(A, [0, len(A)], B, [0, len(B)], k)[0][0]
        assert abs(float(loss[i]) - want) <= 1e-5 * max(want, 1e-30), (i, float(loss[i]), want)


def test_batched_tiny_clouds_and_padding(api):
    a = synth.uniform(1 + 3 + 40, 3, 11)
    b = synth.uniform(2 + 1 + 17, 3, 12)
    a_off = np.array([0, 1, 4, 44])
    b_off = np.array([0, 2, 3, 20])
    k = 5
    loss, iab, iba, dab, dba = api.pg_batched_chamfer(_cuda(a), a_off, _cuda(b), b_off, k, want_dist=True)
    iab = iab.cpu().numpy()
    assert np.all(iab[0, 2:] == -1) and np.all(iab[1:4, 1:] == -1)      # B_0 has 2 points, B_1 has 1
    _check_against_oracle(a, a_off, b, b_off, k, iab, dab.cpu().numpy(), iba.cpu().numpy(), dba.cpu().numpy(),
                          loss.cpu().numpy())


def _grad_bound(X, Y, idx_xy, Xoff, Yoff, g, idx_yx, k):
    """Per-element sum of |terms| of the gradient of X rows (float64)."""
    bx = np.zeros(X.shape)
    for i in range(len(Xoff) - 1):
        xs = slice(Xoff[i], Xoff[i + 1])
        ys = slice(Yoff[i], Yoff[i + 1])
        Xi, Yi = X[xs].astype(np.float64), Y[ys].astype(np.float64)
        for j in range(k):
            t = idx_xy[xs, j]
            ok = t >= 0
            bx[xs][ok] += np.abs(2 * g[i] * (Xi[ok] - Yi[t[ok]]))
            t = idx_yx[ys, j]
            ok = t >= 0
            np.add.at(bx[xs], t[ok], np.abs(2 * g[i] * (Yi[ok] - Xi[t[ok]])))
    return bx


@pytest.mark.parametrize("k", [1, 8])
def test_batched_backward_matches_oracle(api, k):
    a, a_off, b, b_off = synth.cloud_pairs(4, seed=20 + k, lo=40, hi=2500)
    A, B = _cuda(a), _cuda(b)
    loss, iab, iba, _, _ = api.pg_batched_chamfer(A, a_off, B, b_off, k)
    g = np.random.default_rng(k).standard_normal(4).astype(np.float32)
    ga, gb = api.pg_batched_chamfer_backward(A, a_off, B, b_off, k, iab, iba, _cuda(g))
    ga2, gb2 = api.pg_batched_chamfer_backward(A, a_off, B, b_off, k, iab, iba, _cuda(g))
    assert torch.equal(ga, ga2) and torch.equal(gb, gb2)                  # deterministic
    iab_n, iba_n = iab.cpu().numpy().astype(np.int64), iba.cpu().numpy().astype(np.int64)
    wa = np.zeros(a.shape)
    wb = np.zeros(b.shape)
    for i in range(4):
        As, Bs = slice(a_off[i], a_off[i + 1]), slice(b_off[i], b_off[i + 1])
        gq, gp = oracle.knn_grad(b[Bs], a[As], iab_n[As], np.full(iab_n[As].shape, float(g[i])))
        wa[As] += gq
        wb[Bs] += gp
        gq, gp = oracle.knn_grad(a[As], b[Bs], iba_n[Bs], np.full(iba_n[Bs].shape, float(g[i])))
        wb[Bs] += gq
        wa[As] += gp
    ba = _grad_bound(a, b, iab_n, a_off, b_off, g.astype(np.float64), iba_n, k)
    bb = _grad_bound(b, a, iba_n, b_off, a_off, g.astype(np.float64), iab_n, k)
    assert np.all(np.abs(ga.cpu().numpy() - wa) <= 1e-5 * ba + 1e-30)
    assert np.all(np.abs(gb.cpu().numpy() - wb) <= 1e-5 * bb + 1e-30)


def test_batched_backward_finite_differences_two_pairs_of_500(api):
    """Gradient of the summed loss vs float64 central differences (h = 1e-4)
    with the selection frozen, on 2 pairs of 500-point clouds."""
    k = 8
    a = np.concatenate([synth.cloud(500, 3, 31), synth.cloud(500, 3, 32)])
    b = np.concatenate([synth.cloud(500, 3, 33), synth.cloud(500, 3, 34)])
    off = np.array([0, 500, 1000])
    A, B = _cuda(a), _cuda(b)
    loss, iab, iba, _, _ = api.pg_batched_chamfer(A, off, B, off, k)
    ga, gb = api.pg_batched_chamfer_backward(A, off, B, off, k, iab, iba, _cuda(np.ones(2)))
    iab_n, iba_n = iab.cpu().numpy().astype(np.int64), iba.cpu().numpy().astype(np.int64)
    ones = np.ones((500, k))

    def L(Af, Bf):
        t = 0.0
        for i in range(2):
            s = slice(500 * i, 500 * (i + 1))
            t += oracle.knn_loss(Bf[s], Af[s], iab_n[s], ones) + oracle.knn_loss(Af[s], Bf[s], iba_n[s], ones)
        return t

    Af, Bf = a.astype(np.float64), b.astype(np.float64)
    h = 1e-4
    err, scale = 0.0, 0.0
    for arr, g in ((Af, ga.cpu().numpy()), (Bf, gb.cpu().numpy())):
        for r in range(0, 1000, 37):
            for c in range(3):
                keep = arr[r, c]
                arr[r, c] = keep + h
                lp = L(Af, Bf)
                arr[r, c] = keep - h
                lm = L(Af, Bf)
                arr[r, c] = keep
                fd = (lp - lm) / (2 * h)
                err = max(err, abs(g[r, c] - fd))
                scale = max(scale, abs(fd))
    print(f"batched backward: max |GPU - FD| / max |FD| = {err / scale:.2e}")
    assert err / scale < 1e-5
    assert abs(float(loss.sum()) - L(Af, Bf)) <= 1e-5 * L(Af, Bf)


@pytest.mark.parametrize("k", [1, 8])
def test_batched_256_pairs_full_size(api, k):
    """256 pairs of 3D clouds, sizes log-uniform in [1,000, 100,000], each from
    its own 8-component mixture: bit-identical to the plain per-cloud path on
    every row, sampled rows against the oracle."""
    a, a_off, b, b_off = synth.cloud_pairs(256, seed=synth.BASE_SEED + 5)
    loss, iab, iba, dab, dba = api.pg_batched_chamfer(_cuda(a), a_off, _cuda(b), b_off, k, want_dist=True)
    p_iab, p_dab, p_iba, p_dba = _plain(api, a, a_off, b, b_off, k)
    assert torch.equal(iab, p_iab) and torch.equal(dab, p_dab)
    assert torch.equal(iba, p_iba) and torch.equal(dba, p_dba)
    sel = synth.pick_rows(256, 6, k)
    sub_a = np.concatenate([a[a_off[i]:a_off[i + 1]] for i in sel])
    sub_b = np.concatenate([b[b_off[i]:b_off[i + 1]] for i in sel])
    sa = np.concatenate([[0], np.cumsum([a_off[i + 1] - a_off[i] for i in sel])])
    sb = np.concatenate([[0], np.cumsum([b_off[i + 1] - b_off[i] for i in sel])])
    rows_a = np.concatenate([np.arange(a_off[i], a_off[i + 1]) for i in sel])
    rows_b = np.concatenate([np.arange(b_off[i], b_off[i + 1]) for i in sel])
    _check_against_oracle(sub_a, sa, sub_b, sb, k, iab.cpu().numpy()[rows_a], dab.cpu().numpy()[rows_a],
                          iba.cpu().numpy()[rows_b], dba.cpu().numpy()[rows_b], None, rows_per_pair=40)
    assert torch.all(torch.isfinite(loss)) and torch.all(loss > 0)


def test_batched_wait_timeout_is_reported(api):
    """A ready flag that nothing sets: every query chunk's bounded wait runs
    out and the call reports PG_ETIMEOUT; the path works again afterwards."""
    from paper_2207_01834_gb300._lib import PG_ETIMEOUT, PgError

    a, a_off, b, b_off = synth.cloud_pairs(2, seed=77, lo=100, hi=400)
    api.debug_batched_faults(True, 2000)
    try:
        with pytest.raises(PgError) as e:
            api.pg_batched_chamfer(_cuda(a), a_off, _cuda(b), b_off, 4)
        assert e.value.status == PG_ETIMEOUT
    finally:
        api.debug_batched_faults(False, 0)
    loss, iab, iba, _, _ = api.pg_batched_chamfer(_cuda(a), a_off, _cuda(b), b_off, 4)
    p = _plain(api, a, a_off, b, b_off, 4)
    assert torch.equal(iab, p[0]) and torch.equal(iba, p[2])
