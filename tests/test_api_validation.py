"""The binding's argument checks run before anything is launched: malformed
gradient calls raise on any machine (no GPU needed), and the library is not
called."""
from __future__ import annotations

import pytest

torch = pytest.importorskip("torch")


@pytest.fixture
def api(monkeypatch):
    from paper_2207_01834_gb300 import api as a

    calls = []
    monkeypatch.setattr(a, "call", lambda *args: calls.append(args))
    a._calls = calls
    return a


def _inputs(n=50, m=20, d=3, k=4):
    return (torch.zeros(n, d), torch.zeros(m, d), torch.zeros(m, k, dtype=torch.int32), torch.zeros(m, k))


@pytest.mark.parametrize("fn", ["pg_knn_backward", "pg_knn_backward_noalloc"])
def test_backward_rejects_mismatched_inputs(api, fn):
    f = getattr(api, fn)
    extra = (None, None) if fn.endswith("noalloc") else ()
    data, q, idx, g = _inputs()
    with pytest.raises(ValueError, match="queries must have shape"):
        f(data, torch.zeros(20, 2), idx, g, *extra)            # wrong dimension
    with pytest.raises(ValueError, match="queries must have shape"):
        f(data, torch.zeros(21, 3), idx, g, *extra)            # wrong count
    with pytest.raises(ValueError, match="grad_dist must have idx's shape"):
        f(data, q, idx, torch.zeros(20, 5), *extra)
    with pytest.raises(TypeError, match="idx must be"):
        f(data, q, idx.long(), g, *extra)
    with pytest.raises(TypeError, match="data must be"):
        f(data.double(), q, idx, g, *extra)
    with pytest.raises(ValueError, match="CUDA"):
        f(data, q, idx, g, *extra)                              # well formed, but not on a GPU
    assert api._calls == []


def test_noalloc_rejects_bad_outputs(api, monkeypatch):
    data, q, idx, g = _inputs()
    # pretend the inputs passed their checks, so that only the outputs are examined
    monkeypatch.setattr(api, "_backward_inputs", lambda *a: (data, q, idx, g, 50, 20, 3, 4))
    dev = data.device
    with pytest.raises(ValueError, match=r"grad_data must have shape \(50, 3\)"):
        api.pg_knn_backward_noalloc(data, q, idx, g, None, torch.zeros(49, 3))      # short: would overrun
    with pytest.raises(TypeError, match="grad_queries must be torch.float32"):
        api.pg_knn_backward_noalloc(data, q, idx, g, torch.zeros(20, 3, dtype=torch.float64), None)
    with pytest.raises(ValueError, match="grad_queries must be contiguous"):
        api.pg_knn_backward_noalloc(data, q, idx, g, torch.zeros(3, 20).t(), None)
    with pytest.raises(ValueError, match="CUDA"):
        api.pg_knn_backward_noalloc(data, q, idx, g, torch.zeros(20, 3, device=dev), None)
    assert api._calls == []
