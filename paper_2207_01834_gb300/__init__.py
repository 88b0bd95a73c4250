"""GB300-native (sm_103a) kd-tree / BDL-tree exact k-NN.

The compute path is the CUDA library libpargeo_gpu.so (C ABI in
include/pargeo_gpu.h), built in-tree by `paper_2207_01834_gb300.build`.
`paper_2207_01834_gb300.api` is the thin Python binding; `autograd` wraps the
k-NN distance and its backward kernel as a torch.autograd.Function.
The binding is imported lazily so that `synth` (seeded inputs) can be used
without CUDA.
"""
from __future__ import annotations

_LAZY = {"api", "autograd", "autotune"}


def __getattr__(name):
    import importlib

    if name in _LAZY:
        return importlib.import_module(f".{name}", __name__)
    api = importlib.import_module(".api", __name__)
    if name in api.__all__:
        return getattr(api, name)
    raise AttributeError(name)
