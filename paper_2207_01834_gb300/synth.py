"""Seeded synthetic point sets shaped like the paper's workloads.

This module is shared by the CUDA path's tests/benchmark and by the CPU
oracle's tests.  It draws random numbers and nothing else: it holds none of the
method's arithmetic (no distances, no selection, no tree logic).

Distributions (paper, Section 6 "Data Sets"):
  * Uniform (U): i.i.d. uniform points in a hypercube.  The paper uses side
    sqrt(n); k-NN indices are invariant under uniform scaling, so the unit cube
    [0,1)^d is used here.
  * Varying-density clustered points: the paper's VisualVar generator is not
    specified in the text, so an isotropic Gaussian mixture stands in for it
    (centres uniform in [0,1)^d, sigma log-uniform, Zipf-like weights).

All generation is done in float64 with numpy's PCG64 and cast to float32 once.
"""
from __future__ import annotations

import numpy as np

BASE_SEED = 20220705


def rng(seed: int) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(seed))


def uniform(n: int, d: int, seed: int) -> np.ndarray:
    """n points i.i.d. uniform in [0,1)^d, float32, row-major (n, d)."""
    return rng(seed).random((n, d)).astype(np.float32)


def gmm_mixture(d: int, seed: int, components: int = 100,
                sigma_lo: float = 1e-3, sigma_hi: float = 1e-1,
                zipf_s: float = 1.2):
    """Parameters of an isotropic Gaussian mixture.

    Centres uniform in [0,1)^d, per-component sigma log-uniform in
    [sigma_lo, sigma_hi], weights proportional to i^-zipf_s (i = 1..components).
    """
    g = rng(seed)
    centres = g.random((components, d))
    sigmas = np.exp(g.uniform(np.log(sigma_lo), np.log(sigma_hi), components))
    w = np.arange(1, components + 1, dtype=np.float64) ** (-zipf_s)
    w /= w.sum()
    return centres, sigmas, w


def gmm_sample(n: int, mixture, seed: int) -> np.ndarray:
    """n float32 points drawn from a mixture returned by gmm_mixture."""
    centres, sigmas, w = mixture
    g = rng(seed)
    comp = g.choice(len(w), size=n, p=w)
    pts = centres[comp] + g.standard_normal((n, centres.shape[1])) * sigmas[comp][:, None]
    return pts.astype(np.float32)


def gmm(n: int, d: int, seed: int, **kw) -> np.ndarray:
    """n points from the mixture seeded by `seed` (mixture and sample share it)."""
    return gmm_sample(n, gmm_mixture(d, seed, **kw), seed + 1)


def cloud_sizes(npairs: int, seed: int, lo: int = 1000, hi: int = 100000) -> np.ndarray:
    """Sizes of 2*npairs clouds, floor(exp(U[ln lo, ln hi])) each."""
    g = rng(seed)
    s = np.floor(np.exp(g.uniform(np.log(lo), np.log(hi), 2 * npairs))).astype(np.int64)
    return np.clip(s, lo, hi)


def cloud(size: int, d: int, seed: int, components: int = 8) -> np.ndarray:
    """One point cloud from its own Gaussian mixture with Dirichlet(1) weights."""
    g = rng(seed)
    centres = g.random((components, d))
    sigmas = np.exp(g.uniform(np.log(1e-3), np.log(1e-1), components))
    w = g.dirichlet(np.ones(components))
    comp = g.choice(components, size=size, p=w)
    pts = centres[comp] + g.standard_normal((size, d)) * sigmas[comp][:, None]
    return pts.astype(np.float32)


def cloud_pairs(npairs: int, seed: int, d: int = 3, lo: int = 1000, hi: int = 100000):
    """npairs (A, B) cloud pairs, concatenated.

    Returns (a, a_off, b, b_off): a is (sum |A_i|, d) float32, a_off is int64 of
    length npairs+1 with a_off[i]:a_off[i+1] the rows of A_i; same for b.
    """
    sizes = cloud_sizes(npairs, seed, lo, hi)
    a_sizes, b_sizes = sizes[0::2], sizes[1::2]
    a = [cloud(int(s), d, seed * 7919 + 2 * i + 1) for i, s in enumerate(a_sizes)]
    b = [cloud(int(s), d, seed * 7919 + 2 * i + 2) for i, s in enumerate(b_sizes)]
    a_off = np.concatenate([[0], np.cumsum(a_sizes)]).astype(np.int64)
    b_off = np.concatenate([[0], np.cumsum(b_sizes)]).astype(np.int64)
    return np.concatenate(a), a_off, np.concatenate(b), b_off


def lattice(shape, spacing: float = 1.0) -> np.ndarray:
    """Integer grid points (exact in float32), row-major over `shape`."""
    axes = [np.arange(s, dtype=np.float64) * spacing for s in shape]
    mesh = np.meshgrid(*axes, indexing="ij")
    return np.stack([m.ravel() for m in mesh], axis=1).astype(np.float32)


def pick_rows(n_live: int, count: int, seed: int) -> np.ndarray:
    """`count` distinct row positions in [0, n_live), uniformly chosen."""
    return rng(seed).choice(n_live, size=count, replace=False)


def bdl_schedule(initial: int = 4_000_000, insert: int = 1_000_000, erase: int = 500_000,
                 rounds: int = 5):
    """The batch-dynamic schedule: an initial insert, then [I, I, D] x rounds."""
    ops = [("I", initial)]
    for _ in range(rounds):
        ops += [("I", insert), ("I", insert), ("D", erase)]
    return ops


# k-NN throughput against k on forests built incrementally: k = 2..11, the
# forest grown by batch inserts of 5% of the data each.
KSWEEP_KS = tuple(range(2, 12))
KSWEEP_BATCHES = 20


def ksweep_points(d: int, n: int = 10_000_000) -> np.ndarray:
    """Data of the k-sweep: 2D clustered (a varying-density Gaussian mixture
    stands in for the paper's 2D VisualVar set) or d-dimensional uniform."""
    if d == 2:
        return gmm_sample(n, gmm_mixture(2, BASE_SEED + 60), BASE_SEED + 61)
    return uniform(n, d, BASE_SEED + 60 + d)


def ksweep_queries(n: int, d: int, count: int = 1_000_000) -> np.ndarray:
    """Rows of the k-sweep data used as queries (the points query the
    structure that holds them)."""
    return pick_rows(n, min(n, count), BASE_SEED + 62 + d)
