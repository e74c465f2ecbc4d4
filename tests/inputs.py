"""Seeded synthetic inputs shared by the oracle side and the CUDA side of the tests.

This module holds no arithmetic of the method (no KL expansion, no assembly,
no solve): only random inputs of the right shapes and value ranges, drawn with
NumPy's PCG64 from explicit seeds.  Values meant for both an FP32 and an FP64
consumer are rounded to FP32 first, so both sides see exactly the same numbers.
"""
import numpy as np


def smooth_lognormal_field(n, S, seed, log_sd=1.0, modes=4, fp32_exact=True):
    """S nodal coefficient fields a[S][(n+1)^2] = exp(g) with g a random smooth
    trigonometric sum of standard deviation about ``log_sd`` (contrast e^{+-3 sd})."""
    rng = np.random.default_rng(seed)
    x = np.arange(n + 1) / n
    X, Y = np.meshgrid(x, x, indexing="xy")
    out = np.empty((S, (n + 1) * (n + 1)))
    for s in range(S):
        g = np.zeros_like(X)
        for _ in range(modes):
            kx, ky = rng.integers(0, 4, size=2)
            ph = rng.uniform(0, 2 * np.pi, size=2)
            g += rng.standard_normal() * np.cos(np.pi * kx * X + ph[0]) * np.cos(np.pi * ky * Y + ph[1])
        g *= log_sd / np.sqrt(modes / 4.0)
        out[s] = np.exp(g).ravel()
    if fp32_exact:
        out = out.astype(np.float32).astype(np.float64)
    return out


def rough_field(n, S, seed, lo=0.05, hi=20.0, fp32_exact=True):
    """Nodal fields with independent log-uniform values in [lo, hi] (no smoothness)."""
    rng = np.random.default_rng(seed)
    out = np.exp(rng.uniform(np.log(lo), np.log(hi), size=(S, (n + 1) * (n + 1))))
    if fp32_exact:
        out = out.astype(np.float32).astype(np.float64)
    return out


def random_vectors(n, S, seed, fp32_exact=True):
    """Random values on all (n+1)^2 nodes of S grids (boundary values included)."""
    rng = np.random.default_rng(seed)
    v = rng.standard_normal((S, (n + 1) * (n + 1)))
    if fp32_exact:
        v = v.astype(np.float32).astype(np.float64)
    return v


def random_normals(S, K, seed):
    return np.random.default_rng(seed).standard_normal((S, K))
