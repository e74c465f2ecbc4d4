"""Helpers shared by the GPU tests (no method arithmetic here)."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")


def device():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return torch.device("cuda:0")


def lib():
    import __graft_entry__
    __graft_entry__.build()
    import paper_2503_05533_gb300 as M
    return M


def to_dev(x, dtype=torch.float64):
    return torch.as_tensor(np.ascontiguousarray(x)).to(device=device(), dtype=dtype)


def fp64_delta(n):
    """Tightest relative residual to ask of an FP64 solve on an n x n grid.

    Cor. 3.4 condition 2 needs c (1 + h^-2) u < delta: merely storing x in FP64
    leaves a residual of order (1 + n^2) 2^-53, so delta must stay above it."""
    return max(1e-13, 2.0 * (1.0 + n * n) * 2.0 ** -53)


def round_storage(a, prec, M):
    """Round nodal values the way the operator's storage type does (inputs are FP32-exact)."""
    a = np.asarray(a, dtype=np.float64)
    if prec == M.MLMC_FP64:
        return a
    if prec == M.MLMC_FP32:
        return a.astype(np.float32).astype(np.float64)
    if prec == M.MLMC_FP16S:
        return a.astype(np.float16).astype(np.float64)
    if prec == M.MLMC_BF16S:
        u = a.astype(np.float32).view(np.uint32).astype(np.uint64)
        u = (u + 0x7FFF + ((u >> 16) & 1)) & 0xFFFF0000
        return u.astype(np.uint32).view(np.float32).astype(np.float64)
    raise ValueError(prec)
