"""The adjoint gradient dQ/dxi (A12) and its torch.autograd wrapper."""
import numpy as np
import pytest

from gpu_common import device, fp64_delta, lib, to_dev, torch
from oracle import adjoint as o_adj
from oracle import kl as o_kl

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def M():
    device()
    return lib()


def _grad(M, h, level, xi_np, prec, delta):
    S, K = xi_np.shape
    Q = torch.empty(S, dtype=torch.float64, device=device())
    g = torch.empty((S, K), dtype=torch.float64, device=device())
    M.mlmc_adjoint_grad(h, level, S, to_dev(xi_np), prec, delta, 200000, Q, g)
    torch.cuda.synchronize()
    return Q.cpu().numpy(), g.cpu().numpy()


@pytest.mark.parametrize("box", [None, (0.25, 0.75, 0.25, 0.75)])
def test_gradient_fp64_matches_cpu_adjoint(M, box):
    kw = dict(n0=16, m=2, L_max=0, kind=0, K=24, sigma2=1.0, corr_len=0.1, seed=0)
    if box:
        kw.update(qoi=1, box=box)
    h = M.mlmc_create(M.make_problem(**kw), 0)
    try:
        xi = np.random.default_rng(5).standard_normal((3, 24))
        Q, g = _grad(M, h, 0, xi, M.MLMC_FP64, fp64_delta(16))
        phi = o_kl.basis(0, 24, 16, 1.0, 0.1)
        for s in range(3):
            Qo, go = o_adj.gradient(16, xi[s], phi, box)
            assert abs(Q[s] - Qo) <= 1e-12 * abs(Qo)
            assert np.max(np.abs(g[s] - go)) <= 1e-10 * np.max(np.abs(go))
    finally:
        M.mlmc_destroy(h)


def test_gradient_matches_central_differences_on_gpu(M):
    h = M.mlmc_create(M.make_problem(n0=32, m=2, L_max=0, kind=0, K=8, sigma2=1.0, corr_len=0.1, seed=0), 0)
    try:
        xi = np.random.default_rng(6).standard_normal((1, 8))
        _, g = _grad(M, h, 0, xi, M.MLMC_FP64, fp64_delta(32))
        eps = 1e-6
        pert = np.repeat(xi, 16, axis=0)
        for k in range(8):
            pert[2 * k, k] += eps
            pert[2 * k + 1, k] -= eps
        a = torch.empty((16, 33 * 33), dtype=torch.float64, device=device())
        M.mlmc_synthesize_fields(h, 0, 16, to_dev(pert), a, M.MLMC_FP64)
        Q = torch.empty(16, dtype=torch.float64, device=device())
        M.mlmc_level_solve(h, 32, 16, a, M.MLMC_FP64, 32, M.MLMC_FP64, M.MLMC_CG, fp64_delta(32), 100000, None, Q)
        torch.cuda.synchronize()
        Qn = Q.cpu().numpy()
        fd = (Qn[0::2] - Qn[1::2]) / (2 * eps)
        assert np.max(np.abs(fd - g[0])) <= 1e-4 * np.max(np.abs(g[0]))
    finally:
        M.mlmc_destroy(h)


@pytest.mark.parametrize("prec", ["FP32", "FP16S"])
def test_gradient_mixed_precision(M, prec):
    h = M.mlmc_create(M.make_problem(n0=16, m=2, L_max=0, kind=0, K=16, sigma2=1.0, corr_len=0.1, seed=0), 0)
    try:
        xi = np.random.default_rng(7).standard_normal((4, 16))
        Q, g = _grad(M, h, 0, xi, getattr(M, "MLMC_" + prec), 1e-9)
        phi = o_kl.basis(0, 16, 16, 1.0, 0.1)
        for s in range(4):
            # FP64 refinement to delta = 1e-9 around the low-precision inner solves, FP64 tensor-core field
            # (about 1e-9 in log a): held to 1e-8 (observed about 6e-11)
            Qo, go = o_adj.gradient(16, xi[s], phi)
            assert abs(Q[s] - Qo) <= 1e-8 * abs(Qo)
            assert np.max(np.abs(g[s] - go)) <= 1e-8 * np.max(np.abs(go))
    finally:
        M.mlmc_destroy(h)


def test_autograd_function(M):
    from paper_2503_05533_gb300 import autograd as AG
    h = M.mlmc_create(M.make_problem(n0=16, m=2, L_max=0, kind=0, K=12, sigma2=1.0, corr_len=0.2, seed=0), 0)
    try:
        xi_np = np.random.default_rng(9).standard_normal((5, 12))
        xi = to_dev(xi_np).requires_grad_(True)
        Q = AG.qoi(xi, h, 0, 16, M.MLMC_FP64, fp64_delta(16))
        w = torch.arange(1, 6, dtype=torch.float64, device=device())
        (Q * w).sum().backward()
        phi = o_kl.basis(0, 12, 16, 1.0, 0.2)
        for s in range(5):
            Qo, go = o_adj.gradient(16, xi_np[s], phi)
            assert abs(Q[s].item() - Qo) <= 1e-12 * abs(Qo)
            assert np.allclose(xi.grad[s].cpu().numpy(), (s + 1) * go, rtol=1e-9, atol=1e-12 * np.abs(go).max())
    finally:
        M.mlmc_destroy(h)
