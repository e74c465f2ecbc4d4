"""KL synthesis on the tensor cores (tcgen05 + TMA, split-FP16 operands, FP32
accumulation) against the FP64 oracle field."""
import numpy as np
import pytest

from gpu_common import device, lib, to_dev, torch
from oracle import kl as o_kl
from oracle import rng as o_rng

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def M():
    device()
    return lib()


@pytest.mark.parametrize("kind,K,n0,sigma2,corr,S", [(0, 16, 8, 1.0, 0.3, 37), (0, 64, 16, 1.0, 0.3, 130),
                                                     (0, 128, 12, 1.0, 0.1, 1), (0, 256, 16, 1.5, 0.1, 300),
                                                     (1, 4, 8, 4.0, 0.3, 129), (2, 1, 6, 0.49, 0.3, 5)])
def test_tensor_core_field_matches_oracle(M, kind, K, n0, sigma2, corr, S):
    h = M.mlmc_create(M.make_problem(n0=n0, m=2, L_max=1, kind=kind, K=K, sigma2=sigma2, corr_len=corr, seed=3), 0)
    try:
        n = 2 * n0
        V = (n + 1) ** 2
        guard = 4096
        buf = torch.full((S * V + guard,), -7.0, dtype=torch.float32, device=device())
        xi = torch.empty((S, K), dtype=torch.float64, device=device())
        M.mlmc_sample_fields(h, 1, 11, S, xi, buf, M.MLMC_FP32)
        torch.cuda.synchronize()
        got = buf[: S * V].cpu().numpy().reshape(S, V).astype(np.float64)
        assert np.all(buf[S * V:].cpu().numpy() == -7.0), "wrote past the end of the output"
        xi_o = o_rng.draw_xi(3, 1, 11, S, K)
        assert np.array_equal(xi.cpu().numpy(), xi_o)
        loga = o_kl.log_coefficient(xi_o, o_kl.basis(kind, K, n, sigma2, corr, 2.0))
        # split-FP16 products (2^-22 relative each) and FP32 accumulation of K terms, then expf
        scale = np.abs(xi_o) @ np.abs(o_kl.basis(kind, K, n, sigma2, corr, 2.0))
        err = np.abs(np.log(got) - loga)
        assert np.all(np.isfinite(got))
        assert np.all(err <= 2e-6 * np.maximum(scale, 1.0)), err.max()
        # FP32 accumulation of K terms: typical error ~ sqrt(K) u_32 |log a|
        rms = float(np.sqrt(np.mean(loga ** 2)))
        assert np.median(err) < max(3e-7, 6e-8 * np.sqrt(K) * max(1.0, rms))
    finally:
        M.mlmc_destroy(h)


def test_tensor_core_field_from_given_xi(M):
    K, n0, S = 64, 16, 64
    h = M.mlmc_create(M.make_problem(n0=n0, m=2, L_max=0, kind=0, K=K, sigma2=1.0, corr_len=0.3), 0)
    try:
        xi_np = np.random.default_rng(8).standard_normal((S, K)) * 2.0
        a = torch.empty((S, (n0 + 1) ** 2), dtype=torch.float32, device=device())
        M.mlmc_synthesize_fields(h, 0, S, to_dev(xi_np), a, M.MLMC_FP32)
        torch.cuda.synchronize()
        ref = o_kl.coefficient(xi_np, o_kl.basis(0, K, n0, 1.0, 0.3))
        assert np.allclose(a.cpu().numpy(), ref, rtol=4e-6, atol=0)
    finally:
        M.mlmc_destroy(h)
