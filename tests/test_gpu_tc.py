"""KL synthesis on the tensor cores (tcgen05 + TMA) against the FP64 oracle
field: the FP32 form (split-FP16 operands, FP32 accumulation) and the FP64 form
(exactly accumulated integer lead slice, float-float exponential)."""
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


def _exact_lead_bound(xi, phi):
    """Bound on |log a_gpu - log a| of the FP64 tensor-core form: slices that represent each scaled
    operand to 2^-23 of |X| <= 512 (2^-32 (2^e_v sum|xi| + 2^e_s sum|Phi|) + K 2^(e_s + e_v - 42)),
    the FP32 accumulation of the correction terms (at most 6 times the first part), the float-float
    exponential (about 1e-13) and the oracle's own FP64 rounding."""
    K = xi.shape[1]
    mx = np.abs(xi).max(axis=1)
    es = np.where(mx > 0, np.frexp(mx)[1], 0).astype(np.float64)          # max|xi_s| 2^-e_s in [1/2, 1)
    mp = np.abs(phi).max(axis=0)
    ev = np.where(mp > 0, np.frexp(mp)[1], 0).astype(np.float64)
    sx = np.abs(xi).sum(axis=1)[:, None]
    sp = np.abs(phi).sum(axis=0)[None, :]
    rep = 2.0 ** -32 * (2.0 ** ev[None, :] * sx + 2.0 ** es[:, None] * sp)
    cross = K * 2.0 ** (es[:, None] + ev[None, :] - 42)
    return 7.0 * rep + cross + 1e-13 + 1e-15 * (np.abs(xi) @ np.abs(phi))


@pytest.mark.parametrize("kind,K,n0,sigma2,corr,S", [(0, 16, 8, 1.0, 0.3, 37), (0, 64, 16, 1.0, 0.3, 130),
                                                     (0, 128, 12, 1.0, 0.1, 1), (0, 256, 16, 1.5, 0.1, 300),
                                                     (1, 4, 8, 4.0, 0.3, 129), (2, 1, 6, 0.49, 0.3, 5)])
def test_fp64_tensor_core_field_matches_oracle(M, kind, K, n0, sigma2, corr, S):
    h = M.mlmc_create(M.make_problem(n0=n0, m=2, L_max=1, kind=kind, K=K, sigma2=sigma2, corr_len=corr, seed=3), 0)
    try:
        n = 2 * n0
        V = (n + 1) ** 2
        guard = 4096
        buf = torch.full((S * V + guard,), -7.0, dtype=torch.float64, device=device())
        xi = torch.empty((S, K), dtype=torch.float64, device=device())
        M.mlmc_sample_fields(h, 1, 11, S, xi, buf, M.MLMC_FP64TC)
        torch.cuda.synchronize()
        got = buf[: S * V].cpu().numpy().reshape(S, V)
        assert np.all(buf[S * V:].cpu().numpy() == -7.0), "wrote past the end of the output"
        xi_o = o_rng.draw_xi(3, 1, 11, S, K)
        assert np.array_equal(xi.cpu().numpy(), xi_o)
        phi = o_kl.basis(kind, K, n, sigma2, corr, 2.0)
        loga = o_kl.log_coefficient(xi_o, phi)
        assert np.all(np.isfinite(got)) and np.all(got > 0)
        err = np.abs(np.log(got) - loga)
        bound = _exact_lead_bound(xi_o, phi)
        assert np.all(err <= bound), (err.max(), (err / bound).max())
        # the rounding errors are not all of one sign: the RMS error is far below the bound
        assert np.sqrt(np.mean(err ** 2)) <= max(1e-9 * np.sqrt(K), 1e-12), np.sqrt(np.mean(err ** 2))
        # and the same numbers as the FP64 form (FP64 contraction and exp on the FP64 pipe) to that accuracy
        a64 = torch.empty((S, V), dtype=torch.float64, device=device())
        M.mlmc_sample_fields(h, 1, 11, S, None, a64, M.MLMC_FP64)
        torch.cuda.synchronize()
        assert np.all(np.abs(np.log(a64.cpu().numpy()) - np.log(got)) <= bound + 1e-13)
    finally:
        M.mlmc_destroy(h)


def test_fp64_tensor_core_field_extreme_coefficients(M):
    # large |xi| (|log a| up to about 40) exercise the exponential's range reduction and table over many
    # binades of a; zero rows give a = 1 exactly
    K, n0, S = 64, 16, 40
    h = M.mlmc_create(M.make_problem(n0=n0, m=2, L_max=0, kind=0, K=K, sigma2=1.0, corr_len=0.3), 0)
    try:
        g = np.random.default_rng(5)
        xi_np = g.standard_normal((S, K)) * np.linspace(0.0, 12.0, S)[:, None]
        xi_np[0] = 0.0
        a = torch.empty((S, (n0 + 1) ** 2), dtype=torch.float64, device=device())
        M.mlmc_synthesize_fields(h, 0, S, to_dev(xi_np), a, M.MLMC_FP64TC)
        torch.cuda.synchronize()
        phi = o_kl.basis(0, K, n0, 1.0, 0.3)
        loga = o_kl.log_coefficient(xi_np, phi)
        got = a.cpu().numpy()
        assert np.all(got[0] == 1.0)
        assert np.abs(loga).max() > 20.0
        err = np.abs(np.log(got) - loga)
        assert np.all(err <= _exact_lead_bound(xi_np, phi))
    finally:
        M.mlmc_destroy(h)


@pytest.mark.parametrize("fprec", ["FP32", "FP64TC", "FP64"])
@pytest.mark.parametrize("n0,S", [(8, 37), (16, 130)])
def test_field_row_pitch_and_offset(M, fprec, n0, S):
    # the same field into dense rows, into rows padded to whole 128-byte lines (the FP32 form's direct store
    # path), into rows padded by 5 elements, and one element past a 128-byte boundary (the staged store path):
    # identical bits everywhere, the gaps and the guard untouched
    K = 64
    p = getattr(M, "MLMC_" + fprec)
    dt = torch.float32 if fprec == "FP32" else torch.float64
    h = M.mlmc_create(M.make_problem(n0=n0, m=2, L_max=1, kind=0, K=K, sigma2=1.0, corr_len=0.3, seed=9), 0)
    try:
        n = 2 * n0
        V = (n + 1) ** 2
        xi = torch.empty((S, K), dtype=torch.float64, device=device())
        dense = torch.empty((S, V), dtype=dt, device=device())
        M.mlmc_sample_fields(h, 1, 0, S, xi, dense, p)
        ref = dense.cpu().numpy()
        for ld, off in (((V + 31) // 32 * 32, 0), (V + 5, 0), (V, 1), (V + 3, 3)):
            buf = torch.full((off + S * ld + 256,), -7.0, dtype=dt, device=device())
            view = buf[off:]
            M.mlmc_synthesize_fields(h, 1, S, xi, view, p, a_ld=ld)
            torch.cuda.synchronize()
            got = buf.cpu().numpy()
            rows = got[off: off + S * ld].reshape(S, ld)
            assert np.array_equal(rows[:, :V], ref), (ld, off)
            assert np.all(rows[:, V:] == -7.0) and np.all(got[:off] == -7.0) and np.all(got[off + S * ld:] == -7.0)
        with pytest.raises(M.MlmcError):
            M.mlmc_synthesize_fields(h, 1, S, xi, dense, p, a_ld=V - 1)
    finally:
        M.mlmc_destroy(h)
