"""The measurement workloads at their full sizes, checked on sampled systems
against the oracle and by properties that hold at any size:

- single-level sweep: 4096 systems on the 512 x 512 grid, K = 128, corr 0.1,
  fixed delta 1e-6, FP32 and FP16-stored inner solves;
- adjoint gradients: 1024 samples on the 256 x 256 grid, K = 256, corr 0.1,
  box QoI over [0.25, 0.75]^2;
- the finest level pair of the 7-level hierarchy (h = 1/1024 and 1/512,
  K = 256, sigma^2 = 1.5, corr 0.1).
"""
import numpy as np
import pytest

from gpu_common import device, lib, to_dev, torch
from oracle import adjoint as o_adj
from oracle import fem as o_fem
from oracle import kl as o_kl
from oracle import rng as o_rng

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def M():
    device()
    return lib()


def _interior(n, u):
    return u.reshape(n + 1, n + 1)[1:n, 1:n].ravel()


def lambda_min_lower(n, a_nodal):
    """A rigorous lower bound on the smallest eigenvalue of the P1 matrix: every
    edge weight is an average of nodal values, so A >= min(a) L with L the
    5-point Laplacian, whose smallest eigenvalue is 8 sin^2(pi h / 2)."""
    return float(np.min(a_nodal)) * 8.0 * np.sin(np.pi / (2.0 * n)) ** 2


def residual_floor(n, a_nodal, x):
    """Rounding floor of an FP64 relative residual ||b - A x|| / ||b||: each entry of A x
    is a sum of a few products, so two evaluations in different orders differ by at most
    a small multiple of u (|A| |x|)_i per entry."""
    A = o_fem.assemble(n, a_nodal)
    b = o_fem.load_vector(n)
    return 16.0 * 2.0 ** -53 * float(np.linalg.norm(abs(A) @ np.abs(x)) / np.linalg.norm(b))


def _solve(M, h, n, a, a_prec, prec, delta, u=False):
    S = a.shape[0]
    U = torch.zeros((S, (n + 1) ** 2), dtype=torch.float64, device=device()) if u else None
    Q = torch.empty(S, dtype=torch.float64, device=device())
    it = torch.zeros(S, dtype=torch.int32, device=device())
    rr = torch.zeros(S, dtype=torch.float64, device=device())
    fl = torch.zeros(S, dtype=torch.int32, device=device())
    M.mlmc_level_solve(h, n, S, a, a_prec, n, prec, M.MLMC_CG, delta, 200000, U, Q, it, rr, fl)
    torch.cuda.synchronize()
    return (U.cpu().numpy() if u else None), Q.cpu().numpy(), it.cpu().numpy(), rr.cpu().numpy(), fl.cpu().numpy()


@pytest.mark.parametrize("prec", ["FP32", "FP16S"])
def test_sweep_4096_systems_n512(M, prec):
    n, S, K, delta = 512, 4096, 128, 1e-6
    p = getattr(M, "MLMC_" + prec)
    h = M.mlmc_create(M.make_problem(n0=n, m=2, L_max=0, kind=0, K=K, sigma2=1.0, corr_len=0.1, seed=11), 0)
    try:
        a = torch.empty((S, (n + 1) ** 2), dtype=torch.float32, device=device())
        xi = torch.empty((S, K), dtype=torch.float64, device=device())
        M.mlmc_sample_fields(h, 0, 0, S, xi, a, M.MLMC_FP32)
        _, Q, it, rr, fl = _solve(M, h, n, a, M.MLMC_FP32, p, delta)
        assert np.all(fl == M.MLMC_F_CONVERGED), np.unique(fl)
        assert np.all(rr < delta) and np.all(np.isfinite(Q)) and np.all(Q > 0) and np.all(it > 0)
        # the inputs are the method's own draws, and the tensor-core field matches the FP64 field
        pick = [0, 2047, 4095]
        xi_o = o_rng.draw_xi(11, 0, 0, S, K)[pick]
        assert np.array_equal(xi[pick].cpu().numpy(), xi_o)
        phi = o_kl.basis(0, K, n, 1.0, 0.1)
        loga = o_kl.log_coefficient(xi_o, phi)
        scale = np.abs(xi_o) @ np.abs(phi)
        got = a[pick].cpu().numpy().astype(np.float64)
        assert np.all(np.abs(np.log(got) - loga) <= 2e-6 * np.maximum(scale, 1.0))
        # sampled systems again, alone and with the solution: a system's result does not
        # depend on the batch it is solved in
        sub = a[pick].contiguous()
        U, Qs, its, rrs, fls = _solve(M, h, n, sub, M.MLMC_FP32, p, delta, u=True)
        assert np.array_equal(Qs, Q[pick]) and np.array_equal(its, it[pick]) and np.array_equal(rrs, rr[pick])
        af = sub.cpu().numpy().astype(np.float64)
        g = o_fem.qoi_weights(n)
        b = o_fem.load_vector(n)
        for i in range(len(pick)):
            x = _interior(n, U[i])
            # the oracle's own assembly certifies the residual; Q is g^T x
            res = o_fem.relative_residual(n, af[i], x)
            assert res < delta * (1 + 1e-6) and abs(res - rrs[i]) <= 1e-6 * res + residual_floor(n, af[i], x)
            assert abs(Qs[i] - g @ x) <= 1e-13 * abs(Qs[i])
        # one sampled system against the oracle's direct solve, within the rigorous bound
        xo, Qo = o_fem.solve_sample(n, af[0])
        bound = np.linalg.norm(g) * rrs[0] * np.linalg.norm(b) / lambda_min_lower(n, af[0])
        assert abs(Qs[0] - Qo) <= bound
    finally:
        M.mlmc_destroy(h)


def test_adjoint_gradients_1024_samples_n256_box(M):
    n, S, K = 256, 1024, 256
    box = (0.25, 0.75, 0.25, 0.75)
    h = M.mlmc_create(M.make_problem(n0=n, m=2, L_max=0, kind=0, K=K, sigma2=1.0, corr_len=0.1, seed=21, qoi=1,
                                     box=box), 0)
    try:
        xi_np = o_rng.draw_xi(21, 0, 0, S, K)
        Q = torch.empty(S, dtype=torch.float64, device=device())
        G = torch.empty((S, K), dtype=torch.float64, device=device())
        M.mlmc_adjoint_grad(h, 0, S, to_dev(xi_np), M.MLMC_FP32, 1e-8, 200000, Q, G)
        torch.cuda.synchronize()
        Qg, Gg = Q.cpu().numpy(), G.cpu().numpy()
        assert np.all(np.isfinite(Qg)) and np.all(np.isfinite(Gg)) and np.all(Qg > 0)
        phi = o_kl.basis(0, K, n, 1.0, 0.1)
        for s in (0, 511, 1023):
            Qo, go = o_adj.gradient(n, xi_np[s], phi, box)
            # the mixed form's field is the FP64 tensor-core synthesis (about 1e-9 in log a) and the state and
            # adjoint solves reach delta = 1e-8: QoI and gradient are held to delta (observed about 2e-10)
            assert abs(Qg[s] - Qo) <= 1e-8 * abs(Qo)
            assert np.max(np.abs(Gg[s] - go)) <= 1e-8 * np.max(np.abs(go))
    finally:
        M.mlmc_destroy(h)


def test_finest_level_pair_of_7_level_hierarchy(M):
    # level 6 of h = 1/16 .. 1/1024: fine member n = 1024, coarse member n = 512 on the even nodes
    n0, L, K, S = 16, 6, 256, 4
    h = M.mlmc_create(M.make_problem(n0=n0, m=2, L_max=L, kind=0, K=K, sigma2=1.5, corr_len=0.1, seed=5), 0)
    try:
        nf, nc = n0 * 2 ** L, n0 * 2 ** (L - 1)
        hs = [1.0 / (n0 * 2 ** l) for l in range(L + 1)]
        deltas, precs = M.mlmc_adapt_precision(hs, 0.05)
        a = torch.empty((S, (nf + 1) ** 2), dtype=torch.float32, device=device())
        M.mlmc_sample_fields(h, L, 0, S, None, a, M.MLMC_FP32)
        Uf = torch.zeros((S, (nf + 1) ** 2), dtype=torch.float64, device=device())
        Uc = torch.zeros((S, (nc + 1) ** 2), dtype=torch.float64, device=device())
        Qf = torch.empty(S, dtype=torch.float64, device=device())
        Qc = torch.empty(S, dtype=torch.float64, device=device())
        flf = torch.zeros(S, dtype=torch.int32, device=device())
        flc = torch.zeros(S, dtype=torch.int32, device=device())
        rrf = torch.zeros(S, dtype=torch.float64, device=device())
        rrc = torch.zeros(S, dtype=torch.float64, device=device())
        M.mlmc_level_solve(h, nf, S, a, M.MLMC_FP32, nf, precs[L], M.MLMC_CG, deltas[L], 200000, Uf, Qf, None,
                           rrf, flf)
        M.mlmc_level_solve(h, nc, S, a, M.MLMC_FP32, nf, precs[L - 1], M.MLMC_CG, deltas[L - 1], 200000, Uc, Qc,
                           None, rrc, flc)
        torch.cuda.synchronize()
        flf, flc = flf.cpu().numpy(), flc.cpu().numpy()
        rrf, rrc = rrf.cpu().numpy(), rrc.cpu().numpy()
        # With the rule's default contrast (1) the finest levels get FP32 inner arithmetic; should
        # the conditions of Cor. 3.4 fail for a rough sample at h = 1/1024, the refinement must say
        # so (STAGNATED, with its true residual) rather than claim convergence; the estimate loop
        # re-runs such solves in FP64.
        ok = M.MLMC_F_CONVERGED
        assert np.all((flf == ok) | (flf == M.MLMC_F_STAGNATED)) and np.all(flc == ok)
        assert np.all(rrf[flf == ok] < deltas[L]) and np.all(rrf[flf != ok] >= deltas[L])
        af = a.cpu().numpy().astype(np.float64)
        Uf, Uc, Qf, Qc = Uf.cpu().numpy(), Uc.cpu().numpy(), Qf.cpu().numpy(), Qc.cpu().numpy()
        gf = o_fem.qoi_weights(nf)
        for s in range(S):
            xf = _interior(nf, Uf[s])
            rf = o_fem.relative_residual(nf, af[s], xf)
            assert abs(rf - rrf[s]) <= 1e-6 * rf + residual_floor(nf, af[s], xf)
            assert abs(Qf[s] - gf @ _interior(nf, Uf[s])) <= 1e-13 * abs(Qf[s])
        for s in (0, S - 1):
            ac, xc = o_fem.coarse_view(af[s], nf), _interior(nc, Uc[s])
            rc = o_fem.relative_residual(nc, ac, xc)
            assert rc < deltas[L - 1] * (1 + 1e-6) and abs(rc - rrc[s]) <= 1e-6 * rc + residual_floor(nc, ac, xc)
        # the level difference is small against the QoI (O(h^2) discretisation error)
        assert np.all(np.abs(Qf - Qc) < 0.02 * np.abs(Qf))
    finally:
        M.mlmc_destroy(h)
