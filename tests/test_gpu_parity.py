"""GPU parity of every stage of the hot path against the CPU FP64 oracle.

All calls go through the C ABI (paper_2503_05533_gb300.capi).  Inputs are either
the method's own random draws (both sides implement the Philox4x32-10 + AS241
generator) or seeded synthetic fields from tests/inputs.py, rounded to FP32 so
that both precisions of the GPU path see exactly the oracle's values.
"""
import numpy as np
import pytest
import scipy.sparse.linalg as spla

from gpu_common import device, fp64_delta, lib, round_storage, to_dev, torch
from inputs import random_vectors, rough_field, smooth_lognormal_field
from oracle import fem as o_fem
from oracle import kl as o_kl
from oracle import mlmc as o_mlmc
from oracle import rng as o_rng

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def M():
    device()
    return lib()


def _ctx(M, **kw):
    base = dict(n0=8, m=2, L_max=2, kind=0, K=16, sigma2=1.0, corr_len=0.3, seed=0)
    base.update(kw)
    return M.mlmc_create(M.make_problem(**base), 0)


# ---------------------------------------------------------------- A1: xi
@pytest.mark.parametrize("seed,level,first,S,K", [(0, 0, 0, 257, 16), (7, 3, 5, 3, 7),
                                                  ((1 << 40) + 3, 1, (1 << 32) - 2, 5, 256),
                                                  (123, 4, 1000, 1000, 64)])
def test_xi_bit_exact(M, seed, level, first, S, K):
    h = _ctx(M, L_max=4, K=K, seed=seed)
    try:
        xi = torch.empty((S, K), dtype=torch.float64, device=device())
        a = torch.empty((S, 9 * 9 * 2 ** (2 * level) * 4), dtype=torch.float64, device=device())
        M.mlmc_sample_fields(h, level, first, S, xi, a, M.MLMC_FP64)
        torch.cuda.synchronize()
        ref = o_rng.draw_xi(seed, level, first, S, K)
        got = xi.cpu().numpy()
        assert np.array_equal(got.view(np.uint64), ref.view(np.uint64))
    finally:
        M.mlmc_destroy(h)


# ---------------------------------------------------------------- A2: field (FP64 form)
@pytest.mark.parametrize("kind,K,n0,sigma2,corr", [(0, 16, 8, 1.0, 0.3), (0, 64, 12, 1.5, 0.1),
                                                   (1, 4, 8, 4.0, 0.3), (2, 1, 6, 0.49, 0.3)])
def test_field_fp64(M, kind, K, n0, sigma2, corr):
    h = _ctx(M, n0=n0, L_max=1, kind=kind, K=K, sigma2=sigma2, corr_len=corr, seed=5)
    try:
        S, n = 37, 2 * n0
        xi = torch.empty((S, K), dtype=torch.float64, device=device())
        a = torch.empty((S, (n + 1) ** 2), dtype=torch.float64, device=device())
        M.mlmc_sample_fields(h, 1, 100, S, xi, a, M.MLMC_FP64)
        torch.cuda.synchronize()
        ref = o_kl.coefficient(o_rng.draw_xi(5, 1, 100, S, K), o_kl.basis(kind, K, n, sigma2, corr, 2.0))
        assert np.allclose(a.cpu().numpy(), ref, rtol=1e-13, atol=0)
    finally:
        M.mlmc_destroy(h)


def test_synthesize_from_given_xi(M):
    h = _ctx(M, L_max=1, K=16)
    try:
        S, n = 9, 16
        xi_np = np.random.default_rng(3).standard_normal((S, 16))
        a = torch.empty((S, (n + 1) ** 2), dtype=torch.float64, device=device())
        M.mlmc_synthesize_fields(h, 1, S, to_dev(xi_np), a, M.MLMC_FP64)
        torch.cuda.synchronize()
        ref = o_kl.coefficient(xi_np, o_kl.basis(0, 16, n, 1.0, 0.3))
        assert np.allclose(a.cpu().numpy(), ref, rtol=1e-13, atol=0)
    finally:
        M.mlmc_destroy(h)


# ---------------------------------------------------------------- A3/A4: operator
def _oracle_apply(n, a_nodal, x_nodal):
    A = o_fem.assemble(n, a_nodal)
    X = x_nodal.reshape(n + 1, n + 1)[1:n, 1:n].ravel()
    y = np.zeros((n + 1, n + 1))
    y[1:n, 1:n] = (A @ X).reshape(n - 1, n - 1)
    return y.ravel()


@pytest.mark.parametrize("n,stride", [(2, 1), (5, 1), (13, 1), (16, 2), (33, 1), (64, 2)])
def test_operator_fp64_matches_element_assembly(M, n, stride):
    S = 3
    a_n = n * stride
    af = rough_field(a_n, S, seed=n)
    x = random_vectors(n, S, seed=n + 1)
    y = torch.empty((S, (n + 1) ** 2), dtype=torch.float64, device=device())
    M.mlmc_apply_operator(n, S, to_dev(af), M.MLMC_FP64, a_n, M.MLMC_FP64, to_dev(x), y, M.MLMC_FP64)
    torch.cuda.synchronize()
    got = y.cpu().numpy()
    for s in range(S):
        ac = af[s].reshape(a_n + 1, a_n + 1)[::stride, ::stride].ravel()
        ref = _oracle_apply(n, ac, x[s])
        assert np.max(np.abs(got[s] - ref)) <= 1e-14 * max(1.0, np.max(np.abs(ref)))


@pytest.mark.parametrize("op", ["FP32", "BF16S", "FP16S"])
def test_operator_storage_precisions(M, op):
    prec = getattr(M, "MLMC_" + op)
    n, S = 31, 2
    af = smooth_lognormal_field(n, S, seed=2)
    x = random_vectors(n, S, seed=3)
    y = torch.empty((S, (n + 1) ** 2), dtype=torch.float32, device=device())
    M.mlmc_apply_operator(n, S, to_dev(af, torch.float32), M.MLMC_FP32, n, prec, to_dev(x, torch.float32), y,
                          M.MLMC_FP32)
    torch.cuda.synchronize()
    got = y.cpu().numpy().astype(np.float64)
    for s in range(S):
        ref = _oracle_apply(n, round_storage(af[s], prec, M), x[s])
        assert np.max(np.abs(got[s] - ref)) <= 2e-6 * np.max(np.abs(ref))


# ---------------------------------------------------------------- A5-A7: solves
def _solve(M, h, n, a_np, a_prec, a_n, prec, delta, max_iters=200000, u=True):
    S = a_np.shape[0]
    dt = torch.float64 if a_prec == M.MLMC_FP64 else torch.float32
    a = to_dev(a_np, dt)
    U = torch.zeros((S, (n + 1) ** 2), dtype=torch.float64, device=device()) if u else None
    Q = torch.empty(S, dtype=torch.float64, device=device())
    it = torch.zeros(S, dtype=torch.int32, device=device())
    rr = torch.zeros(S, dtype=torch.float64, device=device())
    fl = torch.zeros(S, dtype=torch.int32, device=device())
    M.mlmc_level_solve(h, n, S, a, a_prec, a_n, prec, M.MLMC_CG, delta, max_iters, U, Q, it, rr, fl)
    torch.cuda.synchronize()
    return (U.cpu().numpy() if u else None), Q.cpu().numpy(), it.cpu().numpy(), rr.cpu().numpy(), fl.cpu().numpy()


def _interior(n, u):
    return u.reshape(n + 1, n + 1)[1:n, 1:n].ravel()


@pytest.mark.parametrize("n", [2, 3, 8, 13, 32, 64])
def test_solve_fp64_matches_cholesky(M, n):
    h = _ctx(M)
    try:
        S = 5
        af = smooth_lognormal_field(n, S, seed=10 + n, log_sd=1.0)
        delta = fp64_delta(n)
        U, Q, it, rr, fl = _solve(M, h, n, af, M.MLMC_FP64, n, M.MLMC_FP64, delta)
        for s in range(S):
            x, Qo = o_fem.solve_sample(n, af[s])
            assert abs(Q[s] - Qo) <= 1e-12 * abs(Qo)
            assert np.max(np.abs(_interior(n, U[s]) - x)) <= 1e-11 * np.max(np.abs(x))
            assert fl[s] == M.MLMC_F_CONVERGED and rr[s] < delta
            assert o_fem.relative_residual(n, af[s], _interior(n, U[s])) < 2 * delta
            # boundary of the returned solution is exactly zero
            B = U[s].reshape(n + 1, n + 1)
            assert not B[0].any() and not B[-1].any() and not B[:, 0].any() and not B[:, -1].any()
    finally:
        M.mlmc_destroy(h)


@pytest.mark.parametrize("prec", ["FP32", "BF16S", "FP16S"])
@pytest.mark.parametrize("delta", [3.5e-3, 1e-6, 1e-9])
def test_solve_mixed_reaches_delta(M, prec, delta):
    p = getattr(M, "MLMC_" + prec)
    h = _ctx(M)
    try:
        n, S = 32, 6
        af = smooth_lognormal_field(n, S, seed=77, log_sd=1.2)
        U, Q, it, rr, fl = _solve(M, h, n, af, M.MLMC_FP32, n, p, delta)
        assert np.all(fl == M.MLMC_F_CONVERGED), fl
        for s in range(S):
            x, Qo = o_fem.solve_sample(n, af[s])
            res = o_fem.relative_residual(n, af[s], _interior(n, U[s]))
            # the two FP64 residual evaluations agree up to their rounding floors (~1e-14 here)
            assert res < delta * (1 + 1e-6) and abs(res - rr[s]) <= 1e-6 * res + 1e-13
            # rigorous QoI bound |dQ| <= ||g|| ||r|| / lambda_min(A)
            A = o_fem.assemble(n, af[s])
            lmin = spla.eigsh(A, k=1, sigma=0, which="LM", return_eigenvectors=False)[0]
            b = o_fem.load_vector(n)
            g = o_fem.qoi_weights(n)
            bound = np.linalg.norm(g) * res * np.linalg.norm(b) / lmin
            assert abs(Q[s] - Qo) <= bound * 1.01
            if delta <= 1e-9:
                assert abs(Q[s] - Qo) <= 1e-6 * abs(Qo)
    finally:
        M.mlmc_destroy(h)


@pytest.mark.parametrize("prec", ["FP64", "FP32", "FP16S"])
@pytest.mark.parametrize("n", [100, 128, 160])
def test_solve_large_systems_row_pipeline(M, prec, n):
    # n >= 91 puts a system on a 512-thread CTA whose CG sweeps stream rows through
    # shared memory; n = 100 and 160 give teams that straddle warps (25 and 40 chunks per row)
    p = getattr(M, "MLMC_" + prec)
    h = _ctx(M)
    try:
        S = 3
        af = smooth_lognormal_field(n, S, seed=300 + n, log_sd=1.0)
        delta = fp64_delta(n) if prec == "FP64" else 1e-7
        ap = M.MLMC_FP64 if prec == "FP64" else M.MLMC_FP32
        U, Q, it, rr, fl = _solve(M, h, n, af, ap, n, p, delta)
        assert np.all(fl == M.MLMC_F_CONVERGED), fl
        b = o_fem.load_vector(n)
        g = o_fem.qoi_weights(n)
        for s in range(S):
            x, Qo = o_fem.solve_sample(n, af[s])
            res = o_fem.relative_residual(n, af[s], _interior(n, U[s]))
            assert res < (2 * delta if prec == "FP64" else delta * (1 + 1e-6))
            A = o_fem.assemble(n, af[s])
            lmin = spla.eigsh(A, k=1, sigma=0, which="LM", return_eigenvectors=False)[0]
            assert abs(Q[s] - Qo) <= np.linalg.norm(g) * res * np.linalg.norm(b) / lmin * 1.01 + 1e-15 * abs(Qo)
            if prec == "FP64":
                assert abs(Q[s] - Qo) <= 1e-10 * abs(Qo)
            B = U[s].reshape(n + 1, n + 1)
            assert not B[0].any() and not B[-1].any() and not B[:, 0].any() and not B[:, -1].any()
    finally:
        M.mlmc_destroy(h)


@pytest.mark.parametrize("prec", ["FP64", "FP32", "FP16S"])
def test_row_pipeline_is_bit_identical_to_plain_loads(M, prec):
    # the pipeline changes where rows come from, not the arithmetic: every ring depth and
    # the plain-load sweeps must give the same bits
    p = getattr(M, "MLMC_" + prec)
    ap = M.MLMC_FP64 if prec == "FP64" else M.MLMC_FP32
    h = _ctx(M)
    try:
        outs = []
        for ring in (0, 2, 3, 4, -1):
            M.mlmc_debug_set_solve_ring(h, ring)
            for n in (100, 128):
                af = smooth_lognormal_field(n, 2, seed=500 + n, log_sd=1.0)
                U, Q, it, rr, fl = _solve(M, h, n, af, ap, n, p, 1e-9 if prec != "FP64" else fp64_delta(n))
                outs.append((ring, n, U, Q, it, rr, fl))
        ref = {o[1]: o for o in outs if o[0] == 0}
        for ring, n, U, Q, it, rr, fl in outs:
            r = ref[n]
            assert np.array_equal(U, r[2]) and np.array_equal(Q, r[3]) and np.array_equal(it, r[4])
            assert np.array_equal(rr, r[5]) and np.array_equal(fl, r[6]) and np.all(fl == M.MLMC_F_CONVERGED)
        with pytest.raises(M.MlmcError):
            M.mlmc_debug_set_solve_ring(h, 1)
    finally:
        M.mlmc_destroy(h)


@pytest.mark.parametrize("prec", ["FP64", "FP32"])
@pytest.mark.parametrize("n", [100, 128])
def test_mid_size_systems_in_quarter_groups(M, prec, n):
    # n = 91..128 on 128-thread quarters (four systems per CTA, the last CTA partly filled), as the
    # estimate's mixed launches place them, and on whole CTAs: both reach delta and the oracle's Q
    p = getattr(M, "MLMC_" + prec)
    ap = M.MLMC_FP64 if prec == "FP64" else M.MLMC_FP32
    h = _ctx(M)
    try:
        S = 5
        af = smooth_lognormal_field(n, S, seed=900 + n, log_sd=1.0)
        delta = fp64_delta(n) if prec == "FP64" else 1e-8
        out = {}
        for items in (4096, 2048):
            M.mlmc_debug_set_medium_items(h, items)
            for pc in (M.MLMC_PC_MG, M.MLMC_PC_JACOBI):
                out[(items, pc)] = _solve_pc(M, h, n, af, ap, p, delta, pc)
        M.mlmc_debug_set_medium_items(h, -1)
        b = o_fem.load_vector(n)
        g = o_fem.qoi_weights(n)
        for s in range(S):
            _, Qo = o_fem.solve_sample(n, af[s])
            A = o_fem.assemble(n, af[s])
            lmin = spla.eigsh(A, k=1, sigma=0, which="LM", return_eigenvectors=False)[0]
            for key, (U, Q, it, rr, fl) in out.items():
                assert fl[s] == M.MLMC_F_CONVERGED, key
                res = o_fem.relative_residual(n, af[s], _interior(n, U[s]))
                assert res < (2 * delta if prec == "FP64" else delta * (1 + 1e-6)), key
                bound = np.linalg.norm(g) * res * np.linalg.norm(b) / lmin
                assert abs(Q[s] - Qo) <= bound * 1.01 + 1e-15 * abs(Qo), key
        for bad in (0, 511, 16385, -2):
            with pytest.raises(M.MlmcError):
                M.mlmc_debug_set_medium_items(h, bad)
    finally:
        M.mlmc_destroy(h)


def test_large_solve_pipeline_timeout_is_reported_and_gpu_stays_usable(M):
    # the row pipeline's first wait of every team expects bytes that never arrive:
    # the solve stops, flags its systems, and the context keeps working afterwards
    h = _ctx(M)
    try:
        n, S = 128, 2
        af = smooth_lognormal_field(n, S, seed=41, log_sd=1.0)
        a = to_dev(af, torch.float32)
        Q = torch.empty(S, dtype=torch.float64, device=device())
        fl = torch.zeros(S, dtype=torch.int32, device=device())
        M.mlmc_set_wait_timeout(h, 0.2)
        M.mlmc_debug_set_wait_extra(h, 1)
        M.mlmc_debug_set_solve_ring(h, 4)     # two systems would not turn the pipeline on by themselves
        # the solve is asynchronous: the wait that ran out is reported by the next synchronising call
        M.mlmc_level_solve(h, n, S, a, M.MLMC_FP32, n, M.MLMC_FP32, M.MLMC_CG, 1e-7, 100000, None, Q, None,
                           None, fl)
        with pytest.raises(M.MlmcError) as ei:
            M.mlmc_sync(h)
        assert ei.value.status == M.MLMC_E_TIMEOUT
        M.mlmc_sync(h)          # the error words were cleared by the read
        torch.cuda.synchronize()
        assert np.all(fl.cpu().numpy() == M.MLMC_F_TIMEOUT)
        M.mlmc_debug_set_wait_extra(h, 0)
        _, Q2, _, _, fl2 = _solve(M, h, n, af, M.MLMC_FP32, n, M.MLMC_FP32, 1e-9, u=False)
        assert np.all(fl2 == M.MLMC_F_CONVERGED)
        for s in range(S):
            assert abs(Q2[s] - o_fem.solve_sample(n, af[s])[1]) <= 1e-6 * abs(Q2[s])
    finally:
        M.mlmc_destroy(h)


def test_coarse_view_solve(M):
    h = _ctx(M)
    try:
        nf, S = 32, 4
        af = smooth_lognormal_field(nf, S, seed=5)
        _, Q, _, _, fl = _solve(M, h, nf // 2, af, M.MLMC_FP32, nf, M.MLMC_FP32, 1e-10, u=False)
        for s in range(S):
            _, Qo = o_fem.solve_sample(nf // 2, o_fem.coarse_view(af[s], nf))
            assert abs(Q[s] - Qo) <= 1e-7 * abs(Qo)
        assert np.all(fl == M.MLMC_F_CONVERGED)
    finally:
        M.mlmc_destroy(h)


def test_box_qoi(M):
    h = _ctx(M, qoi=1, box=(0.25, 0.75, 0.25, 0.75))
    try:
        n, S = 16, 3
        af = smooth_lognormal_field(n, S, seed=9)
        _, Q, _, _, _ = _solve(M, h, n, af, M.MLMC_FP64, n, M.MLMC_FP64, fp64_delta(n), u=False)
        for s in range(S):
            _, Qo = o_fem.solve_sample(n, af[s], box=(0.25, 0.75, 0.25, 0.75))
            assert abs(Q[s] - Qo) <= 1e-12 * abs(Qo)
    finally:
        M.mlmc_destroy(h)


def test_solve_edge_cases(M):
    h = _ctx(M)
    try:
        # S = 0 is a no-op
        Q = torch.zeros(1, dtype=torch.float64, device=device())
        M.mlmc_level_solve(h, 8, 0, Q, M.MLMC_FP64, 8, M.MLMC_FP64, M.MLMC_CG, 1e-8, 10, None, Q)
        # max_iters = 1 stops early with MAXIT
        af = smooth_lognormal_field(32, 2, seed=4)
        _, _, it, rr, fl = _solve(M, h, 32, af, M.MLMC_FP64, 32, M.MLMC_FP64, 1e-12, max_iters=1, u=False)
        assert np.all(fl == M.MLMC_F_MAXIT) and np.all(it <= 1) and np.all(rr > 1e-12)
        # a NaN in the coefficient is reported, not propagated silently
        bad = af.copy()
        bad[1, 100] = np.nan
        _, Qb, _, _, flb = _solve(M, h, 32, bad, M.MLMC_FP64, 32, M.MLMC_FP64, 1e-10, u=False)
        assert flb[1] == M.MLMC_F_NONFINITE and flb[0] == M.MLMC_F_CONVERGED
        # delta above 1: x = 0 already satisfies the criterion
        _, Q0, it0, _, fl0 = _solve(M, h, 8, af[:, : 81], M.MLMC_FP64, 8, M.MLMC_FP64, 2.0, u=False)
        assert np.all(Q0 == 0.0) and np.all(it0 == 0) and np.all(fl0 == M.MLMC_F_CONVERGED)
        # argument errors
        with pytest.raises(M.MlmcError):
            M.mlmc_level_solve(h, 1, 1, Q, M.MLMC_FP64, 1, M.MLMC_FP64, M.MLMC_CG, 1e-8, 10, None, Q)
        with pytest.raises(M.MlmcError):
            M.mlmc_level_solve(h, 8, 1, Q, M.MLMC_FP64, 12, M.MLMC_FP64, M.MLMC_CG, 1e-8, 10, None, Q)
    finally:
        M.mlmc_destroy(h)


def test_mixed_batch_many_sizes_one_launch(M):
    # several grid sizes in one resident-solve launch through the estimate scheduler's path
    h = _ctx(M, n0=6, L_max=3)
    try:
        for n in (6, 12, 24, 48):
            af = smooth_lognormal_field(n, 3, seed=n)
            _, Q, _, _, fl = _solve(M, h, n, af, M.MLMC_FP32, n, M.MLMC_FP16S, 1e-7, u=False)
            assert np.all(fl == M.MLMC_F_CONVERGED)
            for s in range(3):
                # FP32-exact coefficient, delta = 1e-7: held to 1e-6 (observed at most 1e-8)
                assert abs(Q[s] - o_fem.solve_sample(n, af[s])[1]) <= 1e-6 * abs(Q[s])
    finally:
        M.mlmc_destroy(h)


def test_bounded_wait_timeout_is_reported_and_gpu_stays_usable(M):
    # the tensor-core synthesis waits on TMA copies with a bounded wait; make it
    # expect bytes that never arrive, check the reported status, then run again
    h = _ctx(M, L_max=1, K=16, seed=4)
    try:
        M.mlmc_set_wait_timeout(h, 0.2)
        M.mlmc_debug_set_wait_extra(h, 1)
        S, n = 5, 16
        a = torch.empty((S, (n + 1) ** 2), dtype=torch.float32, device=device())
        M.mlmc_sample_fields(h, 1, 0, S, None, a, M.MLMC_FP32)
        with pytest.raises(M.MlmcError) as ei:
            M.mlmc_profile_get(h)
        assert ei.value.status == M.MLMC_E_TIMEOUT
        M.mlmc_debug_set_wait_extra(h, 0)
        M.mlmc_sample_fields(h, 1, 0, S, None, a, M.MLMC_FP32)
        M.mlmc_profile_get(h)
        ref = o_kl.coefficient(o_rng.draw_xi(4, 1, 0, S, 16), o_kl.basis(0, 16, n, 1.0, 0.3))
        assert np.allclose(a.cpu().numpy(), ref, rtol=5e-6, atol=0)
    finally:
        M.mlmc_destroy(h)


# ---------------------------------------------------------------- A8: statistics
def test_level_stats(M):
    h = _ctx(M)
    try:
        for S in (1, 2, 255, 1000, 4097):
            g = np.random.default_rng(S)
            Qf = g.standard_normal(S) * 1e-3 + 0.05
            Qc = Qf - (g.standard_normal(S) * 1e-5 + 2e-4)
            acc = M.mlmc_level_stats(h, S, to_dev(Qf), to_dev(Qc))
            Y = Qf - Qc
            m, v = o_mlmc.mean_var(Y)
            assert acc.n == S
            assert abs(acc.mean - m) <= 1e-13 * abs(m)
            assert abs(acc.m2 / S - v) <= 1e-9 * v + 1e-30
            assert abs((acc.sum + acc.sum_c) - np.sum(Y)) <= 1e-13 * abs(np.sum(Y))
        acc0 = M.mlmc_level_stats(h, 3, to_dev(np.ones(3)), None)
        assert acc0.n == 3 and acc0.mean == 1.0 and acc0.m2 == 0.0
    finally:
        M.mlmc_destroy(h)


# ---------------------------------------------------------------- pipeline A1-A8
def test_level_pipeline_matches_oracle_sampler(M):
    seed = 21
    h = _ctx(M, n0=8, L_max=2, K=16, seed=seed)
    P = o_mlmc.Problem(n0=8, m=2, L_max=2, field_kind=0, K=16, sigma2=1.0, corr_len=0.3, seed=seed)
    try:
        for level in (0, 1, 2):
            S, n = 40, 8 * 2 ** level
            a = torch.empty((S, (n + 1) ** 2), dtype=torch.float64, device=device())
            M.mlmc_sample_fields(h, level, 3, S, None, a, M.MLMC_FP64)
            Qf = torch.empty(S, dtype=torch.float64, device=device())
            M.mlmc_level_solve(h, n, S, a, M.MLMC_FP64, n, M.MLMC_FP64, M.MLMC_CG, fp64_delta(n), 100000, None, Qf)
            Qc = torch.zeros(S, dtype=torch.float64, device=device())
            if level > 0:
                M.mlmc_level_solve(h, n // 2, S, a, M.MLMC_FP64, n, M.MLMC_FP64, M.MLMC_CG, fp64_delta(n), 100000,
                                   None, Qc)
            acc = M.mlmc_level_stats(h, S, Qf, Qc if level > 0 else None)
            qf_o, qc_o = P.level_samples(level, 3, S)
            assert np.allclose(Qf.cpu().numpy(), qf_o, rtol=1e-11, atol=0)
            assert np.allclose(Qc.cpu().numpy(), qc_o, rtol=1e-11, atol=0)
            m, v = o_mlmc.mean_var(qf_o - qc_o)
            assert abs(acc.mean - m) <= 1e-9 * abs(m) and abs(acc.m2 / S - v) <= 1e-6 * v
    finally:
        M.mlmc_destroy(h)


# ---------------------------------------------------------------- A5: MINRES
def _solve_minres(M, h, n, a_np, a_prec, prec, delta):
    S = a_np.shape[0]
    dt = torch.float64 if a_prec == M.MLMC_FP64 else torch.float32
    U = torch.zeros((S, (n + 1) ** 2), dtype=torch.float64, device=device())
    Q = torch.empty(S, dtype=torch.float64, device=device())
    it = torch.zeros(S, dtype=torch.int32, device=device())
    rr = torch.zeros(S, dtype=torch.float64, device=device())
    fl = torch.zeros(S, dtype=torch.int32, device=device())
    M.mlmc_level_solve(h, n, S, to_dev(a_np, dt), a_prec, n, prec, M.MLMC_MINRES, delta, 200000, U, Q, it, rr, fl)
    torch.cuda.synchronize()
    return U.cpu().numpy(), Q.cpu().numpy(), it.cpu().numpy(), rr.cpu().numpy(), fl.cpu().numpy()


@pytest.mark.parametrize("n", [2, 8, 13, 32, 64])
def test_minres_fp64_matches_cholesky(M, n):
    h = _ctx(M)
    try:
        af = smooth_lognormal_field(n, 4, seed=200 + n, log_sd=1.0)
        delta = fp64_delta(n)
        U, Q, it, rr, fl = _solve_minres(M, h, n, af, M.MLMC_FP64, M.MLMC_FP64, delta)
        for s in range(4):
            x, Qo = o_fem.solve_sample(n, af[s])
            assert fl[s] == M.MLMC_F_CONVERGED and rr[s] < delta
            assert abs(Q[s] - Qo) <= 1e-12 * abs(Qo)
            assert np.max(np.abs(_interior(n, U[s]) - x)) <= 1e-11 * np.max(np.abs(x))
    finally:
        M.mlmc_destroy(h)


@pytest.mark.parametrize("prec", ["FP32", "FP16S"])
@pytest.mark.parametrize("delta", [3.5e-3, 1e-7])
def test_minres_mixed_reaches_delta(M, prec, delta):
    p = getattr(M, "MLMC_" + prec)
    h = _ctx(M)
    try:
        n, S = 48, 5
        af = smooth_lognormal_field(n, S, seed=31, log_sd=1.2)
        U, Q, it, rr, fl = _solve_minres(M, h, n, af, M.MLMC_FP32, p, delta)
        assert np.all(fl == M.MLMC_F_CONVERGED), fl
        for s in range(S):
            x, Qo = o_fem.solve_sample(n, af[s])
            res = o_fem.relative_residual(n, af[s], _interior(n, U[s]))
            assert res < delta * (1 + 1e-6)
            A = o_fem.assemble(n, af[s])
            lmin = spla.eigsh(A, k=1, sigma=0, which="LM", return_eigenvectors=False)[0]
            bound = np.linalg.norm(o_fem.qoi_weights(n)) * res * np.linalg.norm(o_fem.load_vector(n)) / lmin
            assert abs(Q[s] - Qo) <= bound * 1.01
    finally:
        M.mlmc_destroy(h)


# ---------------------------------------------------------------- A5: multigrid preconditioner
def _solve_pc(M, h, n, af, a_prec, prec, delta, pc, nu=0, coarse=0, omega=0.0):
    M.mlmc_set_precond(h, pc, nu, coarse, omega)
    try:
        return _solve(M, h, n, af, a_prec, n, prec, delta)
    finally:
        M.mlmc_set_precond(h, M.MLMC_PC_MG, 1, 8, 0.8)


@pytest.mark.parametrize("prec", ["FP64", "FP32", "FP16S"])
def test_multigrid_and_jacobi_reach_the_same_solution(M, prec):
    p = getattr(M, "MLMC_" + prec)
    ap = M.MLMC_FP64 if prec == "FP64" else M.MLMC_FP32
    h = _ctx(M)
    try:
        n, S = 128, 3
        af = smooth_lognormal_field(n, S, seed=640, log_sd=1.2)
        delta = fp64_delta(n) if prec == "FP64" else 1e-7
        Um, Qm, itm, rrm, flm = _solve_pc(M, h, n, af, ap, p, delta, M.MLMC_PC_MG)
        Uj, Qj, itj, rrj, flj = _solve_pc(M, h, n, af, ap, p, delta, M.MLMC_PC_JACOBI)
        assert np.all(flm == M.MLMC_F_CONVERGED) and np.all(flj == M.MLMC_F_CONVERGED)
        # a V-cycle per iteration: iterations no longer grow like h^-1
        assert np.all(itm * 10 < itj), (itm, itj)
        b = o_fem.load_vector(n)
        g = o_fem.qoi_weights(n)
        for s in range(S):
            A = o_fem.assemble(n, af[s])
            lmin = spla.eigsh(A, k=1, sigma=0, which="LM", return_eigenvectors=False)[0]
            _, Qo = o_fem.solve_sample(n, af[s])
            for U, Q, rr in ((Um, Qm, rrm), (Uj, Qj, rrj)):
                res = o_fem.relative_residual(n, af[s], _interior(n, U[s]))
                assert res < (2 * delta if prec == "FP64" else delta * (1 + 1e-6))
                assert abs(Q[s] - Qo) <= np.linalg.norm(g) * res * np.linalg.norm(b) / lmin * 1.01 + 1e-15 * abs(Qo)
    finally:
        M.mlmc_destroy(h)


@pytest.mark.parametrize("n", [6, 24, 60, 100, 192])
def test_multigrid_hierarchies_that_stop_early(M, n):
    # coarsening halves while the grid is even and the half has >= 4 cells:
    # 6 has no coarse grid, 24 -> 12 -> 6, 60 -> 30 -> 15, 100 -> 50 -> 25, 192 -> ... -> 6
    h = _ctx(M)
    try:
        af = smooth_lognormal_field(n, 2, seed=700 + n, log_sd=1.0)
        delta = fp64_delta(n)
        U, Q, it, rr, fl = _solve_pc(M, h, n, af, M.MLMC_FP64, M.MLMC_FP64, delta, M.MLMC_PC_MG)
        assert np.all(fl == M.MLMC_F_CONVERGED)
        for s in range(2):
            x, Qo = o_fem.solve_sample(n, af[s])
            assert abs(Q[s] - Qo) <= 1e-11 * abs(Qo)
            assert np.max(np.abs(_interior(n, U[s]) - x)) <= 1e-10 * np.max(np.abs(x))
    finally:
        M.mlmc_destroy(h)


@pytest.mark.parametrize("nu,coarse,omega", [(1, 2, 0.8), (2, 16, 0.6), (1, 8, 0.9)])
def test_multigrid_parameters(M, nu, coarse, omega):
    h = _ctx(M)
    try:
        n = 64
        af = smooth_lognormal_field(n, 3, seed=77, log_sd=1.0)
        U, Q, it, rr, fl = _solve_pc(M, h, n, af, M.MLMC_FP32, M.MLMC_FP32, 1e-8, M.MLMC_PC_MG, nu, coarse, omega)
        assert np.all(fl == M.MLMC_F_CONVERGED) and np.all(rr < 1e-8)
        for s in range(3):
            assert o_fem.relative_residual(n, af[s], _interior(n, U[s])) < 1e-8 * (1 + 1e-6)
        with pytest.raises(M.MlmcError):
            M.mlmc_set_precond(h, M.MLMC_PC_MG, 3, 0, 0.0)     # nu is 1 or 2
        with pytest.raises(M.MlmcError):
            M.mlmc_set_precond(h, M.MLMC_PC_MG, 0, 3, 0.0)     # coarse sweeps even
        with pytest.raises(M.MlmcError):
            M.mlmc_set_inner_tolerance(h, 1.5, 0.0)
    finally:
        M.mlmc_destroy(h)


@pytest.mark.parametrize("prec", ["FP64", "FP32"])
def test_minres_with_multigrid_and_jacobi(M, prec):
    p = getattr(M, "MLMC_" + prec)
    ap = M.MLMC_FP64 if prec == "FP64" else M.MLMC_FP32
    h = _ctx(M)
    try:
        n, S = 128, 2
        af = smooth_lognormal_field(n, S, seed=810, log_sd=1.0)
        delta = fp64_delta(n) if prec == "FP64" else 1e-7
        out = {}
        for pc in (M.MLMC_PC_MG, M.MLMC_PC_JACOBI):
            M.mlmc_set_precond(h, pc, 0, 0, 0.0)
            out[pc] = _solve_minres(M, h, n, af, ap, p, delta)
        M.mlmc_set_precond(h, M.MLMC_PC_MG, 0, 0, 0.0)
        Um, Qm, itm, rrm, flm = out[M.MLMC_PC_MG]
        Uj, Qj, itj, rrj, flj = out[M.MLMC_PC_JACOBI]
        assert np.all(flm == M.MLMC_F_CONVERGED) and np.all(flj == M.MLMC_F_CONVERGED)
        assert np.all(itm * 10 < itj), (itm, itj)
        for s in range(S):
            for U in (Um, Uj):
                res = o_fem.relative_residual(n, af[s], _interior(n, U[s]))
                assert res < (2 * delta if prec == "FP64" else delta * (1 + 1e-6))
    finally:
        M.mlmc_destroy(h)


def test_two_asynchronous_solves_on_a_user_stream(M):
    # mlmc_level_solve enqueues its launch and returns: two calls on a stream of the caller's, with no
    # host synchronisation between them, share the context's workspace in call order on the device
    h = _ctx(M)
    try:
        st = torch.cuda.Stream()
        S, cases = 4, [(32, 71, M.MLMC_FP64, M.MLMC_FP64), (64, 72, M.MLMC_FP32, M.MLMC_FP32)]
        outs = []
        with torch.cuda.stream(st):
            for n, seed, ap, prec in cases:
                af = smooth_lognormal_field(n, S, seed=seed, log_sd=1.0)
                a = to_dev(af, torch.float64 if ap == M.MLMC_FP64 else torch.float32)
                Q = torch.empty(S, dtype=torch.float64, device=device())
                fl = torch.zeros(S, dtype=torch.int32, device=device())
                delta = fp64_delta(n) if prec == M.MLMC_FP64 else 1e-9
                M.mlmc_level_solve(h, n, S, a, ap, n, prec, M.MLMC_CG, delta, 100000, None, Q, None, None, fl,
                                   stream=st)
                outs.append((n, af, a, Q, fl, prec))
        M.mlmc_sync(h, st)
        for n, af, a, Q, fl, prec in outs:
            assert np.all(fl.cpu().numpy() == M.MLMC_F_CONVERGED)
            tol = 1e-11 if prec == M.MLMC_FP64 else 1e-7
            for s in range(S):
                Qo = o_fem.solve_sample(n, af[s])[1]
                assert abs(Q[s].item() - Qo) <= tol * abs(Qo)
    finally:
        M.mlmc_destroy(h)


@pytest.mark.parametrize("solver", ["CG", "CHOLESKY"])
def test_level_solve_reads_padded_rows(M, solver):
    # rows of the master coefficient a_ld apart (here padded to whole 128-byte lines, with garbage in the gap)
    # give the same bits as the dense layout, for the fine grid and for a coarse view (a_n = 2 n)
    S, n = 5, 32
    af = smooth_lognormal_field(2 * n, S, seed=77, log_sd=1.0)
    V2 = (2 * n + 1) ** 2
    ld = (V2 + 31) // 32 * 32
    padded = np.full((S, ld), 1e30)
    padded[:, :V2] = af
    sv = getattr(M, "MLMC_" + solver)
    h = _ctx(M)
    try:
        outs = []
        for a_np, a_ld in ((af, 0), (padded, ld)):
            a = to_dev(a_np, torch.float64)
            Q = torch.empty(S, dtype=torch.float64, device=device())
            it = torch.zeros(S, dtype=torch.int32, device=device())
            fl = torch.zeros(S, dtype=torch.int32, device=device())
            M.mlmc_level_solve(h, n, S, a, M.MLMC_FP64, 2 * n, M.MLMC_FP32, sv, 1e-9, 100000, None, Q, it, None, fl,
                               a_ld=a_ld)
            M.mlmc_sync(h)
            outs.append((Q.cpu().numpy(), it.cpu().numpy(), fl.cpu().numpy()))
        assert np.array_equal(outs[0][0], outs[1][0]) and np.array_equal(outs[0][1], outs[1][1])
        assert np.all(outs[0][2] == M.MLMC_F_CONVERGED) and np.array_equal(outs[0][2], outs[1][2])
        for s in range(S):
            Qo = o_fem.solve_sample(n, af[s].reshape(2 * n + 1, 2 * n + 1)[::2, ::2].ravel())[1]
            assert abs(outs[1][0][s] - Qo) <= 1.5e-9 * abs(Qo) + 1e-15
        with pytest.raises(M.MlmcError):
            M.mlmc_level_solve(h, n, S, to_dev(af, torch.float64), M.MLMC_FP64, 2 * n, M.MLMC_FP32, sv, 1e-9, 100,
                               None, torch.empty(S, dtype=torch.float64, device=device()), a_ld=V2 - 1)
    finally:
        M.mlmc_destroy(h)


@pytest.mark.parametrize("mg_min,coarse", [(2, 8), (8, 16), (16, 4), (64, 16)])
def test_multigrid_depth_choices_meet_delta(M, mg_min, coarse):
    # the coarsest grid of the V-cycle (mlmc_set_mg_coarsest) and its sweeps only change the preconditioner:
    # every choice still certifies delta on the FP64 residual and agrees with the oracle within c_u delta
    n, S, delta = 128, 4, 1e-8
    af = smooth_lognormal_field(n, S, seed=61, log_sd=1.0)
    h = _ctx(M)
    try:
        M.mlmc_set_mg_coarsest(h, mg_min)
        M.mlmc_set_precond(h, M.MLMC_PC_MG, 0, coarse, 0.0)
        U, Q, it, rr, fl = _solve(M, h, n, af, M.MLMC_FP64, n, M.MLMC_FP32, delta)
        with pytest.raises(M.MlmcError):
            M.mlmc_set_mg_coarsest(h, 1)
    finally:
        M.mlmc_destroy(h)
    assert np.all(fl == M.MLMC_F_CONVERGED) and np.all(rr < delta)
    for s in range(S):
        x, Qo = o_fem.solve_sample(n, af[s])
        assert abs(Q[s] - Qo) <= 1.5 * delta * abs(Qo)


@pytest.mark.parametrize("n,prec,solver,pc,ring", [
    (160, "FP32", "CG", "MG", -1), (64, "FP16S", "CG", "MG", -1), (24, "FP32", "CG", "JACOBI", -1),
    (160, "FP32", "MINRES", "MG", -1), (100, "FP64", "CG", "MG", -1), (128, "FP32", "CG", "JACOBI", 4),
    (96, "BF16S", "MINRES", "JACOBI", -1)])
def test_solve_in_a_reused_workspace_is_bit_identical(M, n, prec, solver, pc, ring):
    # a batch solved in the workspace that another batch of the same shape has just used (its values left in
    # place) gives bit for bit what a new context gives: nothing of a solve is read before it is written,
    # except what the launch clears
    S = 6
    p = getattr(M, "MLMC_" + prec)
    fa, fb = smooth_lognormal_field(n, S, seed=11), smooth_lognormal_field(n, S, seed=12)

    def run(h, af):
        dt = torch.float64 if p == M.MLMC_FP64 else torch.float32
        a = to_dev(af, dt)
        U = torch.zeros((S, (n + 1) ** 2), dtype=torch.float64, device=device())
        Q = torch.empty(S, dtype=torch.float64, device=device())
        it = torch.zeros(S, dtype=torch.int32, device=device())
        rr = torch.zeros(S, dtype=torch.float64, device=device())
        fl = torch.zeros(S, dtype=torch.int32, device=device())
        M.mlmc_level_solve(h, n, S, a, M.MLMC_FP64 if p == M.MLMC_FP64 else M.MLMC_FP32, n, p,
                           getattr(M, "MLMC_" + solver), 1e-9 if p == M.MLMC_FP64 else 1e-7, 200000, U, Q, it,
                           rr, fl)
        torch.cuda.synchronize()
        return [x.cpu().numpy() for x in (U, Q, it, rr, fl)]

    hs = [_ctx(M), _ctx(M)]
    try:
        for h in hs:
            M.mlmc_set_precond(h, getattr(M, "MLMC_PC_" + pc))
            M.mlmc_debug_set_solve_ring(h, ring)
        run(hs[0], fa)
        got, ref = run(hs[0], fb), run(hs[1], fb)
        assert np.all(ref[4] == M.MLMC_F_CONVERGED)
        for x, y in zip(got, ref):
            assert np.array_equal(x.view(np.uint8), y.view(np.uint8))
    finally:
        for h in hs:
            M.mlmc_destroy(h)


@pytest.mark.parametrize("n,prec", [(160, "FP32"), (256, "FP32"), (96, "FP16S"), (100, "FP64")])
def test_full_multigrid_start(M, n, prec):
    # the first inner CG solve from the nested-iteration guess: the same certified accuracy against the
    # oracle as from zero, in fewer inner iterations
    S = 4
    p = getattr(M, "MLMC_" + prec)
    af = smooth_lognormal_field(n, S, seed=21)
    a_prec = M.MLMC_FP64 if p == M.MLMC_FP64 else M.MLMC_FP32
    delta = 1e-10 if p == M.MLMC_FP64 else 1e-7
    out = {}
    h = _ctx(M)
    try:
        for on in (True, False):
            M.mlmc_set_full_multigrid(h, on)
            out[on] = _solve(M, h, n, af, a_prec, n, p, delta, u=False)
    finally:
        M.mlmc_destroy(h)
    for on in (True, False):
        _, Q, it, rr, fl = out[on]
        assert np.all(fl == M.MLMC_F_CONVERGED) and np.all(rr < delta)
        for s in range(S):
            xo, Qo = o_fem.solve_sample(n, af[s])
            assert abs(Q[s] - Qo) <= 1e-6 * abs(Qo)
    assert out[True][2].sum() < out[False][2].sum()
