"""The low-precision direct solver with iterative refinement (Sec. 5.2; Alg. 2.1
with the factorisation reused; Table 1 right) against the oracle's FP64
banded Cholesky solves, for each precision quadruple (u_f = u_s, u, u_r)."""
import ctypes

import numpy as np
import pytest

from gpu_common import device, lib, to_dev, torch
from inputs import smooth_lognormal_field
from oracle import fem as o_fem
from oracle import mlmc as o_mlmc

pytestmark = pytest.mark.gpu

PAPER = dict(n0=8, m=2, L_max=3, kind=1, K=4, sigma2=4.0, q=2.0, corr_len=0.3, seed=17)


@pytest.fixture(scope="module")
def M():
    device()
    return lib()


def _solve(M, h, n, af, prec, u, ur, delta, with_u=True):
    S = af.shape[0]
    M.mlmc_set_cholesky_precision(h, u, ur)
    a = to_dev(af, torch.float64)
    U = torch.zeros((S, (n + 1) ** 2), dtype=torch.float64, device=device()) if with_u else None
    Q = torch.empty(S, dtype=torch.float64, device=device())
    it = torch.empty(S, dtype=torch.int32, device=device())
    rr = torch.empty(S, dtype=torch.float64, device=device())
    fl = torch.empty(S, dtype=torch.int32, device=device())
    M.mlmc_level_solve(h, n, S, a, M.MLMC_FP64, n, prec, M.MLMC_CHOLESKY, delta, 1000, U, Q, it, rr, fl)
    M.mlmc_sync(h)
    return (U.cpu().numpy() if with_u else None), Q.cpu().numpy(), it.cpu().numpy(), rr.cpu().numpy(), fl.cpu().numpy()


@pytest.mark.parametrize("n,quad,delta,log_sd", [(8, "hhss", 3.5e-3, 1.5), (16, "ssss", 8.7e-4, 1.5),
                                                 (32, "ssdd", 2.2e-4, 1.5), (64, "ssdd", 5.5e-5, 1.5),
                                                 (16, "bbss", 8.7e-4, 0.5), (32, "dddd", 1e-12, 1.5),
                                                 (4, "qhhh", 2e-2, 0.5), (8, "qhhh", 1e-2, 0.5),
                                                 (16, "hhss", 8.7e-4, 1.0)])
def test_cholesky_refinement_matches_oracle(M, n, quad, delta, log_sd):
    # (bfloat16 keeps 8 significant bits: the refinement contracts only while kappa u_bf16 stays well below
    # one (Cor. 3.4), hence the milder field for it; test_bfloat16_factor_reports_stagnation covers the rest)
    code = {"q": M.MLMC_FP8S, "h": M.MLMC_FP16S, "b": M.MLMC_BF16S, "s": M.MLMC_FP32, "d": M.MLMC_FP64}
    prec, u, ur = code[quad[0]], code[quad[2]], code[quad[3]]
    S = 12
    af = smooth_lognormal_field(n, S, seed=300 + n, log_sd=log_sd)
    h = M.mlmc_create(M.make_problem(n0=n, m=2, L_max=0, kind=0, K=4, sigma2=1.0, corr_len=0.3), 0)
    try:
        U, Q, it, rr, fl = _solve(M, h, n, af, prec, u, ur, delta)
    finally:
        M.mlmc_destroy(h)
    assert np.all(fl == M.MLMC_F_CONVERGED), fl
    assert np.all(rr < delta) and np.all(it >= 1)
    for s in range(S):
        x, Qo = o_fem.solve_sample(n, af[s])
        xg = U[s].reshape(n + 1, n + 1)[1:n, 1:n].ravel()
        # the residual the refinement tested was computed in u_r: its FP64 value agrees to u_r's accuracy
        res = o_fem.relative_residual(n, af[s], xg)
        tol_r = {M.MLMC_FP64: 1e-12, M.MLMC_FP32: 2e-5, M.MLMC_FP16S: 1e-2 * delta}[ur]
        assert res < delta * (1 + 1e-6) + tol_r
        # the QoI within c_u delta |Q| (c_u = rms(u) / mean(u) <= 1.5, see test_gpu_estimate) and the working
        # precision's rounding of x (half: 2^-11 relative per entry)
        tol_q = 1.5 * delta + {M.MLMC_FP64: 1e-13, M.MLMC_FP32: 2e-6, M.MLMC_FP16S: 1e-3}[u]
        assert abs(Q[s] - Qo) <= tol_q * abs(Qo), (s, Q[s], Qo)


def test_bfloat16_factor_reports_stagnation(M):
    # on the rougher field a bfloat16 factor can stop contracting the residual: the solve must say so and
    # report its true (above-delta) residual, never claim convergence
    n, S, delta = 16, 12, 8.7e-4
    af = smooth_lognormal_field(n, S, seed=316, log_sd=1.5)
    h = M.mlmc_create(M.make_problem(n0=n, m=2, L_max=0, kind=0, K=4, sigma2=1.0, corr_len=0.3), 0)
    try:
        U, Q, it, rr, fl = _solve(M, h, n, af, M.MLMC_BF16S, M.MLMC_FP32, M.MLMC_FP32, delta)
    finally:
        M.mlmc_destroy(h)
    assert np.all((fl == M.MLMC_F_CONVERGED) | (fl == M.MLMC_F_STAGNATED))
    assert np.all(rr[fl == M.MLMC_F_CONVERGED] < delta) and np.all(rr[fl == M.MLMC_F_STAGNATED] >= delta)
    for s in np.nonzero(fl == M.MLMC_F_STAGNATED)[0]:
        xg = U[s].reshape(n + 1, n + 1)[1:n, 1:n].ravel()
        assert o_fem.relative_residual(n, af[s], xg) >= 0.9 * delta


def test_cholesky_iterations_and_memory_counter(M):
    # a half-precision factor needs more refinement steps than a single one for the same delta; the
    # profile's bit count follows the cost model of Sec. 5.2
    n, S, delta = 16, 8, 1e-6
    af = smooth_lognormal_field(n, S, seed=44, log_sd=1.0)
    h = M.mlmc_create(M.make_problem(n0=n, m=2, L_max=0, kind=0, K=4, sigma2=1.0, corr_len=0.3), 0)
    try:
        M.mlmc_profile_enable(h, True)
        out = {}
        for prec in (M.MLMC_FP16S, M.MLMC_FP32, M.MLMC_FP64):
            M.mlmc_profile_reset(h)
            _, Q, it, rr, fl = _solve(M, h, n, af, prec, M.MLMC_FP64, M.MLMC_FP64, delta, with_u=False)
            out[prec] = (it, M.mlmc_profile_get(h)["chol_bits"], fl)
    finally:
        M.mlmc_destroy(h)
    m = n - 1
    N = m * m
    nnz = N * (m + 1) - m * (m + 1) // 2
    for prec, bf in ((M.MLMC_FP16S, 16), (M.MLMC_FP32, 32), (M.MLMC_FP64, 64)):
        it, bits, fl = out[prec]
        assert np.all(fl == M.MLMC_F_CONVERGED)
        expect = sum(nnz * bf + N * 64 + (k + 1) * N * 64 + k * 2 * N * 64 for k in it)
        assert bits == pytest.approx(expect, rel=1e-12)
    assert out[M.MLMC_FP16S][0].mean() > out[M.MLMC_FP32][0].mean() >= out[M.MLMC_FP64][0].mean()


def test_half_factor_overflow_is_reported(M):
    # a coefficient of 1e10 puts factor entries near 1e5, beyond IEEE half's 65504: the solve reports a
    # non-finite value (Sec. 5.2 notes the overflow of low-precision formats) and the context keeps working
    n, S = 8, 3
    af = np.full((S, (n + 1) ** 2), 1e10)
    h = M.mlmc_create(M.make_problem(n0=n, m=2, L_max=0, kind=0, K=4, sigma2=1.0, corr_len=0.3), 0)
    try:
        _, Q, it, rr, fl = _solve(M, h, n, af, M.MLMC_FP16S, M.MLMC_FP64, M.MLMC_FP64, 1e-6, with_u=False)
        assert np.all(fl == M.MLMC_F_NONFINITE)
        _, Q2, _, _, fl2 = _solve(M, h, n, af, M.MLMC_FP32, M.MLMC_FP64, M.MLMC_FP64, 1e-10, with_u=False)
        assert np.all(fl2 == M.MLMC_F_CONVERGED)
        Qo = o_fem.solve_sample(n, af[0])[1]
        assert abs(Q2[0] - Qo) <= 1e-9 * abs(Qo)
    finally:
        M.mlmc_destroy(h)


def test_cholesky_estimate_paper_setting(M):
    # Sec. 5.2: the paper's field, h_0 = 1/8, MPML with Table 1 (right) -- hhss on level 0, ssss on level 1,
    # ssdd above -- against standard MLMC with an FP64 factor (dddd) on the same samples; level means within
    # the solves' accuracy and the memory cost model lower for MPML
    N = [200, 80, 40, 20]
    arr = (ctypes.c_int64 * 4)(*N)
    out = {}
    for form in (M.MLMC_FORM_MIXED, M.MLMC_FORM_FP64_FIXED):
        h = M.mlmc_create(M.make_problem(**PAPER), 0)
        try:
            M.mlmc_profile_enable(h, True)
            o = M.mlmc_default_options()
            o.form, o.solver, o.L_start, o.fixed_delta = form, M.MLMC_CHOLESKY, 3, 1e-10
            o.fixed_N = ctypes.cast(arr, ctypes.POINTER(ctypes.c_int64))
            r = M.result_dict(M.mlmc_estimate(h, o))
            out[form] = (r, M.mlmc_profile_get(h)["chol_bits"])
        finally:
            M.mlmc_destroy(h)
    (mp, bits_mp), (ml, bits_ml) = out[M.MLMC_FORM_MIXED], out[M.MLMC_FORM_FP64_FIXED]
    assert mp["N"] == N and ml["N"] == N
    assert mp["flags_or"] & ~M.MLMC_F_CONVERGED == 0 and ml["flags_or"] & ~M.MLMC_F_CONVERGED == 0
    deltas = np.array(mp["delta"])
    for l in range(4):
        dc = deltas[l - 1] if l > 0 else 0.0
        assert abs(mp["Yhat"][l] - ml["Yhat"][l]) <= 1.5 * (deltas[l] + dc) * 0.1 + 1e-7, l
    # the FP64 form against the oracle's own FP64 Cholesky on the two coarsest levels
    P = o_mlmc.Problem(n0=8, m=2, L_max=3, field_kind=1, K=4, sigma2=4.0, q=2.0, seed=17)
    for l in range(2):
        Qf, Qc = P.level_samples(l, 0, N[l])
        assert abs(ml["Yhat"][l] - float(np.mean(Qf - Qc))) <= 1e-9 * 0.1
    assert bits_mp < bits_ml


def test_quarter_factor_overflow_and_memory_counter(M):
    # FP8 E4M3 holds at most 448: a coefficient of 1e6 puts the factor's diagonal near 2e3 and the solve reports
    # the non-finite factor; on an ordinary field the q43 factor is counted at 8 bits an entry, half vectors at 16
    n, S = 8, 4
    h = M.mlmc_create(M.make_problem(n0=n, m=2, L_max=0, kind=0, K=4, sigma2=1.0, corr_len=0.3), 0)
    try:
        _, _, _, _, fl = _solve(M, h, n, np.full((S, (n + 1) ** 2), 1e6), M.MLMC_FP8S, M.MLMC_FP16S,
                                M.MLMC_FP16S, 1e-2, with_u=False)
        assert np.all(fl == M.MLMC_F_NONFINITE)
        M.mlmc_profile_enable(h, True)
        M.mlmc_profile_reset(h)
        af = smooth_lognormal_field(n, S, seed=77, log_sd=0.5)
        _, Q, it, rr, fl = _solve(M, h, n, af, M.MLMC_FP8S, M.MLMC_FP16S, M.MLMC_FP16S, 1e-2, with_u=False)
        bits = M.mlmc_profile_get(h)["chol_bits"]
    finally:
        M.mlmc_destroy(h)
    assert np.all(fl == M.MLMC_F_CONVERGED)
    m = n - 1
    N = m * m
    nnz = N * (m + 1) - m * (m + 1) // 2
    assert bits == pytest.approx(sum(nnz * 8 + N * 16 + (k + 1) * N * 16 + k * 2 * N * 16 for k in it), rel=1e-12)


def test_fp8_factor_only_with_the_cholesky_solver(M):
    n, S = 8, 2
    h = M.mlmc_create(M.make_problem(n0=n, m=2, L_max=0, kind=0, K=4, sigma2=1.0, corr_len=0.3), 0)
    try:
        a = to_dev(np.ones((S, (n + 1) ** 2)), torch.float64)
        Q = torch.empty(S, dtype=torch.float64, device=device())
        with pytest.raises(RuntimeError):
            M.mlmc_level_solve(h, n, S, a, M.MLMC_FP64, n, M.MLMC_FP8S, M.MLMC_CG, 1e-6, 100, None, Q, None,
                               None, None)
        with pytest.raises(RuntimeError):
            M.mlmc_set_cholesky_precision(h, M.MLMC_FP16S, M.MLMC_FP32)
    finally:
        M.mlmc_destroy(h)


def test_quarter_precision_estimate(M):
    # the quarter-precision setting of Sec. 5.2 (s = 1, sigma = 1, h_0 = 1/4, k_p = 0.4): qhhh on level 0,
    # hhss above, every solve converged, level means within the solves' accuracy of the dddd run on the same
    # samples, and the memory model's bits at most a third of dddd's (the paper reports about 3.5x)
    N = [400, 100, 40, 16]
    arr = (ctypes.c_int64 * 4)(*N)
    kw = dict(n0=4, m=2, L_max=3, kind=1, K=1, sigma2=1.0, q=2.0, corr_len=0.3, seed=5)
    out = {}
    for form in (M.MLMC_FORM_MIXED, M.MLMC_FORM_FP64_FIXED):
        h = M.mlmc_create(M.make_problem(**kw), 0)
        try:
            M.mlmc_profile_enable(h, True)
            o = M.mlmc_default_options()
            o.form, o.solver, o.L_start, o.fixed_delta = form, M.MLMC_CHOLESKY, 3, 1e-10
            o.kp, o.tol, o.chol_table = 0.4, 2e-6 ** 0.5, 1
            o.fixed_N = ctypes.cast(arr, ctypes.POINTER(ctypes.c_int64))
            r = M.result_dict(M.mlmc_estimate(h, o))
            out[form] = (r, M.mlmc_profile_get(h)["chol_bits"])
        finally:
            M.mlmc_destroy(h)
    (mp, bits_mp), (ml, bits_ml) = out[M.MLMC_FORM_MIXED], out[M.MLMC_FORM_FP64_FIXED]
    assert mp["N"] == N and mp["flags_or"] & ~M.MLMC_F_CONVERGED == 0
    assert mp["prec"][:4] == [M.MLMC_FP8S, M.MLMC_FP16S, M.MLMC_FP16S, M.MLMC_FP16S]
    deltas = np.array(mp["delta"])
    for l in range(4):
        dc = deltas[l - 1] if l > 0 else 0.0
        # delta_l >= 1e-3 here: the half working precision's rounding of x (2^-11) adds about 1e-3 |Q|
        assert abs(mp["Yhat"][l] - ml["Yhat"][l]) <= (1.5 * (deltas[l] + dc) + 2e-3) * 0.1, l
    assert bits_ml / bits_mp > 2.5
