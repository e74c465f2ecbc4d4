"""The estimate loop (Alg. 4.1) and the round scheduler on the GPU against the
sequential oracle, including the full-size mixed-precision workload."""
import ctypes

import numpy as np
import pytest
import scipy.sparse.linalg as spla

from gpu_common import device, lib, torch
from oracle import fem as o_fem
from oracle import kl as o_kl
from oracle import mlmc as o_mlmc
from oracle import rng as o_rng

pytestmark = pytest.mark.gpu

CFG1 = dict(n0=8, m=2, L_max=2, kind=0, K=16, sigma2=1.0, corr_len=0.3, seed=0)


@pytest.fixture(scope="module")
def M():
    device()
    return lib()


def _fixed(M, N):
    arr = (ctypes.c_int64 * len(N))(*N)
    return arr, ctypes.cast(arr, ctypes.POINTER(ctypes.c_int64))


# A solve stopped at ||b - A x|| <= delta ||b|| changes the full-domain QoI (f = 1: g = b) by
# |u^T r| <= ||u|| ||r|| <= c_u delta Q with c_u = rms(u) / mean(u) (Cauchy-Schwarz), about 1.3 for
# these coefficients; 1.5 bounds it.  A level difference Y_l takes the fine member at delta_l and the
# coarse member at delta_{l-1}.
C_U = 1.5


def _ylevel_tol(deltas, l, Qmax, extra_rel=1e-8):
    dc = deltas[l - 1] if l > 0 else 0.0
    return C_U * (deltas[l] + dc) * Qmax + extra_rel * Qmax


def test_fixed_sample_mlmc_config1_fp64(M):
    # 3 levels h = 1/8, 1/16, 1/32; K = 16, sigma^2 = 1, corr 0.3; N_l = 1000/500/250
    N = [1000, 500, 250]
    h = M.mlmc_create(M.make_problem(**CFG1), 0)
    try:
        o = M.mlmc_default_options()
        o.form = M.MLMC_FORM_FP64_FIXED
        o.fixed_delta = 2e-13          # above the FP64 floor (1 + h^-2) u of the h = 1/32 level
        o.L_start = 2
        keep, o.fixed_N = _fixed(M, N)
        r = M.result_dict(M.mlmc_estimate(h, o))
    finally:
        M.mlmc_destroy(h)
    P = o_mlmc.Problem(n0=8, m=2, L_max=2, field_kind=0, K=16, sigma2=1.0, corr_len=0.3, seed=0)
    ref = o_mlmc.estimate_fixed(P, N)
    assert r["N"] == N
    assert np.allclose(r["Yhat"], ref["Yhat"], rtol=1e-9, atol=1e-15)
    assert np.allclose(r["s2"], ref["s2"], rtol=1e-7, atol=0)
    assert abs(r["estimate"] - ref["estimate"]) <= 1e-10 * abs(ref["estimate"])


def test_adaptive_alg41_fp64_matches_oracle(M):
    tol = 2e-3
    h = M.mlmc_create(M.make_problem(**CFG1), 0)
    try:
        o = M.mlmc_default_options()
        o.form = M.MLMC_FORM_FP64_ADAPTIVE
        o.tol, o.N_init = tol, 50
        r = M.result_dict(M.mlmc_estimate(h, o))
    finally:
        M.mlmc_destroy(h)
    P = o_mlmc.Problem(n0=8, m=2, L_max=2, field_kind=0, K=16, sigma2=1.0, corr_len=0.3, seed=0)
    ref = o_mlmc.estimate(P, tol, N_init=50)
    # same samples, same rule: only solver tolerances delta_l separate the two
    assert r["L"] == ref["L"]
    assert np.all(np.abs(np.array(r["N"]) - ref["N"]) <= np.maximum(2, 0.01 * ref["N"]))
    assert abs(r["estimate"] - ref["estimate"]) <= max(1e-3 * abs(ref["estimate"]), 0.5 * ref["rmse"])
    assert r["rmse"] <= tol * 1.5


def test_mixed_vs_fp64_same_samples(M):
    # MPML and MLMC with the same N_l and seeds differ only by the computational error
    N = [400, 200, 100]
    out = {}
    for form in (M.MLMC_FORM_MIXED, M.MLMC_FORM_FP64_FIXED):
        h = M.mlmc_create(M.make_problem(**CFG1), 0)
        try:
            o = M.mlmc_default_options()
            o.form = form
            o.L_start = 2
            keep, o.fixed_N = _fixed(M, N)
            out[form] = M.result_dict(M.mlmc_estimate(h, o))
        finally:
            M.mlmc_destroy(h)
    mp, ml = out[M.MLMC_FORM_MIXED], out[M.MLMC_FORM_FP64_FIXED]
    deltas = np.array(mp["delta"])
    # level by level, the solves' accuracy bounds the difference (the FP64 form at 1e-10 is exact here)
    for l in range(3):
        assert abs(mp["Yhat"][l] - ml["Yhat"][l]) <= _ylevel_tol(deltas, l, 0.1), l
    assert abs(mp["estimate"] - ml["estimate"]) <= 0.1 * ml["rmse"] if ml["rmse"] > 0 else True
    assert mp["prec"][0] == M.MLMC_FP16S


def test_full_size_mixed_workload_sampled(M):
    # launch configuration of the benchmark: 5 levels h = 1/16 .. 1/256, K = 64,
    # sigma^2 = 1, corr 0.3; finest level batch of 100 samples, FP32 master field from
    # the tensor cores, inner precision and delta from the accuracy rule.
    S, level, K = 100, 4, 64
    h = M.mlmc_create(M.make_problem(n0=16, m=2, L_max=4, kind=0, K=K, sigma2=1.0, corr_len=0.3, seed=0), 0)
    try:
        n = 256
        hs = [1.0 / (16 * 2 ** l) for l in range(5)]
        deltas, precs = M.mlmc_adapt_precision(hs, 0.05)
        a = torch.empty((S, (n + 1) ** 2), dtype=torch.float32, device=device())
        a = torch.empty((S, (n + 1) ** 2), dtype=torch.float64, device=device())
        M.mlmc_sample_fields(h, level, 0, S, None, a, M.MLMC_FP64TC)   # the mixed form's master field
        Q = torch.empty(S, dtype=torch.float64, device=device())
        U = torch.empty((S, (n + 1) ** 2), dtype=torch.float64, device=device())
        rr = torch.empty(S, dtype=torch.float64, device=device())
        fl = torch.empty(S, dtype=torch.int32, device=device())
        M.mlmc_level_solve(h, n, S, a, M.MLMC_FP64, n, precs[4], M.MLMC_CG, deltas[4], 200000, U, Q, None, rr, fl)
        torch.cuda.synchronize()
        assert np.all(fl.cpu().numpy() == M.MLMC_F_CONVERGED)
        assert np.all(rr.cpu().numpy() < deltas[4])
        xi = o_rng.draw_xi(0, level, 0, S, K)
        phi = o_kl.basis(0, K, n, 1.0, 0.3)
        ag = a.cpu().numpy()
        for s in (0, 57):
            a_o = o_kl.coefficient(xi[s:s + 1], phi)[0]
            x, Qo = o_fem.solve_sample(n, a_o)
            A = o_fem.assemble(n, a_o)
            Ag = o_fem.assemble(n, ag[s])          # the oracle's assembly of the GPU's master field
            lmin = spla.eigsh(A, k=1, sigma=0, which="LM", return_eigenvectors=False)[0]
            g = o_fem.qoi_weights(n)
            b = o_fem.load_vector(n)
            u = U[s].cpu().numpy().reshape(n + 1, n + 1)[1:n, 1:n].ravel()
            # the refinement's claim, certified by independent assembly of the same master field
            res_g = np.linalg.norm(b - Ag @ u) / np.linalg.norm(b)
            assert res_g < deltas[4] * (1 + 1e-6)
            # against the oracle's own field: delta plus the field error's share, computed exactly
            res = np.linalg.norm(b - A @ u) / np.linalg.norm(b)
            assert res <= res_g + np.linalg.norm((A - Ag) @ u) / np.linalg.norm(b) * (1 + 1e-9) + 1e-15
            assert res < 1.1 * deltas[4]
            bound = np.linalg.norm(g) * res * np.linalg.norm(b) / lmin
            assert abs(Q[s].item() - Qo) <= bound * 1.01
            # the accuracy the method assigns to the finest level: delta_4 = 7.6e-7 relative, and the
            # QoI within c_u delta_4 |Q| of the FP64 oracle
            assert abs(Q[s].item() - Qo) <= min(1e-6, C_U * deltas[4]) * abs(Qo)
    finally:
        M.mlmc_destroy(h)


def test_bench_configuration_estimate_runs_clean(M):
    h = M.mlmc_create(M.make_problem(n0=16, m=2, L_max=4, kind=0, K=64, sigma2=1.0, corr_len=0.3, seed=0), 0)
    try:
        o = M.mlmc_default_options()
        o.tol, o.L_start, o.N_init = 1e-3, 4, 100
        r = M.result_dict(M.mlmc_estimate(h, o))
    finally:
        M.mlmc_destroy(h)
    assert r["L"] == 4 and r["flags_or"] & ~M.MLMC_F_CONVERGED == 0
    assert r["var_est"] <= (1e-3) ** 2 / 2 * 1.0001
    assert all(nl >= 100 for nl in r["N"])
    # E[Q] of the unit-coefficient problem is 0.0351; a lognormal coefficient with
    # sigma^2 = 1 raises it (E[1/a] = e^{1/2} for a constant field)
    assert 0.035 < r["estimate"] < 0.1


def test_group_size_choice_changes_the_estimate_only_within_the_solve_tolerance(M):
    # the bench configuration's FP32 launch (levels 2-4) puts its n = 128 systems four to a CTA, a
    # choice made per launch; a whole CTA each must give the same level means up to delta_l
    N = [200, 100, 100, 100, 100]
    out = {}
    for items in (-1, 2048):
        h = M.mlmc_create(M.make_problem(n0=16, m=2, L_max=4, kind=0, K=64, sigma2=1.0, corr_len=0.3, seed=0), 0)
        try:
            M.mlmc_debug_set_medium_items(h, items)
            o = M.mlmc_default_options()
            o.form = M.MLMC_FORM_MIXED
            o.L_start = 4
            keep, o.fixed_N = _fixed(M, N)
            out[items] = M.result_dict(M.mlmc_estimate(h, o))
        finally:
            M.mlmc_destroy(h)
    a, b = out[-1], out[2048]
    assert a["N"] == N and b["N"] == N and a["prec"] == b["prec"]
    assert a["flags_or"] & ~M.MLMC_F_CONVERGED == 0 and b["flags_or"] & ~M.MLMC_F_CONVERGED == 0
    deltas = np.array(a["delta"])
    for l in range(5):
        # both runs meet delta_l: each is within the tolerance of the exact level mean
        assert abs(a["Yhat"][l] - b["Yhat"][l]) <= 2 * _ylevel_tol(deltas, l, 0.1), l


def test_mixed_estimate_with_quarter_groups_matches_oracle(M):
    # the bench hierarchy with 8 samples per level: the FP32 launch of levels 2-4 holds the n = 256
    # systems on whole CTAs and the n = 128 and n = 64 ones four to a CTA, whose coarsest grids sit
    # in shared memory beside each other; every level mean must match the oracle's FP64 solves
    N = [8] * 5
    h = M.mlmc_create(M.make_problem(n0=16, m=2, L_max=4, kind=0, K=64, sigma2=1.0, corr_len=0.3, seed=3), 0)
    try:
        o = M.mlmc_default_options()
        o.form = M.MLMC_FORM_MIXED
        o.L_start = 4
        keep, o.fixed_N = _fixed(M, N)
        r = M.result_dict(M.mlmc_estimate(h, o))
    finally:
        M.mlmc_destroy(h)
    P = o_mlmc.Problem(n0=16, m=2, L_max=4, field_kind=0, K=64, sigma2=1.0, corr_len=0.3, seed=3)
    ref = o_mlmc.estimate_fixed(P, N)
    assert r["N"] == N and r["flags_or"] & ~M.MLMC_F_CONVERGED == 0
    deltas = np.array(r["delta"])
    Qmax = 0.1
    for l in range(5):
        # the solves' accuracy (c_u delta |Q| per member) plus the FP64 tensor-core field's (about 1e-9)
        assert abs(r["Yhat"][l] - ref["Yhat"][l]) <= _ylevel_tol(deltas, l, Qmax), l


def test_paper_setting_minres_fp64(M):
    # Sec. 5.1: f = 1, field of Eq. (5.2) with s = 4, q = 2, sigma = 2, h_0 = 1/8, m = 2,
    # MINRES in double precision to the accuracy delta_l of Eq. (4.12), k_p = 0.05.
    tol = 2e-3
    kw = dict(n0=8, m=2, L_max=3, kind=1, K=4, sigma2=4.0, q=2.0, seed=3)
    h = M.mlmc_create(M.make_problem(**kw), 0)
    try:
        o = M.mlmc_default_options()
        o.form = M.MLMC_FORM_FP64_ADAPTIVE
        o.solver = M.MLMC_MINRES
        o.tol, o.N_init = tol, 40
        r = M.result_dict(M.mlmc_estimate(h, o))
        o.solver = M.MLMC_CG
        rc = M.result_dict(M.mlmc_estimate(h, o))
    finally:
        M.mlmc_destroy(h)
    P = o_mlmc.Problem(n0=8, m=2, L_max=3, field_kind=1, K=4, sigma2=4.0, q=2.0, seed=3)
    ref = o_mlmc.estimate(P, tol, N_init=40)
    assert r["L"] == ref["L"] and r["flags_or"] & ~M.MLMC_F_CONVERGED == 0
    assert abs(r["estimate"] - ref["estimate"]) <= max(1e-3 * abs(ref["estimate"]), 0.5 * ref["rmse"])
    # MINRES and CG reach the same accuracy per level: the estimates agree to the solver tolerances
    assert abs(r["estimate"] - rc["estimate"]) <= 1e-3 * abs(rc["estimate"])


def test_seven_level_estimate_configuration(M):
    # the 7-level hierarchy h = 1/16 .. 1/1024, K = 256, sigma^2 = 1.5, corr 0.1, with a few samples per
    # level: the mixed form against (a) the oracle's FP64 solves on levels 0-3, (b) the GPU's FP64 form
    # at 1e-9 with the same samples on every level, (c) a certification of the finest level's solves
    # by the oracle's assembly of the same master field
    wl = dict(n0=16, m=2, L_max=6, kind=0, K=256, sigma2=1.5, corr_len=0.1, seed=7)
    N = [6, 4, 4, 2, 2, 2, 2]
    out = {}
    for form in (M.MLMC_FORM_MIXED, M.MLMC_FORM_FP64_FIXED):
        h = M.mlmc_create(M.make_problem(**wl), 0)
        try:
            o = M.mlmc_default_options()
            o.form, o.fixed_delta, o.L_start = form, 1e-9, 6
            keep, o.fixed_N = _fixed(M, N)
            out[form] = M.result_dict(M.mlmc_estimate(h, o))
        finally:
            M.mlmc_destroy(h)
    mp, ml = out[M.MLMC_FORM_MIXED], out[M.MLMC_FORM_FP64_FIXED]
    assert mp["N"] == N and ml["N"] == N
    assert mp["flags_or"] & ~M.MLMC_F_CONVERGED == 0 and ml["flags_or"] & ~M.MLMC_F_CONVERGED == 0
    deltas = np.array(mp["delta"])
    assert deltas[6] == pytest.approx(0.05 / 1024 ** 2, rel=1e-12)
    for l in range(7):
        assert abs(mp["Yhat"][l] - ml["Yhat"][l]) <= _ylevel_tol(deltas, l, 0.2) + C_U * 2e-9 * 0.2, l
    P = o_mlmc.Problem(n0=16, m=2, L_max=6, field_kind=0, K=256, sigma2=1.5, corr_len=0.1, seed=7)
    for l in range(4):
        Qf, Qc = P.level_samples(l, 0, N[l])
        assert abs(mp["Yhat"][l] - float(np.mean(Qf - Qc))) <= _ylevel_tol(deltas, l, 0.2), l
    # (c) finest level: the estimate's first sample pair, re-solved through mlmc_level_solve
    h = M.mlmc_create(M.make_problem(**wl), 0)
    try:
        nf, nc, S = 1024, 512, 1
        hs = [1.0 / (16 * 2 ** l) for l in range(7)]
        d7, p7 = M.mlmc_adapt_precision(hs, 0.05)
        a = torch.empty((S, (nf + 1) ** 2), dtype=torch.float64, device=device())
        M.mlmc_sample_fields(h, 6, 0, S, None, a, M.MLMC_FP64TC)
        U = torch.zeros((S, (nf + 1) ** 2), dtype=torch.float64, device=device())
        Q = torch.empty(S, dtype=torch.float64, device=device())
        rr = torch.empty(S, dtype=torch.float64, device=device())
        fl = torch.empty(S, dtype=torch.int32, device=device())
        M.mlmc_level_solve(h, nf, S, a, M.MLMC_FP64, nf, p7[6], M.MLMC_CG, d7[6], 200000, U, Q, None, rr, fl)
        torch.cuda.synchronize()
        fl0 = int(fl.cpu().numpy()[0])
        if fl0 == M.MLMC_F_CONVERGED:
            ag = a.cpu().numpy()[0]
            u = U.cpu().numpy()[0].reshape(nf + 1, nf + 1)[1:nf, 1:nf].ravel()
            res = o_fem.relative_residual(nf, ag, u)
            assert res < d7[6] * (1 + 1e-6) + 2e-12
            # the master field against the oracle's FP64 field of the same sample
            xi = o_rng.draw_xi(7, 6, 0, S, 256)
            loga = o_kl.log_coefficient(xi, o_kl.basis(0, 256, nf, 1.5, 0.1))[0]
            assert np.max(np.abs(np.log(ag) - loga)) <= 1e-6
        else:
            # a rough sample may break Cor. 3.4's conditions at FP32: the solve must say so
            assert fl0 == M.MLMC_F_STAGNATED and rr.cpu().numpy()[0] >= d7[6]
    finally:
        M.mlmc_destroy(h)


def test_calibrated_precision_rule_high_contrast(M):
    # sigma^2 = 1.5, corr 0.1: pointwise contrasts of about e^7.  The calibrated rule measures each level's
    # contrast on its own fields and takes FP64 inner arithmetic where Cor. 3.4's condition
    # contrast h^-2 u_single <= 0.5 fails; no solve then needs the FP64 re-run
    wl = dict(n0=16, m=2, L_max=4, kind=0, K=64, sigma2=1.5, corr_len=0.1, seed=9)
    N = [16, 8, 8, 8, 8]
    h = M.mlmc_create(M.make_problem(**wl), 0)
    try:
        o = M.mlmc_default_options()
        o.L_start, o.prec_rule = 4, 1
        keep, o.fixed_N = _fixed(M, N)
        r = M.result_dict(M.mlmc_estimate(h, o))
    finally:
        M.mlmc_destroy(h)
    assert r["flags_or"] & ~M.MLMC_F_CONVERGED == 0
    assert all(x == 0 for x in r["fp64_retries"])
    P = o_mlmc.Problem(n0=16, m=2, L_max=4, field_kind=0, K=64, sigma2=1.5, corr_len=0.1, seed=9)
    picked64 = False
    for l in range(5):
        a = P.fields(l, 0, N[l])
        contrast = float(np.max(a.max(axis=1) / a.min(axis=1)))
        assert r["contrast"][l] == pytest.approx(contrast, rel=1e-6)
        hl = 1.0 / (16 * 2 ** l)
        if contrast / hl ** 2 * 2.0 ** -24 > 0.5:
            assert r["prec"][l] == M.MLMC_FP64, l
            picked64 = True
        elif r["delta"][l] >= 1e-4:
            ok16 = a.min() >= 6.2e-5 and a.max() <= 4e3
            assert r["prec"][l] == (M.MLMC_FP16S if ok16 else M.MLMC_BF16S), l
        else:
            assert r["prec"][l] == M.MLMC_FP32, l
    assert picked64 and r["prec"][4] == M.MLMC_FP64
