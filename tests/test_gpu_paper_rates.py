"""The paper's Sec. 5.1 setting on the GPU: the decay of the computational
error with the effective precision (Fig. 1; Lemma 4.6) and the library's
operation counter.

Lemma 4.6 bounds the computational part of the bias by O(delta) (through
||G(u_h) - G(u~_h)||_{L1(Omega)} <= C delta) and of the variance of the level
difference by O(delta^2).  With the paper's solver (FP64 MINRES, here Jacobi-
preconditioned) stopped at relative residual delta on the fine member and
4 delta on the coarse one (the ratio delta_{l-1} / delta_l of Eq. (4.12) for
m = 2), the measured rates over delta in [1e-6, 1e-2] are at least 1 and 2
for the paper's QoI (int u, which converges faster: its error is quadratic in
the residual) and near 1 and 2 for a box QoI.  The exact solutions come from
the oracle's banded Cholesky solves.
"""
import numpy as np
import pytest

from gpu_common import device, lib, torch
from oracle import fem as o_fem
from oracle import kl as o_kl
from oracle import rng as o_rng

pytestmark = pytest.mark.gpu

PAPER = dict(n0=8, m=2, L_max=2, kind=1, K=4, sigma2=4.0, q=2.0, corr_len=0.3, seed=11)


@pytest.fixture(scope="module")
def M():
    device()
    return lib()


def _slope(x, y):
    return float(np.polyfit(np.log(x), np.log(y), 1)[0])


def _rates(M, qoi, box):
    """Computational errors of the level-2 pair of the paper's field against delta: the mean absolute
    QoI error of the fine member (it bounds the bias) and Var[Y~_l - Y_l]; slopes of their logs."""
    level, S = 2, 256
    nf, nc = 32, 16
    xi = o_rng.draw_xi(PAPER["seed"], level, 0, S, 4)
    phi = o_kl.basis(1, 4, nf, 4.0, 0.3, 2.0)
    a_np = o_kl.coefficient(xi, phi)
    Qf = np.array([o_fem.solve_sample(nf, a_np[s], box)[1] for s in range(S)])
    Qc = np.array([o_fem.solve_sample(nc, o_fem.coarse_view(a_np[s], nf), box)[1] for s in range(S)])
    kw = dict(PAPER, qoi=qoi)
    if box is not None:
        kw["box"] = box
    h = M.mlmc_create(M.make_problem(**kw), 0)
    try:
        M.mlmc_set_precond(h, M.MLMC_PC_JACOBI)
        a = torch.empty((S, (nf + 1) ** 2), dtype=torch.float64, device=device())
        M.mlmc_sample_fields(h, level, 0, S, None, a, M.MLMC_FP64)
        deltas = np.logspace(-2, -6, 9)
        l1, var, bias = [], [], []
        for d in deltas:
            qf = torch.empty(S, dtype=torch.float64, device=device())
            qc = torch.empty(S, dtype=torch.float64, device=device())
            ff = torch.empty(S, dtype=torch.int32, device=device())
            fc = torch.empty(S, dtype=torch.int32, device=device())
            M.mlmc_level_solve(h, nf, S, a, M.MLMC_FP64, nf, M.MLMC_FP64, M.MLMC_MINRES, d, 100000, None, qf,
                               None, None, ff)
            M.mlmc_level_solve(h, nc, S, a, M.MLMC_FP64, nf, M.MLMC_FP64, M.MLMC_MINRES, 4 * d, 100000, None, qc,
                               None, None, fc)
            torch.cuda.synchronize()
            assert np.all(ff.cpu().numpy() == M.MLMC_F_CONVERGED) and np.all(fc.cpu().numpy() == M.MLMC_F_CONVERGED)
            ef = qf.cpu().numpy() - Qf
            ey = ef - (qc.cpu().numpy() - Qc)
            l1.append(np.mean(np.abs(ef)))
            bias.append(abs(np.mean(ef)))
            var.append(np.mean((ey - ey.mean()) ** 2))
    finally:
        M.mlmc_destroy(h)
    l1, var, bias = np.array(l1), np.array(var), np.array(bias)
    assert np.all(bias <= l1 * (1 + 1e-12))
    return deltas, l1, var, Qf


def test_computational_error_rates_fig1_paper_qoi(M):
    # Q = int u with f = 1, as in Fig. 1.  Lemma 4.6 gives rates of at least 1 (bias) and 2 (variance).
    # For this QoI g = b, so Q - Q~ = b^T e = e^T A u ... = r^T A^-1 r for the Galerkin iterate: the
    # error is quadratic in the residual, and the measured rates are about 2 and 4.
    deltas, l1, var, Qf = _rates(M, 0, None)
    assert np.all(l1 <= 1.5 * deltas * np.abs(Qf).max())
    sl, sv = _slope(deltas, l1), _slope(deltas, var)
    assert sl >= 0.9, (sl, l1)
    assert sv >= 1.8, (sv, var)


def test_computational_error_rates_fig1_box_qoi(M):
    # Q = int over [0.25, 0.75]^2 of u: the QoI error is linear in the residual, and the measured
    # rates are the lemma's, 1 for the bias and 2 for the variance of the level difference
    deltas, l1, var, Qf = _rates(M, 1, (0.25, 0.75, 0.25, 0.75))
    sl, sv = _slope(deltas, l1), _slope(deltas, var)
    assert 0.75 <= sl <= 1.25, (sl, l1)
    assert 1.5 <= sv <= 2.5, (sv, var)


def test_operation_counter_of_the_minres_solve(M):
    # FP64 Jacobi-MINRES: 2 stencil sweeps from stored FP64 weights (12 operations a point) and 18 more
    # per iteration and unknown; the refinement residuals and set-up add a bounded amount per unknown
    n, S = 32, 16
    h = M.mlmc_create(M.make_problem(**PAPER), 0)
    try:
        M.mlmc_set_precond(h, M.MLMC_PC_JACOBI)
        a = torch.empty((S, (n + 1) ** 2), dtype=torch.float64, device=device())
        M.mlmc_sample_fields(h, 2, 0, S, None, a, M.MLMC_FP64)
        M.mlmc_profile_enable(h, True)
        M.mlmc_profile_reset(h)
        Q = torch.empty(S, dtype=torch.float64, device=device())
        M.mlmc_level_solve(h, n, S, a, M.MLMC_FP64, n, M.MLMC_FP64, M.MLMC_MINRES, 1e-8, 100000, None, Q)
        p = M.mlmc_profile_get(h)
    finally:
        M.mlmc_destroy(h)
    unk = S * (n - 1) ** 2
    per_it = 18.0 + 2 * 12.0
    assert p["solve_flops"] >= per_it * p["unknown_iters"]
    # at most 12 refinement steps of 21 operations and 38 for set-up and the QoI, per unknown
    assert p["solve_flops"] <= per_it * p["unknown_iters"] + unk * (12 * 21 + 38)
