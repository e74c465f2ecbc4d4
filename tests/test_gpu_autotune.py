"""The launch-setting autotuner (mlmc_set_autotune): it times candidate settings
for each new launch shape, caches the fastest in the context, never picks a
setting slower than the library's own rules, and changes results only within
the solves' tolerance, whatever it picks."""
import ctypes

import numpy as np
import pytest

from gpu_common import device, lib, to_dev, torch
from inputs import smooth_lognormal_field
from oracle import fem as o_fem

pytestmark = pytest.mark.gpu

WL = dict(n0=16, m=2, L_max=4, kind=0, K=64, sigma2=1.0, corr_len=0.3, seed=4)


@pytest.fixture(scope="module")
def M():
    device()
    return lib()


def _estimate(M, tune, N):
    arr = (ctypes.c_int64 * len(N))(*N)
    h = M.mlmc_create(M.make_problem(**WL), 0)
    try:
        M.mlmc_set_autotune(h, tune)
        o = M.mlmc_default_options()
        o.L_start = len(N) - 1
        o.fixed_N = ctypes.cast(arr, ctypes.POINTER(ctypes.c_int64))
        r1 = M.result_dict(M.mlmc_estimate(h, o))
        n1 = M.mlmc_autotune_count(h)
        r2 = M.result_dict(M.mlmc_estimate(h, o))
        entries = [M.mlmc_autotune_entry(h, i) for i in range(M.mlmc_autotune_count(h))]
        n2 = len(entries)
    finally:
        M.mlmc_destroy(h)
    return r1, r2, n1, n2, entries


def test_autotuned_estimate_agrees_with_the_default_settings(M):
    N = [64, 32, 32, 32, 32]
    base, _, n0, _, _ = _estimate(M, False, N)
    r1, r2, n1, n2, entries = _estimate(M, True, N)
    assert n0 == 0 and n1 >= 2 and n2 == n1          # one entry per launch shape, reused afterwards
    for e in entries:
        assert e["trials"] >= 2 and 0 < e["best_ms"] <= e["default_ms"]
        assert e["shape"].startswith("prec ")
    deltas = np.array(base["delta"])
    for r in (r1, r2):
        assert r["N"] == N and r["flags_or"] & ~M.MLMC_F_CONVERGED == 0
        for l in range(5):
            # both runs meet delta_l on every solve: level means agree within twice the bound
            # 1.5 (delta_l + delta_{l-1}) max|Q| of each against the exact solves
            dc = deltas[l - 1] if l > 0 else 0.0
            assert abs(r["Yhat"][l] - base["Yhat"][l]) <= 2 * 1.5 * (deltas[l] + dc) * 0.1 + 1e-9, l


def test_autotuned_jacobi_level_solve_matches_oracle(M):
    # Jacobi-preconditioned CG on n = 128: the tuner also tries the row pipeline's depth
    n, S = 128, 6
    af = smooth_lognormal_field(n, S, seed=91, log_sd=1.0)
    h = M.mlmc_create(M.make_problem(n0=n, m=2, L_max=0, kind=0, K=4, sigma2=1.0, corr_len=0.3), 0)
    try:
        M.mlmc_set_precond(h, M.MLMC_PC_JACOBI)
        M.mlmc_set_autotune(h, True)
        a = to_dev(af, torch.float32)
        for _ in range(2):
            Q = torch.empty(S, dtype=torch.float64, device=device())
            fl = torch.empty(S, dtype=torch.int32, device=device())
            M.mlmc_level_solve(h, n, S, a, M.MLMC_FP32, n, M.MLMC_FP32, M.MLMC_CG, 1e-9, 200000, None, Q, None,
                               None, fl)
            M.mlmc_sync(h)
            assert np.all(fl.cpu().numpy() == M.MLMC_F_CONVERGED)
            for s in range(S):
                Qo = o_fem.solve_sample(n, af[s])[1]
                assert abs(Q[s].item() - Qo) <= 1e-7 * abs(Qo)
        assert M.mlmc_autotune_count(h) == 1
        e = M.mlmc_autotune_entry(h, 0)
        assert e["precond"] == M.MLMC_PC_JACOBI and e["trials"] >= 8
    finally:
        M.mlmc_destroy(h)
