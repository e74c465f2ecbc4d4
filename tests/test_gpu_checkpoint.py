"""Checkpoint and resume of the Alg. 4.1 state, the per-round log, and the
forced-allocation-failure hook, on the GPU estimate."""
import ctypes
import json

import numpy as np
import pytest

from gpu_common import device, lib, to_dev, torch
from inputs import smooth_lognormal_field

pytestmark = pytest.mark.gpu

WL = dict(n0=8, m=2, L_max=3, kind=0, K=16, sigma2=1.0, corr_len=0.3, seed=21)


@pytest.fixture(scope="module")
def M():
    device()
    return lib()


def _opts(M, **kw):
    o = M.mlmc_default_options()
    o.tol, o.N_init, o.L_start = 2e-3, 32, 1
    for k, v in kw.items():
        setattr(o, k, v)
    return o


@pytest.mark.parametrize("prec_rule", [0, 1])
def test_resumed_estimate_equals_uninterrupted(M, tmp_path, prec_rule):
    h = M.mlmc_create(M.make_problem(**WL), 0)
    try:
        full = M.mlmc_estimate(h, _opts(M, prec_rule=prec_rule))
        assert full.rounds >= 2
        part = M.mlmc_estimate(h, _opts(M, prec_rule=prec_rule, max_rounds=full.rounds - 1))
        M.save_result(part, str(tmp_path / "ck.bin"))
        o = _opts(M, prec_rule=prec_rule)
        M.set_resume(o, M.load_result(str(tmp_path / "ck.bin")))
        res = M.mlmc_estimate(h, o)
    finally:
        M.mlmc_destroy(h)
    a, b = M.result_dict(res), M.result_dict(full)
    # the same samples, solved by the same launches: identical bits and counters
    for key in ("L", "N", "Yhat", "s2", "estimate", "rmse", "rounds", "prec", "inner_iters", "dofs", "delta",
                "fp64_retries", "contrast"):
        assert a[key] == b[key], key


def test_round_log_of_the_gpu_estimate(M, tmp_path):
    path = tmp_path / "rounds.jsonl"
    h = M.mlmc_create(M.make_problem(**WL), 0)
    try:
        o = _opts(M)
        M.set_log_path(o, str(path))
        r = M.result_dict(M.mlmc_estimate(h, o))
    finally:
        M.mlmc_destroy(h)
    lines = [json.loads(x) for x in path.read_text().splitlines()]
    assert len(lines) == r["rounds"]
    assert lines[-1]["N"] == r["N"] and lines[-1]["Yhat"] == r["Yhat"] and lines[-1]["delta"] == r["delta"]


def test_forced_allocation_failure(M):
    clean = None
    h = M.mlmc_create(M.make_problem(**WL), 0)
    try:
        clean = M.result_dict(M.mlmc_estimate(h, _opts(M)))
    finally:
        M.mlmc_destroy(h)
    try:
        # creation: the first basis buffer cannot be had
        M.mlmc_debug_fail_allocation(0)
        with pytest.raises(M.MlmcError) as ei:
            M.mlmc_create(M.make_problem(**WL), 0)
        assert "out of memory" in str(ei.value)
        # an estimate whose workspace cannot grow fails cleanly; the context works afterwards
        h = M.mlmc_create(M.make_problem(**WL), 0)
        try:
            M.mlmc_debug_fail_allocation(2)
            with pytest.raises(M.MlmcError) as ei:
                M.mlmc_estimate(h, _opts(M))
            assert "out of memory" in str(ei.value)
            again = M.result_dict(M.mlmc_estimate(h, _opts(M)))
            assert again["N"] == clean["N"] and again["Yhat"] == clean["Yhat"]
        finally:
            M.mlmc_destroy(h)
        # the allocation-free entry point allocates nothing: an armed hook does not touch it
        M.mlmc_debug_fail_allocation(0)
        n, S = 32, 3
        af = smooth_lognormal_field(n, S, seed=3, log_sd=0.5)
        Q = torch.empty(S, dtype=torch.float64, device=device())
        fl = torch.empty(S, dtype=torch.int32, device=device())
        M.mlmc_level_solve_noalloc(0, n, S, to_dev(af, torch.float64), M.MLMC_FP64, n, M.MLMC_FP32, 1e-8, 10000, 0,
                                   (0.0, 1.0, 0.0, 1.0), 1.0, Q, flags=fl)
        torch.cuda.synchronize()
        assert np.all(fl.cpu().numpy() == M.MLMC_F_CONVERGED)
    finally:
        M.mlmc_debug_fail_allocation(-1)


def test_set_seed_reuses_the_context(M):
    # a new Philox key on a live context gives exactly the estimate of a context created with that key
    h = M.mlmc_create(M.make_problem(**WL), 0)
    try:
        r1 = M.result_dict(M.mlmc_estimate(h, _opts(M)))
        M.mlmc_set_seed(h, WL["seed"] + 1)
        r2 = M.result_dict(M.mlmc_estimate(h, _opts(M)))
        M.mlmc_set_seed(h, WL["seed"])
        r3 = M.result_dict(M.mlmc_estimate(h, _opts(M)))
    finally:
        M.mlmc_destroy(h)
    h = M.mlmc_create(M.make_problem(**dict(WL, seed=WL["seed"] + 1)), 0)
    try:
        r2f = M.result_dict(M.mlmc_estimate(h, _opts(M)))
    finally:
        M.mlmc_destroy(h)
    assert r3["Yhat"] == r1["Yhat"] and r3["N"] == r1["N"]
    assert r2f["Yhat"] == r2["Yhat"] and r2f["N"] == r2["N"]
    assert r2["Yhat"] != r1["Yhat"]


_RESULT_KEYS = ("L", "rounds", "N", "Yhat", "s2", "estimate", "var_est", "rmse", "inner_iters", "dofs",
                "fp64_retries", "prec", "flags_or")


def _same(r, q):
    return all(np.array_equal(np.asarray(r[k]), np.asarray(q[k])) for k in _RESULT_KEYS)


@pytest.mark.parametrize("L_start,form", [(3, "MIXED"), (1, "MIXED"), (3, "FP64_ADAPTIVE")])
def test_samples_solved_ahead_leave_the_estimate_unchanged(M, L_start, form):
    # the second estimate on a context solves samples ahead of the rounds that ask for them (up to the
    # first estimate's counts); it equals the first bit for bit, and so does one with it switched off
    kw = dict(L_start=L_start, form=getattr(M, "MLMC_FORM_" + form))
    h = M.mlmc_create(M.make_problem(**WL), 0)
    try:
        M.mlmc_profile_enable(h, True)
        r1 = M.result_dict(M.mlmc_estimate(h, _opts(M, **kw)))
        p1 = M.mlmc_profile_get(h)
        M.mlmc_profile_reset(h)
        r2 = M.result_dict(M.mlmc_estimate(h, _opts(M, **kw)))
        p2 = M.mlmc_profile_get(h)
        M.mlmc_set_sample_ahead(h, False)
        r3 = M.result_dict(M.mlmc_estimate(h, _opts(M, **kw)))
    finally:
        M.mlmc_destroy(h)
    assert r1["rounds"] >= 2
    assert _same(r2, r1) and _same(r3, r1)
    if L_start == 3:
        # the finest level is fixed: the later rounds' samples were all solved in the first round
        assert p2["solve_launches"] < p1["solve_launches"]


def test_samples_solved_ahead_for_new_seeds(M):
    # the counts to solve ahead come from another seed's estimate, so rounds ask for more or fewer samples than
    # were solved ahead and later rounds take the ones left over; every result equals a fresh context's
    kw = dict(L_start=3)
    h = M.mlmc_create(M.make_problem(**WL), 0)
    got = []
    try:
        M.mlmc_estimate(h, _opts(M, **kw))
        for seed in (WL["seed"] + 1, WL["seed"] + 2, WL["seed"] + 3):
            M.mlmc_set_seed(h, seed)
            got.append(M.result_dict(M.mlmc_estimate(h, _opts(M, **kw))))
    finally:
        M.mlmc_destroy(h)
    for k, r in enumerate(got):
        h = M.mlmc_create(M.make_problem(**dict(WL, seed=WL["seed"] + 1 + k)), 0)
        try:
            M.mlmc_set_sample_ahead(h, False)
            ref = M.result_dict(M.mlmc_estimate(h, _opts(M, **kw)))
        finally:
            M.mlmc_destroy(h)
        assert _same(r, ref)


def test_destroy_returns_the_device_memory(M):
    # a context that used every workspace (estimate with samples solved ahead, direct solver, adjoint
    # contraction) gives all of its device memory back on destroy
    def cycle():
        h = M.mlmc_create(M.make_problem(**WL), 0)
        try:
            M.mlmc_estimate(h, _opts(M, L_start=3))
            M.mlmc_estimate(h, _opts(M, L_start=3))
            M.mlmc_estimate(h, _opts(M, L_start=3, solver=M.MLMC_CHOLESKY, form=M.MLMC_FORM_FP64_FIXED,
                                     fixed_delta=1e-10))
            xi = torch.zeros((4, WL["K"]), dtype=torch.float64, device=device())
            Q = torch.empty(4, dtype=torch.float64, device=device())
            G = torch.empty((4, WL["K"]), dtype=torch.float64, device=device())
            M.mlmc_adjoint_grad(h, 1, 4, xi, M.MLMC_FP32, 1e-8, 100000, Q, G)
            torch.cuda.synchronize()
        finally:
            M.mlmc_destroy(h)
        torch.cuda.synchronize()

    cycle()   # first use: the runtime's and the kernels' own one-time allocations
    torch.cuda.empty_cache()
    free0 = torch.cuda.mem_get_info()[0]
    for _ in range(3):
        cycle()
    torch.cuda.empty_cache()
    assert free0 - torch.cuda.mem_get_info()[0] <= 16 << 20
