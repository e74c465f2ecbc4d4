"""C-ABI boundary checks that need no GPU: the library loads, exports every
symbol include/libmlmc.h declares, and its pure-host logic (accuracy rule,
Algorithm 4.1 loop, accumulator merge) agrees with the oracle."""
import ctypes
import math
import os
import re

import numpy as np
import pytest

from conftest import ROOT, golden_rows
from oracle import mlmc as o_mlmc


@pytest.fixture(scope="session")
def L():
    import __graft_entry__
    __graft_entry__.build()
    import paper_2503_05533_gb300 as M
    return M


def _declared_functions():
    text = open(os.path.join(ROOT, "include", "libmlmc.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    names = set(re.findall(r"\b(mlmc_[a-z0-9_]+)\s*\(", text))
    typedef_fn = set(re.findall(r"\(\s*\*\s*(mlmc_[a-z0-9_]+)\s*\)", text))
    return sorted(names - typedef_fn)


def test_library_exports_every_declared_symbol(L):
    names = _declared_functions()
    assert len(names) >= 17
    so = ctypes.CDLL(L.capi.LIB_PATH)
    missing = [n for n in names if not hasattr(so, n)]
    assert not missing, missing
    # and the binding wraps each of them under the same name
    assert all(hasattr(L.capi, n) for n in names)
    assert "sm_103a" in L.mlmc_version()


def test_struct_layouts_match_header(L):
    # offsets of the C structs as compiled by the host compiler
    import ctypes as C
    assert C.sizeof(L.capi.mlmc_acc) == 56
    assert C.sizeof(L.capi.mlmc_field) == 32
    assert L.capi.mlmc_problem.seed.offset == C.sizeof(L.capi.mlmc_problem) - 8


def test_accuracy_rule_matches_table_1_and_oracle(L):
    rows = golden_rows("table1_delta.txt")
    for Lf in range(1, 5):
        h = [(1.0 / 8.0) * 2.0 ** -l for l in range(Lf + 1)]
        d, prec = L.mlmc_adapt_precision(h, 0.05)
        assert np.allclose(d, o_mlmc.delta_rule_fem(h, 0.05), rtol=1e-14)
        for r in rows:
            if int(r[0]) == Lf:
                e = math.floor(math.log10(float(r[2])))
                assert abs(d[int(r[1])] - float(r[2])) <= 10.0 ** (e - 1) * 1.0001
    # precision choice: 16-bit storage while delta >= 1e-4, FP32 below, FP64 only for huge kappa
    d, prec = L.mlmc_adapt_precision([1 / 16, 1 / 32, 1 / 64, 1 / 128, 1 / 256], 0.05)
    assert prec[0] == L.MLMC_FP16S and prec[-1] == L.MLMC_FP32
    _, p64 = L.mlmc_adapt_precision([1 / 1024], 0.05, contrast=1e3)
    assert p64 == [L.MLMC_FP64]
    with pytest.raises(L.MlmcError):
        L.mlmc_adapt_precision([0.0], 0.05)


class _Mock:
    def __init__(self, mu, sd, seed):
        self.mu, self.sd, self.seed = mu, sd, seed
        self.calls = []

    def draws(self, l, first, count):
        # values depend only on (level, sample index): both loops see the same Y
        out = np.empty(count)
        for i in range(count):
            g = np.random.default_rng([self.seed, l, first + i])
            out[i] = self.mu[l] + self.sd[l] * g.standard_normal()
        return out

    def __call__(self, l, first, count, deltas):
        self.calls.append((l, first, count))
        return self.draws(l, first, count)


class _P:
    def __init__(self, L_max, n0, m=2):
        self.L_max, self.n0, self.m = L_max, n0, m

    def h(self, l):
        return 1.0 / (self.n0 * self.m ** l)


@pytest.mark.parametrize("L_start", [1, 3])
def test_algorithm_4_1_host_loop_matches_oracle(L, L_start):
    tol = 1e-3
    thr = o_mlmc.bias_threshold(2, 2.0, tol)
    mu = [0.05, 4 * thr, thr, thr / 8, thr / 30]
    sd = [2e-2, 2e-3, 4e-4, 1e-4, 3e-5]
    o = L.mlmc_default_options()
    o.tol, o.N_init, o.L_start = tol, 40, L_start
    mock_c = _Mock(mu, sd, 3)
    res = L.mlmc_estimate_host(2, 4, 8, o, mock_c)
    mock_o = _Mock(mu, sd, 3)
    ref = o_mlmc.estimate(_P(4, 8), tol, N_init=40, L_start=L_start, sampler=mock_o)
    r = L.result_dict(res)
    assert r["L"] == ref["L"] and r["N"] == list(ref["N"]) and r["rounds"] == ref["rounds"]
    assert mock_c.calls == mock_o.calls
    assert np.allclose(r["Yhat"], ref["Yhat"], rtol=1e-12, atol=1e-15)
    assert np.allclose(r["s2"], ref["s2"], rtol=1e-10, atol=0)
    assert abs(r["estimate"] - ref["estimate"]) < 1e-13
    assert abs(r["rmse"] - ref["rmse"]) <= 1e-12 * ref["rmse"]


def test_fixed_samples_mode(L):
    o = L.mlmc_default_options()
    o.L_start = 2
    N = (ctypes.c_int64 * 3)(30, 20, 10)
    o.fixed_N = ctypes.cast(N, ctypes.POINTER(ctypes.c_int64))
    mock = _Mock([1.0, 0.1, 0.01], [0.1, 0.01, 0.001], 9)
    r = L.result_dict(L.mlmc_estimate_host(2, 2, 4, o, mock))
    assert r["N"] == [30, 20, 10] and r["rounds"] == 1
    Y0 = mock.draws(0, 0, 30)
    assert abs(r["Yhat"][0] - Y0.mean()) < 1e-14


def test_acc_merge_matches_two_pass(L):
    g = np.random.default_rng(4)
    Y = g.standard_normal(1001) * 3e-3 + 0.2
    parts = np.split(Y, [1, 17, 500, 999])
    total = L.capi.mlmc_acc()
    for p in parts:
        a = L.capi.mlmc_acc()
        a.n, a.mean = len(p), float(p.mean())
        a.m2 = float(((p - p.mean()) ** 2).sum())
        a.sum, a.sumsq = float(p.sum()), float((p * p).sum())
        L.mlmc_acc_merge(total, a)
    m, v = o_mlmc.mean_var(Y)
    assert total.n == len(Y)
    assert abs(total.mean - m) < 1e-15 and abs(total.m2 / total.n - v) < 1e-12 * v


def test_host_loop_rejects_bad_options(L):
    o = L.mlmc_default_options()
    o.tol = -1.0
    with pytest.raises(L.MlmcError):
        L.mlmc_estimate_host(2, 2, 4, o, _Mock([0, 0, 0], [1, 1, 1], 0))


class _Alternating:
    """Y_l = mu_l + sd_l (-1)^k for sample k: mean mu_l and 1/N variance sd_l^2 for even counts."""

    def __init__(self, mu, sd):
        self.mu, self.sd = mu, sd

    def __call__(self, l, first, count, deltas):
        k = np.arange(first, first + count)
        return self.mu[l] + self.sd[l] * np.where(k % 2 == 0, 1.0, -1.0)


@pytest.mark.parametrize("yl, grows", [(2.1220e-3, True), (2.1205e-3, False)])
def test_host_loop_bias_test_constant(L, yl, grows):
    # m = 2, alpha = 2, r = 1, TOL = 1e-3: the bias test passes iff |Y_hat_L| <= 2.1213203435596424e-3
    o = L.mlmc_default_options()
    o.tol, o.N_init, o.L_start = 1e-3, 10, 1
    r = L.result_dict(L.mlmc_estimate_host(2, 2, 4, o, _Alternating([0.05, yl, 0.0], [1e-4, 1e-5, 1e-6])))
    assert r["L"] == (2 if grows else 1)


def test_host_loop_rmse_hand_computed(L):
    # fixed N = 100/10/2, means 0.03/0.003/9e-4, variances 1e-5/5e-7/2e-8: bias 9e-4/3 = 3e-4,
    # variance of the estimator 1.6e-7, RMSE sqrt(9e-8 + 1.6e-7) = 5e-4; estimate 0.0339
    o = L.mlmc_default_options()
    o.L_start = 2
    N = (ctypes.c_int64 * 3)(100, 10, 2)
    o.fixed_N = ctypes.cast(N, ctypes.POINTER(ctypes.c_int64))
    sampler = _Alternating([0.03, 0.003, 9e-4], [math.sqrt(1e-5), math.sqrt(5e-7), math.sqrt(2e-8)])
    r = L.result_dict(L.mlmc_estimate_host(2, 2, 4, o, sampler))
    assert r["rmse"] == pytest.approx(5e-4, rel=1e-12)
    assert r["estimate"] == pytest.approx(0.0339, rel=1e-13)
    assert r["var_est"] == pytest.approx(1.6e-7, rel=1e-12)


def test_host_loop_sample_targets_hand_computed(L):
    # level variances exactly 4e-4 and 1e-6 (alternating samples), TOL = 1.1e-3, m = 2, gamma = 2: the optimal
    # counts are 728 and 19 (727.27 and 18.18 rounded up); level 1 keeps its 100 initial samples
    o = L.mlmc_default_options()
    o.tol, o.N_init, o.L_start = 1.1e-3, 100, 1
    r = L.result_dict(L.mlmc_estimate_host(2, 1, 4, o, _Alternating([0.05, 0.0], [0.02, 0.001])))
    assert r["N"] == [728, 100] and r["rounds"] == 2 and r["L"] == 1
    assert r["var_est"] == pytest.approx(4e-4 / 728 + 1e-6 / 100, rel=1e-12)


@pytest.mark.parametrize("cut", [1, 2, 3])
def test_resume_from_checkpoint_equals_uninterrupted_run(L, tmp_path, cut):
    # Alg. 4.1 stopped after `cut` rounds, its result saved to disk, read back and resumed: the same samples
    # (indices continue from the checkpoint's counts), the same decisions, the same final state bit for bit
    tol = 1e-3
    thr = o_mlmc.bias_threshold(2, 2.0, tol)
    mu = [0.05, 4 * thr, thr, thr / 8, thr / 30]
    sd = [2e-2, 2e-3, 4e-4, 1e-4, 3e-5]
    o = L.mlmc_default_options()
    o.tol, o.N_init, o.L_start = tol, 40, 1
    full_mock = _Mock(mu, sd, 5)
    full = L.mlmc_estimate_host(2, 4, 8, o, full_mock)
    assert full.rounds > cut
    o.max_rounds = cut
    first_mock = _Mock(mu, sd, 5)
    part = L.mlmc_estimate_host(2, 4, 8, o, first_mock)
    assert part.rounds == cut
    L.save_result(part, str(tmp_path / "ckpt.bin"))
    ck = L.load_result(str(tmp_path / "ckpt.bin"))
    o.max_rounds = 100
    L.set_resume(o, ck)
    second_mock = _Mock(mu, sd, 5)
    res = L.mlmc_estimate_host(2, 4, 8, o, second_mock)
    assert first_mock.calls + second_mock.calls == full_mock.calls
    a, b = L.result_dict(res), L.result_dict(full)
    for key in ("L", "N", "Yhat", "s2", "estimate", "rmse", "rounds", "bias_failed"):
        assert a[key] == b[key], key


def test_resume_rejects_fixed_samples_and_bad_checkpoints(L):
    o = L.mlmc_default_options()
    o.L_start = 1
    prev = L.mlmc_result()
    prev.L, prev.rounds = 1, 1
    N = (ctypes.c_int64 * 2)(10, 10)
    o.fixed_N = ctypes.cast(N, ctypes.POINTER(ctypes.c_int64))
    L.set_resume(o, prev)
    with pytest.raises(L.MlmcError):
        L.mlmc_estimate_host(2, 2, 4, o, _Mock([0, 0, 0], [1, 1, 1], 0))
    o.fixed_N = None
    prev.L = 7
    with pytest.raises(L.MlmcError):
        L.mlmc_estimate_host(2, 2, 4, o, _Mock([0, 0, 0], [1, 1, 1], 0))


def test_round_log_lines(L, tmp_path):
    # one JSON line per round; the last line's state is the result's
    import json
    tol = 1e-3
    thr = o_mlmc.bias_threshold(2, 2.0, tol)
    o = L.mlmc_default_options()
    o.tol, o.N_init, o.L_start = tol, 40, 1
    path = tmp_path / "rounds.jsonl"
    L.set_log_path(o, str(path))
    res = L.result_dict(L.mlmc_estimate_host(2, 4, 8, o, _Mock([0.05, 4 * thr, thr, thr / 8, thr / 30],
                                                                [2e-2, 2e-3, 4e-4, 1e-4, 3e-5], 7)))
    lines = [json.loads(x) for x in path.read_text().splitlines()]
    assert len(lines) == res["rounds"] and [x["round"] for x in lines] == list(range(1, res["rounds"] + 1))
    last = lines[-1]
    assert last["L"] == res["L"] and last["N"] == res["N"] and last["Yhat"] == res["Yhat"]
    assert last["enough"] and last["bias_ok"] and last["rmse"] == res["rmse"]
    assert all(len(x["N"]) == x["L"] + 1 == len(x["Yhat"]) for x in lines)
    assert all(b["seconds"] >= a["seconds"] for a, b in zip(lines, lines[1:]))
    o.log_path = b"/nonexistent-dir/x.jsonl"
    with pytest.raises(L.MlmcError):
        L.mlmc_estimate_host(2, 4, 8, o, _Mock([0.0] * 5, [1.0] * 5, 7))
