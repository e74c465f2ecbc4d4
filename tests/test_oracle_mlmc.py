"""Pins for the oracle's estimator, accuracy rule and adaptive algorithm (oracle/mlmc.py)."""
import math
from fractions import Fraction

import numpy as np
import pytest

from conftest import golden_rows
from oracle import fem, mlmc


def test_accuracy_rule_reproduces_table_1():
    rows = golden_rows("table1_delta.txt")
    for L in range(1, 5):
        h = [(1.0 / 8.0) * 2.0 ** -l for l in range(L + 1)]
        d = mlmc.delta_rule_fem(h, 0.05)
        dg = mlmc.delta_rule(h, 0.05, alpha1=2, alpha2=1, beta1=4, beta2=2)
        assert np.allclose(d, dg, rtol=1e-15)
        for r in rows:
            if int(r[0]) == L:
                l, printed = int(r[1]), float(r[2])
                e = math.floor(math.log10(printed))
                assert abs(d[l] - printed) <= 10.0 ** (e - 1) * 1.0001, (L, l, d[l], printed)


def test_accuracy_rule_general_rates():
    h = np.array([0.5, 0.25, 0.125])
    d = mlmc.delta_rule(h, 0.1, alpha1=1, alpha2=2, beta1=2, beta2=1)
    assert np.allclose(d[:2], 0.1 * h[:2] ** 2)
    assert np.isclose(d[2], min(0.1 * h[2] ** 2, math.sqrt(0.1 * h[2])))


def test_cost_prediction_cor_4_4():
    q, m, beta, gamma, ratio, gain = [float(v) for v in golden_rows("cost_model.txt")[0]]
    r = mlmc.cost_ratio_bound(q, m, beta, gamma)
    assert abs(r - ratio) < 1e-15
    assert round(1.0 / r, 1) == gain
    # finite-L bound: L = 1 leaves only the coarse gain, and it tends to the limit
    assert math.isclose(mlmc.cost_ratio_bound(q, m, beta, gamma, L=1), q)
    assert abs(mlmc.cost_ratio_bound(q, m, beta, gamma, L=60) - r) < 1e-12
    # direct sum: levels with C_{l+1}N_{l+1} = c C_l N_l, level 0 made q times cheaper
    c = m ** ((gamma - beta) / 2.0)
    L = 5
    ml = sum(c ** l for l in range(L))
    mp = q + sum(c ** l for l in range(1, L))
    assert math.isclose(mp / ml, mlmc.cost_ratio_bound(q, m, beta, gamma, L=L), rel_tol=1e-14)


def test_mean_var_exact_rationals():
    g = np.random.default_rng(3)
    for N in (1, 2, 5, 33):
        Y = g.standard_normal(N) * 1e-3 + 0.7
        F = [Fraction(float(y)) for y in Y]
        mean = sum(F) / N
        var = sum((f - mean) ** 2 for f in F) / N
        m, v = mlmc.mean_var(Y)
        assert abs(m - float(mean)) <= 1e-15 * abs(float(mean))
        assert abs(v - float(var)) <= 1e-12 * float(var) + 1e-300


def test_optimal_samples_formula():
    V = np.array([1e-3 * 2.0 ** (-4 * l) for l in range(4)])
    C = np.array([2.0 ** (2 * l) for l in range(4)])
    tol = 1e-3
    N = mlmc.optimal_samples(V, C, tol)
    raw = np.sqrt(V / C) * (2 / tol ** 2) * np.sum(np.sqrt(V * C))
    assert np.all(N == np.ceil(raw))
    assert np.allclose(raw[1:] / raw[:-1], 2.0 ** -3)      # m^(-(beta+gamma)/2)
    assert np.sum(V / N) <= tol ** 2 / 2 * (1 + 1e-12)


def test_optimal_samples_hand_computed():
    # V = (4e-4, 1e-6), C = (1, 4) (m = 2, gamma = 2), TOL = 1.1e-3: sum sqrt(V C) = 0.02 + 0.002 = 0.022 and
    # 2 / TOL^2 = 1652892.56, so N_0 = 0.02 * 1652892.56 * 0.022 = 727.27 -> 728 and
    # N_1 = sqrt(1e-6 / 4) * 1652892.56 * 0.022 = 18.18 -> 19
    N = mlmc.optimal_samples(np.array([4e-4, 1e-6]), np.array([1.0, 4.0]), 1.1e-3)
    assert list(N) == [728, 19]


class _MockSampler:
    """Y_l = mu_l + sd_l z with prescribed bias and variance decay (no PDE)."""

    def __init__(self, mu, sd, seed=0):
        self.mu, self.sd = mu, sd
        self.g = np.random.default_rng(seed)
        self.calls = []

    def __call__(self, l, first, count, deltas):
        self.calls.append((l, first, count))
        return self.mu[l] + self.sd[l] * self.g.standard_normal(count)


class _P:
    def __init__(self, L_max, n0=8, m=2):
        self.L_max, self.n0, self.m = L_max, n0, m

    def h(self, l):
        return 1.0 / (self.n0 * self.m ** l)


def test_algorithm_4_1_adds_levels_until_bias_small():
    tol = 1e-3
    thr = mlmc.bias_threshold(2, 2.0, tol)
    mu = [0.05, 8 * thr, 2 * thr, thr / 4, thr / 16, thr / 64]
    sd = [2e-2, 1e-3, 3e-4, 1e-4, 3e-5, 1e-5]
    s = _MockSampler(mu, sd)
    out = mlmc.estimate(_P(5), tol, N_init=50, sampler=s)
    assert out["L"] == 3 and not out["bias_failed"]
    # variance test holds with the final sample counts
    assert np.sum(out["s2"] / out["N"]) <= tol ** 2 / 2 * (1 + 1e-12)
    # each level was started with N_init samples, and samples are never recomputed
    firsts = {}
    for l, first, count in s.calls:
        assert first == firsts.get(l, 0)
        firsts[l] = first + count
    assert [c for c in s.calls if c[1] == 0] == [(l, 0, 50) for l in range(4)]


def test_algorithm_4_1_stops_at_L_max_and_fixed_start():
    tol = 1e-3
    big = 10 * mlmc.bias_threshold(2, 2.0, tol)
    s = _MockSampler([0.05, big, big], [1e-2, 1e-3, 1e-3])
    out = mlmc.estimate(_P(2), tol, N_init=20, sampler=s)
    assert out["L"] == 2 and out["bias_failed"]
    s2 = _MockSampler([0.05, 0.0, 0.0, 0.0], [1e-2, 1e-4, 1e-5, 1e-6])
    out2 = mlmc.estimate(_P(3), tol, N_init=30, L_start=3, sampler=s2)
    assert out2["L"] == 3 and [c for c in s2.calls if c[1] == 0] == [(l, 0, 30) for l in range(4)]


def test_lognormal_constant_field_level_statistics():
    # a = exp(sigma z) in space gives Q_l = Q_{h_l}(1) e^{-sigma z}, so
    # E[Y_l] = dQ e^{sigma^2/2} and Var[Y_l] = dQ^2 (e^{2 sigma^2} - e^{sigma^2}).
    sigma = 0.5
    P = mlmc.Problem(n0=4, m=2, L_max=2, field_kind=2, K=1, sigma2=sigma ** 2, seed=7)
    Q1 = [fem.solve_sample(P.n(l), np.ones((P.n(l) + 1) ** 2))[1] for l in range(3)]
    N = 4000
    for l in range(3):
        Qf, Qc = P.level_samples(l, 0, N)
        dQ = Q1[l] - (Q1[l - 1] if l > 0 else 0.0)
        Y = Qf - Qc
        m, v = mlmc.mean_var(Y)
        Ev = dQ * math.exp(sigma ** 2 / 2)
        Vv = dQ ** 2 * (math.exp(2 * sigma ** 2) - math.exp(sigma ** 2))
        assert abs(m - Ev) < 5 * math.sqrt(Vv / N)
        assert abs(v / Vv - 1.0) < 6 * math.sqrt(2.0 / N) * 2   # lognormal kurtosis margin
        # the sample-wise relation is exact
        z = P.xi(l, 0, N)[:, 0]
        assert np.allclose(Y, dQ * np.exp(-sigma * z), rtol=1e-12)


def test_fixed_sample_mlmc_telescopes():
    P = mlmc.Problem(n0=4, m=2, L_max=2, field_kind=0, K=4, sigma2=1.0, corr_len=0.3, seed=0)
    out = mlmc.estimate_fixed(P, [40, 20, 10])
    # level l's fine member and level l+1's coarse member solve the same grid but with
    # independent draws; their means agree only statistically -- the estimator is a sum
    assert np.isclose(out["estimate"], np.sum(out["Yhat"]))
    Qf0, _ = P.level_samples(0, 0, 40)
    assert np.isclose(out["Yhat"][0], Qf0.mean())


def test_bias_threshold_literal_values():
    # Alg. 4.1 bias test |Y_hat_L| <= (r m^alpha - 1) TOL / sqrt(2): with m = 2, alpha = 2, r = 1 the
    # constant is 3 / sqrt(2) = 2.1213203435596424; with r = 1.5 it is 5 / sqrt(2) = 3.5355339059327373
    assert mlmc.bias_threshold(2, 2.0, 1e-3) == pytest.approx(2.1213203435596424e-3, rel=1e-15)
    assert mlmc.bias_threshold(2, 2.0, 1e-3, r=1.5) == pytest.approx(3.5355339059327373e-3, rel=1e-15)
    # m = 4, alpha = 1: (4 - 1) TOL / sqrt(2) again
    assert mlmc.bias_threshold(4, 1.0, 2e-4) == pytest.approx(4.242640687119285e-4, rel=1e-15)


def test_rmse_hand_computed():
    # bias = 9e-4 / (2^2 - 1) = 3e-4; variance 1e-5/100 + 5e-7/10 + 2e-8/2 = 1.6e-7;
    # sqrt(9e-8 + 1.6e-7) = sqrt(2.5e-7) = 5e-4 exactly
    r = mlmc.rmse([0.03, 0.003, 9e-4], [1e-5, 5e-7, 2e-8], [100, 10, 2], 2, 2.0)
    assert r == pytest.approx(5e-4, rel=1e-13)
    # the sign of the finest mean does not matter: one level with mean -0.02 has bias 0.02 / 3 and
    # variance 0.04 / 100 = 4e-4, so the RMSE is sqrt(4/9 1e-4 + 4e-4) = 0.0210818510677891...
    r1 = mlmc.rmse([-0.02], [0.04], [100], 2, 2.0)
    assert r1 == pytest.approx(0.021081851067789197, rel=1e-14)
