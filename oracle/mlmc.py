"""Oracle: the MLMC / MPML estimator and the adaptive algorithm.

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__.py``).

* Estimator, Sec. 4.1 Eq. (4.1): Q_hat = sum_l Y_hat_l with
  Y_l = Q_l - Q_{l-1} evaluated on the same omega (Q_{-1} = 0).
* Sample variance, Eq. (4.2): s_l^2 = (1/N_l) sum_k (Y_l^(k) - Y_hat_l)^2.
* Accuracy rule, Eq. (4.7) (general rates) and Eq. (4.12) (P1 FEM:
  delta_l = sqrt(k_p) h_l^2 for l < L, delta_L = k_p h_L^2).
* Adaptive MPML, Algorithm 4.1, with these readings of points the paper
  leaves open: the loop stops once the bias test and the variance test both
  hold; "compute N_l new samples" computes max(0, N_l - N_l^done) more; the
  bias test is |Y_hat_L| <= (r m^alpha - 1) TOL / sqrt 2 with r = 1;
  V_l = s_l^2; the cost is the model C_l = m^(gamma l); N_l = ceil(formula).
  ``L_start`` lets the loop start at a fixed finest level (standard MLMC with
  a given number of levels).
* Cost analysis, Sec. 4.2: the finite-L ratio bound and Cor. 4.4.

The level sampler solves every system exactly (banded Cholesky in FP64), so
this is the FP64 reference against which inexact solves are measured.
"""
import math

import numpy as np

from . import fem, kl, rng


# ---------------------------------------------------------------------------
# Accuracy rule
def delta_rule(h, kp, alpha1=2.0, alpha2=1.0, beta1=4.0, beta2=2.0):
    """Eq. (4.7): delta_l = (k_p h_l^beta1)^(1/beta2), l < L, and
    delta_L = min((k_p h_L^beta1)^(1/beta2), (k_p h_L^alpha1)^(1/alpha2))."""
    h = np.asarray(h, dtype=np.float64)
    d = (kp * h ** beta1) ** (1.0 / beta2)
    d[-1] = min(d[-1], (kp * h[-1] ** alpha1) ** (1.0 / alpha2))
    return d


def delta_rule_fem(h, kp):
    """Eq. (4.12): the same rule with alpha1=2, alpha2=1, beta1=4, beta2=2."""
    h = np.asarray(h, dtype=np.float64)
    d = math.sqrt(kp) * h ** 2
    d[-1] = kp * h[-1] ** 2
    return d


# ---------------------------------------------------------------------------
# Statistics
def mean_var(Y):
    """Two-pass (Y_hat, s^2) with the 1/N normalisation of Eq. (4.2)."""
    Y = np.asarray(Y, dtype=np.float64)
    if Y.size == 0:
        return 0.0, 0.0
    m = float(np.sum(Y) / Y.size)
    return m, float(np.sum((Y - m) ** 2) / Y.size)


def optimal_samples(V, C, tol):
    """Algorithm 4.1 update: N_l = sqrt(V_l / C_l) (2 / TOL^2) sum_k sqrt(V_k C_k), ceil."""
    V = np.asarray(V, dtype=np.float64)
    C = np.asarray(C, dtype=np.float64)
    s = float(np.sum(np.sqrt(V * C)))
    return np.ceil(np.sqrt(V / C) * (2.0 / tol ** 2) * s).astype(np.int64)


def bias_threshold(m, alpha, tol, r=1.0):
    """(r m^alpha - 1) TOL / sqrt(2), the bias test of Algorithm 4.1."""
    return (r * m ** alpha - 1.0) * tol / math.sqrt(2.0)


def rmse(Yhat, s2, N, m, alpha):
    """Root-mean-square error estimate of the MLMC estimator (Sec. 4.1): the
    squared bias, estimated by Richardson extrapolation from the finest level
    mean as |Y_hat_L| / (m^alpha - 1), plus the estimator variance
    sum_l s_l^2 / N_l of Eq. (4.2)."""
    Yhat = np.asarray(Yhat, dtype=np.float64)
    bias = abs(float(Yhat[-1])) / (m ** alpha - 1.0)
    var = float(np.sum(np.asarray(s2, dtype=np.float64) / np.asarray(N, dtype=np.float64)))
    return math.sqrt(bias ** 2 + var)


def cost_ratio_bound(q, m, beta, gamma, L=None):
    """Sec. 4.2: bound on C^MPML / C^ML.  L None gives the L -> infinity limit
    q + m^((gamma-beta)/2) (1 - q) of Cor. 4.4; otherwise the finite-L form
    q (1-c)/(1-c^L) + c (1-c^(L-1))/(1-c^L) with c = m^((gamma-beta)/2)."""
    c = m ** ((gamma - beta) / 2.0)
    if L is None:
        return q + c * (1.0 - q)
    return q * (1.0 - c) / (1.0 - c ** L) + c * (1.0 - c ** (L - 1)) / (1.0 - c ** L)


# ---------------------------------------------------------------------------
# Level sampler (exact FP64 solves)
class Problem:
    """-div(a grad u) = 1 on (0,1)^2, u = 0 on the boundary, log a from a KL basis.

    Grid of level l: n_l = n0 m^l cells per side, h_l = 1 / n_l."""

    def __init__(self, n0, m, L_max, field_kind=0, K=16, sigma2=1.0, corr_len=0.3, q=2.0,
                 seed=0, box=None):
        self.n0, self.m, self.L_max = n0, m, L_max
        self.field_kind, self.K = field_kind, K
        self.sigma2, self.corr_len, self.q = sigma2, corr_len, q
        self.seed, self.box = seed, box
        self._phi = {}

    def n(self, l):
        return self.n0 * self.m ** l

    def h(self, l):
        return 1.0 / self.n(l)

    def phi(self, n):
        if n not in self._phi:
            self._phi[n] = kl.basis(self.field_kind, self.K, n, self.sigma2, self.corr_len, self.q)
        return self._phi[n]

    def xi(self, level, first, count):
        return rng.draw_xi(self.seed, level, first, count, self.K)

    def fields(self, level, first, count):
        """Nodal a on the level's fine grid for samples [first, first + count)."""
        return kl.coefficient(self.xi(level, first, count), self.phi(self.n(level)))

    def level_samples(self, level, first, count):
        """(Q_fine, Q_coarse) for samples [first, first+count) of level l (Q_coarse = 0 at l = 0)."""
        nf = self.n(level)
        a = self.fields(level, first, count)
        Qf = np.empty(count)
        Qc = np.zeros(count)
        for s in range(count):
            _, Qf[s] = fem.solve_sample(nf, a[s], self.box)
            if level > 0:
                _, Qc[s] = fem.solve_sample(nf // self.m, fem.coarse_view(a[s], nf), self.box)
        return Qf, Qc


def estimate(problem, tol, N_init=100, kp=0.05, alpha=2.0, gamma=2.0, L_start=1, r=1.0,
             sampler=None, max_rounds=100):
    """Algorithm 4.1 (sequential).  Returns a dict with the estimate, N_l, Y_hat_l, s_l^2,
    delta_l and the number of rounds.  ``sampler(l, first, count, deltas)`` returns the Y
    values; by default the exact FP64 level sampler of ``problem``."""
    m = problem.m
    if sampler is None:
        def sampler(l, first, count, deltas):
            Qf, Qc = problem.level_samples(l, first, count)
            return Qf - Qc
    L = L_start
    N = [N_init] * (L + 1)
    Y = [np.empty(0) for _ in range(L + 1)]
    rounds = 0
    bias_failed = False
    while rounds < max_rounds:
        rounds += 1
        h = [problem.h(l) for l in range(L + 1)]
        deltas = delta_rule_fem(h, kp)
        for l in range(L + 1):
            extra = N[l] - len(Y[l])
            if extra > 0:
                Y[l] = np.concatenate([Y[l], sampler(l, len(Y[l]), extra, deltas)])
        stats = [mean_var(y) for y in Y]
        V = [s[1] for s in stats]
        C = [m ** (gamma * l) for l in range(L + 1)]
        Nopt = optimal_samples(V, C, tol)
        N = [max(int(Nopt[l]), len(Y[l])) for l in range(L + 1)]
        bias_failed = abs(stats[L][0]) > bias_threshold(m, alpha, tol, r)
        if bias_failed and L < problem.L_max:
            L += 1
            N.append(N_init)
            Y.append(np.empty(0))
            continue
        if all(len(Y[l]) >= Nopt[l] for l in range(L + 1)):
            break
    stats = [mean_var(y) for y in Y]
    Yhat = np.array([s[0] for s in stats])
    s2 = np.array([s[1] for s in stats])
    Nl = np.array([len(y) for y in Y])
    return {
        "estimate": float(np.sum(Yhat)),
        "L": L,
        "N": Nl,
        "Yhat": Yhat,
        "s2": s2,
        "delta": delta_rule_fem([problem.h(l) for l in range(L + 1)], kp),
        "rmse": rmse(Yhat, s2, Nl, m, alpha),
        "bias_failed": bool(bias_failed),
        "rounds": rounds,
        "Y": Y,
    }


def estimate_fixed(problem, N):
    """Standard MLMC with fixed samples per level (no adaptivity)."""
    Y = []
    for l, nl in enumerate(N):
        Qf, Qc = problem.level_samples(l, 0, nl)
        Y.append(Qf - Qc)
    stats = [mean_var(y) for y in Y]
    return {"estimate": float(sum(s[0] for s in stats)),
            "Yhat": np.array([s[0] for s in stats]),
            "s2": np.array([s[1] for s in stats]), "Y": Y}
