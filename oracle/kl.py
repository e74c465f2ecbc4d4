"""Oracle: truncated Karhunen-Loeve bases for log a(x, omega).

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__.py``).

log a(x) = sum_k xi_k Phi_k(x) with xi_k ~ N(0, 1) (``oracle.rng``), so
sigma and the eigenvalues are folded into Phi_k.  Three kinds:

* kind 0 -- separable exponential covariance on [0,1]^2,
  C(x, y) = sigma^2 exp(-|x1-y1|/lam) exp(-|x2-y2|/lam).  The paper does not
  define this field (it uses Eq. (5.2)); it is the covariance named by the
  workloads.  1D eigenpairs of exp(-|s-t|/lam) on [0,1]: theta = 2 lam /
  (1 + lam^2 w^2), b(t) = sin(w t) + lam w cos(w t) with w the positive roots
  of (lam^2 w^2 - 1) sin w = 2 lam w cos w, normalised in L^2(0,1).  2D modes are
  products, sorted by sigma^2 theta_i theta_j descending, ties broken by
  (i + j) ascending then i ascending; the first K are kept.
* kind 1 -- the paper's field, Sec. 5.1 Eq. (5.2):
  Phi_j(x) = sigma j^-q sin(2 pi j x1) cos(2 pi j x2), j = 1..K.
* kind 2 -- a single spatially constant mode Phi_0 = sigma (a = exp(sigma xi)),
  for closed-form checks.

Here the roots are bracketed by a sign scan and refined by Brent's method and
the eigenfunctions are normalised by composite Gauss-Legendre quadrature
(64 panels of 24 points: exact to rounding for every oscillation frequency
used here, unlike a single high-order rule whose weights lose ~1e-13).
"""
import numpy as np
from scipy.optimize import brentq


def _char_eq(w, lam):
    return (lam * lam * w * w - 1.0) * np.sin(w) - 2.0 * lam * w * np.cos(w)


def expcov_roots(lam, count):
    """The first ``count`` positive roots w of (lam^2 w^2 - 1) sin w = 2 lam w cos w."""
    roots = []
    step = np.pi / 64.0
    lo = 1e-9
    flo = _char_eq(lo, lam)
    while len(roots) < count:
        hi = lo + step
        fhi = _char_eq(hi, lam)
        if flo == 0.0:
            roots.append(lo)
        elif np.sign(flo) != np.sign(fhi):
            roots.append(brentq(_char_eq, lo, hi, args=(lam,), xtol=1e-15, rtol=8.9e-16, maxiter=200))
        lo, flo = hi, fhi
    return np.array(roots[:count])


def composite_gauss(panels=64, points=24):
    """Nodes and weights of a composite Gauss-Legendre rule on [0, 1]."""
    t, wt = np.polynomial.legendre.leggauss(points)
    nodes, weights = [], []
    for p in range(panels):
        a, b = p / panels, (p + 1) / panels
        nodes.append(a + (b - a) * 0.5 * (t + 1.0))
        weights.append((b - a) * 0.5 * wt)
    return np.concatenate(nodes), np.concatenate(weights)


def expcov_1d(lam, count, panels=64):
    """(theta[count], w[count], norm[count]) with b_i(t) = (sin(w t) + lam w cos(w t)) / norm."""
    w = expcov_roots(lam, count)
    theta = 2.0 * lam / (1.0 + lam * lam * w * w)
    t, wt = composite_gauss(panels)
    vals = np.sin(np.outer(w, t)) + (lam * w)[:, None] * np.cos(np.outer(w, t))
    norm = np.sqrt((vals * vals) @ wt)
    return theta, w, norm


def expcov_1d_eval(lam, w, norm, t):
    """b_i(t) for all modes i (rows) at points t (columns)."""
    t = np.asarray(t, dtype=np.float64)
    return (np.sin(np.outer(w, t)) + (lam * w)[:, None] * np.cos(np.outer(w, t))) / norm[:, None]


TIE_RTOL = 1e-12


def expcov_modes(sigma2, lam, K):
    """The K leading 2D modes: list of (i, j) and their eigenvalues sigma^2 theta_i theta_j.

    Order: theta_i theta_j descending; values within TIE_RTOL (relative) of the
    first value of a run count as tied -- (i, j) and (j, i) are exact ties of
    the true eigenvalues -- and a run of ties is ordered by (i + j, i)."""
    m1 = max(K, 8)
    theta, w, norm = expcov_1d(lam, m1)
    cand = sorted(((theta[i] * theta[j], i, j) for i in range(m1) for j in range(m1)), key=lambda c: -c[0])
    ordered = []
    start = 0
    while start < len(cand):
        end = start + 1
        while end < len(cand) and cand[start][0] - cand[end][0] <= TIE_RTOL * cand[start][0]:
            end += 1
        ordered.extend(sorted(cand[start:end], key=lambda c: (c[1] + c[2], c[1])))
        start = end
    modes = [(c[1], c[2]) for c in ordered[:K]]
    lam2d = np.array([sigma2 * c[0] for c in ordered[:K]])
    return modes, lam2d, (theta, w, norm)


def basis(kind, K, n, sigma2=1.0, corr_len=0.3, q=2.0):
    """Phi[K][(n+1)^2] at the grid nodes (x_i, y_j) = (i/n, j/n), node index j*(n+1) + i."""
    x = np.arange(n + 1, dtype=np.float64) / n
    if kind == 0:
        modes, lam2d, (theta, w, norm) = expcov_modes(sigma2, corr_len, K)
        b = expcov_1d_eval(corr_len, w, norm, x)            # b[i][node coordinate]
        phi = np.empty((K, (n + 1) * (n + 1)))
        for k, (i, j) in enumerate(modes):
            phi[k] = np.sqrt(lam2d[k]) * np.outer(b[j], b[i]).ravel()   # rows: y index
        return phi
    if kind == 1:
        sigma = np.sqrt(sigma2)
        phi = np.empty((K, (n + 1) * (n + 1)))
        for jj in range(1, K + 1):
            sx = np.sin(2.0 * np.pi * jj * x)
            cy = np.cos(2.0 * np.pi * jj * x)
            phi[jj - 1] = sigma * jj ** (-q) * np.outer(cy, sx).ravel()
        return phi
    if kind == 2:
        if K != 1:
            raise ValueError("the constant field has exactly one mode")
        return np.full((1, (n + 1) * (n + 1)), np.sqrt(sigma2))
    raise ValueError("unknown field kind %r" % kind)


def log_coefficient(xi, phi):
    """log a[s][v] = sum_k xi[s][k] Phi[k][v] (plain matrix product)."""
    return np.asarray(xi, dtype=np.float64) @ phi


def coefficient(xi, phi):
    return np.exp(log_coefficient(xi, phi))
