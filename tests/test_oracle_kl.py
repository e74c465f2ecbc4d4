"""Pins for the oracle's KL bases (oracle/kl.py)."""
import numpy as np
import pytest

from oracle import kl


def _piecewise_nystrom_residual(lam, w, norm, theta, xs, npts=60):
    """max_x |int_0^1 exp(-|x-y|/lam) b(y) dy - theta b(x)|, integrating [0,x] and
    [x,1] separately with Gauss-Legendre so the kink at y = x costs no accuracy."""
    t, wt = np.polynomial.legendre.leggauss(npts)
    worst = 0.0
    for x in xs:
        total = np.zeros(len(w))
        for lo, hi in ((0.0, x), (x, 1.0)):
            if hi - lo <= 0.0:
                continue
            y = lo + (hi - lo) * 0.5 * (t + 1.0)
            wy = (hi - lo) * 0.5 * wt
            # many panels for high modes
            by = kl.expcov_1d_eval(lam, w, norm, y)
            total += by @ (wy * np.exp(-np.abs(x - y) / lam))
        bx = kl.expcov_1d_eval(lam, w, norm, [x])[:, 0]
        worst = max(worst, float(np.max(np.abs(total - theta * bx))))
    return worst


@pytest.mark.parametrize("lam", [0.1, 0.3, 1.0])
def test_expcov_eigenpairs_satisfy_integral_equation(lam):
    theta, w, norm = kl.expcov_1d(lam, 8)
    res = _piecewise_nystrom_residual(lam, w, norm, theta, np.linspace(0.0, 1.0, 13), npts=80)
    assert res < 1e-10


@pytest.mark.parametrize("lam", [0.1, 0.3])
def test_expcov_orthonormal_and_one_root_per_interval(lam):
    # normalisation against the closed form of int_0^1 (sin wt + lam w cos wt)^2 dt
    th, ww, nn = kl.expcov_1d(lam, 12)
    closed = np.sqrt(0.5 - np.sin(2 * ww) / (4 * ww) + lam * np.sin(ww) ** 2 +
                     lam ** 2 * ww ** 2 * (0.5 + np.sin(2 * ww) / (4 * ww)))
    assert np.max(np.abs(nn - closed) / closed) < 2e-15
    M = 40
    theta, w, norm = kl.expcov_1d(lam, M)
    t, wt = kl.composite_gauss(128, 24)
    B = kl.expcov_1d_eval(lam, w, norm, t)
    assert np.max(np.abs((B * wt) @ B.T - np.eye(M))) < 1e-12
    # a missed or duplicated root breaks this: exactly one root in (i pi, (i+1) pi)
    assert np.all((w > np.arange(M) * np.pi) & (w < (np.arange(M) + 1) * np.pi))
    assert np.all(np.diff(theta) < 0)


def test_expcov_trace():
    # sum of all 1D eigenvalues = int_0^1 C(t, t) dt = 1; the tail beyond M modes is
    # about sum 2 / (lam w^2) ~ 2 / (lam pi^2 M)
    lam, M = 0.3, 400
    theta, w, _ = kl.expcov_1d(lam, M, panels=4)
    s = theta.sum()
    assert s < 1.0
    assert 1.0 - s < 2.0 / (lam * np.pi ** 2 * (M - 1))
    assert 1.0 - s > 2.0 / (lam * np.pi ** 2 * (M + 2)) * 0.5


def test_expcov_2d_modes_sorted_and_bounded():
    sigma2, lam, K = 1.5, 0.1, 64
    modes, lam2d, (theta, _, _) = kl.expcov_modes(sigma2, lam, K)
    assert np.all(np.diff(lam2d) <= 0)
    assert modes[0] == (0, 0)
    assert modes[1] == (0, 1) and modes[2] == (1, 0)       # tie broken by i ascending
    assert np.allclose(lam2d, [sigma2 * theta[i] * theta[j] for i, j in modes], rtol=1e-15)
    # no omitted mode: every pair outside the kept set is not larger than the smallest kept
    kept = set(modes)
    for i in range(K):
        for j in range(K):
            if (i, j) not in kept:
                assert sigma2 * theta[i] * theta[j] <= lam2d[-1] * (1 + 1e-15)


def test_basis_pointwise_variance_and_orthogonality():
    sigma2, lam, K, n = 1.0, 0.3, 16, 32
    phi = kl.basis(0, K, n, sigma2, lam)
    # partial Mercer sums never exceed C(x, x) = sigma^2
    assert np.all((phi ** 2).sum(axis=0) <= sigma2 * (1 + 1e-12))
    # the constant-in-mean variance integral equals the sum of eigenvalues
    _, lam2d, _ = kl.expcov_modes(sigma2, lam, K)
    t, wt = kl.composite_gauss(32, 24)
    modes, _, (theta, w, norm) = kl.expcov_modes(sigma2, lam, K)
    B = kl.expcov_1d_eval(lam, w, norm, t)
    gram = np.empty((K, K))
    for a, (ia, ja) in enumerate(modes):
        for c, (ic, jc) in enumerate(modes):
            gram[a, c] = np.sqrt(lam2d[a] * lam2d[c]) * ((B[ia] * wt) @ B[ic]) * ((B[ja] * wt) @ B[jc])
    assert np.allclose(gram, np.diag(lam2d), atol=1e-12)
    # node layout: Phi_k(x_i, y_j) = sqrt(lam_k) b_{i_k}(x_i) b_{j_k}(y_j) at index j (n+1) + i
    i_k, j_k = modes[3]
    bx = kl.expcov_1d_eval(lam, w, norm, [5 / n])[:, 0]
    by = kl.expcov_1d_eval(lam, w, norm, [7 / n])[:, 0]
    assert np.isclose(phi[3, 7 * (n + 1) + 5], np.sqrt(lam2d[3]) * bx[i_k] * by[j_k], rtol=1e-14)


def test_paper_field_structure():
    # Eq. (5.2) with s = 4 on h = 1/8: sin(2 pi 4 x) vanishes at every node
    phi = kl.basis(1, 4, 8, sigma2=4.0, q=2.0)
    assert np.max(np.abs(phi[3])) < 1e-14
    assert np.max(np.abs(phi[0])) > 0.5
    # amplitudes sigma j^-q at a node where sin = cos = +-1 for j = 1 (x = 1/4, y = 0)
    n = 8
    assert np.isclose(phi[0, 0 * (n + 1) + 2], 2.0 * 1.0)
    phi16 = kl.basis(1, 4, 16, sigma2=4.0, q=2.0)
    assert np.isclose(np.max(np.abs(phi16[1])), 2.0 / 4.0)


def test_constant_field():
    phi = kl.basis(2, 1, 4, sigma2=0.49)
    assert np.all(phi == 0.7)
    a = kl.coefficient(np.array([[1.0], [-2.0]]), phi)
    assert np.allclose(a[0], np.exp(0.7)) and np.allclose(a[1], np.exp(-1.4))
