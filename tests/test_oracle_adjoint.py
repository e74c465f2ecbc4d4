"""Pins for the oracle's QoI gradient (oracle/adjoint.py)."""
import numpy as np
import pytest

from oracle import adjoint, kl


@pytest.mark.parametrize("box", [None, (0.25, 0.75, 0.25, 0.75)])
def test_gradient_matches_central_differences(box):
    n, K = 16, 6
    phi = kl.basis(0, K, n, 1.0, 0.1)
    xi = np.random.default_rng(1).standard_normal(K)
    Q, g = adjoint.gradient(n, xi, phi, box)
    fd = np.array([adjoint.finite_difference(n, xi, phi, k, 1e-6, box) for k in range(K)])
    assert np.max(np.abs(g - fd)) <= 1e-6 * np.max(np.abs(g))


def test_full_domain_adjoint_equals_primal():
    # f = 1 and Q = int u give g = b, so the adjoint solution is the primal one
    n = 12
    a = kl.coefficient(np.random.default_rng(2).standard_normal((1, 5)), kl.basis(0, 5, n))[0]
    _, x, lam, _ = adjoint.nodal_sensitivity(n, a)
    assert np.allclose(lam, x, rtol=1e-13, atol=0)


def test_constant_field_gradient_closed_form():
    # a = exp(sigma xi) gives Q = Q(1) e^{-sigma xi}, dQ/dxi = -sigma Q
    n, sigma = 8, 0.6
    phi = kl.basis(2, 1, n, sigma2=sigma ** 2)
    for z in (-0.7, 1.9):
        Q, g = adjoint.gradient(n, np.array([z]), phi)
        assert np.isclose(g[0], -sigma * Q, rtol=1e-12)
