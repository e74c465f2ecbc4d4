"""Pins for the oracle's P1 finite-element layer (oracle/fem.py)."""
import numpy as np
import pytest
import scipy.sparse as sps

from inputs import rough_field, smooth_lognormal_field
from oracle import fem, kl


def _laplacian_5pt(n):
    T = sps.diags([-1.0, 2.0, -1.0], [-1, 0, 1], shape=(n - 1, n - 1))
    return sps.kronsum(T, T).tocsr()


@pytest.mark.parametrize("n", [2, 3, 8, 13])
def test_unit_coefficient_gives_5_point_laplacian(n):
    A = fem.assemble(n, np.ones((n + 1) ** 2))
    assert abs(A - _laplacian_5pt(n)).max() < 1e-14
    b = fem.load_vector(n)
    assert np.allclose(b, 1.0 / n ** 2, rtol=1e-14, atol=0)


def test_constant_coefficient_scales_operator():
    n = 9
    A1 = fem.assemble(n, np.ones((n + 1) ** 2))
    A3 = fem.assemble(n, np.full((n + 1) ** 2, 3.25))
    assert abs(A3 - 3.25 * A1).max() < 1e-14


def test_energy_identity_independent_gradients():
    # x^T A_full x = sum_T a_T |T| |grad x_T|^2, gradients taken from the legs of each
    # right triangle (not from the barycentric formula the assembly uses)
    n = 7
    h = 1.0 / n
    a = rough_field(n, 1, seed=3)[0]
    x = np.random.default_rng(4).standard_normal((n + 1) ** 2)
    A = fem.assemble_full(n, a)
    energy = 0.0
    X = x.reshape(n + 1, n + 1)
    Aa = a.reshape(n + 1, n + 1)
    for j in range(n):
        for i in range(n):
            sw, se, ne, nw = X[j, i], X[j, i + 1], X[j + 1, i + 1], X[j + 1, i]
            # T1 = (SW, SE, NE): right angle at SE
            gx, gy = (se - sw) / h, (ne - se) / h
            aT = (Aa[j, i] + Aa[j, i + 1] + Aa[j + 1, i + 1]) / 3.0
            energy += aT * 0.5 * h * h * (gx * gx + gy * gy)
            # T2 = (SW, NE, NW): right angle at NW
            gx, gy = (ne - nw) / h, (nw - sw) / h
            aT = (Aa[j, i] + Aa[j + 1, i + 1] + Aa[j + 1, i]) / 3.0
            energy += aT * 0.5 * h * h * (gx * gx + gy * gy)
    assert np.isclose(x @ (A @ x), energy, rtol=1e-13)


def test_operator_structure_for_any_coefficient():
    n = 10
    a = rough_field(n, 1, seed=8)[0]
    Af = fem.assemble_full(n, a)
    assert abs(Af - Af.T).max() < 1e-15
    assert np.max(np.abs(Af @ np.ones((n + 1) ** 2))) < 1e-13     # constants in the kernel
    A = fem.assemble(n, a)
    assert np.all(np.linalg.eigvalsh(A.toarray()) > 0)
    # 5-point sparsity: no coupling across the SW-NE hypotenuse or to far nodes
    Ad = A.tocoo()
    di = Ad.row % (n - 1) - Ad.col % (n - 1)
    dj = Ad.row // (n - 1) - Ad.col // (n - 1)
    far = np.abs(di) + np.abs(dj) > 1
    assert np.all(np.abs(Ad.data[far]) <= 1e-14 * np.abs(Ad.data).max())
    # with constant a the patch test holds: linear functions are discrete-harmonic
    Af1 = fem.assemble_full(n, np.full((n + 1) ** 2, 2.0))
    xs, ys = fem.node_coords(n)
    lin = 0.3 + 1.7 * xs - 0.9 * ys
    interior = (xs > 0) & (xs < 1) & (ys > 0) & (ys < 1)
    assert np.max(np.abs((Af1 @ lin)[interior])) < 1e-12


def test_dense_lu_matches_banded_cholesky():
    n = 8
    for s, a in enumerate(smooth_lognormal_field(n, 3, seed=11, log_sd=1.5)):
        A = fem.assemble(n, a)
        b = fem.load_vector(n)
        xd = fem.solve_dense(A, b)
        xc = fem.solve_cholesky(n, A, b)
        assert np.max(np.abs(xd - xc)) <= 1e-14 * np.max(np.abs(xd))


def _qh_closed_form(n):
    """Q_h = h^4 1^T A^{-1} 1 for a = 1 from the discrete sine eigenbasis of A."""
    h = 1.0 / n
    idx = np.arange(1, n)
    lam = 4.0 - 2.0 * np.cos(idx[:, None] * np.pi * h) - 2.0 * np.cos(idx[None, :] * np.pi * h)
    s = np.sin(np.outer(idx, idx) * np.pi * h).sum(axis=1) * np.sqrt(2.0 * h)   # 1^T v_p
    return h ** 4 * np.sum(np.outer(s, s) ** 2 / lam)


@pytest.mark.parametrize("n", [2, 8, 16, 32])
def test_unit_coefficient_qoi_closed_form(n):
    _, Q = fem.solve_sample(n, np.ones((n + 1) ** 2))
    assert abs(Q - _qh_closed_form(n)) < 1e-14


def test_unit_coefficient_qoi_converges_to_continuum():
    # int u for -Lap u = 1 on the unit square: (64/pi^6) sum_{p,q odd} 1/(p^2 q^2 (p^2+q^2))
    p = np.arange(1, 4001, 2, dtype=np.float64)
    cont = 64.0 / np.pi ** 6 * np.sum(1.0 / (np.outer(p * p, p * p) * (p[:, None] ** 2 + p[None, :] ** 2)))
    errs = [cont - fem.solve_sample(n, np.ones((n + 1) ** 2))[1] for n in (8, 16, 32, 64)]
    rates = np.log2(np.array(errs[:-1]) / np.array(errs[1:]))
    assert abs(cont - 0.0351442) < 1e-6
    assert np.all(np.array(errs) > 0) and np.all(np.abs(rates - 2.0) < 0.05)


def test_manufactured_solution_second_order():
    u = lambda x, y: np.sin(np.pi * x) * np.sin(np.pi * y)
    f = lambda x, y: 2.0 * np.pi ** 2 * u(x, y)
    errs = []
    for n in (8, 16, 32, 64):
        A = fem.assemble(n, np.ones((n + 1) ** 2))
        x = fem.solve_cholesky(n, A, fem.load_vector(n, f))
        xs, ys = np.meshgrid(np.arange(1, n) / n, np.arange(1, n) / n, indexing="xy")
        errs.append(np.max(np.abs(x - u(xs, ys).ravel())))
    rates = np.log2(np.array(errs[:-1]) / np.array(errs[1:]))
    assert np.all(rates > 1.8) and np.all(rates < 2.3)


def test_constant_lognormal_coefficient_scales_qoi():
    n = 16
    _, Q1 = fem.solve_sample(n, np.ones((n + 1) ** 2))
    phi = kl.basis(2, 1, n, sigma2=0.64)
    for z in (-1.3, 0.0, 2.1):
        a = kl.coefficient(np.array([[z]]), phi)[0]
        assert np.isclose(fem.solve_sample(n, a)[1], Q1 * np.exp(-0.8 * z), rtol=1e-13)


def test_qoi_weights():
    n = 16
    g = fem.qoi_weights(n)
    assert np.allclose(g, 1.0 / n ** 2)
    gb = fem.qoi_weights(n, (0.25, 0.75, 0.25, 0.75))
    assert np.isclose(gb.sum(), 0.25, rtol=1e-14)           # partition of unity inside the box
    h2 = 1.0 / n ** 2
    G = gb.reshape(n - 1, n - 1)
    # interior of the box h^2, edge points h^2/2, corners h^2/3 (SW, NE) and h^2/6 (SE, NW)
    assert np.isclose(G[7, 7], h2)
    assert np.isclose(G[7, 3], h2 / 2) and np.isclose(G[3, 7], h2 / 2)
    assert np.isclose(G[3, 3], h2 / 3) and np.isclose(G[11, 11], h2 / 3)
    assert np.isclose(G[3, 11], h2 / 6) and np.isclose(G[11, 3], h2 / 6)
    assert G[2, 7] == 0.0


def test_coarse_view_is_the_same_points():
    nf = 8
    xs, ys = fem.node_coords(nf)
    v = 10 * xs + ys
    c = fem.coarse_view(v, nf)
    xc, yc = fem.node_coords(nf // 2)
    assert np.allclose(c, 10 * xc + yc)
