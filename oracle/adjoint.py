"""Oracle: gradient of the QoI with respect to the KL coefficients.

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__.py``).

Q = g^T x with A(a) x = b (Sec. 3.1, Problem 4.5), A = sum_T a_T Khat_T where
Khat_T is the unit-coefficient P1 element stiffness and a_T the mean of the
vertex values of a, and a_v = exp(sum_k xi_k Phi_k(x_v)) (Eq. (5.2) form).
With the adjoint A lambda = g (A is symmetric),
  dQ = -lambda^T dA x = -sum_T da_T |T| grad(lambda_h) . grad(u_h),
so dQ/dxi_k = sum_v Phi_k(v) a_v G_v with
  G_v = -(1/3) sum_{T contains v} |T| grad(lambda_h)|_T . grad(u_h)|_T.
Solves are exact (banded Cholesky).  ``finite_difference`` is the central
difference of the same exact Q, used to check the formula.
"""
import numpy as np

from . import fem, kl


def _full(n, x_interior):
    v = np.zeros((n + 1) * (n + 1))
    i, j = np.meshgrid(np.arange(1, n), np.arange(1, n), indexing="xy")
    v[(j * (n + 1) + i).ravel()] = x_interior
    return v


def nodal_sensitivity(n, a_nodal, box=None):
    """(Q, x, lam, G): G_v = dQ/da_T chain-ruled onto nodes, before the factor a_v."""
    A = fem.assemble(n, a_nodal)
    b = fem.load_vector(n)
    g = fem.qoi_weights(n, box)
    x = fem.solve_cholesky(n, A, b)
    lam = fem.solve_cholesky(n, A, g)
    xf, lf = _full(n, x), _full(n, lam)
    tris = fem.triangles(n)
    area, grads = fem.element_geometry(n, tris)
    gu = np.einsum("ta,tad->td", xf[tris], grads)
    gl = np.einsum("ta,tad->td", lf[tris], grads)
    eT = area * np.einsum("td,td->t", gl, gu)
    G = -np.bincount(tris.ravel(), weights=np.repeat(eT / 3.0, 3), minlength=(n + 1) * (n + 1))
    return float(g @ x), x, lam, G


def gradient(n, xi, phi, box=None):
    """(Q, dQ/dxi[K]) for one sample."""
    a = kl.coefficient(np.asarray(xi)[None, :], phi)[0]
    Q, _, _, G = nodal_sensitivity(n, a, box)
    return Q, phi @ (a * G)


def qoi(n, xi, phi, box=None):
    a = kl.coefficient(np.asarray(xi)[None, :], phi)[0]
    return fem.solve_sample(n, a, box)[1]


def finite_difference(n, xi, phi, k, step=1e-6, box=None):
    xp = np.array(xi, dtype=np.float64)
    xm = np.array(xi, dtype=np.float64)
    xp[k] += step
    xm[k] -= step
    return (qoi(n, xp, phi, box) - qoi(n, xm, phi, box)) / (2.0 * step)
