"""Oracle: P1 finite elements for Problem 3.1 on the unit square.

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__.py``).

Problem 3.1 (Sec. 3.1): find u in H^1_0(D) with int a grad u . grad v = int f v.
Sec. 5.1 uses D = (0,1)^2, u = 0 on the boundary, f = 1 (Eq. (5.1)).  The
paper discretises with conforming P1 Lagrange elements on a quasi-uniform
triangulation (Sec. 3.1) and does not say which; the reading here is the
uniform grid with h = 1/n whose cells are split along the SW-NE diagonal.
The coefficient is P1-interpolated from its nodal values, so the element
stiffness is exact with a_T = mean of the three vertex values.

Nodes: (x_i, y_j) = (i h, j h), flat index j (n+1) + i.  Unknowns: the
(n-1)^2 interior nodes, index (j-1)(n-1) + (i-1).

Assembly is element by element from the gradients of the barycentric
coordinates; the 5-point structure of the result is a consequence that the
tests check, not an input.  Solves use LAPACK through SciPy / NumPy: banded
Cholesky (bandwidth n-1) and, for small grids, dense LU.
"""
import numpy as np
import scipy.sparse as sps
from scipy.linalg import solveh_banded


def triangles(n):
    """Vertex node indices of all 2 n^2 triangles: T1 = (SW, SE, NE), T2 = (SW, NE, NW)."""
    i, j = np.meshgrid(np.arange(n), np.arange(n), indexing="xy")
    sw = (j * (n + 1) + i).ravel()
    se = sw + 1
    nw = sw + (n + 1)
    ne = nw + 1
    t1 = np.stack([sw, se, ne], axis=1)
    t2 = np.stack([sw, ne, nw], axis=1)
    return np.concatenate([t1, t2], axis=0)


def node_coords(n):
    idx = np.arange((n + 1) * (n + 1))
    return (idx % (n + 1)) / n, (idx // (n + 1)) / n


def element_geometry(n, tris):
    """Per triangle: area and the gradients (3 x 2) of the three barycentric coordinates."""
    x, y = node_coords(n)
    x0, x1, x2 = x[tris[:, 0]], x[tris[:, 1]], x[tris[:, 2]]
    y0, y1, y2 = y[tris[:, 0]], y[tris[:, 1]], y[tris[:, 2]]
    D = np.empty((len(tris), 2, 2))
    D[:, 0, 0] = x1 - x0
    D[:, 0, 1] = x2 - x0
    D[:, 1, 0] = y1 - y0
    D[:, 1, 1] = y2 - y0
    det = D[:, 0, 0] * D[:, 1, 1] - D[:, 0, 1] * D[:, 1, 0]
    area = 0.5 * np.abs(det)
    Dinv = np.linalg.inv(D)                   # rows: grad lambda_1, grad lambda_2
    g = np.empty((len(tris), 3, 2))
    g[:, 1, :] = Dinv[:, 0, :]
    g[:, 2, :] = Dinv[:, 1, :]
    g[:, 0, :] = -(g[:, 1, :] + g[:, 2, :])
    return area, g


def element_stiffness(n, a_nodal, tris=None):
    """K_T[a][b] = a_T |T| grad phi_a . grad phi_b with a_T = mean of vertex values."""
    tris = triangles(n) if tris is None else tris
    area, g = element_geometry(n, tris)
    a_nodal = np.asarray(a_nodal, dtype=np.float64).ravel()
    aT = a_nodal[tris].mean(axis=1)
    KT = np.einsum("t,tad,tbd->tab", aT * area, g, g)
    return tris, KT, area, g


def _interior_map(n):
    m = np.full((n + 1) * (n + 1), -1, dtype=np.int64)
    i, j = np.meshgrid(np.arange(1, n), np.arange(1, n), indexing="xy")
    m[(j * (n + 1) + i).ravel()] = np.arange((n - 1) * (n - 1))
    return m


def assemble_full(n, a_nodal):
    """Stiffness on all (n+1)^2 nodes (no boundary condition applied), CSR."""
    tris, KT, _, _ = element_stiffness(n, a_nodal)
    rows = np.repeat(tris, 3, axis=1).ravel()
    cols = np.tile(tris, (1, 3)).ravel()
    N = (n + 1) * (n + 1)
    return sps.coo_matrix((KT.ravel(), (rows, cols)), shape=(N, N)).tocsr()


def assemble(n, a_nodal):
    """Stiffness on the interior unknowns (homogeneous Dirichlet data), CSR."""
    tris, KT, _, _ = element_stiffness(n, a_nodal)
    m = _interior_map(n)
    rows = m[np.repeat(tris, 3, axis=1).ravel()]
    cols = m[np.tile(tris, (1, 3)).ravel()]
    keep = (rows >= 0) & (cols >= 0)
    N = (n - 1) * (n - 1)
    return sps.coo_matrix((KT.ravel()[keep], (rows[keep], cols[keep])), shape=(N, N)).tocsr()


def load_vector(n, f=None):
    """b_i = int f phi_i.  f = None means f = 1 (exact: |T|/3 per triangle).

    A callable f(x, y) is integrated with the 3-point edge-midpoint rule
    (exact for quadratics)."""
    tris = triangles(n)
    area, _ = element_geometry(n, tris)
    m = _interior_map(n)
    bT = np.empty((len(tris), 3))
    if f is None:
        bT[:] = (area / 3.0)[:, None]
    else:
        x, y = node_coords(n)
        X, Y = x[tris], y[tris]
        # midpoints of edges (0,1), (1,2), (2,0); phi_a = 1/2 at both ends' midpoints
        mids = [((0, 1), 2), ((1, 2), 0), ((2, 0), 1)]
        bT[:] = 0.0
        for (p, r), opp in mids:
            fm = f(0.5 * (X[:, p] + X[:, r]), 0.5 * (Y[:, p] + Y[:, r]))
            for a in range(3):
                if a != opp:
                    bT[:, a] += (area / 3.0) * fm * 0.5
    rows = m[tris.ravel()]
    keep = rows >= 0
    return np.bincount(rows[keep], weights=bT.ravel()[keep], minlength=(n - 1) * (n - 1))


def qoi_weights(n, box=None):
    """g_i = int_B phi_i for B = D (box None) or an axis-aligned box
    (x0, x1, y0, y1) whose sides lie on grid lines: a triangle counts when it
    lies inside B, contributing |T|/3 to each of its vertices."""
    tris = triangles(n)
    area, _ = element_geometry(n, tris)
    keep_t = np.ones(len(tris), dtype=bool)
    if box is not None:
        x, y = node_coords(n)
        cx, cy = x[tris].mean(axis=1), y[tris].mean(axis=1)   # centroid inside <=> triangle inside
        x0, x1, y0, y1 = box
        keep_t = (cx > x0) & (cx < x1) & (cy > y0) & (cy < y1)
    m = _interior_map(n)
    rows = m[tris[keep_t].ravel()]
    w = np.repeat(area[keep_t] / 3.0, 3)
    keep = rows >= 0
    return np.bincount(rows[keep], weights=w[keep], minlength=(n - 1) * (n - 1))


def to_banded_upper(A, bw):
    """Upper banded storage ab[bw + i - j, j] = A[i, j] for j - bw <= i <= j."""
    A = A.tocoo()
    N = A.shape[0]
    ab = np.zeros((bw + 1, N))
    up = A.row <= A.col
    ab[bw + A.row[up] - A.col[up], A.col[up]] = A.data[up]
    return ab


def solve_cholesky(n, A, b):
    """Banded Cholesky solve (LAPACK pbsv), bandwidth n - 1."""
    if n == 2:
        return np.asarray(b, dtype=np.float64) / A.toarray()[0, 0]
    return solveh_banded(to_banded_upper(A, n - 1), b, lower=False, check_finite=True)


def solve_dense(A, b):
    """Dense LU solve (LAPACK gesv)."""
    return np.linalg.solve(A.toarray(), b)


def solve_sample(n, a_nodal, box=None, f=None):
    """(x, Q): the P1 solution on the interior nodes and Q = g^T x."""
    A = assemble(n, a_nodal)
    b = load_vector(n, f)
    x = solve_cholesky(n, A, b)
    return x, float(qoi_weights(n, box) @ x)


def coarse_view(a_fine, n_fine):
    """Nodal values of the coarse grid (n_fine / 2) taken from the fine field:
    coarse node (i, j) is fine node (2i, 2j), the same point in D."""
    a = np.asarray(a_fine).reshape(n_fine + 1, n_fine + 1)
    return a[::2, ::2].ravel().copy()


def relative_residual(n, a_nodal, x, f=None):
    """||b - A x||_2 / ||b||_2 with the oracle's own A and b (Eq. (2.1))."""
    A = assemble(n, a_nodal)
    b = load_vector(n, f)
    return float(np.linalg.norm(b - A @ x) / np.linalg.norm(b))
