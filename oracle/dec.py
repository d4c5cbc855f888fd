"""DEC operators of the paper, assembled in FP64 with plain numpy / scipy.sparse.

TEST INFRASTRUCTURE ONLY (see the package docstring).

Notation follows the paper: N0 vertices, N1 edges, N2 triangles; ``D0`` is the
incidence matrix d0 (N1 x N0), ``D1`` is d1 (N2 x N1), ``H0`` the diagonal of the
barycentric Hodge star *0, ``H1`` the Galerkin Hodge star *1 (N1 x N1).

A 1D mesh (segments) is handled by the same definitions one dimension down:
the dual cell of a vertex gets half of each adjacent segment, and the Whitney
1-form of a segment is its constant gradient form.
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp


def cell_measures(coords: np.ndarray, cells: np.ndarray) -> np.ndarray:
    """|t|: triangle areas (2D) or segment lengths (1D)."""
    if cells.shape[1] == 2:
        return np.abs(coords[cells[:, 1], 0] - coords[cells[:, 0], 0])
    p0, p1, p2 = coords[cells[:, 0]], coords[cells[:, 1]], coords[cells[:, 2]]
    return 0.5 * np.abs((p1[:, 0] - p0[:, 0]) * (p2[:, 1] - p0[:, 1])
                        - (p1[:, 1] - p0[:, 1]) * (p2[:, 0] - p0[:, 0]))


def edges(cells: np.ndarray) -> np.ndarray:
    """Edges [v_a, v_b] with the canonical orientation a < b (Sec. "DEC
    computational framework": lower-dimensional simplices are oriented by
    increasing vertex index).  Sorted lexicographically, unique."""
    if cells.shape[1] == 2:
        e = np.sort(cells, axis=1)
    else:
        e = np.concatenate([cells[:, [0, 1]], cells[:, [1, 2]], cells[:, [2, 0]]])
        e = np.sort(e, axis=1)
    return np.unique(e, axis=0).astype(np.int64)


def d0(E: np.ndarray, n0: int) -> sp.csr_matrix:
    """Incidence matrix d0 (N1 x N0): +1 at the head v_b, -1 at the tail v_a
    of edge [v_a, v_b], so (d0 psi)_e = psi(v_b) - psi(v_a) (discrete Stokes
    theorem, Eq. 7 and the definition of [d0]_kl that follows it)."""
    n1 = len(E)
    rows = np.repeat(np.arange(n1), 2)
    cols = E.reshape(-1)
    vals = np.tile([-1.0, 1.0], n1)
    return sp.csr_matrix((vals, (rows, cols)), shape=(n1, n0))


def d1(tris: np.ndarray, E: np.ndarray) -> sp.csr_matrix:
    """Incidence matrix d1 (N2 x N1) of counter-clockwise triangles: the
    boundary of [v1, v2, v3] is the cycle v1->v2->v3->v1; an edge enters with
    +1 when its canonical orientation (a < b) agrees with the cycle."""
    index = {(int(a), int(b)): k for k, (a, b) in enumerate(E)}
    rows, cols, vals = [], [], []
    for t, (a, b, c) in enumerate(tris):
        for u, v in ((a, b), (b, c), (c, a)):
            u, v = int(u), int(v)
            rows.append(t)
            if u < v:
                cols.append(index[(u, v)])
                vals.append(1.0)
            else:
                cols.append(index[(v, u)])
                vals.append(-1.0)
    return sp.csr_matrix((vals, (rows, cols)), shape=(len(tris), len(E)))


def star0(coords: np.ndarray, cells: np.ndarray, f_cell: np.ndarray | None = None) -> np.ndarray:
    """Diagonal of the barycentric Hodge star *0, or of *0(f) for a
    piecewise-constant cell function f (Sec. "Discrete Hodge star"):
    [*0(f)]_pp = (1/3) sum_{t ni p} f_t |t|  (1/2 for segments in 1D)."""
    n0 = coords.shape[0]
    k = cells.shape[1]                    # vertices per cell: share of the measure is 1/k
    meas = cell_measures(coords, cells)
    w = meas if f_cell is None else meas * f_cell
    out = np.zeros(n0)
    for j in range(k):
        np.add.at(out, cells[:, j], w / k)
    return out


def _barycentric_gradients(coords: np.ndarray, cells: np.ndarray) -> np.ndarray:
    """grad lambda_i for every cell and local vertex i: [Nc, k, dim].
    lambda_i(r) = G[i, 0] + G[i, 1:] . r with G = inverse of [[1 ... 1], [r_1 ... r_k]]."""
    nc, k = cells.shape
    dim = coords.shape[1]
    Mx = np.ones((nc, k, k))
    Mx[:, 1:, :] = np.transpose(coords[cells], (0, 2, 1))      # rows: 1, x, y
    G = np.linalg.inv(Mx)                                       # [nc, k (lambda), k]
    return G[:, :, 1:1 + dim]


def galerkin_star1(coords: np.ndarray, cells: np.ndarray, E: np.ndarray, xi: np.ndarray | None = None
                   ) -> sp.csr_matrix:
    """Galerkin Hodge star *1 (Eq. 9): [*1]_pq = int xi W_p . W_q over the
    domain, with the Whitney 1-form proxy of edge [v_a, v_b] (Eq. 8)
    W = lambda_a grad lambda_b - lambda_b grad lambda_a.  Products of
    barycentric coordinates integrate exactly over a simplex of dimension n:
    int lambda_i lambda_j = |t| (1 + delta_ij) / ((n+1)(n+2)).
    xi is per cell (the paper leaves it unspecified; 1 gives the Laplacian)."""
    nc, k = cells.shape
    n = k - 1
    meas = cell_measures(coords, cells)
    if xi is None:
        xi = np.ones(nc)
    grad = _barycentric_gradients(coords, cells)
    # local edges of a cell: pairs (i, j) of local vertices, oriented so the
    # global index of i is below the one of j
    pairs = [(i, j) for i in range(k) for j in range(i + 1, k)]
    index = {(int(a), int(b)): e for e, (a, b) in enumerate(E)}
    loc_a = np.zeros((nc, len(pairs)), dtype=np.int64)
    loc_b = np.zeros((nc, len(pairs)), dtype=np.int64)
    eid = np.zeros((nc, len(pairs)), dtype=np.int64)
    for l, (i, j) in enumerate(pairs):
        gi, gj = cells[:, i], cells[:, j]
        swap = gi > gj
        loc_a[:, l] = np.where(swap, j, i)
        loc_b[:, l] = np.where(swap, i, j)
        lo, hi = np.minimum(gi, gj), np.maximum(gi, gj)
        eid[:, l] = [index[(int(u), int(v))] for u, v in zip(lo, hi)]

    def mass(x, y):       # int lambda_x lambda_y over each cell
        return meas * (1.0 + (x == y)) / ((n + 1) * (n + 2))

    def dot(x, y):        # grad lambda_x . grad lambda_y per cell
        gx = grad[np.arange(nc), x]
        gy = grad[np.arange(nc), y]
        return np.sum(gx * gy, axis=1)

    rows, cols, vals = [], [], []
    for l in range(len(pairs)):
        a, b = loc_a[:, l], loc_b[:, l]
        for m in range(len(pairs)):
            c, d = loc_a[:, m], loc_b[:, m]
            # (l_a gb - l_b ga) . (l_c gd - l_d gc) integrated over the cell
            v = (mass(a, c) * dot(b, d) - mass(a, d) * dot(b, c)
                 - mass(b, c) * dot(a, d) + mass(b, d) * dot(a, c))
            rows.append(eid[:, l])
            cols.append(eid[:, m])
            vals.append(xi * v)
    n1 = len(E)
    return sp.csr_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))), shape=(n1, n1))


def projection_Q(cells: np.ndarray, D1: sp.csr_matrix, D0: sp.csr_matrix) -> sp.csr_matrix:
    """Q = (1/6) |d1| |d0| (Eq. 13): maps vertex values to triangle averages."""
    return (abs(D1) @ abs(D0)) / 6.0


class Operators:
    """All operators the method needs for one mesh, in the paper's notation.

    K    = d0^T *1 d0           (N0 x N0, the DEC stiffness)
    A    = *0^{-1} K            (so that the transverse Laplacian is -A, Table I)
    v    = *0^{-1} *0(V) 1      (per-vertex potential, lumped)
    chib = *0^{-1} *0(chi) 1    (per-vertex Kerr coefficient, lumped)
    QtDQ = Q^T diag(chi_t |t|) Q (element-averaged Kerr, Eq. 14; 2D only)
    """

    def __init__(self, coords, cells, V_cell=None, chi_cell=None):
        coords = np.asarray(coords, dtype=np.float64)
        cells = np.asarray(cells, dtype=np.int64)
        self.coords, self.cells = coords, cells
        self.n0 = coords.shape[0]
        nc = cells.shape[0]
        V_cell = np.zeros(nc) if V_cell is None else np.asarray(V_cell, dtype=np.float64)
        chi_cell = np.ones(nc) if chi_cell is None else np.asarray(chi_cell, dtype=np.float64)
        self.E = edges(cells)
        self.D0 = d0(self.E, self.n0)
        self.H0 = star0(coords, cells)
        self.H1 = galerkin_star1(coords, cells, self.E)
        self.K = (self.D0.T @ self.H1 @ self.D0).tocsr()
        self.A = (sp.diags(1.0 / self.H0) @ self.K).tocsr()
        self.v = star0(coords, cells, V_cell) / self.H0
        self.chib = star0(coords, cells, chi_cell) / self.H0
        self.chi_cell, self.V_cell = chi_cell, V_cell
        self._QtDQ = None
        # infinity-norm of A: max row sum of |A| (also a Gershgorin bound on
        # the spectrum of A, which is real and >= 0 since K is PSD)
        self.rho = float(np.max(np.asarray(abs(self.A).sum(axis=1)).ravel()))

    @property
    def QtDQ(self) -> sp.csr_matrix:
        if self._QtDQ is None:
            D1 = d1(self.cells, self.E)
            Q = projection_Q(self.cells, D1, self.D0)
            D = sp.diags(self.chi_cell * cell_measures(self.coords, self.cells))
            self._QtDQ = (Q.T @ D @ Q).tocsr()
        return self._QtDQ
