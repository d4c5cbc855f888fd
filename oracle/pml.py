"""Perfectly matched layer by complex stretching of the discrete Hodge stars
(the paper's "natural next step" in the Conclusion: a complex-stretched
metric, in the spirit of exterior complex scaling), FP64, plain numpy.

TEST INFRASTRUCTURE ONLY (see the package docstring).

Reading (the paper gives no formulas): radial exterior complex scaling about
a centre c.  Outside r_in the radius is continued into the complex plane,
    r~(r) = r + i int_{r_in}^r sigma,   s(r) = dr~/dr = 1 + i sigma(r),
    sigma(r) = sigma_max ((r - r_in) / (R - r_in))^order   (0 inside r_in).
The Laplacian in the stretched metric is (1/J) div(Lambda grad) with, per
triangle (evaluated at its centroid),
    Lambda = (r~ / (s r)) e_r e_r^T + (s r / r~) e_t e_t^T,   J = s r~ / r,
i.e. *1 becomes the Galerkin star of Eq. 9 with the tensor Lambda in the
inner product of the Whitney forms, and *0 becomes sum_t J_t |t| / 3.
Then K~ = d0^T *1~ d0 (complex symmetric, K~ 1 = 0) and A~ = *0~^{-1} K~;
the potential and Kerr coefficient keep their lumped definitions with the
stretched *0 (an average of V_t, chi_t with weights J_t |t|).  The
propagation equation is unchanged: i dPsi/dz = p1 A~ Psi - v Psi - N Psi.
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp

from .dec import _barycentric_gradients, cell_measures, d0, edges


def stretch(coords, cells, center=(0.0, 0.0), r_in=3.0, R=4.0, sigma_max=2.0, order=2):
    """Per triangle: Lambda [nt, 2, 2] (complex) and J [nt] (complex)."""
    c = coords[cells].mean(axis=1) - np.asarray(center)[None, :]
    r = np.hypot(c[:, 0], c[:, 1])
    u = np.clip((r - r_in) / (R - r_in), 0.0, None)
    sig = sigma_max * u ** order if order > 0 else np.where(r > r_in, sigma_max, 0.0)
    s = 1.0 + 1j * sig
    rt = r + 1j * sigma_max * (R - r_in) * u ** (order + 1) / (order + 1)
    safe = np.where(r > 0, r, 1.0)
    er = np.where(r[:, None] > 0, c / safe[:, None], np.array([1.0, 0.0])[None, :])
    et = np.stack([-er[:, 1], er[:, 0]], axis=1)
    a_r = np.where(r > 0, rt / (s * safe), 1.0)
    a_t = np.where(r > 0, s * safe / np.where(r > 0, rt, 1.0), 1.0)
    Lam = a_r[:, None, None] * er[:, :, None] * er[:, None, :] + a_t[:, None, None] * et[:, :, None] * et[:, None, :]
    J = np.where(r > 0, s * rt / safe, 1.0)
    return Lam, J


def stiffness(coords, cells, Lam):
    """P1 stiffness with the tensor Lambda: K_ij = sum_t |t| grad l_i . Lambda_t grad l_j."""
    n0 = coords.shape[0]
    meas = cell_measures(coords, cells)
    g = _barycentric_gradients(coords, cells)                    # [nt, 3, 2]
    Kt = np.einsum("tia,tab,tjb->tij", g, Lam, g) * meas[:, None, None]
    rows = np.repeat(cells, 3, axis=1).reshape(-1)
    cols = np.tile(cells, (1, 3)).reshape(-1)
    return sp.csr_matrix((Kt.reshape(-1), (rows, cols)), shape=(n0, n0))


def whitney_star1(coords, cells, E, Lam):
    """The Galerkin *1 of Eq. 9 with the inner product of the Whitney 1-forms
    weighted by Lambda: [*1]_pq = int W_p . Lambda W_q (exact quadrature of
    products of barycentric coordinates)."""
    nc = cells.shape[0]
    meas = cell_measures(coords, cells)
    grad = _barycentric_gradients(coords, cells)
    pairs = [(0, 1), (0, 2), (1, 2)]
    index = {(int(a), int(b)): e for e, (a, b) in enumerate(E)}
    rows, cols, vals = [], [], []
    la, lb, ids = [], [], []
    for i, j in pairs:
        gi, gj = cells[:, i], cells[:, j]
        swap = gi > gj
        la.append(np.where(swap, j, i))
        lb.append(np.where(swap, i, j))
        lo, hi = np.minimum(gi, gj), np.maximum(gi, gj)
        ids.append(np.array([index[(int(u), int(v))] for u, v in zip(lo, hi)]))
    t = np.arange(nc)

    def mass(x, y):
        return meas * (1.0 + (x == y)) / 12.0

    def dot(x, y):
        return np.einsum("ta,tab,tb->t", grad[t, x], Lam, grad[t, y])

    for l in range(3):
        a, b = la[l], lb[l]
        for m in range(3):
            c, d = la[m], lb[m]
            v = (mass(a, c) * dot(b, d) - mass(a, d) * dot(b, c) - mass(b, c) * dot(a, d) + mass(b, d) * dot(a, c))
            rows.append(ids[l])
            cols.append(ids[m])
            vals.append(v)
    n1 = len(E)
    return sp.csr_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))), shape=(n1, n1))


class StretchedOperators:
    """The attributes the oracle's RK45 (bpm.dopri5 / bpm.dec_rhs, lumped
    Kerr) and Taylor march use, for the complex-stretched metric:
    A (complex), v, chib (complex lumped averages), rho (inf-norm of A).
    H0 is the physical (unstretched) *0, used only by the error norms;
    H0s is the stretched one."""

    def __init__(self, coords, cells, V_cell, chi_cell, **pml):
        self.coords, self.cells, self.n0 = coords, cells, coords.shape[0]
        Lam, J = stretch(coords, cells, **pml)
        meas = cell_measures(coords, cells)
        self.E = edges(cells)
        self.D0 = d0(self.E, self.n0)
        self.H1s = whitney_star1(coords, cells, self.E, Lam)
        self.K = (self.D0.T @ self.H1s @ self.D0).tocsr()
        wt = J * meas / 3.0
        self.H0s = np.zeros(self.n0, dtype=complex)
        num_v = np.zeros(self.n0, dtype=complex)
        num_c = np.zeros(self.n0, dtype=complex)
        for j in range(3):
            np.add.at(self.H0s, cells[:, j], wt)
            np.add.at(num_v, cells[:, j], wt * V_cell)
            np.add.at(num_c, cells[:, j], wt * chi_cell)
        self.v = num_v / self.H0s
        self.chib = num_c / self.H0s
        self.A = (sp.diags(1.0 / self.H0s) @ self.K).tocsr()
        self.H0 = np.zeros(self.n0)
        for j in range(3):
            np.add.at(self.H0, cells[:, j], meas / 3.0)
        self.rho = float(np.max(np.asarray(abs(self.A).sum(axis=1)).ravel()))


# --------------------------------------------------------------------------
# split-step march with the layer
# --------------------------------------------------------------------------
def diagonal_flow_stretched(ops, psi, h, sigma=None):
    """Exact flow over h of dpsi_p/dz = i (v_p + chib_p |psi_p|^2) psi_p - sigma_p psi_p
    with the complex lumped v and chib of the stretched metric (lumped Kerr).

    The intensity I = |psi|^2 obeys dI/dz = -alpha I - beta I^2 with
    alpha = 2 (Im v + sigma), beta = 2 Im chib (a Bernoulli equation):
        I(h) = I0 e^{-alpha h} / D,   D = 1 + beta I0 q,   q = (1 - e^{-alpha h}) / alpha,
    and the phase is the integral of Re v + Re chib I(z):
        theta = Re v h + Re chib ln(D) / beta   (-> Re chib I0 q as beta -> 0),
    so psi(h) = psi0 sqrt(e^{-alpha h} / D) e^{i theta}.  With real v and chib
    this is the flow of bpm.diagonal_flow."""
    n0 = ops.n0
    sigma = np.zeros(n0) if sigma is None else np.asarray(sigma, dtype=np.float64)
    psi = np.asarray(psi, dtype=np.complex128)
    v = np.asarray(ops.v, dtype=np.complex128)
    c = np.asarray(ops.chib, dtype=np.complex128)
    if psi.ndim == 2:
        v, c, sigma = v[:, None], c[:, None], sigma[:, None]
    I0 = np.abs(psi) ** 2
    alpha = 2.0 * (v.imag + sigma)
    beta = 2.0 * c.imag
    ah = alpha * h
    with np.errstate(divide="ignore", invalid="ignore"):
        q = np.where(np.abs(ah) > 1e-300, -np.expm1(-ah) / np.where(alpha == 0, 1.0, alpha), h)
        x = beta * I0 * q
        # ln(1 + x) / beta = I0 q log1p(x) / x, the ratio -> 1 as x -> 0
        ratio = np.where(np.abs(x) > 1e-300, np.log1p(x) / np.where(x == 0, 1.0, x), 1.0)
    integral = I0 * q * ratio
    theta = v.real * h + c.real * integral
    amp = np.sqrt(np.exp(-ah) / (1.0 + x))
    return psi * amp * np.exp(1j * theta)


def propagate_stretched(ops, p, psi0, h, n_steps, sigma=None):
    """n_steps Strang steps D_{h/2} E_h D_{h/2} on the stretched operators:
    E_h = exp(-i h L_diff) with the complex A~ (bpm.linear_step, Taylor with
    substeps: the series holds for any matrix), D the flow above.  Half steps
    are applied as written (no merging)."""
    from . import bpm
    psi = np.array(psi0, dtype=np.complex128, copy=True)
    for _ in range(n_steps):
        psi = diagonal_flow_stretched(ops, psi, 0.5 * h, sigma)
        psi = bpm.linear_step(ops, p, psi, h)
        psi = diagonal_flow_stretched(ops, psi, 0.5 * h, sigma)
    return psi
