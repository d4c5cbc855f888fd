"""Split-step z-march of the DEC NLSE, FP64, plain and slow.

TEST INFRASTRUCTURE ONLY (see the package docstring).

The equation (Eq. 1 in normalized form, discretized as Eqs. 10-12) is read as

    i dPsi/dz = -sum_n p_n (-A)^n Psi - v Psi - chib |Psi|^2 Psi  (- i sigma Psi)

with A = *0^{-1} d0^T *1 d0, so that the transverse Laplacian is -A (Table I).
This follows Eq. 1 and Table I; Eq. 11 as printed puts the stiffness and the
potential under one minus sign, which would flip the relative sign of
diffraction against the potential and the Kerr term (the exact sech soliton
is stationary only with the reading used here).  sigma >= 0 is the absorber
(a damping rate per vertex; the paper names absorbing layers but gives no
formula).

One step of length h is the Strang composition D_{h/2} E_h D_{h/2}:
  E_h  exact action of exp(i h sum_n p_n (-A)^n)       (linear diffraction)
  D_h  exact flow of dpsi/dz = i (v + N(|psi|^2)) psi - sigma psi per vertex
The oracle applies every half step as written (no merging of adjacent half
steps), so that a fused implementation can be checked against it.
"""
from __future__ import annotations

import math

import numpy as np
import scipy.sparse as sp

from .dec import Operators


# --------------------------------------------------------------------------
# linear operator of the diffraction part
# --------------------------------------------------------------------------
def apply_Ldiff(ops: Operators, p, psi: np.ndarray) -> np.ndarray:
    """L_diff psi = -sum_n p_n (-A)^n psi: the higher-order terms are the
    cascaded powers of the DEC Laplacian (Table I, 'Higher-order' row)."""
    out = np.zeros_like(psi)
    term = psi
    for n, pn in enumerate(p, start=1):
        term = -(ops.A @ term)            # (-A)^n psi
        if pn != 0.0:
            out = out - pn * term
    return out


def Ldiff_norm_bound(ops: Operators, p) -> float:
    """Bound on the infinity norm of L_diff: sum_n |p_n| ||A||_inf^n."""
    return float(sum(abs(pn) * ops.rho ** n for n, pn in enumerate(p, start=1)))


def linear_step(ops: Operators, p, psi: np.ndarray, h: float, tol: float = 1e-18) -> np.ndarray:
    """E_h psi = exp(-i h L_diff) psi by its Taylor series, with the step
    split into s substeps so that ||(h/s) L_diff||_inf <= 1; each series is
    summed until the last term is below tol times the partial sum (both in
    the infinity norm).  This is a different algorithm from the library's
    Chebyshev expansion on purpose."""
    bound = Ldiff_norm_bound(ops, p) * abs(h)
    s = max(1, int(math.ceil(bound)))
    hs = h / s
    psi = np.array(psi, dtype=np.complex128, copy=True)
    for _ in range(s):
        acc = psi.copy()
        term = psi
        k = 0
        while True:
            k += 1
            term = (-1j * hs / k) * apply_Ldiff(ops, p, term)
            acc = acc + term
            if np.max(np.abs(term)) <= tol * max(np.max(np.abs(acc)), 1e-300) or k > 200:
                break
        psi = acc
    return psi


# --------------------------------------------------------------------------
# diagonal (potential + Kerr + absorber) flow
# --------------------------------------------------------------------------
def _phi(sigma: np.ndarray, h: float) -> np.ndarray:
    """int_0^h exp(-2 sigma z) dz = (1 - exp(-2 sigma h)) / (2 sigma), -> h as sigma -> 0."""
    sigma = np.asarray(sigma, dtype=np.float64)
    out = np.full(sigma.shape, float(h))
    nz = sigma > 0
    out[nz] = -np.expm1(-2.0 * sigma[nz] * h) / (2.0 * sigma[nz])
    return out


def diagonal_flow(ops: Operators, psi: np.ndarray, h: float, sigma: np.ndarray | None = None,
                  kerr: str = "lumped") -> np.ndarray:
    """Exact flow over h of dpsi_p/dz = i (v_p + N_p) psi_p - sigma_p psi_p.

    |psi_p|^2 decays as exp(-2 sigma_p z) and the phase is the integral of
    the rate:  theta_p = v_p h + sum_q c_pq |psi_q(0)|^2 phi(sigma_q, h).
    kerr="lumped":  N_p = chib_p |psi_p|^2 (c = diag(chib)).
    kerr="element": N_p = [*0^{-1} Q^T D Q |psi|^2]_p, the triangle-averaged
                    intensity of Eq. 14 (the phase flow stays exact because
                    every |psi_q| only decays at its own rate).
    """
    n0 = ops.n0
    sigma = np.zeros(n0) if sigma is None else np.asarray(sigma, dtype=np.float64)
    psi = np.asarray(psi, dtype=np.complex128)
    I0 = np.abs(psi) ** 2
    ph = _phi(sigma, h)
    if psi.ndim == 2:
        ph2 = ph[:, None]
        v = ops.v[:, None]
        sig = sigma[:, None]
    else:
        ph2, v, sig = ph, ops.v, sigma
    if kerr == "lumped":
        chib = ops.chib[:, None] if psi.ndim == 2 else ops.chib
        theta = v * h + chib * I0 * ph2
    elif kerr == "element":
        C = sp.diags(1.0 / ops.H0) @ ops.QtDQ
        theta = v * h + C @ (I0 * ph2)
    else:
        raise ValueError(kerr)
    return psi * np.exp(-sig * h) * np.exp(1j * theta)


# --------------------------------------------------------------------------
# Strang split-step march
# --------------------------------------------------------------------------
def strang_step(ops, p, psi, h, sigma=None, kerr="lumped"):
    psi = diagonal_flow(ops, psi, 0.5 * h, sigma, kerr)
    psi = linear_step(ops, p, psi, h)
    return diagonal_flow(ops, psi, 0.5 * h, sigma, kerr)


def propagate(ops: Operators, p, psi0: np.ndarray, h: float, n_steps: int, sigma=None, kerr="lumped",
              callback=None) -> np.ndarray:
    """n_steps Strang steps of length h.  psi0 is [N0] or [N0, B] (fields
    are independent).  callback(step, psi) runs after every step if given."""
    psi = np.array(psi0, dtype=np.complex128, copy=True)
    for n in range(n_steps):
        psi = strang_step(ops, p, psi, h, sigma, kerr)
        if callback is not None:
            callback(n + 1, psi)
    return psi


# --------------------------------------------------------------------------
# diagnostics
# --------------------------------------------------------------------------
def power(ops: Operators, psi: np.ndarray) -> np.ndarray:
    """P = Psi^H *0 Psi = sum_p m_p |psi_p|^2 (conserved without absorber)."""
    w = ops.H0 if psi.ndim == 1 else ops.H0[:, None]
    return np.sum(w * np.abs(psi) ** 2, axis=0)


def hamiltonian(ops: Operators, p, psi: np.ndarray) -> np.ndarray:
    """H = Psi^H *0 L_diff Psi - sum_p m_p v_p |psi_p|^2 - (1/2) sum_p m_p chib_p |psi_p|^4,
    the conserved energy of the lumped DEC system (i *0 dPsi/dz = dH/dPsi^*)."""
    psi2 = psi if psi.ndim == 2 else psi[:, None]
    Lpsi = apply_Ldiff(ops, p, psi2)
    m = ops.H0[:, None]
    lin = np.real(np.sum(np.conj(psi2) * m * Lpsi, axis=0))
    I = np.abs(psi2) ** 2
    pot = np.sum(m * ops.v[:, None] * I, axis=0)
    kerr = 0.5 * np.sum(m * ops.chib[:, None] * I * I, axis=0)
    out = lin - pot - kerr
    return out if psi.ndim == 2 else out[0]


def relative_error(ops: Operators, psi: np.ndarray, ref: np.ndarray) -> float:
    """*0-weighted relative L2 error of the complex field."""
    w = ops.H0 if psi.ndim == 1 else ops.H0[:, None]
    return float(math.sqrt(np.sum(w * np.abs(psi - ref) ** 2) / np.sum(w * np.abs(ref) ** 2)))


def intensity_error(ops: Operators, psi: np.ndarray, ref: np.ndarray) -> float:
    """E_rel of Eq. 15 on intensities, with the L2 norm taken *0-weighted
    over the mesh (the paper does not state the quadrature)."""
    w = ops.H0 if psi.ndim == 1 else ops.H0[:, None]
    a, b = np.abs(psi) ** 2, np.abs(ref) ** 2
    return float(math.sqrt(np.sum(w * (a - b) ** 2) / np.sum(w * b * b)))


# --------------------------------------------------------------------------
# the paper's own integrator (cross-check of the split-step march)
# --------------------------------------------------------------------------
def rk45_reference(ops: Operators, p, psi0: np.ndarray, z: float, rtol=1e-11, atol=1e-13,
                   kerr="lumped") -> np.ndarray:
    """Integrate the DEC ODE of Eq. 10, i dPsi/dz = L Psi + N(|psi|^2) Psi,
    with adaptive Dormand-Prince RK45 (scipy's solve_ivp, as in the paper,
    which used rtol 1e-9 / atol 1e-11).  L = L_diff - diag(v) and
    N = -diag(chib |psi|^2) (lumped) or -*0^{-1} diag(Q^T D Q |psi|^2) (Eq. 14).
    No absorber: the paper's runs have none."""
    from scipy.integrate import solve_ivp

    C = sp.diags(1.0 / ops.H0) @ ops.QtDQ if kerr == "element" else None

    def rhs(_z, y):
        psi = y[: ops.n0] + 1j * y[ops.n0:]
        I = np.abs(psi) ** 2
        Nterm = ops.chib * I if kerr == "lumped" else C @ I
        dpsi = -1j * (apply_Ldiff(ops, p, psi) - ops.v * psi - Nterm * psi)
        return np.concatenate([dpsi.real, dpsi.imag])

    y0 = np.concatenate([np.real(psi0), np.imag(psi0)])
    sol = solve_ivp(rhs, (0.0, z), y0, method="RK45", rtol=rtol, atol=atol)
    y = sol.y[:, -1]
    return y[: ops.n0] + 1j * y[ops.n0:]


# --------------------------------------------------------------------------
# exact discrete adjoint of the split-step march (lumped Kerr)
# --------------------------------------------------------------------------
def overlap_objective(ops: Operators, phi: np.ndarray, psi: np.ndarray):
    """J = |<phi, psi>_{*0}|^2 = |sum_p m_p conj(phi_p) psi_p|^2 and its
    Euclidean gradient G (dJ = Re sum conj(G_p) dpsi_p): G = 2 c m phi."""
    c = np.sum(ops.H0 * np.conj(phi) * psi)
    return float(abs(c) ** 2), 2.0 * c * ops.H0 * phi


def adjoint_diagonal(ops: Operators, psi_in: np.ndarray, gt: np.ndarray, h: float, sigma=None):
    """Backward through D_h (lumped Kerr).  psi_in is the input state of the
    flow, gt the *0-weighted cotangent of its output.  With u = e^{-sigma h} e^{i theta}
    and theta = v h + chib |psi_in|^2 phi(sigma, h):
        ghat = conj(u) gt,   g_in = ghat - 2 chib phi Im(conj(ghat) psi_in) psi_in,
        dJ/dv_p = -h m_p Im(conj(ghat_p) psi_in_p).
    Returns (g_in, dJ/dv contribution)."""
    sigma = np.zeros(ops.n0) if sigma is None else np.asarray(sigma, dtype=np.float64)
    I0 = np.abs(psi_in) ** 2
    ph = _phi(sigma, h)
    theta = ops.v * h + ops.chib * I0 * ph
    u = np.exp(-sigma * h) * np.exp(1j * theta)
    ghat = np.conj(u) * gt
    im = np.imag(np.conj(ghat) * psi_in)
    return ghat - 2.0 * ops.chib * ph * im * psi_in, -h * ops.H0 * im


def vjp(ops: Operators, p, psi0: np.ndarray, gN: np.ndarray, h: float, n_steps: int, sigma=None):
    """Vector-Jacobian product of the whole march psi_N = (D_{h/2} E_h D_{h/2})^N psi0.
    gN is the Euclidean cotangent of psi_N.  Returns (Euclidean gradient
    w.r.t. psi0, dJ/dv for a per-vertex potential offset v).  Every
    intermediate state is stored (small problems only)."""
    pre, mid = [], []
    psi = np.array(psi0, dtype=np.complex128, copy=True)
    for _ in range(n_steps):
        pre.append(psi)
        a = diagonal_flow(ops, psi, 0.5 * h, sigma)
        b = linear_step(ops, p, a, h)
        mid.append(b)
        psi = diagonal_flow(ops, b, 0.5 * h, sigma)
    gt = gN / ops.H0
    gv = np.zeros(ops.n0)
    for n in reversed(range(n_steps)):
        gt, d1 = adjoint_diagonal(ops, mid[n], gt, 0.5 * h, sigma)
        gt = linear_step(ops, p, gt, -h)          # E^H in the *0 inner product is E^{-1}
        gt, d2 = adjoint_diagonal(ops, pre[n], gt, 0.5 * h, sigma)
        gv += d1 + d2
    return ops.H0 * gt, gv


# --------------------------------------------------------------------------
# the paper's integrator: adaptive Dormand-Prince 5(4) on the DEC ODE
# --------------------------------------------------------------------------
# Butcher tableau of Dormand & Prince (1980), 5th-order solution with an
# embedded 4th-order estimate, first-same-as-last.
DP_C = [0.0, 1 / 5, 3 / 10, 4 / 5, 8 / 9, 1.0, 1.0]
DP_A = [[],
        [1 / 5],
        [3 / 40, 9 / 40],
        [44 / 45, -56 / 15, 32 / 9],
        [19372 / 6561, -25360 / 2187, 64448 / 6561, -212 / 729],
        [9017 / 3168, -355 / 33, 46732 / 5247, 49 / 176, -5103 / 18656],
        [35 / 384, 0.0, 500 / 1113, 125 / 192, -2187 / 6784, 11 / 84]]
DP_B4 = [5179 / 57600, 0.0, 7571 / 16695, 393 / 640, -92097 / 339200, 187 / 2100, 1 / 40]
DP_E = [b5 - b4 for b5, b4 in zip(DP_A[6] + [0.0], DP_B4)]


def dec_rhs(ops: Operators, p, psi: np.ndarray, sigma=None, kerr="lumped") -> np.ndarray:
    """Right-hand side of Eq. 10, dPsi/dz = -i (L Psi + N Psi), with
    L = L_diff - diag(v) (the potential inside L as in Eq. 11, sign per Eq. 1)
    and N = -chib |psi|^2 (lumped) or -*0^{-1} Q^T D Q |psi|^2 (Eq. 14); the
    absorber adds -sigma psi (zero for the paper's runs)."""
    I = np.abs(psi) ** 2
    if kerr == "lumped":
        Nr = ops.chib * I
    else:
        Nr = (sp.diags(1.0 / ops.H0) @ ops.QtDQ) @ I
    out = -1j * (apply_Ldiff(ops, p, psi) - ops.v * psi - Nr * psi)
    if sigma is not None:
        out = out - np.asarray(sigma) * psi
    return out


def _rms_error(err, y, y_new, rtol, atol):
    """sqrt(mean((err / (atol + rtol max(|y|, |y_new|)))^2)) over the real and
    imaginary components (the field viewed as a real vector of length 2 N0)."""
    e = np.concatenate([err.real, err.imag])
    a = np.concatenate([y.real, y.imag])
    b = np.concatenate([y_new.real, y_new.imag])
    sc = atol + rtol * np.maximum(np.abs(a), np.abs(b))
    return float(np.sqrt(np.mean((e / sc) ** 2)))


def dopri5(ops: Operators, p, psi0: np.ndarray, z_end: float, rtol=1e-9, atol=1e-11, h0=0.0, sigma=None,
           kerr="lumped", max_steps=10_000_000):
    """Adaptive Dormand-Prince integration of Eq. 10 from z = 0 to z_end.

    Step control: accept when the RMS error norm E <= 1; the next step is
    h * min(10, 0.9 E^(-1/5)) after an accept (no growth right after a
    rejection) and h * max(0.2, 0.9 E^(-1/5)) after a reject.  h0 = 0 picks
    the first step as 0.01 * ||y|| / ||f(y)|| (RMS norms scaled as above),
    limited by the fifth-root rule on a trial Euler step.
    Returns (psi(z_end), stats dict)."""
    y = np.array(psi0, dtype=np.complex128, copy=True)
    f = lambda v: dec_rhs(ops, p, v, sigma, kerr)
    k1 = f(y)
    n_rhs = 1
    if h0 <= 0.0:
        sc = atol + rtol * np.abs(np.concatenate([y.real, y.imag]))
        d0 = float(np.sqrt(np.mean((np.concatenate([y.real, y.imag]) / sc) ** 2)))
        d1 = float(np.sqrt(np.mean((np.concatenate([k1.real, k1.imag]) / sc) ** 2)))
        h_try = 1e-6 if (d0 < 1e-5 or d1 < 1e-5) else 0.01 * d0 / d1
        y1 = y + h_try * k1
        k_try = f(y1)
        n_rhs += 1
        d2 = float(np.sqrt(np.mean((np.concatenate([(k_try - k1).real, (k_try - k1).imag]) / sc) ** 2))) / h_try
        h1 = max(1e-6, h_try * 1e-3) if max(d1, d2) <= 1e-15 else (0.01 / max(d1, d2)) ** (1 / 5)
        h = min(100 * h_try, h1)
    else:
        h = h0
    z = 0.0
    h_last = 0.0
    n_acc = n_rej = 0
    while z < z_end and n_acc + n_rej < max_steps:
        h = min(h, z_end - z)
        rejected = False
        while True:
            ks = [k1]
            for s in range(1, 7):
                ys = y + h * sum(a * k for a, k in zip(DP_A[s], ks))
                ks.append(f(ys))
                n_rhs += 1
            y_new = ys                                   # stage 7 input is the 5th-order solution
            err = h * sum(e * k for e, k in zip(DP_E, ks))
            E = _rms_error(err, y, y_new, rtol, atol)
            if E <= 1.0:
                factor = 10.0 if E == 0.0 else min(10.0, 0.9 * E ** (-0.2))
                if rejected:
                    factor = min(1.0, factor)
                z = z + h
                y = y_new
                k1 = ks[6]
                n_acc += 1
                h_last = h
                h = h * factor
                break
            n_rej += 1
            rejected = True
            h = h * max(0.2, 0.9 * E ** (-0.2))
    return y, {"n_accepted": n_acc, "n_rejected": n_rej, "n_rhs": n_rhs, "h_last": h_last}


# --------------------------------------------------------------------------
# discrete soliton: self-consistent nonlinear eigenmode
# --------------------------------------------------------------------------
def soliton_operator(ops: Operators, p, phi: np.ndarray, kerr="lumped") -> sp.csr_matrix:
    """*0 H(phi) with H(phi) = p1 A - diag(v + N(|phi|^2)): the generator of
    Eq. 10 with the nonlinearity frozen at phi, so that a stationary field
    psi(z) = phi e^{-i mu z} solves  H(phi) phi = mu phi.  Multiplied by *0 it
    is a symmetric matrix (K symmetric, *0 diagonal): the generalized
    eigenproblem  (*0 H) phi = mu *0 phi  is symmetric-definite."""
    if len(p) != 1:
        raise ValueError("the soliton solver takes p_1 only")
    I = np.abs(phi) ** 2
    if kerr == "lumped":
        Nr = ops.chib * I
    else:
        Nr = (sp.diags(1.0 / ops.H0) @ ops.QtDQ) @ I
    return (p[0] * ops.K - sp.diags(ops.H0 * (ops.v + Nr))).tocsr()


def soliton(ops: Operators, p, power: float, phi0=None, kerr="lumped", tol=1e-12, max_iter=500, mix=0.5):
    """Fundamental discrete soliton of power P = sum_p m_p |phi_p|^2 (the
    paper's self-consistent nonlinear eigenmode, Supp. Note 4, whose text is
    not available): repeat
        mu, u <- lowest eigenpair of (*0 H(phi)) u = mu *0 u   (scipy eigsh)
        u     <- u scaled to power P, sign fixed by sum m u > 0
        phi   <- u  (with the intensity entering H mixed:  I <- mix |u|^2 + (1 - mix) I)
    until the intensity changes by less than tol (relative, *0-weighted).
    The start is phi0 if given, else the linear fundamental mode (which is
    localized only where the potential traps it: a homogeneous medium needs
    a localized phi0).  Returns (phi (real), mu, iterations)."""
    from scipy.sparse.linalg import eigsh

    M = sp.diags(ops.H0).tocsc()
    n = ops.n0

    def lowest(Hm, guess):
        vals, vecs = eigsh(Hm.tocsc(), k=1, M=M, sigma=guess, which="LM", tol=1e-14, v0=None)
        return float(vals[0]), vecs[:, 0]

    def scaled(u):
        u = np.asarray(u, dtype=np.float64)
        u = u * math.sqrt(power / float(np.sum(ops.H0 * u * u)))
        return u if float(np.sum(ops.H0 * u)) >= 0 else -u

    # start: the linear fundamental mode (or the given guess)
    if phi0 is None:
        H_lin = (p[0] * ops.K - sp.diags(ops.H0 * ops.v)).tocsr()
        lo = float(np.min(-ops.v)) - 1.0
        _, u = lowest(H_lin, lo)
        phi = scaled(u)
    else:
        phi = scaled(np.real(phi0))
    I = phi * phi
    mu = None
    for it in range(1, max_iter + 1):
        Hm = soliton_operator(ops, p, np.sqrt(I), kerr)
        shift = float(np.min(-(ops.v + (ops.chib * I if kerr == "lumped" else
                                         (sp.diags(1.0 / ops.H0) @ ops.QtDQ) @ I)))) - 1.0
        mu, u = lowest(Hm, shift)
        phi_new = scaled(u)
        I_new = mix * phi_new ** 2 + (1.0 - mix) * I
        change = math.sqrt(float(np.sum(ops.H0 * (I_new - I) ** 2)) / float(np.sum(ops.H0 * I ** 2)))
        I, phi = I_new, phi_new
        if change < tol:
            break
    # final eigenpair at the converged intensity
    Hm = soliton_operator(ops, p, phi, kerr)
    shift = float(np.min(-(ops.v + (ops.chib * phi ** 2 if kerr == "lumped" else
                                     (sp.diags(1.0 / ops.H0) @ ops.QtDQ) @ (phi ** 2))))) - 1.0
    mu, u = lowest(Hm, shift)
    return scaled(u), mu, it


def soliton_residual(ops: Operators, p, phi: np.ndarray, mu: float, kerr="lumped") -> float:
    """|| H(phi) phi - mu phi ||_*0 / ||phi||_*0."""
    Hm = soliton_operator(ops, p, phi, kerr)
    r = Hm @ phi / ops.H0 - mu * phi
    return math.sqrt(float(np.sum(ops.H0 * np.abs(r) ** 2)) / float(np.sum(ops.H0 * np.abs(phi) ** 2)))
