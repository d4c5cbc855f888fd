"""Pins of the oracle's discrete adjoint: central finite differences of the
(pinned) forward march, for the input field and for a per-vertex potential
offset, and the inner-product identity of the linear step."""
import numpy as np
import pytest

from oracle import bpm, dec
from paper_2608_03587_b300 import workloads as W


@pytest.fixture(scope="module")
def setup():
    coords, tris = W.mesh_disk_graded(2.5, 400, 2.0, interfaces=(1.0,), seed=13, grade_from=1.0)
    V, chi = W.step_index_materials(coords, tris, V_clad=-6.0, chi_clad=0.6)
    ops = dec.Operators(coords, tris, V, chi)
    sigma = W.absorber_profile(coords, 2.5, 8.0)
    psi0 = W.elliptic_gaussian(coords, A=2.2, wx=0.7, wy=0.4)
    phi = W.gaussian(coords, w=0.6) * np.exp(0.3j)
    return ops, sigma, psi0, phi


def _J(ops, sigma, psi0, phi, h, n, dv=None):
    v0 = ops.v.copy()
    if dv is not None:
        ops.v = v0 + dv
    try:
        out = bpm.propagate(ops, (1.0,), psi0, h, n, sigma)
    finally:
        ops.v = v0
    return bpm.overlap_objective(ops, phi, out)[0]


def test_adjoint_gradient_wrt_input_field(setup):
    ops, sigma, psi0, phi = setup
    h, n = 4e-3, 6
    out = bpm.propagate(ops, (1.0,), psi0, h, n, sigma)
    J, G = bpm.overlap_objective(ops, phi, out)
    g0, gv = bpm.vjp(ops, (1.0,), psi0, G, h, n, sigma)
    rng = np.random.default_rng(1)
    for _ in range(3):
        d = rng.standard_normal(ops.n0) + 1j * rng.standard_normal(ops.n0)
        eps = 1e-6
        fd = (_J(ops, sigma, psi0 + eps * d, phi, h, n) - _J(ops, sigma, psi0 - eps * d, phi, h, n)) / (2 * eps)
        ad = np.real(np.sum(np.conj(g0) * d))
        assert ad == pytest.approx(fd, rel=1e-7, abs=1e-12 * abs(J))


def test_adjoint_gradient_wrt_potential(setup):
    ops, sigma, psi0, phi = setup
    h, n = 4e-3, 6
    out = bpm.propagate(ops, (1.0,), psi0, h, n, sigma)
    J, G = bpm.overlap_objective(ops, phi, out)
    _, gv = bpm.vjp(ops, (1.0,), psi0, G, h, n, sigma)
    rng = np.random.default_rng(2)
    idx = rng.choice(ops.n0, 6, replace=False)
    idx = np.concatenate([idx, [int(np.argmax(np.abs(psi0)))]])
    for p in idx:
        e = np.zeros(ops.n0)
        e[p] = 1.0
        eps = 1e-5
        fd = (_J(ops, sigma, psi0, phi, h, n, eps * e) - _J(ops, sigma, psi0, phi, h, n, -eps * e)) / (2 * eps)
        assert gv[p] == pytest.approx(fd, rel=1e-6, abs=1e-7 * np.max(np.abs(gv)))


def test_linear_step_adjoint_identity(setup):
    """<y, E x> = <E^H y, x> (Euclidean) with E^H = *0 E_{-h} *0^{-1}."""
    ops, _, _, _ = setup
    rng = np.random.default_rng(3)
    x = rng.standard_normal(ops.n0) + 1j * rng.standard_normal(ops.n0)
    y = rng.standard_normal(ops.n0) + 1j * rng.standard_normal(ops.n0)
    Ex = bpm.linear_step(ops, (1.0, 1e-4), x, 5e-3)
    EHy = ops.H0 * bpm.linear_step(ops, (1.0, 1e-4), y / ops.H0, -5e-3)
    assert np.vdot(y, Ex) == pytest.approx(np.vdot(EHy, x), rel=1e-12)
