"""Pins of the oracle's complex-stretched PML operators (radial exterior
complex scaling of the Hodge stars)."""
import numpy as np
import pytest
import scipy.linalg as sla
import scipy.sparse as sp

from oracle import bpm, dec, pml
from paper_2608_03587_b300 import workloads as W


@pytest.fixture(scope="module")
def fiber():
    coords, tris = W.mesh_disk_graded(4.0, 700, 3.0, interfaces=(1.0,), seed=9, grade_from=1.0)
    V, chi = W.step_index_materials(coords, tris)
    return coords, tris, V, chi


def test_zero_stretch_is_the_plain_operator(fiber):
    coords, tris, V, chi = fiber
    plain = dec.Operators(coords, tris, V, chi)
    st = pml.StretchedOperators(coords, tris, V, chi, r_in=3.0, R=4.0, sigma_max=0.0)
    assert abs(st.A - plain.A).max() < 1e-12 * abs(plain.A).max()
    assert np.max(np.abs(st.v - plain.v)) < 1e-12 * np.max(np.abs(plain.v))
    assert np.max(np.abs(st.chib - plain.chib)) < 1e-14


def test_whitney_star_equals_tensor_stiffness(fiber):
    """d0^T *1~ d0 with the Lambda-weighted Whitney inner product is the P1
    stiffness with Lambda (the gradient of a P1 field is the Whitney
    interpolant of its d0); complex symmetric with zero row sums."""
    coords, tris, V, chi = fiber
    st = pml.StretchedOperators(coords, tris, V, chi, r_in=2.5, R=4.0, sigma_max=3.0, order=2)
    Lam, _ = pml.stretch(coords, tris, r_in=2.5, R=4.0, sigma_max=3.0, order=2)
    Kd = pml.stiffness(coords, tris, Lam)
    assert abs(st.K - Kd).max() < 1e-12 * abs(Kd).max()
    assert abs(st.K - st.K.T).max() < 1e-12 * abs(Kd).max()
    assert np.max(np.abs(st.K @ np.ones(st.n0))) < 1e-12 * abs(Kd).max()
    assert abs(st.K.imag).max() > 1e-3 * abs(st.K.real).max()        # really stretched


def test_uniform_complex_scaling_divides_by_s_squared(fiber):
    """Stretching every radius by the same s (r~ = s r) leaves Lambda = I and
    makes J = s^2: the operator is exactly A / s^2."""
    coords, tris, V, chi = fiber
    s = 1.0 + 0.3j
    plain = dec.Operators(coords, tris, V, chi)
    st = pml.StretchedOperators(coords, tris, V, chi, r_in=0.0, R=4.0, sigma_max=0.3, order=0)
    assert abs(st.A - plain.A / s ** 2).max() < 1e-12 * abs(plain.A).max()


def test_exterior_scaling_keeps_the_guided_mode_and_damps_the_rest(fiber):
    """Bound states are invariant under exterior complex scaling beyond the
    mode's reach: the LP01 eigenvalue of p1 A - v stays put, while the
    radiation continuum moves into the lower half-plane (damped modes of
    i dpsi/dz = (p1 A - v) psi)."""
    coords, tris, V, chi = fiber
    plain = dec.Operators(coords, tris, V, chi)
    st = pml.StretchedOperators(coords, tris, V, chi, r_in=3.0, R=4.0, sigma_max=2.0, order=2)
    Hp = (plain.K - sp.diags(plain.H0 * plain.v)).toarray()
    lam_p = sla.eigh(Hp, np.diag(plain.H0), eigvals_only=True)
    Hs = (st.K - sp.diags(st.H0s * st.v)).toarray()
    lam_s = sla.eig(Hs, np.diag(st.H0s), right=False)
    ground_s = lam_s[np.argmin(lam_s.real)]
    assert abs(ground_s - lam_p[0]) < 1e-6 * abs(lam_p[0])
    assert np.min(lam_s.imag) < -1e-2 * np.max(np.abs(lam_s))       # the layer does damp
    # the radiation continuum (above the cladding cutoff V#^2) is damped; guided
    # modes keep real eigenvalues up to a discretization error that grows
    # with the part of their evanescent tail inside the layer (largest just
    # below cutoff) and stays far below the layer's damping
    V0 = -W.FIBER_V_CLAD
    scale = np.max(np.abs(lam_s))
    assert np.max(lam_s.imag[lam_s.real > V0 + 0.5]) < 1e-9 * scale
    assert np.all(lam_s.real[lam_s.imag > 1e-9 * scale] < V0)
    assert np.max(lam_s.imag) < 1e-4 * scale


def test_layer_absorbs_an_outgoing_beam():
    """A Gaussian with transverse momentum k = 4 leaves the centre towards the
    rim (linear, no absorber).  On a disk of radius 4 with Neumann walls it
    comes back; with the PML (r > 3, sigma_max = 4, quadratic) it leaves.  At
    z = 0.7 the field inside r < 2.5 is compared with the same launch on a
    disk of radius 8 (same resolution), from which nothing has returned:
    error relative to the launch norm 0.66 with walls, 0.015 with the layer
    (the remainder is the meshes' own difference: it halves with 2x the
    vertices)."""
    from scipy.interpolate import LinearNDInterpolator

    def run(R, n, pml_kw=None):
        coords, tris = W.mesh_disk_graded(R, n, 1.0, seed=3)
        V, chi = np.zeros(len(tris)), np.zeros(len(tris))
        ops = (dec.Operators(coords, tris, V, chi) if pml_kw is None
               else pml.StretchedOperators(coords, tris, V, chi, **pml_kw))
        x, y = coords[:, 0], coords[:, 1]
        psi0 = np.exp(-((x + 0.5) ** 2 + y ** 2) / 0.5 + 4.0j * x).astype(complex)
        out, _ = bpm.dopri5(ops, (1.0,), psi0, 0.7, rtol=1e-8, atol=1e-10)
        return coords, out, psi0, ops

    cb, big, _, _ = run(8.0, 16000)
    errs = {}
    for name, kw in (("neumann", None), ("pml", dict(r_in=3.0, R=4.0, sigma_max=4.0, order=2))):
        cs, small, psi0, ops = run(4.0, 4000, kw)
        ref = LinearNDInterpolator(cb, big)(cs[:, 0], cs[:, 1])
        inner = np.hypot(cs[:, 0], cs[:, 1]) < 2.5
        w = ops.H0[inner]
        errs[name] = np.sqrt(np.sum(w * np.abs(small[inner] - ref[inner]) ** 2) / np.sum(ops.H0 * np.abs(psi0) ** 2))
    assert errs["neumann"] > 0.3, errs
    assert errs["pml"] < 0.03 and errs["pml"] < 0.05 * errs["neumann"], errs


def test_stretched_diagonal_flow_matches_ode_integration(fiber):
    """The exact flow with complex lumped v and chib (Bernoulli equation for
    the intensity, closed-form phase integral) against DOP853 on the vertex
    ODE dpsi/dz = i (v + chib |psi|^2) psi - sigma psi, with damping and
    gaining imaginary parts and an absorber; and equal to bpm.diagonal_flow
    when the coefficients are real."""
    from scipy.integrate import solve_ivp
    coords, tris, V, chi = fiber
    ops = pml.StretchedOperators(coords, tris, V, chi, r_in=3.0, R=4.0, sigma_max=2.0, order=2)
    rng = np.random.default_rng(5)
    n = 12
    idx = rng.choice(ops.n0, n, replace=False)
    class Fake:
        pass
    f = Fake()
    f.n0 = n
    f.v = rng.uniform(-8, 3, n) + 1j * rng.uniform(-0.5, 2.0, n)
    f.chib = rng.uniform(0.2, 1.5, n) + 1j * rng.uniform(-0.05, 0.4, n)
    sigma = np.where(rng.random(n) < 0.5, rng.uniform(0.0, 5.0, n), 0.0)
    psi = (rng.standard_normal(n) + 1j * rng.standard_normal(n)) * 1.2
    h = 0.09
    out = pml.diagonal_flow_stretched(f, psi, h, sigma)
    for p in range(n):
        def rhs(_z, y, p=p):
            c = y[0] + 1j * y[1]
            d = 1j * (f.v[p] + f.chib[p] * abs(c) ** 2) * c - sigma[p] * c
            return [d.real, d.imag]
        sol = solve_ivp(rhs, (0, h), [psi[p].real, psi[p].imag], method="DOP853", rtol=1e-13, atol=1e-15)
        ref = sol.y[0, -1] + 1j * sol.y[1, -1]
        assert abs(out[p] - ref) <= 1e-10 * abs(psi[p]), p
    plain = dec.Operators(coords, tris, V, chi)
    psi2 = (rng.standard_normal(plain.n0) + 1j * rng.standard_normal(plain.n0)) * 1.5
    sig2 = W.absorber_profile(coords, 4.0, 6.0)
    a = pml.diagonal_flow_stretched(plain, psi2, 0.05, sig2)
    b = bpm.diagonal_flow(plain, psi2, 0.05, sig2)
    assert np.max(np.abs(a - b)) <= 1e-14 * np.max(np.abs(psi2))
    _ = idx


def test_split_step_with_layer_converges_to_the_rk45_integration(fiber):
    """The Strang march on the stretched operators converges at second order
    in dz to the oracle's Dormand-Prince integration of the same equation
    with the layer (linear and Kerr launches)."""
    coords, tris, V, chi = fiber
    ops = pml.StretchedOperators(coords, tris, V, chi, r_in=3.0, R=4.0, sigma_max=4.0, order=2)
    x, y = coords[:, 0], coords[:, 1]
    psi0 = 2.0 * np.exp(-((x - 0.3) ** 2 + y ** 2) / 0.5 + 3.0j * x)
    z = 0.02
    ref, _ = bpm.dopri5(ops, (1.0,), psi0, z, rtol=1e-12, atol=1e-14)
    errs = []
    for n in (10, 20, 40):
        out = pml.propagate_stretched(ops, (1.0,), psi0, z / n, n)
        errs.append(bpm.relative_error(ops, out, ref))
    assert errs[-1] < 1e-4
    for e1, e2 in zip(errs, errs[1:]):
        assert 3.3 < e1 / e2 < 4.8, errs


def test_split_step_with_layer_on_several_fields_is_each_field_alone(fiber):
    """The fields of a [vertex, field] array march independently: the march
    on three fields at once (Taylor action on the block, flow per element)
    equals the march of each field alone, so the GPU tests can hold a
    multi-field run against one oracle call."""
    coords, tris, V, chi = fiber
    ops = pml.StretchedOperators(coords, tris, V, chi, r_in=3.0, R=4.0, sigma_max=4.0, order=2)
    x, y = coords[:, 0], coords[:, 1]
    psi0 = np.stack([a * np.exp(-((x - x0) ** 2 + y ** 2) / 0.5 + 1j * k * x)
                     for a, x0, k in ((2.0, 0.3, 3.0), (0.5, -0.2, -1.0), (1.2, 0.0, 4.0))], axis=1)
    block = pml.propagate_stretched(ops, (1.0,), psi0, 1e-3, 12)
    for f in range(3):
        alone = pml.propagate_stretched(ops, (1.0,), psi0[:, f], 1e-3, 12)
        assert bpm.relative_error(ops, block[:, f], alone) <= 1e-13, f
