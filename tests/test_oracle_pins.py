"""Pins of the CPU oracle against what the paper and the mathematics fix.

Each test ties an oracle function to something other than itself: exact
identities of the DEC operators, closed-form solutions, textbook eigenvalues,
dense brute force, an independent ODE integrator, conservation laws and
convergence orders.  A plausible slip in the oracle (a dropped term, a wrong
sign, a swapped index, a wrong Hodge factor) fails at least one of them.
"""
import json
import math
import os

import numpy as np
import pytest
import scipy.linalg as sla
import scipy.sparse as sp
import scipy.sparse.linalg as spla
from scipy.integrate import solve_ivp
from scipy.spatial import ConvexHull, Delaunay
from scipy.special import jnp_zeros

from oracle import bpm, dec
from paper_2608_03587_b300 import workloads as W

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


# ---------------------------------------------------------------- fixtures
@pytest.fixture(scope="module")
def fiber_small():
    coords, tris = W.mesh_disk_graded(4.0, 1500, 3.0, interfaces=(1.0,), seed=7, grade_from=1.0)
    V, chi = W.step_index_materials(coords, tris)
    return coords, tris, V, chi


@pytest.fixture(scope="module")
def fiber_ops(fiber_small):
    coords, tris, V, chi = fiber_small
    return dec.Operators(coords, tris, V, chi)


@pytest.fixture(scope="module")
def tiny():
    """<= 500 vertices: small enough for dense matrix exponentials."""
    coords, tris = W.mesh_disk_graded(2.0, 300, 2.0, interfaces=(1.0,), seed=9, grade_from=1.0)
    V, chi = W.step_index_materials(coords, tris, V_clad=-8.0, chi_clad=0.5)
    sigma = W.absorber_profile(coords, 2.0, 5.0)
    return dec.Operators(coords, tris, V, chi), sigma


def boundary_vertices(tris, n0):
    e = np.sort(np.concatenate([tris[:, [0, 1]], tris[:, [1, 2]], tris[:, [2, 0]]]), axis=1)
    uniq, cnt = np.unique(e, axis=0, return_counts=True)
    b = np.zeros(n0, dtype=bool)
    b[uniq[cnt == 1].ravel()] = True
    return b


# ------------------------------------------------------ topology / d^2 = 0
def test_d1_d0_is_exactly_zero(fiber_small):
    """d1 d0 = 0 holds exactly (the discrete d^2 = 0 of Sec. 'Conceptual
    framework' / Table I), with integer arithmetic."""
    coords, tris, _, _ = fiber_small
    E = dec.edges(tris)
    D0 = dec.d0(E, len(coords))
    D1 = dec.d1(tris, E)
    assert (abs(D1 @ D0)).max() == 0
    # each edge row has one head (+1) and one tail (-1); each triangle row three edges
    assert np.all(np.asarray(D0.sum(axis=1)).ravel() == 0)
    assert np.all(np.asarray(abs(D0).sum(axis=1)).ravel() == 2)
    assert np.all(np.asarray(abs(D1).sum(axis=1)).ravel() == 3)
    # Euler characteristic of a disk: V - E + F = 1
    assert len(coords) - len(E) + len(tris) == 1


def test_d1_d0_zero_on_pcf():
    coords, tris, _ = W.mesh_pcf(4000)
    E = dec.edges(tris)
    assert (abs(dec.d1(tris, E) @ dec.d0(E, len(coords)))).max() == 0


def test_d0_orientation_head_minus_tail():
    """(d0 psi)_e = psi(v_b) - psi(v_a) for edge [v_a, v_b], a < b."""
    tris = np.array([[0, 1, 2], [2, 1, 3]])
    E = dec.edges(tris)
    psi = np.array([1.0, 10.0, 100.0, 1000.0])
    out = dec.d0(E, 4) @ psi
    expect = {(0, 1): 9.0, (0, 2): 99.0, (1, 2): 90.0, (1, 3): 990.0, (2, 3): 900.0}
    for (a, b), val in zip(E, out):
        assert val == expect[(int(a), int(b))]


# --------------------------------------------------------------- Hodge stars
def test_star0_partitions_area(fiber_small):
    coords, tris, V, _ = fiber_small
    m = dec.star0(coords, tris)
    assert m.sum() == pytest.approx(ConvexHull(coords).volume, rel=1e-12)
    # *0(V) carries the integral of the piecewise-constant V
    mv = dec.star0(coords, tris, V)
    assert mv.sum() == pytest.approx(np.sum(V * dec.cell_measures(coords, tris)), rel=1e-12)


def test_star0_1d_partitions_length():
    x, cells = W.mesh_1d_jittered(64, seed=3)
    assert dec.star0(x, cells).sum() == pytest.approx(40.0, rel=1e-14)


def test_galerkin_star1_gives_cotangent_stiffness(fiber_small):
    """d0^T *1 d0 with the Galerkin (Whitney) *1 of Eq. 9 (xi = 1) equals the
    cotangent stiffness d0^T diag(w) d0, w_e = (1/2) sum cot(opposite angle),
    assembled here by a separate formula.  *1 itself is not diagonal."""
    coords, tris, _, _ = fiber_small
    n0 = len(coords)
    E = dec.edges(tris)
    D0 = dec.d0(E, n0)
    H1 = dec.galerkin_star1(coords, tris, E)
    K_gal = (D0.T @ H1 @ D0).tocsr()
    rows, cols, vals = [], [], []
    for i in range(3):
        a, b, c = tris[:, i], tris[:, (i + 1) % 3], tris[:, (i + 2) % 3]
        u = coords[b] - coords[a]
        v = coords[c] - coords[a]
        cot = (u * v).sum(1) / np.abs(u[:, 0] * v[:, 1] - u[:, 1] * v[:, 0])
        w = 0.5 * cot                              # angle at a is opposite edge (b, c)
        rows += [b, c, b, c]
        cols += [c, b, b, c]
        vals += [-w, -w, w, w]
    K_cot = sp.csr_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))), shape=(n0, n0))
    diff = abs(K_gal - K_cot).max()
    assert diff <= 1e-12 * abs(K_cot).max()
    offdiag = H1 - sp.diags(H1.diagonal())
    assert abs(offdiag).max() > 0.01 * abs(H1).max()


def test_stiffness_annihilates_constants_and_linears(fiber_ops, fiber_small):
    coords, tris, _, _ = fiber_small
    K = fiber_ops.K
    scale = abs(K).max()
    assert np.max(np.abs(K @ np.ones(len(coords)))) <= 1e-13 * scale
    interior = ~boundary_vertices(tris, len(coords))
    for col in range(2):
        r = K @ coords[:, col]
        assert np.max(np.abs(r[interior])) <= 1e-12 * scale * 4.0
    # K is symmetric (to rounding of the summation order) and positive semi-definite
    assert abs(K - K.T).max() <= 1e-15 * scale
    assert np.linalg.eigvalsh(0.5 * (K + K.T).toarray()).min() > -1e-12 * scale


def test_1d_quadratic_exact():
    """-A x^2 = (x^2)'' = 2 at every interior node of a jittered 1D mesh."""
    x, cells = W.mesh_1d_jittered(200, seed=4)
    ops = dec.Operators(x, cells)
    r = ops.A @ (x[:, 0] ** 2)
    assert np.max(np.abs(r[1:-1] + 2.0)) < 1e-9


def test_2d_equilateral_quadratic_exact():
    """On a uniform equilateral mesh -A (x^2+y^2) = lap(x^2+y^2) = 4 at every
    interior vertex."""
    h = 0.1
    pts = []
    for j in range(-15, 16):
        for i in range(-15, 16):
            pts.append((h * (i + 0.5 * (j % 2)), h * math.sqrt(3) / 2 * j))
    pts = np.array(pts)
    tris = Delaunay(pts).simplices.astype(np.int64)
    P = pts[tris]
    cross = (P[:, 1, 0] - P[:, 0, 0]) * (P[:, 2, 1] - P[:, 0, 1]) - (P[:, 1, 1] - P[:, 0, 1]) * (P[:, 2, 0] - P[:, 0, 0])
    tris[cross < 0] = tris[cross < 0][:, [0, 2, 1]]
    ops = dec.Operators(pts, tris)
    r = ops.A @ (pts[:, 0] ** 2 + pts[:, 1] ** 2)
    # vertices well inside the lattice patch (the hull of the zigzag patch
    # adds obtuse triangles along its rim)
    interior = (np.abs(pts[:, 0]) < 1.2) & (np.abs(pts[:, 1]) < 1.1)
    assert interior.sum() > 400
    assert np.max(np.abs(r[interior] + 4.0)) < 1e-9


def test_neumann_eigenvalue_converges_second_order():
    """Lowest nonzero eigenvalue of K phi = lambda *0 phi on the unit disk
    tends to the Neumann eigenvalue (j'_{1,1})^2 at O(h^2)."""
    exact = jnp_zeros(1, 1)[0] ** 2
    errs, ns = [], []
    for n in (600, 2400, 9600):
        coords, tris = W.mesh_disk_graded(1.0, n, 1.0, seed=21)
        ops = dec.Operators(coords, tris)
        vals = spla.eigsh(ops.K, k=3, M=sp.diags(ops.H0), sigma=-1e-3, which="LM",
                          return_eigenvectors=False)
        lam = np.sort(vals)[1]
        errs.append(abs(lam - exact))
        ns.append(ops.n0)
    orders = [-2 * math.log(errs[i + 1] / errs[i]) / math.log(ns[i + 1] / ns[i]) for i in range(2)]
    assert errs[-1] < 2e-3 * exact
    assert all(1.6 < o < 2.6 for o in orders), (errs, orders)


def test_free_gaussian_beam_second_order_in_h():
    """Linear diffraction (p1 = 1, V = chi = 0) of a Gaussian beam has the
    closed form psi = exp(-r^2/(w^2 q))/q, q = 1 + 4 i z / w^2; the DEC march
    converges to it at O(h^2) (the second-order accuracy the paper reports)."""
    z, w = 0.05, 0.8

    def exact(c, zz):
        q = 1 + 4j * zz / w ** 2
        return np.exp(-(c[:, 0] ** 2 + c[:, 1] ** 2) / (w ** 2 * q)) / q

    errs, ns = [], []
    for n in (500, 2000, 8000):
        coords, tris = W.mesh_disk_graded(4.0, n, 1.0, seed=11)
        nt = len(tris)
        ops = dec.Operators(coords, tris, np.zeros(nt), np.zeros(nt))
        out = bpm.propagate(ops, (1.0,), exact(coords, 0.0), z / 10, 10)
        errs.append(bpm.relative_error(ops, out, exact(coords, z)))
        ns.append(ops.n0)
    orders = [-2 * math.log(errs[i + 1] / errs[i]) / math.log(ns[i + 1] / ns[i]) for i in range(2)]
    assert all(1.7 < o < 2.4 for o in orders), (errs, orders)
    assert errs[-1] < 3e-3


# ------------------------------------------------------- linear propagator
@pytest.mark.parametrize("p", [(1.0,), (0.5,), (1.0, 2e-3), (1.0, 0.0, 1e-6)])
def test_linear_step_matches_dense_expm(tiny, p):
    """Taylor-substep action vs the dense exponential exp(i h sum p_n (-A)^n)."""
    ops, _ = tiny
    A = ops.A.toarray()
    G = np.zeros_like(A)
    Ak = np.eye(len(A))
    for pn in p:
        Ak = Ak @ (-A)
        G = G + pn * Ak
    rng = np.random.default_rng(0)
    psi = rng.standard_normal(ops.n0) + 1j * rng.standard_normal(ops.n0)
    h = 3e-3
    ref = sla.expm(1j * h * G) @ psi
    out = bpm.linear_step(ops, p, psi, h)
    assert np.linalg.norm(out - ref) <= 1e-12 * np.linalg.norm(ref)


def test_linear_step_is_star0_unitary(tiny):
    ops, _ = tiny
    rng = np.random.default_rng(1)
    psi = rng.standard_normal(ops.n0) + 1j * rng.standard_normal(ops.n0)
    out = bpm.linear_step(ops, (1.0,), psi, 0.01)
    assert bpm.power(ops, out) == pytest.approx(bpm.power(ops, psi), rel=1e-13)


# ----------------------------------------------------------- diagonal flow
def test_diagonal_flow_matches_ode_integration(tiny):
    """Closed-form flow of dpsi/dz = i (v + chib|psi|^2) psi - sigma psi vs
    an independent high-order ODE integration, vertex by vertex."""
    ops, _ = tiny
    rng = np.random.default_rng(2)
    idx = rng.choice(ops.n0, 12, replace=False)
    sigma = np.zeros(ops.n0)
    sigma[idx[:6]] = rng.uniform(0.5, 40.0, 6)
    psi = (rng.standard_normal(ops.n0) + 1j * rng.standard_normal(ops.n0)) * 1.5
    h = 0.07
    out = bpm.diagonal_flow(ops, psi, h, sigma)
    for p in idx:
        def rhs(_z, y, p=p):
            c = y[0] + 1j * y[1]
            d = 1j * (ops.v[p] + ops.chib[p] * abs(c) ** 2) * c - sigma[p] * c
            return [d.real, d.imag]
        sol = solve_ivp(rhs, (0, h), [psi[p].real, psi[p].imag], method="DOP853", rtol=1e-13, atol=1e-15)
        ref = sol.y[0, -1] + 1j * sol.y[1, -1]
        assert abs(out[p] - ref) <= 1e-10 * max(abs(psi[p]), 1e-3)


def test_element_kerr_flow_with_absorber_matches_ode_integration(tiny):
    """Element-averaged Kerr (Eq. 14) together with the absorber: the closed
    form theta_p = v_p h + sum_q c_pq |psi_q(0)|^2 phi(sigma_q, h) against a
    DOP853 integration of the coupled vertex system
        dpsi_p/dz = i (v_p + N_p(|psi|^2)) psi_p - sigma_p psi_p,
        N_p = (1 / m_p) sum_{t ni p} chi_t |t| / 3 * (mean of |psi|^2 over t),
    with the triangle averaging written out here from the cells (not from the
    oracle's Q^T D Q), and absorbing rates that differ between neighbouring
    vertices, so that phi(sigma_p) in place of phi(sigma_q), a missing decay of
    the neighbours' intensity or a transposed coupling all fail."""
    ops, _ = tiny
    rng = np.random.default_rng(21)
    n0 = ops.n0
    tris = np.asarray(ops.cells)
    area = 0.5 * np.abs((ops.coords[tris[:, 1], 0] - ops.coords[tris[:, 0], 0])
                        * (ops.coords[tris[:, 2], 1] - ops.coords[tris[:, 0], 1])
                        - (ops.coords[tris[:, 1], 1] - ops.coords[tris[:, 0], 1])
                        * (ops.coords[tris[:, 2], 0] - ops.coords[tris[:, 0], 0]))
    m = np.zeros(n0)
    np.add.at(m, tris.ravel(), np.repeat(area / 3.0, 3))
    chi_t = np.asarray(ops.chi_cell)
    # strongly varying absorber: random rates on a third of the vertices
    sigma = np.where(rng.random(n0) < 0.35, rng.uniform(1.0, 30.0, n0), 0.0)
    psi = (rng.standard_normal(n0) + 1j * rng.standard_normal(n0)) * 1.3
    h = 0.05

    def rate(I):
        tmean = I[tris].mean(axis=1)
        out = np.zeros(n0)
        np.add.at(out, tris.ravel(), np.repeat(chi_t * area * tmean / 3.0, 3))
        return out / m

    def rhs(_z, y):
        c = y[:n0] + 1j * y[n0:]
        d = 1j * (ops.v + rate(np.abs(c) ** 2)) * c - sigma * c
        return np.concatenate([d.real, d.imag])

    sol = solve_ivp(rhs, (0, h), np.concatenate([psi.real, psi.imag]), method="DOP853", rtol=1e-12, atol=1e-14)
    ref = sol.y[:n0, -1] + 1j * sol.y[n0:, -1]
    out = bpm.diagonal_flow(ops, psi, h, sigma, kerr="element")
    assert np.max(np.abs(out - ref)) <= 1e-9 * np.max(np.abs(psi))
    # the absorber does change the answer here (the pin is not vacuous)
    plain = bpm.diagonal_flow(ops, psi, h, None, kerr="element")
    assert np.max(np.abs(plain - ref)) > 1e-2


def test_diagonal_flow_semigroup(tiny):
    ops, sigma = tiny
    rng = np.random.default_rng(3)
    psi = rng.standard_normal(ops.n0) + 1j * rng.standard_normal(ops.n0)
    a = bpm.diagonal_flow(ops, bpm.diagonal_flow(ops, psi, 0.02, sigma), 0.03, sigma)
    b = bpm.diagonal_flow(ops, psi, 0.05, sigma)
    assert np.max(np.abs(a - b)) < 1e-13


def test_element_kerr_consistency(fiber_ops):
    """Q (Eq. 13) averages vertex values over triangles (rows sum to 1) and
    Q^T D Q 1 = *0(chi) 1; for a uniform intensity the element-averaged Kerr
    rate of Eq. 14 equals the lumped one."""
    ops = fiber_ops
    Q = dec.projection_Q(ops.cells, dec.d1(ops.cells, ops.E), ops.D0)
    assert np.allclose(np.asarray(Q.sum(axis=1)).ravel(), 1.0, atol=1e-15)
    assert np.allclose(ops.QtDQ @ np.ones(ops.n0), ops.chib * ops.H0, rtol=1e-12)
    psi = np.full(ops.n0, 0.7 + 0.2j)
    a = bpm.diagonal_flow(ops, psi, 0.1, kerr="element")
    b = bpm.diagonal_flow(ops, psi, 0.1, kerr="lumped")
    assert np.max(np.abs(a - b)) < 1e-13


# ------------------------------------------------------------ whole march
def test_power_conserved_without_absorber(fiber_ops):
    rng = np.random.default_rng(4)
    ops = fiber_ops
    psi0 = W.elliptic_gaussian(ops.coords, A=2.0) + 0.1 * rng.standard_normal(ops.n0)
    out = bpm.propagate(ops, (1.0,), psi0, 2e-3, 40)
    assert bpm.power(ops, out) == pytest.approx(bpm.power(ops, psi0), rel=1e-12)


def test_absorber_only_removes_power(tiny):
    ops, sigma = tiny
    rng = np.random.default_rng(5)
    psi = rng.standard_normal(ops.n0) + 1j * rng.standard_normal(ops.n0)
    P = [bpm.power(ops, psi)]
    for _ in range(10):
        psi = bpm.strang_step(ops, (1.0,), psi, 5e-3, sigma)
        P.append(bpm.power(ops, psi))
    assert np.all(np.diff(P) < 0)


def test_hamiltonian_exact_for_linear_free_propagation(fiber_small):
    coords, tris, _, _ = fiber_small
    nt = len(tris)
    ops = dec.Operators(coords, tris, np.zeros(nt), np.zeros(nt))
    rng = np.random.default_rng(6)
    psi0 = W.elliptic_gaussian(coords) + 0.05 * (rng.standard_normal(ops.n0) + 1j * rng.standard_normal(ops.n0))
    H0 = bpm.hamiltonian(ops, (1.0,), psi0)
    out = bpm.propagate(ops, (1.0,), psi0, 3e-3, 20)
    assert bpm.hamiltonian(ops, (1.0,), out) == pytest.approx(H0, rel=1e-11)


def test_hamiltonian_error_is_second_order_in_dz(fiber_ops):
    """With Kerr and potential the split-step conserves H only up to O(dz^2):
    halving dz divides the largest deviation by about 4."""
    ops = fiber_ops
    psi0 = W.elliptic_gaussian(ops.coords, A=2.5)
    H0 = bpm.hamiltonian(ops, (1.0,), psi0)
    devs = []
    for dz in (4e-3, 2e-3):
        d = []
        bpm.propagate(ops, (1.0,), psi0, dz, int(round(0.04 / dz)),
                      callback=lambda n, psi: d.append(abs(bpm.hamiltonian(ops, (1.0,), psi) - H0)))
        devs.append(max(d))
    assert 3.3 < devs[0] / devs[1] < 4.8, devs


def test_strang_second_order_in_dz(fiber_ops):
    ops = fiber_ops
    psi0 = W.elliptic_gaussian(ops.coords, A=2.5)
    sigma = W.absorber_profile(ops.coords, 4.0, 10.0)
    z = 0.04
    ref = bpm.propagate(ops, (1.0,), psi0, z / 64, 64, sigma)
    e = [bpm.relative_error(ops, bpm.propagate(ops, (1.0,), psi0, z / n, n, sigma), ref) for n in (4, 8)]
    assert 3.5 < e[0] / e[1] < 4.6, e


def test_split_step_converges_to_paper_rk45(tiny):
    """The paper integrates the DEC ODE (Eq. 10, with V inside L as in Eq. 11)
    by adaptive RK45; the split-step march, which moves V to the diagonal
    step, converges to that solution at O(dz^2)."""
    ops, _ = tiny
    psi0 = W.elliptic_gaussian(ops.coords, A=2.0, wx=0.6, wy=0.3)
    z = 0.02
    ref = bpm.rk45_reference(ops, (1.0,), psi0, z)
    e = [bpm.relative_error(ops, bpm.propagate(ops, (1.0,), psi0, z / n, n), ref) for n in (4, 8, 16)]
    assert 3.5 < e[0] / e[1] < 4.5 and 3.5 < e[1] / e[2] < 4.5, e


def test_split_step_converges_to_paper_rk45_element_kerr(tiny):
    ops, _ = tiny
    psi0 = W.elliptic_gaussian(ops.coords, A=2.0, wx=0.6, wy=0.3)
    z = 0.02
    ref = bpm.rk45_reference(ops, (1.0,), psi0, z, kerr="element")
    e = [bpm.relative_error(ops, bpm.propagate(ops, (1.0,), psi0, z / n, n, kerr="element"), ref)
         for n in (4, 8)]
    assert 3.5 < e[0] / e[1] < 4.5, e


def test_exact_sech_soliton_1d():
    """i psi_z + psi_xx/2 + |psi|^2 psi = 0 has the exact solution
    sech(x) e^{iz/2}; on the jittered 1024-node mesh with dz = 1e-3 the march
    stays within O(h^2) of it, and the error falls ~4x when h halves."""
    errs = []
    for n in (512, 1024):
        wl = W.soliton_1d(n=n, seed=1)
        m = wl.meshes[0]
        ops = dec.Operators(m.coords, m.cells, m.V_cell, m.chi_cell)
        z, nst = 0.5, 500
        out = bpm.propagate(ops, wl.p, wl.psi0[0][:, 0], z / nst, nst)
        exact = W.sech_1d(m.coords) * np.exp(0.5j * z)
        errs.append(bpm.relative_error(ops, out, exact))
    assert errs[1] < 1e-4
    assert 3.0 < errs[0] / errs[1] < 5.0, errs


def test_multifield_equals_single_fields(tiny):
    ops, sigma = tiny
    rng = np.random.default_rng(8)
    psi = rng.standard_normal((ops.n0, 3)) + 1j * rng.standard_normal((ops.n0, 3))
    out = bpm.propagate(ops, (1.0,), psi, 2e-3, 3, sigma)
    for b in range(3):
        one = bpm.propagate(ops, (1.0,), psi[:, b], 2e-3, 3, sigma)
        assert np.max(np.abs(out[:, b] - one)) < 1e-14
    P = bpm.power(ops, psi)
    assert P.shape == (3,)
    assert P[1] == pytest.approx(bpm.power(ops, psi[:, 1]), rel=1e-15)


def test_error_metrics_on_known_cases(tiny):
    ops, _ = tiny
    rng = np.random.default_rng(9)
    psi = rng.standard_normal(ops.n0) + 1j * rng.standard_normal(ops.n0)
    assert bpm.relative_error(ops, psi, 2 * psi) == pytest.approx(0.5, rel=1e-14)
    assert bpm.intensity_error(ops, 2 * psi, psi) == pytest.approx(3.0, rel=1e-14)
    assert bpm.relative_error(ops, psi * np.exp(0.3j), psi) == pytest.approx(abs(np.exp(0.3j) - 1), rel=1e-13)


# ------------------------------------------------- the paper's constants
def test_table_II_normalization():
    """The workloads' normalization reproduces the paper's printed L_d and
    V-number from Table II: L_d = 2 k0 n_core R0^2, V = k0 R0 sqrt(n_core^2 - n_clad^2);
    the LP31 cutoff it quotes is the first zero of J_2."""
    from scipy.special import jn_zeros
    g = json.load(open(os.path.join(GOLDEN, "paper_constants.json")))
    t = g["table_II"]
    k0 = 2 * math.pi / t["wavelength_um"]
    Ld = 2 * k0 * t["n_core"] * t["core_radius_um"] ** 2
    assert Ld == pytest.approx(t["L_d_um"], abs=0.01)
    V = k0 * t["core_radius_um"] * math.sqrt(t["n_core"] ** 2 - t["n_clad"] ** 2)
    assert V == pytest.approx(g["fiber_V_number"]["V"], abs=0.005)
    assert W.FIBER_V_NUMBER == g["fiber_V_number"]["V"]
    assert jn_zeros(2, 1)[0] == pytest.approx(g["fiber_V_number"]["LP31_cutoff"], abs=0.005)
    assert W.FIBER_CHI_CLAD == pytest.approx(t["n2_clad"] / t["n2_core"])


def test_launch_fields_follow_paper_parameters():
    g = json.load(open(os.path.join(GOLDEN, "paper_constants.json")))
    eg = g["elliptic_gaussian_launch"]
    c = np.array([[eg["x0"], eg["y0"]], [eg["x0"] + eg["wx"] * math.cos(eg["theta"]),
                                          eg["y0"] + eg["wx"] * math.sin(eg["theta"])]])
    psi = W.elliptic_gaussian(c)
    assert psi[0] == pytest.approx(eg["A"])
    assert psi[1] == pytest.approx(eg["A"] * math.exp(-1.0))
    ev = g["elliptic_vortex_launch"]
    th = ev["theta"]
    c = np.array([[0.0, 0.0], [ev["wx"] * math.cos(th), ev["wx"] * math.sin(th)],
                  [-ev["wy"] * math.sin(th), ev["wy"] * math.cos(th)]])
    psi = W.elliptic_vortex(c)
    assert abs(psi[0]) == 0.0
    assert psi[1] == pytest.approx(math.exp(-1.0))            # rho = 1, Phi = 0
    assert psi[2] == pytest.approx(1j * math.exp(-1.0))       # rho = 1, Phi = pi/2


# ------------------------------------------------------- the paper's RK45
def test_dopri5_matches_scipy_rk45(tiny):
    """The oracle's Dormand-Prince integration of Eq. 10 agrees with scipy's
    solve_ivp RK45 (an independent implementation of the same method) to the
    tolerance level, and with the split-step march at small dz."""
    ops, _ = tiny
    psi0 = W.elliptic_gaussian(ops.coords, A=2.0, wx=0.6, wy=0.3)
    z = 0.01
    out, st = bpm.dopri5(ops, (1.0,), psi0, z, rtol=1e-10, atol=1e-12)
    ref = bpm.rk45_reference(ops, (1.0,), psi0, z, rtol=1e-10, atol=1e-12)
    assert bpm.relative_error(ops, out, ref) < 1e-8
    assert st["n_accepted"] > 10
    split = bpm.propagate(ops, (1.0,), psi0, z / 64, 64)
    assert bpm.relative_error(ops, out, split) < 1e-4
    # the error estimate behaves as a 5th-order method: tighter tolerance, more steps
    _, st2 = bpm.dopri5(ops, (1.0,), psi0, z, rtol=1e-12, atol=1e-14)
    assert st2["n_accepted"] > st["n_accepted"]


def test_dec_rhs_is_the_ode_of_the_split_step(tiny):
    """dec_rhs is the generator of both split pieces: for small h,
    (D_h E_h psi - psi)/h -> dec_rhs(psi)."""
    ops, sigma = tiny
    rng = np.random.default_rng(12)
    psi = W.elliptic_gaussian(ops.coords, A=1.5) + 0.1 * rng.standard_normal(ops.n0)
    f = bpm.dec_rhs(ops, (1.0,), psi, sigma)
    errs = []
    for h in (1e-5, 5e-6):
        step = bpm.strang_step(ops, (1.0,), psi, h, sigma)
        errs.append(np.linalg.norm((step - psi) / h - f) / np.linalg.norm(f))
    # first-order difference quotient: the error halves with h
    assert errs[1] < 2e-3 and 0.4 < errs[1] / errs[0] < 0.6


# ------------------------------------------------------------------ discrete soliton
def test_soliton_1d_converges_to_sech():
    """i psi_z + psi_xx/2 + |psi|^2 psi = 0: the fundamental soliton of power
    P is a sech(a x) with a = P/2 and mu = -P^2/8 (psi = phi e^{-i mu z}).
    The discrete self-consistent eigenmode reaches it at O(h^2): the
    eigenvalue error falls ~4x when h halves, for two powers (this pins the
    sign and the scale of the Kerr term against diffraction)."""
    for P in (2.0, 3.0):
        errs = []
        for n in (513, 1025):
            # a uniform, symmetric mesh: a homogeneous medium has a neutral
            # translation mode, which a jittered mesh would let drift
            coords, cells = W.mesh_1d_jittered(n, jitter=0.0)
            ne = len(cells)
            ops = dec.Operators(coords, cells, np.zeros(ne), np.ones(ne))
            # a localized start: from the constant (the linear ground state of
            # a homogeneous medium) the iteration stays uniform
            phi, mu, _ = bpm.soliton(ops, (0.5,), P, phi0=np.exp(-coords[:, 0] ** 2))
            assert bpm.power(ops, phi) == pytest.approx(P, rel=1e-12)
            assert bpm.soliton_residual(ops, (0.5,), phi, mu) < 1e-9
            a = P / 2.0
            exact = a / np.cosh(a * coords[:, 0])
            assert bpm.relative_error(ops, phi.astype(complex), exact.astype(complex)) < 2e-3
            errs.append(abs(mu + P * P / 8.0))
        assert errs[1] < 1e-3 * P * P / 8.0
        assert 3.0 < errs[0] / errs[1] < 5.0, (P, errs)


def _lp01_eigenvalue(V0):
    """Lowest eigenvalue u^2 of -lap + V0 1_{r > 1} in the plane (the LP01
    mode of a step-index fiber of core radius 1): u solves
    u J1(u) / J0(u) = w K1(w) / K0(w), u^2 + w^2 = V0."""
    from scipy.optimize import brentq
    from scipy.special import j0, j1, k0, k1

    def f(u):
        w = math.sqrt(V0 - u * u)
        return u * j1(u) / j0(u) - w * k1(w) / k0(w)

    u = brentq(f, 1e-6, min(2.404825557695773, math.sqrt(V0)) - 1e-9)
    return u * u


def test_soliton_linear_limit_is_the_lp01_mode():
    """Without the Kerr term the self-consistent mode is the fundamental
    guided mode; its eigenvalue converges at O(h^2) to the Bessel-function
    LP01 eigenvalue of the step-index fiber (Table II V-number)."""
    V0 = -W.FIBER_V_CLAD
    lam = _lp01_eigenvalue(V0)
    errs = []
    for n in (3000, 12000):
        coords, tris = W.mesh_disk_graded(4.0, n, 3.0, interfaces=(1.0,), seed=5, grade_from=1.0)
        V, chi = W.step_index_materials(coords, tris)
        ops = dec.Operators(coords, tris, V, 0.0 * chi)
        phi, mu, _ = bpm.soliton(ops, (1.0,), 1.0)
        errs.append(abs(mu - lam) / lam)
    assert errs[1] < 3e-3
    assert errs[0] / errs[1] > 2.5, errs


def test_soliton_is_stationary_under_the_paper_integrator():
    """A computed nonlinear mode keeps its intensity under the paper's RK45
    integration of Eq. 10 (the eigen-equation and the ODE use one sign
    convention), for lumped and element-averaged Kerr."""
    coords, tris = W.mesh_disk_graded(4.0, 800, 3.0, interfaces=(1.0,), seed=7, grade_from=1.0)
    V, chi = W.step_index_materials(coords, tris)
    ops = dec.Operators(coords, tris, V, chi)
    for kerr in ("lumped", "element"):
        phi, mu, _ = bpm.soliton(ops, (1.0,), 6.0, kerr=kerr)
        assert bpm.soliton_residual(ops, (1.0,), phi, mu, kerr) < 1e-9
        out, _ = bpm.dopri5(ops, (1.0,), phi.astype(complex), 0.3, rtol=1e-11, atol=1e-13, kerr=kerr)
        assert bpm.intensity_error(ops, out, phi.astype(complex)) < 1e-8
        # and the phase advances as e^{-i mu z}
        ph = np.angle(np.sum(ops.H0 * out * phi) / np.sum(ops.H0 * phi * phi))
        assert ph == pytest.approx(np.angle(np.exp(-1j * mu * 0.3)), abs=1e-8)
