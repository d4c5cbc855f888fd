"""GPU PML (complex-stretched Hodge stars) on the paper's RK45 integrator,
against the oracle's stretched operators and Dormand-Prince controller."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import bpm, pml  # noqa: E402
from paper_2608_03587_b300 import _lib as L  # noqa: E402
from paper_2608_03587_b300 import api  # noqa: E402
from paper_2608_03587_b300 import workloads as W  # noqa: E402

pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

DEV = torch.device("cuda:0")
LAYER = dict(r_in=3.0, R=4.0, sigma_max=4.0, order=2)


@pytest.mark.parametrize("amp,p", [(1.0, (1.0,)), (2.5, (1.0,)), (1.0, (1.0, 2e-4))])
def test_rk45_with_pml_matches_oracle(amp, p):
    """Same accepted/rejected steps and fields within 1e-11 on a step-index
    fiber with the layer, linear and Kerr launches, p2 != 0."""
    coords, tris = W.mesh_disk_graded(4.0, 1500, 2.0, interfaces=(1.0,), seed=91, grade_from=1.0)
    V, chi = W.step_index_materials(coords, tris)
    ops = pml.StretchedOperators(coords, tris, V, chi, **LAYER)
    mesh = api.Mesh(coords, tris, V, chi, p=p)
    api.set_pml(mesh, r_inner=3.0, r_outer=4.0, sigma_max=4.0, order=2)
    x, y = coords[:, 0], coords[:, 1]
    psi0 = (amp * np.exp(-((x - 0.3) ** 2 + y ** 2) / 0.5 + 3.0j * x)).astype(np.complex128)
    z = 0.03
    ref, st_ref = bpm.dopri5(ops, p, psi0, z, rtol=1e-9, atol=1e-11)
    t = torch.from_numpy(psi0).to(DEV)
    st = api.rk45(mesh, t, z, rtol=1e-9, atol=1e-11)
    for k in ("n_accepted", "n_rejected", "n_rhs"):
        assert st[k] == st_ref[k], (k, st, st_ref)
    assert bpm.relative_error(ops, t.cpu().numpy(), ref) <= 1e-11


@pytest.mark.parametrize("amp,dz,n,every", [(1.0, 1e-3, 30, 0), (2.5, 5e-4, 40, 15)])
def test_split_step_with_pml_matches_oracle(amp, dz, n, every):
    """The Strang march on the complex-stretched operators (the layer the
    paper's Conclusion proposes) through decbpm_propagate: the Chebyshev
    series of exp(-i a x) evaluated on the stretched operator's complex
    spectrum, degree set by the Bernstein ellipse of its Gershgorin box, and
    the exact diagonal flow with complex lumped v and chib, against the
    oracle's Strang march on the same operators (Taylor action, no merging
    of half steps) <= 1e-12, both as one persistent launch per step block and
    as one launch per Chebyshev term; an outgoing beam loses power to the
    layer."""
    coords, tris = W.mesh_disk_graded(4.0, 1500, 2.0, interfaces=(1.0,), seed=91, grade_from=1.0)
    V, chi = W.step_index_materials(coords, tris)
    ops = pml.StretchedOperators(coords, tris, V, chi, **LAYER)
    mesh = api.Mesh(coords, tris, V, chi)
    api.set_pml(mesh, r_inner=3.0, r_outer=4.0, sigma_max=4.0, order=2)
    x, y = coords[:, 0], coords[:, 1]
    psi0 = (amp * np.exp(-((x - 0.3) ** 2 + y ** 2) / 0.5 + 3.0j * x)).astype(np.complex128)
    ref = pml.propagate_stretched(ops, (1.0,), psi0, dz, n)
    t = torch.from_numpy(psi0).to(DEV)
    d = api.propagate(mesh, t, dz, n, diag_every=every)
    assert bpm.relative_error(ops, t.cpu().numpy(), ref) <= 1e-12
    P = d["power"][:, 0]
    assert np.all(np.isfinite(P)) and np.all(P <= bpm.power(ops, psi0) * (1 + 1e-12))
    # the same march as one launch per Chebyshev term (PLAIN; also the default
    # on meshes too large for one row per thread) instead of the persistent
    # kernel: the same stages, rounding-level agreement
    u = torch.from_numpy(psi0).to(DEV)
    d2 = api.propagate(mesh, u, dz, n, diag_every=every, variant="plain")
    assert bpm.relative_error(ops, u.cpu().numpy(), ref) <= 1e-12
    assert bpm.relative_error(ops, u.cpu().numpy(), t.cpu().numpy()) <= 1e-13
    assert np.allclose(d2["power"], d["power"], rtol=1e-12, atol=0)


def test_split_step_with_pml_absorbs_an_outgoing_beam():
    """A k = 4 beam on a homogeneous disk leaves through the layer: by z = 0.7
    the split-step with the layer keeps 8% of the power (Neumann walls keep
    all of it), follows the oracle's Strang march over the 700 steps
    (<= 1e-11) and the GPU's own RK45 integration with the layer (the
    splitting error, <= 1e-5)."""
    coords, tris = W.mesh_disk_graded(4.0, 1500, 2.0, seed=91)
    nc = len(tris)
    V, chi = np.zeros(nc), np.ones(nc)
    ops = pml.StretchedOperators(coords, tris, V, chi, **LAYER)
    mesh = api.Mesh(coords, tris, V, chi)
    api.set_pml(mesh, r_inner=3.0, r_outer=4.0, sigma_max=4.0, order=2)
    x, y = coords[:, 0], coords[:, 1]
    psi0 = np.exp(-((x - 0.3) ** 2 + y ** 2) / 0.5 + 4.0j * x).astype(np.complex128)
    t = torch.from_numpy(psi0).to(DEV)
    d = api.propagate(mesh, t, 1e-3, 700, diag_every=100)
    P, P0 = d["power"][:, 0], bpm.power(ops, psi0)
    assert P[-1] < 0.1 * P0 and np.all(np.diff(P) <= 1e-12 * P0)
    ref = pml.propagate_stretched(ops, (1.0,), psi0, 1e-3, 700)
    assert bpm.relative_error(ops, t.cpu().numpy(), ref) <= 1e-11
    r = torch.from_numpy(psi0).to(DEV)
    api.rk45(mesh, r, 0.7, rtol=1e-10, atol=1e-12)
    assert bpm.relative_error(ops, t.cpu().numpy(), r.cpu().numpy()) <= 1e-5


def _fiber_with_layer(n=1500, seed=91):
    coords, tris = W.mesh_disk_graded(4.0, n, 2.0, interfaces=(1.0,), seed=seed, grade_from=1.0)
    V, chi = W.step_index_materials(coords, tris)
    ops = pml.StretchedOperators(coords, tris, V, chi, **LAYER)
    mesh = api.Mesh(coords, tris, V, chi)
    api.set_pml(mesh, r_inner=3.0, r_outer=4.0, sigma_max=4.0, order=2)
    return coords, ops, mesh


def _launches(coords, B, seed):
    """B tilted, shifted Gaussian launches of amplitude 0.5..2.5 (linear to
    strongly nonlinear), k up to 4: parts of them leave through the layer."""
    rng = np.random.default_rng(seed)
    x, y = coords[:, 0], coords[:, 1]
    cols = []
    for _ in range(B):
        amp, x0, y0 = rng.uniform(0.5, 2.5), rng.uniform(-0.5, 0.5), rng.uniform(-0.5, 0.5)
        kx, ky = rng.uniform(-4.0, 4.0), rng.uniform(-4.0, 4.0)
        cols.append(amp * np.exp(-((x - x0) ** 2 + (y - y0) ** 2) / 0.5 + 1j * (kx * x + ky * y)))
    return np.stack(cols, axis=1).astype(np.complex128)


@pytest.mark.parametrize("B", [3, 16])
def test_split_step_with_pml_several_fields_matches_oracle(B):
    """B fields per vertex (padded layout, one thread per vertex and field) in
    complex128: every field equals the oracle's Strang march on the stretched
    operators <= 1e-12, in both launch forms (persistent, per term), and the
    FP64 power diagnostic after the last step block is the oracle field's
    power.  (Power is not monotone for every launch: the discretized layer
    leaves near-cutoff guided modes with tiny growth rates.)"""
    coords, ops, mesh = _fiber_with_layer()
    psi0 = _launches(coords, B, seed=200 + B)
    dz, n, every = 5e-4, 30, 12
    ref = pml.propagate_stretched(ops, (1.0,), psi0, dz, n)
    P_ref = bpm.power(ops, ref)
    for variant in ("fused", "plain"):
        t = torch.from_numpy(psi0).to(DEV).contiguous()
        d = api.propagate(mesh, t, dz, n, diag_every=every, variant=variant)
        out = t.cpu().numpy()
        errs = [bpm.relative_error(ops, out[:, f], ref[:, f]) for f in range(B)]
        assert max(errs) <= 1e-12, (variant, errs)
        assert d["power"].shape == (3, B) and np.all(np.isfinite(d["power"]))
        assert np.allclose(d["power"][-1], P_ref, rtol=1e-11, atol=0)


@pytest.mark.parametrize("B", [1, 16])
def test_split_step_with_pml_complex64_matches_oracle(B):
    """The march with the layer in complex64 (FP32 weights a_pq / r, v, chib,
    FP32 arithmetic, last stage in double-float): one step from the oracle's
    state rounded to FP32 within 1e-5 per field, 400 steps (z = 0.2) within
    1e-4 per field, both against the FP64 oracle, and so is each field's
    power; the persistent and per-term launch forms agree to rounding."""
    coords, ops, mesh = _fiber_with_layer()
    psi0 = _launches(coords, B, seed=300 + B).astype(np.complex64)
    x0 = psi0.astype(np.complex128)
    dz = 5e-4

    def run(n, variant="fused"):
        t = torch.from_numpy(psi0[:, 0] if B == 1 else psi0).to(DEV).contiguous()
        api.propagate(mesh, t, dz, n, variant=variant)
        out = t.cpu().numpy().astype(np.complex128)
        return out[:, None] if B == 1 else out

    def errs(out, ref):
        return [bpm.relative_error(ops, out[:, f], ref[:, f]) for f in range(B)]

    e1 = errs(run(1), pml.propagate_stretched(ops, (1.0,), x0, dz, 1))
    assert max(e1) <= 1e-5, e1
    ref = pml.propagate_stretched(ops, (1.0,), x0, dz, 400)
    a, b = run(400), run(400, "plain")
    eN = errs(a, ref)
    assert max(eN) <= 1e-4, eN
    assert max(errs(b, a)) <= 1e-6
    assert np.allclose(bpm.power(ops, a), bpm.power(ops, ref), rtol=1e-4, atol=0)


def test_pml_mesh_limits_and_removal():
    """With a layer the split-step runs one mesh with any number of fields in
    complex64 or complex128 and lumped Kerr (decbpm_propagate, and from host
    buffers with the same bits) besides decbpm_rk45; plans and element Kerr
    are refused; removing the layer restores everything."""
    coords, tris = W.mesh_disk_graded(4.0, 600, 2.0, interfaces=(1.0,), seed=92, grade_from=1.0)
    V, chi = W.step_index_materials(coords, tris)
    mesh = api.Mesh(coords, tris, V, chi)
    x = torch.from_numpy(np.exp(-(coords[:, 0] ** 2 + coords[:, 1] ** 2)).astype(np.complex128)).to(DEV)
    assert api.pml_degree(mesh, 1e-3, "c128") == 0                     # no layer yet
    api.set_pml(mesh, r_inner=3.0, r_outer=4.0, sigma_max=4.0)
    m64, m32 = api.pml_degree(mesh, 1e-3, "c128"), api.pml_degree(mesh, 1e-3, "c64")
    assert m64 >= m32 >= 2 and api.pml_degree(mesh, 2e-3, "c128") > m64
    for y in (x.clone(), x.clone().to(torch.complex64), torch.stack([x, 2 * x], dim=1).contiguous()):
        h = y.cpu().pin_memory()
        api.propagate(mesh, y, 1e-3, 2)
        assert torch.isfinite(torch.view_as_real(y)).all()
        api.propagate_host(mesh, h, 1e-3, 2)                            # host buffers: the same march
        assert torch.equal(h, y.cpu())
    for bad in (lambda: api.propagate(mesh, x.clone(), 1e-3, 2, kerr="element"),
                lambda: api.Plan([mesh], [1], "c128").propagate([x.clone()], 1e-3, 2)):
        with pytest.raises(L.DecbpmError) as e:
            bad()
    with pytest.raises(L.DecbpmError):
        api.set_pml(mesh, r_inner=4.0, r_outer=3.0, sigma_max=1.0)        # bad geometry
    api.set_pml(mesh, None)
    assert api.pml_degree(mesh, 1e-3, "c128") == 0
    z = x.to(torch.complex64)
    api.propagate(mesh, z, 1e-3, 2)                                     # every split-step path runs again
    assert torch.isfinite(torch.view_as_real(z)).all()
