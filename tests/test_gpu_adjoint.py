"""GPU adjoint (decbpm_vjp) against the oracle's exact discrete adjoint, against
central finite differences of the GPU forward march (FP64), and through
torch.autograd.  Objective: J = |<phi_t, psi_N>_{*0}|^2, the overlap of the
output field with a target mode, as in the PCF workload."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import bpm, dec  # noqa: E402
from paper_2608_03587_b300 import api  # noqa: E402
from paper_2608_03587_b300 import workloads as W  # noqa: E402

pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

DEV = "cuda:0"


def _setup(n=1500, seed=13):
    coords, tris, centres = W.mesh_pcf(n, R=3.0, rings=2, seed=seed)
    c = W.centroids(coords, tris)
    d = np.full(len(c), np.inf)
    for cx, cy in centres:
        d = np.minimum(d, np.hypot(c[:, 0] - cx, c[:, 1] - cy))
    hole = d < 0.25
    V = np.where(hole, -30.0, 0.0)
    chi = np.where(hole, 0.0, 1.0)
    sigma = W.absorber_profile(coords, 3.0, 10.0)
    return coords, tris, V, chi, sigma


def _rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def test_vjp_matches_oracle_adjoint():
    coords, tris, V, chi, sigma = _setup()
    ops = dec.Operators(coords, tris, V, chi)
    mesh = api.Mesh(coords, tris, V, chi, sigma)
    psi0 = W.gaussian(coords, w=0.7, A=2.0)
    phi = W.gaussian(coords, w=0.5) * np.exp(0.4j)
    dz, n = 2e-3, 11
    out = bpm.propagate(ops, (1.0,), psi0, dz, n, sigma)
    J, G = bpm.overlap_objective(ops, phi, out)
    g0_ref, gv_ref = bpm.vjp(ops, (1.0,), psi0, G, dz, n, sigma)
    t0 = torch.from_numpy(psi0).to(DEV, torch.complex128)
    tG = torch.from_numpy(G).to(DEV, torch.complex128)
    for ck in (0, 3, 11, 20):
        psiN, g0, gv = api.vjp(mesh, t0, tG, dz, n, checkpoint_every=ck)
        assert _rel(psiN.cpu().numpy(), out) <= 1e-12
        assert _rel(g0.cpu().numpy(), g0_ref) <= 1e-10, ck
        assert _rel(gv.cpu().numpy(), gv_ref) <= 1e-10, ck


def test_vjp_fp32_close_to_fp64():
    coords, tris, V, chi, sigma = _setup(seed=4)
    mesh = api.Mesh(coords, tris, V, chi, sigma)
    psi0 = W.gaussian(coords, w=0.7, A=2.0)
    rng = np.random.default_rng(0)
    G = (rng.standard_normal(len(coords)) + 1j * rng.standard_normal(len(coords))) * W.gaussian(coords, 1.0).real
    res = {}
    for dt in (torch.complex64, torch.complex128):
        _, g0, gv = api.vjp(mesh, torch.from_numpy(psi0).to(DEV, dt), torch.from_numpy(G).to(DEV, dt), 2e-3, 40)
        res[dt] = (g0.cpu().numpy().astype(np.complex128), gv.cpu().numpy())
    assert _rel(res[torch.complex64][0], res[torch.complex128][0]) <= 1e-4
    assert _rel(res[torch.complex64][1], res[torch.complex128][1]) <= 1e-4


def test_adjoint_entry_point_matches_oracle():
    """decbpm_adjoint, whose overlap objective J_f = |<phi_f, psi_N,f>_{*0}|^2
    and its cotangent are formed on the device (FP64 overlap), against the
    oracle's overlap_objective + vjp: J, dJ/dpsi_0 and d(sum J)/dv, two fields
    with their own targets, several checkpoint intervals."""
    coords, tris, V, chi, sigma = _setup(seed=21)
    ops = dec.Operators(coords, tris, V, chi)
    mesh = api.Mesh(coords, tris, V, chi, sigma)
    psi0 = np.stack([W.gaussian(coords, w=0.7, A=2.0), W.elliptic_gaussian(coords, A=1.5)], axis=1)
    phi = np.stack([W.gaussian(coords, w=0.5) * np.exp(0.4j), W.gaussian(coords, w=0.8) * np.exp(-1.1j)], axis=1)
    dz, n = 2e-3, 11
    J_ref, g0_ref, gv_ref = [], [], np.zeros(len(coords))
    for f in range(2):
        out = bpm.propagate(ops, (1.0,), psi0[:, f], dz, n, sigma)
        J, G = bpm.overlap_objective(ops, phi[:, f], out)
        g0, gv = bpm.vjp(ops, (1.0,), psi0[:, f], G, dz, n, sigma)
        J_ref.append(J)
        g0_ref.append(g0)
        gv_ref = gv_ref + gv
    g0_ref = np.stack(g0_ref, axis=1)
    t0 = torch.from_numpy(psi0).to(DEV, torch.complex128).contiguous()
    tp = torch.from_numpy(phi).to(DEV, torch.complex128).contiguous()
    for ck in (0, 4, 11):
        J, gv, g0 = api.adjoint(mesh, t0, tp, dz, n, checkpoint_every=ck)
        assert np.max(np.abs(J - np.asarray(J_ref)) / np.asarray(J_ref)) <= 1e-10, (ck, J, J_ref)
        assert _rel(g0.cpu().numpy(), g0_ref) <= 1e-10, ck
        assert _rel(gv.cpu().numpy(), gv_ref) <= 1e-10, ck
    # complex64: the same objective within the FP32 run budget
    J32, gv32, g032 = api.adjoint(mesh, t0.to(torch.complex64), tp.to(torch.complex64), dz, n)
    assert np.max(np.abs(J32 - np.asarray(J_ref)) / np.asarray(J_ref)) <= 1e-5
    assert _rel(gv32.cpu().numpy(), gv_ref) <= 1e-4
    assert _rel(g032.cpu().numpy().astype(np.complex128), g0_ref) <= 1e-4


def test_device_potential_offset_equals_host_potential():
    """decbpm_mesh_set_potential_offset (v = base + dv on the device) gives the
    same field, bit for bit, as setting base + dv from the host; NULL restores
    the base."""
    coords, tris, V, chi, sigma = _setup(seed=5)
    mesh = api.Mesh(coords, tris, V, chi, sigma)
    v0 = api.assemble_host(coords, tris, V, chi, sigma)["v"]
    dv = np.random.default_rng(8).standard_normal(len(coords)) * 0.3
    psi0 = torch.from_numpy(W.gaussian(coords, w=0.7, A=2.0)).to(DEV, torch.complex128)
    outs = []
    for mode in ("host", "device"):
        if mode == "host":
            api.set_potential(mesh, v0 + dv)
        else:
            api.set_potential(mesh, None)
            api.set_potential_offset(mesh, torch.from_numpy(dv).to(DEV))
        t = psi0.clone()
        api.propagate(mesh, t, 2e-3, 9)
        outs.append(t)
    assert torch.equal(outs[0], outs[1])
    api.set_potential_offset(mesh, None)
    a, b = psi0.clone(), psi0.clone()
    api.propagate(mesh, a, 2e-3, 9)
    api.set_potential(mesh, None)
    api.propagate(mesh, b, 2e-3, 9)
    assert torch.equal(a, b) and not torch.equal(a, outs[0])


def _objective(mesh, psi0_t, phi_m, dz, n, v):
    api.set_potential(mesh, v)
    t = psi0_t.clone()
    api.propagate(mesh, t, dz, n)
    c = np.sum(np.conj(phi_m) * t.cpu().numpy())
    return float(abs(c) ** 2)


@pytest.mark.parametrize("n_vertices,n_steps", [(6000, 200), (300_000, 2000)])
def test_vjp_potential_gradient_vs_central_differences(n_vertices, n_steps):
    """dJ/dv at 32 random vertices of the field's support: adjoint vs central
    differences of the FP64 GPU forward march (Richardson-extrapolated on the
    small mesh; plain, eps = 5e-3, on the full-size one, where the O(eps^2)
    truncation error is ~1e-6 relative)."""
    if n_vertices >= 300_000:
        wl = W.pcf(n_target=n_vertices)
        m = wl.meshes[0]
        coords, tris, V, chi, sigma = m.coords, m.cells, m.V_cell, m.chi_cell, m.sigma
    else:
        coords, tris, V, chi, sigma = _setup(n_vertices, seed=7)
    dz = 5e-4
    mesh = api.Mesh(coords, tris, V, chi, sigma)
    a = api.assemble_host(coords, tris, V, chi, sigma)
    v0, m = a["v"], a["m"]
    psi0 = W.gaussian(coords, w=0.7)
    # target: the forward output of the unperturbed guide (C128)
    t0 = torch.from_numpy(psi0).to(DEV, torch.complex128)
    ref = t0.clone()
    api.propagate(mesh, ref, dz, n_steps)
    phi = ref.cpu().numpy() * np.exp(0.2j) + 0.1 * W.gaussian(coords, w=0.4)
    phi_m = m * phi
    c = np.sum(np.conj(phi_m) * ref.cpu().numpy())
    G = 2.0 * c * phi_m                                       # Euclidean gradient of J at psi_N
    _, _, gv = api.vjp(mesh, t0, torch.from_numpy(G).to(DEV, torch.complex128), dz, n_steps)
    gv = gv.cpu().numpy()
    rng = np.random.default_rng(11)
    support = np.flatnonzero(np.abs(psi0) > 0.3 * np.abs(psi0).max())
    idx = rng.choice(support, 32, replace=False)
    errs = []
    for p in idx:
        def J(e):
            v = v0.copy()
            v[p] += e
            return _objective(mesh, t0, phi_m, dz, n_steps, v)
        if n_vertices >= 300_000:
            eps = 5e-3
            fd = (J(eps) - J(-eps)) / (2 * eps)
        else:
            eps = 1e-2
            d1 = (J(eps) - J(-eps)) / (2 * eps)
            d2 = (J(eps / 2) - J(-eps / 2)) / eps
            fd = (4 * d2 - d1) / 3
        errs.append(abs(gv[p] - fd) / max(abs(fd), 1e-300))
    api.set_potential(mesh, None)
    assert max(errs) <= 1e-4, (max(errs), np.median(errs))



def test_autograd_function_matches_vjp():
    coords, tris, V, chi, sigma = _setup(seed=9)
    mesh = api.Mesh(coords, tris, V, chi, sigma)
    a = api.assemble_host(coords, tris, V, chi, sigma)
    m = torch.from_numpy(a["m"]).to(DEV)
    psi0 = torch.from_numpy(W.gaussian(coords, w=0.7, A=1.5)).to(DEV, torch.complex128).requires_grad_(True)
    dv = torch.zeros(len(coords), dtype=torch.float64, device=DEV, requires_grad=True)
    phi = torch.from_numpy(W.gaussian(coords, w=0.5)).to(DEV, torch.complex128)
    out = api.march(mesh, psi0, dv, 2e-3, 25, checkpoint_every=4)
    J = torch.abs(torch.sum(m * torch.conj(phi) * out)) ** 2
    J.backward()
    c = torch.sum(m * torch.conj(phi) * out.detach())
    Gt = 2 * c * m * phi
    _, g0, gv = api.vjp(mesh, psi0.detach(), Gt, 2e-3, 25)
    assert _rel(psi0.grad.cpu().numpy(), g0.cpu().numpy()) <= 1e-12
    assert _rel(dv.grad.cpu().numpy(), gv.cpu().numpy()) <= 1e-12
    # first-order check of the chain through torch: J(psi0 + eps d) against the gradient
    gen = torch.Generator(device=DEV).manual_seed(3)
    d = torch.randn(len(coords), dtype=torch.complex128, device=DEV, generator=gen) * 1e-4
    with torch.no_grad():
        o1 = api.march(mesh, psi0.detach() + d, dv.detach(), 2e-3, 25)
        o2 = api.march(mesh, psi0.detach() - d, dv.detach(), 2e-3, 25)
        J1 = torch.abs(torch.sum(m * torch.conj(phi) * o1)) ** 2
        J2 = torch.abs(torch.sum(m * torch.conj(phi) * o2)) ** 2
    fd = float((J1 - J2) / 2)
    ad = float(torch.real(torch.sum(torch.conj(psi0.grad) * d)))
    assert ad == pytest.approx(fd, rel=1e-6)


def test_fp32_adjoint_full_size_pcf():
    """The complex64 adjoint (FP32 forward, recomputation and backward march;
    FP64 accumulation of dJ/dv) of the full photonic-crystal-fiber workload
    (300k vertices, 2000 steps) against the FP64 one, with the objective of
    the finite-difference test.  The forward field and dJ/dpsi_0 stay within
    the FP32 run bar (1e-4; measured 7.6e-6 and 3.9e-5).  dJ/dv does not: it
    is 1.8e-3 from FP64 (236 x the field's FP32 error, 11 x the change of the
    FP64 dJ/dv under a 1e-5 white-noise perturbation of the launch field),
    so the potential gradient of a march this long is taken in complex128,
    which matches central differences to 1e-4 (the test above).  The bound
    here (3e-3) records the measured level so that a regression shows."""
    wl = W.pcf()
    m = wl.meshes[0]
    mesh = api.Mesh.from_workload(m, p=wl.p)
    a = api.assemble_host(m.coords, m.cells, m.V_cell, m.chi_cell, m.sigma)
    dz, N = wl.dz, wl.n_steps
    psi0 = W.gaussian(m.coords, w=0.7)
    t0 = torch.from_numpy(psi0).to(DEV, torch.complex128)
    ref = t0.clone()
    api.propagate(mesh, ref, dz, N)
    phi = ref.cpu().numpy() * np.exp(0.2j) + 0.1 * W.gaussian(m.coords, w=0.4)
    c = np.sum(a["m"] * np.conj(phi) * ref.cpu().numpy())
    G = 2.0 * c * a["m"] * phi
    psiN64, g064, gv64 = api.vjp(mesh, t0, torch.from_numpy(G).to(DEV, torch.complex128), dz, N)
    psiN32, g032, gv32 = api.vjp(mesh, t0.to(torch.complex64), torch.from_numpy(G).to(DEV, torch.complex64), dz, N)
    e_psi = _rel(psiN32.cpu().numpy().astype(np.complex128), psiN64.cpu().numpy())
    e_g0 = _rel(g032.cpu().numpy().astype(np.complex128), g064.cpu().numpy())
    e_gv = _rel(gv32.cpu().numpy(), gv64.cpu().numpy())
    rng = np.random.default_rng(12)
    noise = (rng.standard_normal(len(psi0)) + 1j * rng.standard_normal(len(psi0))) * np.abs(psi0) * 1e-5 / np.sqrt(2)
    _, _, gvp = api.vjp(mesh, torch.from_numpy(psi0 + noise).to(DEV, torch.complex128),
                        torch.from_numpy(G).to(DEV, torch.complex128), dz, N)
    sens = _rel(gvp.cpu().numpy(), gv64.cpu().numpy())
    print("fp32 adjoint at 300k/2000 steps: psi_N %.2e, dJ/dpsi0 %.2e, dJ/dv %.2e; FP64 dJ/dv change for a 1e-5 "
          "launch perturbation %.2e" % (e_psi, e_g0, e_gv, sens))
    assert e_psi <= 1e-4 and e_g0 <= 1e-4, (e_psi, e_g0)
    assert e_gv <= 3e-3, (e_gv, sens)
