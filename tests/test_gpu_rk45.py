"""GPU parity for the paper's integrator: adaptive Dormand-Prince 5(4) on the
DEC ODE (Eq. 10, the potential inside L as in Eq. 11) against the oracle's
dopri5 with the same step controller.  Both sides take the same accept/reject
decisions, so the step counts must match exactly and the fields to rounding
(1e-11 relative, *0-weighted L2) after tens of adaptive steps."""
import math

import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import bpm, dec  # noqa: E402
from paper_2608_03587_b300 import _lib as L  # noqa: E402
from paper_2608_03587_b300 import api  # noqa: E402
from paper_2608_03587_b300 import workloads as W  # noqa: E402

pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

DEV = torch.device("cuda:0")


@pytest.fixture(scope="module")
def fiber():
    coords, tris = W.mesh_disk_graded(4.0, 1500, 3.0, interfaces=(1.0,), seed=41, grade_from=1.0)
    V, chi = W.step_index_materials(coords, tris)
    sigma = W.absorber_profile(coords, 4.0, 20.0)
    return coords, tris, V, chi, sigma


def field(coords, A=2.0):
    return W.elliptic_gaussian(coords, A=A, x0=0.2, y0=-0.1, theta=0.4) * np.exp(0.3j)


@pytest.mark.parametrize("kerr,p,use_sigma", [("lumped", (1.0,), True), ("element", (1.0,), False),
                                              ("lumped", (1.0, 2e-4), True)])
def test_rk45_matches_oracle_dopri5(fiber, kerr, p, use_sigma):
    coords, tris, V, chi, sigma = fiber
    sg = sigma if use_sigma else np.zeros_like(sigma)
    ops = dec.Operators(coords, tris, V, chi)
    mesh = api.Mesh(coords, tris, V, chi, sg, p=p)
    psi0 = field(coords)
    z_end = 0.02
    ref, st_ref = bpm.dopri5(ops, p, psi0, z_end, rtol=1e-9, atol=1e-11, sigma=sg, kerr=kerr)
    t = torch.from_numpy(psi0).to(DEV)
    st = api.rk45(mesh, t, z_end, rtol=1e-9, atol=1e-11, kerr=kerr)
    assert st["n_accepted"] >= 5
    for k in ("n_accepted", "n_rejected", "n_rhs"):
        assert st[k] == st_ref[k], (k, st, st_ref)
    assert st["h_last"] == pytest.approx(st_ref["h_last"], rel=1e-9)
    assert st["z"] == pytest.approx(z_end, rel=1e-14)
    out = t.cpu().numpy()
    assert bpm.relative_error(ops, out, ref) <= 1e-11


def test_rk45_fixed_first_step_and_rejections(fiber):
    """A first step far too large forces rejections: the controller's shrink
    rule and the no-growth-after-rejection rule take the same path as the
    oracle's."""
    coords, tris, V, chi, sigma = fiber
    ops = dec.Operators(coords, tris, V, chi)
    mesh = api.Mesh(coords, tris, V, chi, sigma)
    psi0 = field(coords, A=3.0)
    ref, st_ref = bpm.dopri5(ops, (1.0,), psi0, 0.01, rtol=1e-8, atol=1e-10, h0=0.01, sigma=sigma)
    t = torch.from_numpy(psi0).to(DEV)
    st = api.rk45(mesh, t, 0.01, rtol=1e-8, atol=1e-10, h0=0.01)
    assert st_ref["n_rejected"] >= 2
    for k in ("n_accepted", "n_rejected", "n_rhs"):
        assert st[k] == st_ref[k]
    assert bpm.relative_error(ops, t.cpu().numpy(), ref) <= 1e-11


def test_split_step_converges_to_rk45(fiber):
    """The fused Strang march converges to the RK45 solution at second order
    (the paper's cross-check of its integrators): halving dz divides the gap
    by about four."""
    coords, tris, V, chi, sigma = fiber
    ops = dec.Operators(coords, tris, V, chi)
    mesh = api.Mesh(coords, tris, V, chi, sigma)
    psi0 = field(coords)
    z_end = 0.04
    t_rk = torch.from_numpy(psi0).to(DEV)
    api.rk45(mesh, t_rk, z_end, rtol=1e-11, atol=1e-13)
    gaps = []
    for n in (20, 40):
        t = torch.from_numpy(psi0).to(DEV)
        api.propagate(mesh, t, z_end / n, n)
        gaps.append(bpm.relative_error(ops, t.cpu().numpy(), t_rk.cpu().numpy()))
    assert 1e-9 < gaps[1] < gaps[0]
    assert 3.3 < gaps[0] / gaps[1] < 4.7, gaps


def test_rk45_zero_length_and_bad_arguments(fiber):
    coords, tris, V, chi, sigma = fiber
    mesh = api.Mesh(coords, tris, V, chi, sigma)
    psi0 = field(coords)
    t = torch.from_numpy(psi0).to(DEV)
    st = api.rk45(mesh, t, 0.0)
    assert st["n_accepted"] == 0 and st["n_rejected"] == 0
    assert np.array_equal(t.cpu().numpy(), psi0)
    with pytest.raises(L.DecbpmError):
        api.rk45(mesh, t, 0.01, rtol=0.0)
    with pytest.raises(L.DecbpmError):
        api.rk45(mesh, t, -1.0)
    with pytest.raises(TypeError):
        api.rk45(mesh, t.to(torch.complex64), 0.01)
    st = api.rk45(mesh, t, 0.05, max_steps=3)
    assert st["n_accepted"] + st["n_rejected"] == 3 and st["z"] < 0.05
