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


def test_pml_mesh_rejects_the_split_step_and_can_be_removed():
    coords, tris = W.mesh_disk_graded(4.0, 600, 2.0, interfaces=(1.0,), seed=92, grade_from=1.0)
    V, chi = W.step_index_materials(coords, tris)
    mesh = api.Mesh(coords, tris, V, chi)
    x = torch.from_numpy(np.exp(-(coords[:, 0] ** 2 + coords[:, 1] ** 2)).astype(np.complex128)).to(DEV)
    api.set_pml(mesh, r_inner=3.0, r_outer=4.0, sigma_max=4.0)
    with pytest.raises(L.DecbpmError) as e:
        api.propagate(mesh, x.clone(), 1e-3, 2)
    assert "PML" in str(e.value)
    with pytest.raises(L.DecbpmError):
        api.Plan([mesh], [1], "c128").propagate([x.clone()], 1e-3, 2)
    with pytest.raises(L.DecbpmError):
        api.set_pml(mesh, r_inner=4.0, r_outer=3.0, sigma_max=1.0)        # bad geometry
    api.set_pml(mesh, None)
    api.propagate(mesh, x, 1e-3, 2)                                     # the split-step runs again
    assert torch.isfinite(torch.view_as_real(x)).all()
