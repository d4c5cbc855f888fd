"""Failure detection on the GPU without faulting or hanging it.

* The persistent kernel's grid barrier spins for a bounded time; the self
  test waits for arrivals that never come (a count nothing reaches) with a
  50 ms limit and must come back with DECBPM_ERR_TIMEOUT, after which the
  context keeps working.
* A non-finite field is caught by the FP64 diagnostics (status NONFINITE).
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from paper_2608_03587_b300 import _lib as L  # noqa: E402
from paper_2608_03587_b300 import api  # noqa: E402
from paper_2608_03587_b300 import workloads as W  # noqa: E402

pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)


def test_barrier_wait_runs_out_and_context_survives():
    assert api.selftest_barrier(0, 50_000_000) == L.OK
    assert api.selftest_barrier(3, 50_000_000) == L.ERR_TIMEOUT
    # the device is still usable afterwards
    x = torch.arange(10, device="cuda:0", dtype=torch.float32)
    assert float(x.sum()) == 45.0
    assert api.selftest_barrier(0, 50_000_000) == L.OK


def test_nonfinite_field_is_reported():
    coords, tris = W.mesh_disk_graded(2.0, 500, 1.0, seed=2)
    mesh = api.Mesh(coords, tris)
    psi = torch.from_numpy(W.gaussian(coords)).to("cuda:0", torch.complex64)
    psi[7] = complex(float("nan"), 0.0)
    with pytest.raises(L.DecbpmError) as e:
        api.propagate(mesh, psi, 1e-3, 3)
    assert e.value.code == L.ERR_NONFINITE
    good = torch.from_numpy(W.gaussian(coords)).to("cuda:0", torch.complex64)
    api.propagate(mesh, good, 1e-3, 3)
    assert torch.isfinite(torch.view_as_real(good)).all()


def test_invalid_parameters_are_rejected_before_launch():
    coords, tris = W.mesh_disk_graded(2.0, 300, 1.0, seed=3)
    mesh = api.Mesh(coords, tris)
    psi = torch.zeros(len(coords), dtype=torch.complex64, device="cuda:0")
    for kw in ({"dz": -1.0}, {"dz": float("nan")}, {"n_steps": -2}):
        args = {"dz": 1e-3, "n_steps": 1}
        args.update(kw)
        with pytest.raises(L.DecbpmError) as e:
            api.propagate(mesh, psi, **args)
        assert e.value.code == L.ERR_INVALID_ARG
    with pytest.raises(L.DecbpmError) as e:
        api.propagate(mesh, psi, 1e-3, 1, variant="plain")     # plain path is FP64 only
    assert e.value.code == L.ERR_UNSUPPORTED
    assert np.isfinite(api.diagnostics(mesh, psi)["power"]).all()
