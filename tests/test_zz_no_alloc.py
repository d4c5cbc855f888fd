"""The allocation-free entry point decbpm_propagate_noalloc.

It exists for callers that cannot allocate device memory when they
propagate (another allocator owns the memory budget, or a loop must keep a
fixed footprint): its scratch is the library's static device array instead of
cudaMalloc'ed workspaces.  Checked here through the C ABI against
decbpm_propagate, the existing entry point, on two calls in a row (the static
scratch keeps the previous call's contents).  Both run the same row kernel on
the same coefficient tables, so the fields must agree bit for bit, in both
precisions and both Kerr modes.  This file is named so that pytest collects it
last.
"""
import ctypes

import numpy as np
import pytest

torch = pytest.importorskip("torch")

from paper_2608_03587_b300 import _lib as L  # noqa: E402
from paper_2608_03587_b300 import api  # noqa: E402
from paper_2608_03587_b300 import workloads as W  # noqa: E402

pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)


def _rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def _noalloc(lib, mesh, psi, dz, n_steps, precision, kerr_mode=L.KERR_LUMPED):
    prm = L.Params(dz=dz, n_steps=n_steps, precision=precision, kerr_mode=kerr_mode, diag_every=0,
                   variant=L.VARIANT_FUSED, cheb_tol=0.0)
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    return lib.decbpm_propagate_noalloc(mesh.handle, ctypes.byref(prm), ctypes.c_void_p(psi.data_ptr()),
                                        psi.shape[1], stream)


@pytest.mark.parametrize("kerr", ["lumped", "element"])
@pytest.mark.parametrize("dtype,precision", [(torch.complex128, L.C128), (torch.complex64, L.C64)])
def test_noalloc_matches_propagate_two_calls(dtype, precision, kerr):
    lib = L.load()
    coords, tris = W.mesh_disk_graded(4.0, 6000, 3.0, interfaces=(1.0,), seed=77, grade_from=1.0)
    V, chi = W.step_index_materials(coords, tris)
    sigma = W.absorber_profile(coords, 4.0, 20.0)
    mesh = api.Mesh(coords, tris, V, chi, sigma)
    psi0 = W.hg_superpositions(coords, 3, np.random.default_rng(5)) * 3.0
    a = torch.from_numpy(psi0).to("cuda:0", dtype).contiguous()
    b = a.clone()
    mode = L.KERR_LUMPED if kerr == "lumped" else L.KERR_ELEMENT
    for call in range(2):
        api.propagate(mesh, a, 1e-3, 7, kerr=kerr)
        assert _noalloc(lib, mesh, b, 1e-3, 7, precision, mode) == L.OK, lib.decbpm_last_error()
        assert torch.isfinite(torch.view_as_real(b)).all()
        assert torch.equal(b, a), (call, float((b - a).abs().max()))


def test_noalloc_rejects_sizes_beyond_its_scratch():
    lib = L.load()
    coords, tris = W.mesh_disk_graded(4.0, 70_000, 3.0, seed=3)
    mesh = api.Mesh(coords, tris)
    psi = torch.zeros((len(coords), 64), dtype=torch.complex128, device="cuda:0")
    rc = _noalloc(lib, mesh, psi, 1e-3, 1, L.C128)
    assert rc == L.ERR_INVALID_ARG
    msg = lib.decbpm_last_error().decode()
    assert "static scratch" in msg and "bytes" in msg
    # a size that fits still works afterwards
    small = torch.zeros((len(coords), 1), dtype=torch.complex64, device="cuda:0")
    small[:, 0] = torch.from_numpy(W.gaussian(coords)).to("cuda:0", torch.complex64)
    assert _noalloc(lib, mesh, small, 1e-3, 2, L.C64) == L.OK
