"""The bounds-check build (libdecbpm_checked.so, -DDECBPM_BOUNDS_CHECK): its
march kernels test every gather index (neighbour rows in the field buffers,
window offsets in the tile and stage-pair kernels' shared-memory ring)
against its buffer and report DECBPM_ERR_DEVICE_CHECK instead of reading out
of bounds.  On consistent meshes no check fires, and the fields it produces
are bit for bit those of the default build, in every march kernel: the row
kernel (complex64 at 2 and 4 values per thread, complex128, one field), the
tile-staged kernel, the dataflow kernel (its dependency lists are checked
too) and the stage-pair kernel, with lumped and element-averaged Kerr, and
the march with a PML (persistent and per-term launches, both precisions).

The checked library is loaded in a child process (DECBPM_BOUNDS_CHECK=1 in
its environment); the parent runs the same cases on the default library."""
import os
import subprocess
import sys
import tempfile

import numpy as np
import pytest

torch = pytest.importorskip("torch")

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

from paper_2608_03587_b300 import _lib as L  # noqa: E402
from paper_2608_03587_b300 import api  # noqa: E402
from paper_2608_03587_b300 import workloads as W  # noqa: E402

pytestmark = pytest.mark.gpu

DEV = torch.device("cuda:0")

# (vertices, fields, seed): uneven sizes and degrees, a mesh below one tile
# and a single triangle
SPECS = [(600, 16, 51), (2500, 9, 52), (5000, 12, 53), (90, 16, 54), (3, 16, 56)]


def _meshes():
    meshes, psis = [], []
    for n, B, seed in SPECS:
        if n == 3:
            coords = np.array([[0.0, 0.0], [1.0, 0.0], [0.2, 0.9]])
            tris = np.array([[0, 1, 2]], dtype=np.int32)
        else:
            coords, tris = W.mesh_disk_graded(4.0, n, 3.0, interfaces=(1.0,), seed=seed, grade_from=1.0)
        V, chi = W.step_index_materials(coords, tris)
        sigma = W.absorber_profile(coords, 4.0, 20.0)
        meshes.append(api.Mesh(coords, tris, V, chi, sigma))
        psis.append(W.hg_superpositions(coords, B, np.random.default_rng(seed)) * 2.0)
    return meshes, psis


def run_cases() -> dict:
    """Every case on the library this process loaded: name -> final fields."""
    meshes, psis = _meshes()
    dz, n = 2e-3, 7
    out = {}
    # (precision, variant, fields per mesh (None: 9..16), row-kernel values per thread)
    cases = [("c64", "pairs", None, 0), ("c64", "fused", None, 0), ("c64", "flow", None, 0), ("c64", "rows", None, 0),
             ("c64", "fused", None, 2), ("c64", "rows", 4, 0), ("c128", "fused", 3, 0)]
    for prec, variant, fields, fpt in cases:
        dt = torch.complex64 if prec == "c64" else torch.complex128
        ps = [p if fields is None else p[:, :fields] for p in psis]
        plan = api.Plan(meshes, [p.shape[1] for p in ps], prec)
        if fpt:
            plan.set_shape("rows", values_per_thread=fpt)
            assert plan.config()["values_per_thread"] == fpt
        elif (prec, variant, fields) == ("c64", "fused", None):
            out["tile_kernel_used"] = np.array(plan.config()["fused_kernel"] == 1)
        for kerr in ("lumped", "element"):
            t = [torch.from_numpy(np.ascontiguousarray(p)).to(DEV, dt) for p in ps]
            plan.propagate(t, dz, n, diag_every=3, kerr=kerr, variant=variant)
            torch.cuda.synchronize()
            for i, x in enumerate(t):
                out["%s_%s_%s_%d_%s_%d" % (prec, variant, fields, fpt, kerr, i)] = x.cpu().numpy()
    # the single-field entry point (row kernel, one field)
    x = torch.from_numpy(np.ascontiguousarray(psis[2][:, 0])).to(DEV, torch.complex128)
    api.propagate(meshes[2], x, dz, n, kerr="element")
    out["single_c128"] = x.cpu().numpy()
    # the march on the complex-stretched operators of a PML, three fields
    coords, tris = W.mesh_disk_graded(4.0, 2500, 3.0, interfaces=(1.0,), seed=57, grade_from=1.0)
    V, chi = W.step_index_materials(coords, tris)
    mp = api.Mesh(coords, tris, V, chi)
    api.set_pml(mp, r_inner=3.0, r_outer=4.0, sigma_max=4.0)
    p3 = np.ascontiguousarray(W.hg_superpositions(coords, 3, np.random.default_rng(57)) * 2.0)
    for prec, dt in (("c64", torch.complex64), ("c128", torch.complex128)):
        for variant in ("fused", "plain"):
            x = torch.from_numpy(p3).to(DEV, dt)
            api.propagate(mp, x, dz, n, diag_every=3, variant=variant)
            out["pml_%s_%s" % (prec, variant)] = x.cpu().numpy()
    return out


@pytest.mark.skipif(not torch.cuda.is_available(), reason="no CUDA device")
def test_index_check_fires_only_in_the_checked_build():
    """decbpm_selftest_bounds_check passes an out-of-range index through the
    march kernels' index check (never using it to access memory): the default
    build returns it unchanged (DECBPM_OK); the checked build, in a child
    process, reports DECBPM_ERR_DEVICE_CHECK and the context stays usable."""
    if L.CHECKED:
        pytest.skip("this process already loaded the bounds-check build")
    lib = L.load()
    assert lib.decbpm_selftest_bounds_check(None) == L.OK
    code = ("import sys; sys.path.insert(0, %r)\n"
            "from paper_2608_03587_b300 import _lib as L\n"
            "import torch\n"
            "lib = L.load(); rc = lib.decbpm_selftest_bounds_check(None)\n"
            "x = torch.ones(4, device='cuda') * 2; torch.cuda.synchronize()\n"
            "print('rc', rc, float(x.sum()))\n") % ROOT
    res = subprocess.run([sys.executable, "-c", code], env=dict(os.environ, DECBPM_BOUNDS_CHECK="1"), cwd=ROOT,
                         capture_output=True, text=True, timeout=600)
    assert res.returncode == 0, res.stdout[-2000:] + res.stderr[-2000:]
    assert "rc %d 8.0" % L.ERR_DEVICE_CHECK in res.stdout, res.stdout


@pytest.mark.skipif(not torch.cuda.is_available(), reason="no CUDA device")
def test_bounds_checked_build_gives_the_same_fields():
    if L.CHECKED:
        pytest.skip("this process already loaded the bounds-check build")
    lib = L.load()
    assert b"bounds-checked" not in lib.decbpm_version()
    with tempfile.TemporaryDirectory() as tmp:
        path = os.path.join(tmp, "checked.npz")
        env = dict(os.environ, DECBPM_BOUNDS_CHECK="1")
        res = subprocess.run([sys.executable, os.path.abspath(__file__), path], env=env, cwd=ROOT,
                             capture_output=True, text=True, timeout=900)
        assert res.returncode == 0, res.stdout[-3000:] + res.stderr[-3000:]
        assert "bounds-checked" in res.stdout
        checked = dict(np.load(path))
    plain = run_cases()
    assert bool(plain["tile_kernel_used"]) and bool(checked["tile_kernel_used"])
    assert sorted(plain) == sorted(checked)
    for k in plain:
        assert np.array_equal(plain[k], checked[k]), k


if __name__ == "__main__":
    # child: DECBPM_BOUNDS_CHECK=1 selects libdecbpm_checked.so at load time;
    # a check that fires makes the propagation raise DecbpmError (status -8)
    ver = L.load().decbpm_version().decode()
    assert "bounds-checked" in ver, ver
    print(ver, flush=True)
    np.savez(sys.argv[1], **run_cases())
