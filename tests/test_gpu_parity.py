"""GPU parity: the CUDA path (through the C ABI) against the FP64 CPU oracle.

Tolerances (relative *0-weighted L2 error of the complex field):
  FP64 (C128) fused and plain paths ........ 1e-12 over whole runs
  FP32 (C64) fused path .................... 1e-5 for one step from the oracle
                                             state, 1e-4 over a whole run
Diagnostics are FP64 on both sides: power 1e-11 relative; Hamiltonian 1e-10,
because its kinetic term psi^H K psi weights the field difference by A: a
1e-12 difference in the stiffest modes (lambda ~ rho = 1.1e3, where the two
propagators' truncation errors sit) against a field whose mean lambda is ~1.5
appears in H amplified by up to 2 sqrt(rho / lambda) ~ 50.
Sizes span many SELL slices and a ragged last slice; edge cases cover a
single triangle, fewer than 32 vertices, the maximum field count, zero steps.
"""
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


def rel(ops, a, b):
    return bpm.relative_error(ops, a, b)


def to_dev(psi, dtype=torch.complex128):
    return torch.from_numpy(np.ascontiguousarray(psi)).to(DEV, dtype)


def from_dev(t):
    return t.detach().cpu().numpy().astype(np.complex128)


@pytest.fixture(scope="module")
def fiber():
    """Step-index fiber (Table II), 3001 vertices: ~94 SELL slices with a ragged tail."""
    coords, tris = W.mesh_disk_graded(4.0, 3000, 3.0, interfaces=(1.0,), seed=31, grade_from=1.0)
    V, chi = W.step_index_materials(coords, tris)
    sigma = W.absorber_profile(coords, 4.0, 20.0)
    ops = dec.Operators(coords, tris, V, chi)
    mesh = api.Mesh(coords, tris, V, chi, sigma)
    return coords, tris, V, chi, sigma, ops, mesh


def launch(coords, B, seed=0, A=2.0):
    rng = np.random.default_rng(seed)
    cols = []
    for b in range(B):
        g = W.elliptic_gaussian(coords, A=A * (1 + 0.2 * b), x0=0.3 * rng.standard_normal(),
                                y0=0.3 * rng.standard_normal(), theta=rng.uniform(0, math.pi))
        cols.append(g * np.exp(1j * rng.uniform(0, 2 * math.pi)))
    return np.stack(cols, axis=1)


# ------------------------------------------------------------------ FP64
@pytest.mark.parametrize("B", [1, 3])
def test_fp64_fused_matches_oracle(fiber, B):
    coords, tris, V, chi, sigma, ops, mesh = fiber
    psi0 = launch(coords, B)
    dz, n = 2e-3, 25
    ref = bpm.propagate(ops, (1.0,), psi0, dz, n, sigma)
    t = to_dev(psi0 if B > 1 else psi0[:, 0])
    diag = api.propagate(mesh, t, dz, n)
    out = from_dev(t).reshape(-1, B)
    assert rel(ops, out, ref) <= 1e-12
    assert diag.shape == (1, B)
    for b in range(B):
        assert diag[0, b]["power"] == pytest.approx(bpm.power(ops, ref[:, b]), rel=1e-11)
        assert diag[0, b]["z"] == pytest.approx(dz * n)


def test_fp64_plain_matches_oracle(fiber):
    coords, tris, V, chi, sigma, ops, mesh = fiber
    psi0 = launch(coords, 1)[:, 0]
    dz, n = 2e-3, 20
    ref = bpm.propagate(ops, (1.0,), psi0, dz, n, sigma)
    t = to_dev(psi0)
    api.propagate(mesh, t, dz, n, variant="plain")
    assert rel(ops, from_dev(t), ref) <= 1e-12


def test_fp64_diagnostics_and_blocks(fiber):
    """diag_every splits the march into blocks (half steps at the block
    edges); results and the per-block power/Hamiltonian match the oracle."""
    coords, tris, V, chi, sigma, ops, mesh = fiber
    nt = len(tris)
    psi0 = launch(coords, 2, seed=3)
    dz, n, every = 1e-3, 10, 4
    m0 = api.Mesh(coords, tris, V, chi, None)     # no absorber: power conserved
    t = to_dev(psi0)
    diag = api.propagate(m0, t, dz, n, diag_every=every)
    ref = psi0.copy()
    zs = []
    steps = [4, 4, 2]
    for k, s in enumerate(steps):
        ref = bpm.propagate(ops, (1.0,), ref, dz, s)
        zs.append(sum(steps[:k + 1]) * dz)
        for b in range(2):
            assert diag[k, b]["z"] == pytest.approx(zs[-1])
            assert diag[k, b]["power"] == pytest.approx(bpm.power(ops, ref[:, b]), rel=1e-11)
            assert diag[k, b]["hamiltonian"] == pytest.approx(bpm.hamiltonian(ops, (1.0,), ref[:, b]), rel=1e-10)
            assert diag[k, b]["max_intensity"] == pytest.approx(np.max(np.abs(ref[:, b]) ** 2), rel=1e-12)
    assert rel(ops, from_dev(t), ref) <= 1e-12
    assert diag[-1, 0]["power"] == pytest.approx(bpm.power(ops, psi0[:, 0]), rel=1e-12)
    del nt


@pytest.mark.parametrize("p2", [2e-5, -3e-5])
def test_fp64_higher_order_diffraction(fiber, p2):
    """p = (p1, p2): exp(i h (p2 A^2 - p1 A)) (Table I's higher-order row) by
    the Chebyshev path whose coefficients come from a cosine transform."""
    coords, tris, V, chi, sigma, ops, mesh = fiber
    p = (1.0, p2)
    m2 = api.Mesh(coords, tris, V, chi, sigma, p=p)
    psi0 = launch(coords, 2, seed=5)
    dz, n = 1e-3, 6
    ref = bpm.propagate(ops, p, psi0, dz, n, sigma)
    t = to_dev(psi0)
    api.propagate(m2, t, dz, n)
    assert rel(ops, from_dev(t), ref) <= 1e-12


def test_fp32_higher_order_diffraction(fiber):
    """The p2 path in FP32: one step from the oracle's state (<= 1e-5) and a
    whole run (<= 1e-4)."""
    coords, tris, V, chi, sigma, ops, mesh = fiber
    p = (1.0, 2e-5)
    m2 = api.Mesh(coords, tris, V, chi, sigma, p=p)
    psi0 = launch(coords, 2, seed=15)
    dz = 1e-3
    state = bpm.propagate(ops, p, psi0, dz, 4, sigma)
    state32 = state.astype(np.complex64).astype(np.complex128)
    ref = bpm.propagate(ops, p, state32, dz, 1, sigma)
    t = to_dev(state32, torch.complex64)
    api.propagate(m2, t, dz, 1)
    assert rel(ops, from_dev(t), ref) <= 1e-5
    n = 300
    ref = bpm.propagate(ops, p, psi0, dz, n, sigma)
    t = to_dev(psi0, torch.complex64)
    api.propagate(m2, t, dz, n)
    assert rel(ops, from_dev(t), ref) <= 1e-4


def test_fp64_element_kerr(fiber):
    coords, tris, V, chi, sigma, ops, mesh = fiber
    psi0 = launch(coords, 2, seed=6, A=3.0)
    dz, n = 2e-3, 12
    ref = bpm.propagate(ops, (1.0,), psi0, dz, n, sigma, kerr="element")
    t = to_dev(psi0)
    api.propagate(mesh, t, dz, n, kerr="element")
    assert rel(ops, from_dev(t), ref) <= 1e-12


def test_fp64_soliton_1d_full_run():
    """Config of the exact sech soliton (1024 jittered nodes, dz = 1e-3,
    2000 steps, C128): GPU equals the oracle, both near sech(x) e^{iz/2}."""
    wl = W.soliton_1d()
    m = wl.meshes[0]
    ops = dec.Operators(m.coords, m.cells, m.V_cell, m.chi_cell)
    psi0 = wl.psi0[0][:, 0]
    ref = bpm.propagate(ops, wl.p, psi0, wl.dz, wl.n_steps)
    mesh = api.Mesh.from_workload(m, p=wl.p)
    t = to_dev(psi0)
    api.propagate(mesh, t, wl.dz, wl.n_steps)
    out = from_dev(t)
    assert rel(ops, out, ref) <= 1e-12
    z = wl.dz * wl.n_steps
    assert rel(ops, out, W.sech_1d(m.coords) * np.exp(0.5j * z)) < 5e-4


# ------------------------------------------------------------------ FP32
@pytest.mark.parametrize("B", [1, 2, 16, 20, 64])
def test_fp32_one_step_from_oracle_state(fiber, B):
    coords, tris, V, chi, sigma, ops, mesh = fiber
    psi0 = launch(coords, B, seed=7)
    dz = 2e-3
    state = bpm.propagate(ops, (1.0,), psi0, dz, 5, sigma)
    state32 = state.astype(np.complex64).astype(np.complex128)
    ref = bpm.propagate(ops, (1.0,), state32, dz, 1, sigma)
    t = to_dev(state32, torch.complex64)
    api.propagate(mesh, t, dz, 1)
    assert rel(ops, from_dev(t).reshape(-1, B), ref) <= 1e-5


def test_fp32_full_run(fiber):
    coords, tris, V, chi, sigma, ops, mesh = fiber
    psi0 = launch(coords, 4, seed=8)
    dz, n = 1e-3, 400
    ref = bpm.propagate(ops, (1.0,), psi0, dz, n, sigma)
    t = to_dev(psi0, torch.complex64)
    diag = api.propagate(mesh, t, dz, n)
    assert rel(ops, from_dev(t), ref) <= 1e-4
    for b in range(4):
        assert diag[0, b]["power"] == pytest.approx(bpm.power(ops, ref[:, b]), rel=1e-4)


def test_fp32_element_kerr(fiber):
    coords, tris, V, chi, sigma, ops, mesh = fiber
    psi0 = launch(coords, 2, seed=9, A=3.0)
    dz, n = 2e-3, 50
    ref = bpm.propagate(ops, (1.0,), psi0, dz, n, sigma, kerr="element")
    t = to_dev(psi0, torch.complex64)
    api.propagate(mesh, t, dz, n, kerr="element")
    assert rel(ops, from_dev(t), ref) <= 1e-4


# ------------------------------------------------------------------ batched plans
@pytest.mark.parametrize("precision,tol", [("c128", 1e-12), ("c64", 1e-4)])
def test_batched_plan_uneven_meshes(precision, tol):
    """Meshes of uneven size (and so different Chebyshev degrees) and
    different field counts advance in one persistent launch."""
    specs = [(600, 3, 41), (2500, 1, 42), (5000, 4, 43), (90, 2, 44)]
    meshes, opss, sigs, psis = [], [], [], []
    for n, B, seed in specs:
        coords, tris = W.mesh_disk_graded(4.0, n, 3.0, interfaces=(1.0,), seed=seed, grade_from=1.0)
        V, chi = W.step_index_materials(coords, tris)
        sigma = W.absorber_profile(coords, 4.0, 20.0)
        meshes.append(api.Mesh(coords, tris, V, chi, sigma))
        opss.append(dec.Operators(coords, tris, V, chi))
        sigs.append(sigma)
        psis.append(W.hg_superpositions(coords, B, np.random.default_rng(seed)))
    dt = torch.complex64 if precision == "c64" else torch.complex128
    plan = api.Plan(meshes, [s[1] for s in specs], precision)
    degs = [plan.degree(i, 2e-3) for i in range(len(specs))]
    assert len(set(degs)) > 1
    ts = [to_dev(p, dt) for p in psis]
    dz, n = 2e-3, 30
    diag = plan.propagate(ts, dz, n)
    assert diag.shape == (1, sum(s[1] for s in specs))
    for ops, sigma, p0, t in zip(opss, sigs, psis, ts):
        ref = bpm.propagate(ops, (1.0,), p0, dz, n, sigma)
        assert rel(ops, from_dev(t), ref) <= tol
    # a second call reuses the captured graph and continues from the new state
    before = [from_dev(t) for t in ts]
    plan.propagate(ts, dz, 3)
    for ops, sigma, p0, t in zip(opss, sigs, before, ts):
        ref = bpm.propagate(ops, (1.0,), p0, dz, 3, sigma)
        assert rel(ops, from_dev(t), ref) <= tol


@pytest.mark.parametrize("kerr", ["lumped", "element"])
def test_tile_staged_kernel_equals_row_kernel(kerr):
    """complex64 plans with 9..16 fields run the tile-staged kernel (operands
    staged in shared memory by bulk copies, neighbour gathers from the tile
    window).  It performs the row kernel's arithmetic in the same order, so
    the two variants agree bit for bit: meshes below one tile, with a ragged
    last tile, a single triangle, several diagnostic launches."""
    specs = [(600, 16, 51), (2500, 9, 52), (5000, 12, 53), (90, 16, 54), (40, 16, 55)]
    meshes, psis = [], []
    for n, B, seed in specs:
        coords, tris = W.mesh_disk_graded(4.0, n, 3.0, interfaces=(1.0,), seed=seed, grade_from=1.0)
        V, chi = W.step_index_materials(coords, tris)
        sigma = W.absorber_profile(coords, 4.0, 20.0)
        meshes.append(api.Mesh(coords, tris, V, chi, sigma))
        psis.append(W.hg_superpositions(coords, B, np.random.default_rng(seed)))
    coords = np.array([[0.0, 0.0], [1.0, 0.0], [0.2, 0.9]])
    meshes.append(api.Mesh(coords, np.array([[0, 1, 2]], dtype=np.int32), np.array([-2.0]), np.array([1.5])))
    psis.append(np.exp(1j * np.arange(3 * 16).reshape(3, 16) * 0.3) * 0.5)
    plan = api.Plan(meshes, [p.shape[1] for p in psis], "c64")
    cfg = plan.config()
    assert cfg["tile_slots"] >= 2 and cfg["tile_grid"] > 0
    dz, n = 2e-3, 5
    a = [to_dev(p, torch.complex64) for p in psis]
    b = [to_dev(p, torch.complex64) for p in psis]
    da = plan.propagate(a, dz, n, diag_every=2, kerr=kerr)
    db = plan.propagate(b, dz, n, diag_every=2, kerr=kerr, variant="rows")
    for x, y in zip(a, b):
        assert torch.equal(x, y)
    assert np.array_equal(da["power"], db["power"])
    assert all(torch.isfinite(torch.view_as_real(x)).all() for x in a)


@pytest.mark.parametrize("kerr", ["lumped", "element"])
def test_tile_staged_ring_wraps_many_times(kerr):
    """A 100k-vertex fiber (782 tiles): every CTA fills and drains its
    shared-memory ring several times per stage and the copy warps' look-ahead
    crosses stage and step boundaries; still bit for bit the row kernel."""
    coords, tris = W.mesh_disk_graded(4.0, 100_000, 3.0, interfaces=(1.0,), seed=61, grade_from=1.0)
    V, chi = W.step_index_materials(coords, tris)
    sigma = W.absorber_profile(coords, 4.0, 20.0)
    mesh = api.Mesh(coords, tris, V, chi, sigma)
    psi0 = W.hg_superpositions(coords, 16, np.random.default_rng(61))
    plan = api.Plan([mesh], [16], "c64")
    assert plan.config()["tile_slots"] >= 2
    a, b = to_dev(psi0, torch.complex64), to_dev(psi0, torch.complex64)
    plan.propagate([a], 5e-4, 3, kerr=kerr)
    plan.propagate([b], 5e-4, 3, kerr=kerr, variant="rows")
    assert torch.equal(a, b)


def test_tile_staged_full_bench_batch_one_step():
    """The bench workload at full size (16 fibers, 20k..500k vertices, 16
    fields): one step of the tile-staged kernel equals the row kernel."""
    wl = W.batched_fibers(n_meshes=16, fields_per_mesh=16, n_min=20_000, ratio=25.0, seed=4)
    meshes = [api.Mesh.from_workload(m, p=wl.p) for m in wl.meshes]
    plan = api.Plan(meshes, [16] * len(meshes), "c64")
    assert plan.config()["tile_slots"] >= 2
    a = [to_dev(p, torch.complex64) for p in wl.psi0]
    b = [x.clone() for x in a]
    plan.propagate(a, wl.dz, 1)
    plan.propagate(b, wl.dz, 1, variant="rows")
    for x, y in zip(a, b):
        assert torch.equal(x, y)


@pytest.mark.parametrize("kerr", ["lumped", "element"])
def test_stage_pair_kernel(kerr):
    """The stage-pair kernel (two Clenshaw stages per grid-wide pass, depth-two
    halos recomputed per tile) on meshes of uneven size and degree (so that a
    mesh's top stage falls in either phase of a pass, and single and final
    passes occur), with 9..16 fields, a single triangle and meshes below one
    tile: against the row kernel (FP32 rounding only: <= 2e-6 relative after
    7 steps in three blocks) and against the FP64 oracle within the FP32
    bars (one step <= 1e-5, the run <= 1e-4)."""
    specs = [(600, 16, 51), (2500, 9, 52), (5000, 12, 53), (90, 16, 54), (40, 16, 55), (3, 16, 56)]
    meshes, opss, sigs, psis = [], [], [], []
    for n, B, seed in specs:
        if n == 3:
            coords = np.array([[0.0, 0.0], [1.0, 0.0], [0.2, 0.9]])
            tris = np.array([[0, 1, 2]], dtype=np.int32)
        else:
            coords, tris = W.mesh_disk_graded(4.0, n, 3.0, interfaces=(1.0,), seed=seed, grade_from=1.0)
        V, chi = W.step_index_materials(coords, tris)
        sigma = W.absorber_profile(coords, 4.0, 20.0)
        meshes.append(api.Mesh(coords, tris, V, chi, sigma))
        opss.append(dec.Operators(coords, tris, V, chi))
        sigs.append(sigma)
        psis.append(W.hg_superpositions(coords, B, np.random.default_rng(seed)) * 2.0)
    plan = api.Plan(meshes, [p.shape[1] for p in psis], "c64")
    cfg = plan.config()
    assert cfg["pair_slots"] >= 2 and cfg["tile_slots"] >= 2
    dz = 2e-3
    degs = [plan.degree(i, dz) for i in range(len(specs))]
    assert len({d % 2 for d in degs}) == 2          # both parities: top stages in both phases
    a = [to_dev(p, torch.complex64) for p in psis]
    b = [x.clone() for x in a]
    plan.propagate(a, dz, 7, diag_every=3, kerr=kerr, variant="pairs")
    plan.propagate(b, dz, 7, diag_every=3, kerr=kerr, variant="rows")
    for x, y in zip(a, b):
        assert torch.isfinite(torch.view_as_real(x)).all()
        d = float(torch.linalg.vector_norm((x - y).to(torch.complex128)) / torch.linalg.vector_norm(y.to(torch.complex128)))
        assert d <= 2e-6, d
    for ops, sigma, p0, t in zip(opss, sigs, psis, a):
        ref = bpm.propagate(ops, (1.0,), p0, dz, 7, sigma, kerr=kerr)
        assert rel(ops, from_dev(t), ref) <= 1e-4
    # one step from the oracle's state rounded to FP32
    states = [bpm.propagate(ops, (1.0,), p0, dz, 3, sigma, kerr=kerr).astype(np.complex64) for ops, sigma, p0 in
              zip(opss, sigs, psis)]
    c = [to_dev(st, torch.complex64) for st in states]
    plan.propagate(c, dz, 1, kerr=kerr, variant="pairs")
    for ops, sigma, st, t in zip(opss, sigs, states, c):
        ref = bpm.propagate(ops, (1.0,), st.astype(np.complex128), dz, 1, sigma, kerr=kerr)
        assert rel(ops, from_dev(t), ref) <= 1e-5


def test_stage_pair_kernel_full_bench_batch():
    """The bench workload at full size: a 3-step launch of the stage-pair
    kernel against the row kernel (FP32 rounding only)."""
    wl = W.batched_fibers(n_meshes=16, fields_per_mesh=16, n_min=20_000, ratio=25.0, seed=4)
    meshes = [api.Mesh.from_workload(m, p=wl.p) for m in wl.meshes]
    plan = api.Plan(meshes, [16] * len(meshes), "c64")
    assert plan.config()["pair_slots"] >= 2
    a = [to_dev(p, torch.complex64) for p in wl.psi0]
    b = [x.clone() for x in a]
    plan.propagate(a, wl.dz, 3, variant="pairs")
    plan.propagate(b, wl.dz, 3, variant="rows")
    for x, y in zip(a, b):
        d = float(torch.linalg.vector_norm((x - y).to(torch.complex128)) / torch.linalg.vector_norm(y.to(torch.complex128)))
        assert d <= 2e-6, d


@pytest.mark.parametrize("kerr", ["lumped", "element"])
def test_dataflow_kernel_matches_tile_kernel(kerr):
    """The dataflow kernel (no grid barrier between Clenshaw stages; a tile
    waits for its neighbour tiles' previous stage) gives the tile-staged
    kernel's fields bit for bit: meshes of uneven size and degree (meshes
    join the march at different stages), 9..16 fields, a mesh below one tile
    and a single triangle, three launches (diagnostics every 3 of 7 steps),
    walk skips from 1 to beyond a CTA's share, either walk, per-CTA chunks or
    the tile kernel's contiguous ranges.  Repeated runs
    of one shape are bitwise equal too (the waits order every read after the
    write it needs, whatever the timing)."""
    specs = [(600, 16, 51), (2500, 9, 52), (5000, 12, 53), (90, 16, 54), (40, 16, 55), (3, 16, 56),
             (20000, 16, 57)]
    meshes, psis = [], []
    for n, B, seed in specs:
        if n == 3:
            coords = np.array([[0.0, 0.0], [1.0, 0.0], [0.2, 0.9]])
            tris = np.array([[0, 1, 2]], dtype=np.int32)
        else:
            coords, tris = W.mesh_disk_graded(4.0, n, 3.0, interfaces=(1.0,), seed=seed, grade_from=1.0)
        V, chi = W.step_index_materials(coords, tris)
        sigma = W.absorber_profile(coords, 4.0, 20.0)
        meshes.append(api.Mesh(coords, tris, V, chi, sigma))
        psis.append(W.hg_superpositions(coords, B, np.random.default_rng(seed)) * 2.0)
    plan = api.Plan(meshes, [p.shape[1] for p in psis], "c64")
    assert plan.config()["flow_grid"] > 0
    dz = 2e-3
    assert len({plan.degree(i, dz) for i in range(len(specs))}) >= 3
    ref = [to_dev(p, torch.complex64) for p in psis]
    plan.set_shape("tile", tile_slots=3)
    plan.propagate(ref, dz, 7, diag_every=3, kerr=kerr)
    for slots, skip, fw, reps, ranges in ((3, 8, 0, 3, 0), (2, 8, 0, 1, 0), (3, 1, 0, 1, 0), (3, 4000, 0, 1, 0),
                                          (3, 8, 1, 1, 0), (3, 8, 0, 2, 1), (3, 8, 1, 1, 1), (2, 1, 0, 1, 1)):
        plan.set_shape("flow", tile_slots=slots, walk_skip=skip, forward_walk=fw, flow_ranges=ranges)
        assert plan.config()["flow_ranges"] == ranges
        for _ in range(reps):
            out = [to_dev(p, torch.complex64) for p in psis]
            plan.propagate(out, dz, 7, diag_every=3, kerr=kerr)
            for x, y in zip(out, ref):
                assert torch.equal(x, y), (slots, skip, fw, ranges)
    # the explicit variant runs it whatever shape the plan holds
    plan.set_shape("tile", tile_slots=3)
    out = [to_dev(p, torch.complex64) for p in psis]
    plan.propagate(out, dz, 7, diag_every=3, kerr=kerr, variant="flow")
    for x, y in zip(out, ref):
        assert torch.equal(x, y)


def test_dataflow_kernel_repeated_launches_are_bitwise_stable():
    """Ordering check of the dataflow kernel's completion protocol: many
    launches of a plan whose meshes join the march at different stages,
    cycling the ring slots, walk skips, walk direction and tile assignment,
    each bit for bit the tile-staged kernel's fields (a tile published before
    all its rows were stored would show up as a last-bit difference)."""
    specs = [(600, 16, 51), (2500, 9, 52), (5000, 12, 53), (90, 16, 54), (40, 16, 55), (20000, 16, 57),
             (9000, 10, 58)]
    meshes, psis = [], []
    for n, B, seed in specs:
        coords, tris = W.mesh_disk_graded(4.0, n, 3.0, interfaces=(1.0,), seed=seed, grade_from=1.0)
        V, chi = W.step_index_materials(coords, tris)
        meshes.append(api.Mesh(coords, tris, V, chi, W.absorber_profile(coords, 4.0, 20.0)))
        psis.append(W.hg_superpositions(coords, B, np.random.default_rng(seed)) * 2.0)
    plan = api.Plan(meshes, [p.shape[1] for p in psis], "c64")
    plan.set_shape("tile", tile_slots=3)
    ref = [to_dev(p, torch.complex64) for p in psis]
    plan.propagate(ref, 2e-3, 40)
    for rep in range(16):
        plan.set_shape("flow", tile_slots=3 if rep % 2 else 2, walk_skip=1 + rep % 9, forward_walk=int(rep % 3 == 0),
                       flow_ranges=rep % 2)
        out = [to_dev(p, torch.complex64) for p in psis]
        plan.propagate(out, 2e-3, 40)
        for x, y in zip(out, ref):
            assert torch.equal(x, y), rep


def test_dataflow_kernel_full_bench_batch():
    """The bench workload at full size: 3-step launches of the dataflow kernel
    (per-CTA chunks and contiguous ranges, several walks) against the
    tile-staged kernel, bit for bit."""
    wl = W.batched_fibers(n_meshes=16, fields_per_mesh=16, n_min=20_000, ratio=25.0, seed=4)
    meshes = [api.Mesh.from_workload(m, p=wl.p) for m in wl.meshes]
    plan = api.Plan(meshes, [16] * len(meshes), "c64")
    assert plan.config()["flow_grid"] > 0
    a = [to_dev(p, torch.complex64) for p in wl.psi0]
    b = [x.clone() for x in a]
    plan.propagate(a, wl.dz, 3, variant="flow")
    plan.set_shape("tile", tile_slots=3)
    plan.propagate(b, wl.dz, 3)
    for x, y in zip(a, b):
        assert torch.equal(x, y)
    # the tile kernel's contiguous ranges: a tile's own rows may come from
    # another CTA's stores of the stage just before (ordering of the async-proxy
    # bulk reads after the completion counters), several walks, repeated
    for skip, fw in ((16, 0), (8, 0), (4, 0), (8, 1), (16, 0)):
        plan.set_shape("flow", tile_slots=3, walk_skip=skip, forward_walk=fw, flow_ranges=1)
        c = [to_dev(p, torch.complex64) for p in wl.psi0]
        plan.propagate(c, wl.dz, 3)
        for x, y in zip(c, b):
            assert torch.equal(x, y), (skip, fw)


@pytest.mark.parametrize("precision", ["c64", "c128"])
def test_autotuner_picks_a_shape_without_changing_results(precision):
    """decbpm_plan_autotune times the FUSED launch shapes (tile-staged kernel
    with 3/2 ring slots, row kernel with 1..max CTAs per SM, walk order) and
    keeps the fastest: the fields it produces are bit for bit those of the
    default shape; a second plan of the same problem takes the cached choice."""
    specs = [(4000, 16, 81), (12000, 16, 82), (600, 9, 83)]
    meshes, psis = [], []
    for n, B, seed in specs:
        coords, tris = W.mesh_disk_graded(4.0, n, 3.0, interfaces=(1.0,), seed=seed, grade_from=1.0)
        V, chi = W.step_index_materials(coords, tris)
        sigma = W.absorber_profile(coords, 4.0, 20.0)
        meshes.append(api.Mesh(coords, tris, V, chi, sigma))
        psis.append(W.hg_superpositions(coords, B, np.random.default_rng(seed)))
    dt = torch.complex64 if precision == "c64" else torch.complex128
    dz = 5e-4
    ref_plan = api.Plan(meshes, [p.shape[1] for p in psis], precision)
    a = [to_dev(p, dt) for p in psis]
    ref_plan.propagate(a, dz, 7)
    plan = api.Plan(meshes, [p.shape[1] for p in psis], precision)
    tune = plan.autotune(dz, trial_steps=2)
    assert tune["from_cache"] == 0 and tune["candidates"] >= 2 and tune["ms_per_step"] > 0
    cfg = plan.config()
    assert cfg["tuned"] == 1
    assert cfg["fused_kernel"] == {"flow": 3, "pairs": 2, "tile": 1, "rows": 0}[tune["kernel"]]
    if precision == "c128":
        assert tune["kernel"] == "rows"
    b = [to_dev(p, dt) for p in psis]
    plan.propagate(b, dz, 7)
    for x, y in zip(a, b):
        if tune["kernel"] == "pairs":       # the stage-pair kernel rounds differently (FP32 level)
            d = float(torch.linalg.vector_norm((x - y).to(torch.complex128)) / torch.linalg.vector_norm(y))
            assert d <= 2e-6, d
        else:
            assert torch.equal(x, y)
    again = api.Plan(meshes, [p.shape[1] for p in psis], precision).autotune(dz, trial_steps=2)
    assert again["from_cache"] == 1
    keys = ("kernel", "ctas_per_sm", "tile_slots", "forward_walk", "walk_skip", "flow_ranges")
    assert {k: again[k] for k in keys} == {k: tune[k] for k in keys}
    with pytest.raises(L.DecbpmError):
        plan.autotune(dz, trial_steps=0)
    with pytest.raises(L.DecbpmError):
        plan.autotune(-1.0)


@pytest.mark.parametrize("B", [4, 8, 16])
def test_every_launch_shape_gives_the_same_fields(B):
    """decbpm_plan_set_shape forces each single-stage launch shape the
    autotuner searches (row kernel with 4 or 2 complex values per thread, i.e.
    8B/4B.. rows per warp item, 1..max CTAs per SM, either walk; the
    tile-staged kernel with 3 or 2 slots; the dataflow kernel with 3 or 2 slots,
    several walk skips and either walk): every one gives the default shape's
    fields bit for bit; shapes a plan cannot run are refused."""
    specs = [(3000, 61), (700, 62)]
    meshes, psis = [], []
    for n, seed in specs:
        coords, tris = W.mesh_disk_graded(4.0, n, 3.0, interfaces=(1.0,), seed=seed, grade_from=1.0)
        V, chi = W.step_index_materials(coords, tris)
        sigma = W.absorber_profile(coords, 4.0, 20.0)
        meshes.append(api.Mesh(coords, tris, V, chi, sigma))
        psis.append(W.hg_superpositions(coords, B, np.random.default_rng(seed)))
    plan = api.Plan(meshes, [B] * len(specs), "c64")
    ref = [to_dev(p, torch.complex64) for p in psis]
    plan.propagate(ref, 1e-3, 5, variant="rows")
    shapes = [dict(kernel="rows", ctas_per_sm=c, values_per_thread=v, forward_walk=f)
              for v in (4, 2) for c in (1, 2) for f in (0, 1)]
    if B == 16:
        shapes += [dict(kernel="tile", tile_slots=t) for t in (2, 3)]
        shapes += [dict(kernel="flow", tile_slots=t, walk_skip=k, forward_walk=f)
                   for t in (2, 3) for k in (1, 8, 1000) for f in (0, 1)]
    for sh in shapes:
        plan.set_shape(**sh)
        cfg = plan.config()
        if sh["kernel"] == "rows":
            assert cfg["values_per_thread"] == sh["values_per_thread"]
            assert cfg["rows_per_item"] == 32 * sh["values_per_thread"] // B
        if sh["kernel"] == "flow":
            assert cfg["fused_kernel"] == 3 and cfg["flow_skip"] == sh["walk_skip"] and cfg["flow_grid"] > 0
        out = [to_dev(p, torch.complex64) for p in psis]
        plan.propagate(out, 1e-3, 5)
        for x, y in zip(out, ref):
            assert torch.equal(x, y), sh
    with pytest.raises(L.DecbpmError):
        plan.set_shape(kernel="rows", values_per_thread=8)
    if B != 16:
        with pytest.raises(L.DecbpmError):
            plan.set_shape(kernel="tile", tile_slots=2)
        with pytest.raises(L.DecbpmError):
            plan.set_shape(kernel="flow", tile_slots=2)
    else:
        with pytest.raises(L.DecbpmError):
            plan.set_shape(kernel="flow", tile_slots=3, walk_skip=-1)


def _group_sizes(B, g=16):
    n = -(-B // g)
    return [B // n + (1 if k < B % n else 0) for k in range(n)]


@pytest.mark.parametrize("kerr", ["lumped", "element"])
def test_field_groups_equal_their_groups_as_meshes(kerr):
    """A complex64 plan with more than 16 fields on a mesh runs that mesh as
    field groups of at most 16 (balanced, consecutive, sharing the operator):
    meshes with 20, 4 and 33 fields make 2 + 1 + 3 entries of padded width 16,
    on the tile-staged kernel.  Fields and diagnostic records are bit for bit
    those of a plan that lists each group as a mesh of its own, through the
    host-buffer call too; one mesh with 32 fields through decbpm_propagate
    equals its two halves propagated separately."""
    specs = [(2000, 20, 61), (600, 4, 62), (5000, 33, 63)]
    meshes, psis = [], []
    for nv, B, seed in specs:
        coords, tris = W.mesh_disk_graded(4.0, nv, 3.0, interfaces=(1.0,), seed=seed, grade_from=1.0)
        V, chi = W.step_index_materials(coords, tris)
        sigma = W.absorber_profile(coords, 4.0, 20.0)
        meshes.append(api.Mesh(coords, tris, V, chi, sigma))
        psis.append(np.ascontiguousarray(W.hg_superpositions(coords, B, np.random.default_rng(seed)) * 2.0))
    dz, n, every = 2e-3, 7, 3
    plan = api.Plan(meshes, [p.shape[1] for p in psis], "c64")
    cfg = plan.config()
    assert (cfg["field_groups"], cfg["n_meshes"], cfg["fields_padded"], cfg["fused_kernel"]) == (6, 3, 16, 1)
    t = [to_dev(p, torch.complex64) for p in psis]
    d = plan.propagate(t, dz, n, diag_every=every, kerr=kerr)
    gm, gp = [], []
    for m, p in zip(meshes, psis):
        f0 = 0
        for b in _group_sizes(p.shape[1]):
            gm.append(m)
            gp.append(np.ascontiguousarray(p[:, f0:f0 + b]))
            f0 += b
    ref_plan = api.Plan(gm, [p.shape[1] for p in gp], "c64")
    assert ref_plan.config()["field_groups"] == 6
    r = [to_dev(p, torch.complex64) for p in gp]
    dr = ref_plan.propagate(r, dz, n, diag_every=every, kerr=kerr)
    k = 0
    for i, p in enumerate(psis):
        g = len(_group_sizes(p.shape[1]))
        assert torch.equal(t[i], torch.cat(r[k:k + g], dim=1)), i
        k += g
    assert d.shape == dr.shape == (3, 57) and np.array_equal(d, dr)
    h = [torch.from_numpy(p.astype(np.complex64)).pin_memory() for p in psis]
    dh = plan.propagate_host(h, dz, n, diag_every=every, kerr=kerr)
    for i in range(len(psis)):
        assert torch.equal(h[i], t[i].cpu()), i
    assert np.array_equal(dh, d)
    # one mesh, 32 fields: the single-mesh entry point groups them too
    m, p32 = meshes[2], np.ascontiguousarray(psis[2][:, :32])
    a = to_dev(p32, torch.complex64)
    api.propagate(m, a, dz, n, kerr=kerr)
    halves = [to_dev(np.ascontiguousarray(p32[:, j:j + 16]), torch.complex64) for j in (0, 16)]
    for x in halves:
        api.propagate(m, x, dz, n, kerr=kerr)
    assert torch.equal(a, torch.cat(halves, dim=1))


@pytest.mark.parametrize("kerr", ["lumped", "element"])
def test_single_field_tile_kernel_matches_row_kernel(kerr):
    """Complex64 plans of one field per mesh can run the single-field
    tile-staged kernel (512-row tiles staged in shared memory, one row per
    thread; the autotuner's choice, the row kernel by default): bit for bit
    the row kernel's fields, on meshes of uneven size
    and degree (several tiles with ragged last tiles, a mesh below one tile,
    a single triangle), with 3 and 2 ring slots, over three launches
    (diagnostics every 3 of 7 steps); and the oracle within the FP32 bars."""
    specs = [(6000, 81), (1500, 82), (300, 83), (3, 84), (40000, 85)]
    meshes, opss, sigs, psis = [], [], [], []
    for n, seed in specs:
        if n == 3:
            coords = np.array([[0.0, 0.0], [1.0, 0.0], [0.2, 0.9]])
            tris = np.array([[0, 1, 2]], dtype=np.int32)
        else:
            coords, tris = W.mesh_disk_graded(4.0, n, 3.0, interfaces=(1.0,), seed=seed, grade_from=1.0)
        V, chi = W.step_index_materials(coords, tris)
        sigma = W.absorber_profile(coords, 4.0, 20.0)
        meshes.append(api.Mesh(coords, tris, V, chi, sigma))
        opss.append(dec.Operators(coords, tris, V, chi))
        sigs.append(sigma)
        psis.append(W.hg_superpositions(coords, 1, np.random.default_rng(seed)) * 2.0)
    plan = api.Plan(meshes, [1] * len(specs), "c64")
    cfg = plan.config()
    assert cfg["fused_kernel"] == 0 and cfg["tile_rows"] == 512 and cfg["tile_slots"] >= 2
    dz = 2e-3
    plan.set_shape("rows", ctas_per_sm=2)
    ref = [to_dev(p, torch.complex64) for p in psis]
    plan.propagate(ref, dz, 7, diag_every=3, kerr=kerr)
    for slots in range(cfg["tile_slots"], 1, -1):
        plan.set_shape("tile", tile_slots=slots)
        assert plan.config()["fused_kernel"] == 1
        out = [to_dev(p, torch.complex64) for p in psis]
        plan.propagate(out, dz, 7, diag_every=3, kerr=kerr)
        for x, y in zip(out, ref):
            assert torch.equal(x, y), slots
    for ops, sigma, p0, t in zip(opss[:4], sigs, psis, out):
        want = bpm.propagate(ops, (1.0,), p0, dz, 7, sigma, kerr=kerr)
        assert rel(ops, from_dev(t), want) <= 1e-4


@pytest.mark.parametrize("precision,B", [("c64", 1), ("c128", 1), ("c64", 4)])
def test_row_kernel_metadata_cache(precision, B):
    """Single-mesh plans cache each CTA's warp-item metadata (columns,
    weights, slice widths) in shared memory once per launch: the fields are
    bit for bit those of the uncached row kernel, at 1..4 CTAs per SM (the
    cache is dropped where it would cost co-residency), both Kerr modes and
    several launches (diagnostics every 4 of 9 steps)."""
    coords, tris = W.mesh_disk_graded(4.0, 6000, 3.0, interfaces=(1.0,), seed=91, grade_from=1.0)
    V, chi = W.step_index_materials(coords, tris)
    sigma = W.absorber_profile(coords, 4.0, 20.0)
    mesh = api.Mesh(coords, tris, V, chi, sigma)
    psi0 = W.hg_superpositions(coords, B, np.random.default_rng(92)) * 2.0
    dt = torch.complex64 if precision == "c64" else torch.complex128
    plan = api.Plan([mesh], [B], precision)
    n_cached = 0
    for kerr in ("lumped", "element"):
        plan.set_shape("rows", ctas_per_sm=1, no_meta_cache=1)
        assert plan.config()["meta_items"] == 0
        ref = to_dev(psi0, dt)
        plan.propagate([ref], 1e-3, 9, diag_every=4, kerr=kerr)
        for per_sm in (1, 2, 4):
            try:
                plan.set_shape("rows", ctas_per_sm=per_sm)
            except L.DecbpmError:
                continue            # more CTAs per SM than this build can hold
            n_cached += plan.config()["meta_items"] > 0
            out = to_dev(psi0, dt)
            plan.propagate([out], 1e-3, 9, diag_every=4, kerr=kerr)
            assert torch.equal(out, ref), (kerr, per_sm)
    assert n_cached >= 2


# ------------------------------------------------------------------ edge cases
def test_single_triangle_and_tiny_meshes():
    coords = np.array([[0.0, 0.0], [1.0, 0.0], [0.2, 0.9]])
    tris = np.array([[0, 1, 2]], dtype=np.int32)
    ops = dec.Operators(coords, tris, np.array([-2.0]), np.array([1.5]))
    mesh = api.Mesh(coords, tris, np.array([-2.0]), np.array([1.5]))
    psi0 = np.array([1.0 + 0.5j, -0.3j, 0.7])
    ref = bpm.propagate(ops, (1.0,), psi0, 0.01, 7)
    t = to_dev(psi0)
    api.propagate(mesh, t, 0.01, 7)
    assert rel(ops, from_dev(t), ref) <= 1e-12
    # 17 vertices: a single partial SELL slice
    coords, tris = W.mesh_disk_graded(1.0, 17, 1.0, seed=3)
    ops = dec.Operators(coords, tris)
    mesh = api.Mesh(coords, tris)
    psi0 = W.gaussian(coords, w=0.5)
    ref = bpm.propagate(ops, (1.0,), psi0, 0.01, 5)
    t = to_dev(psi0)
    api.propagate(mesh, t, 0.01, 5)
    assert rel(ops, from_dev(t), ref) <= 1e-12


def test_zero_steps_and_max_fields(fiber):
    coords, tris, V, chi, sigma, ops, mesh = fiber
    psi0 = launch(coords, 64, seed=10)
    t = to_dev(psi0)
    diag = api.propagate(mesh, t, 1e-3, 0)
    assert np.array_equal(from_dev(t), psi0)
    assert diag.shape == (1, 64)
    assert diag[0, 63]["power"] == pytest.approx(bpm.power(ops, psi0[:, 63]), rel=1e-12)
    ref = bpm.propagate(ops, (1.0,), psi0, 1e-3, 2, sigma)
    api.propagate(mesh, t, 1e-3, 2)
    assert rel(ops, from_dev(t), ref) <= 1e-12


def test_fields_beyond_maximum_are_rejected(fiber):
    from paper_2608_03587_b300 import _lib as L
    coords, tris, V, chi, sigma, ops, mesh = fiber
    t = torch.zeros((len(coords), 65), dtype=torch.complex64, device=DEV)
    with pytest.raises(L.DecbpmError) as e:
        api.propagate(mesh, t, 1e-3, 1)
    assert e.value.code == L.ERR_UNSUPPORTED


def test_host_buffer_entry_point(fiber):
    coords, tris, V, chi, sigma, ops, mesh = fiber
    psi0 = launch(coords, 2, seed=11)
    ref = bpm.propagate(ops, (1.0,), psi0, 2e-3, 5, sigma)
    h = torch.from_numpy(psi0.copy()).pin_memory()
    api.propagate_host(mesh, h, 2e-3, 5)
    assert rel(ops, h.numpy(), ref) <= 1e-12


def test_deterministic_bitwise(fiber):
    coords, tris, V, chi, sigma, ops, mesh = fiber
    psi0 = launch(coords, 2, seed=12)
    outs, diags = [], []
    for _ in range(2):
        t = to_dev(psi0, torch.complex64)
        diags.append(api.propagate(mesh, t, 2e-3, 15))
        outs.append(from_dev(t))
    assert np.array_equal(outs[0], outs[1])
    assert diags[0]["power"].tolist() == diags[1]["power"].tolist()


# ------------------------------------------------------------------ full size
def test_full_size_gaussian_disk_one_step_sampled():
    """The 200k-vertex graded-disk workload at full size, in the launch
    configuration of the benchmark (C64, fused): one step from the launch
    field against the oracle's step, on all vertices."""
    wl = W.gaussian_disk()
    m = wl.meshes[0]
    ops = dec.Operators(m.coords, m.cells, m.V_cell, m.chi_cell)
    psi0 = wl.psi0[0][:, 0]
    ref = bpm.propagate(ops, wl.p, psi0, wl.dz, 1, m.sigma)
    mesh = api.Mesh.from_workload(m)
    assert mesh.n_vertices >= 196_000
    t = to_dev(psi0.astype(np.complex64), torch.complex64)
    api.propagate(mesh, t, wl.dz, 1)
    assert rel(ops, from_dev(t), ref) <= 1e-5
    t = to_dev(psi0)
    api.propagate(mesh, t, wl.dz, 1)
    assert rel(ops, from_dev(t), ref) <= 1e-12
