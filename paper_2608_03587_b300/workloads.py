"""Seeded synthetic inputs shaped like the paper's workloads.

This module makes meshes, per-cell material data, absorber profiles and launch
fields.  It holds none of the method's arithmetic: no Hodge star, no cotangent
weight, no exterior derivative and no propagation.  Both the CUDA path and the
CPU oracle take its arrays as plain inputs.

Geometry conventions
--------------------
* 1D meshes: ``coords`` is ``[N0, 1]`` float64, ``cells`` is ``[N0-1, 2]`` int32.
* 2D meshes: ``coords`` is ``[N0, 2]`` float64, ``cells`` is ``[N2, 3]`` int32,
  every triangle counter-clockwise (the consistent orientation the paper assumes
  for 2-simplices, Sec. "DEC computational framework").
* Material data is per cell, evaluated at the cell centroid (the paper assigns
  the potential of each triangle its value at the centroid, Sec. "Discrete
  Hodge star").  The absorber strength ``sigma`` is per vertex.

Workload recipes (sizes, launches) follow the paper's benchmarks: the
off-axis elliptic Gaussian (Eq. for psi_0(U,V) with U,V rotated coordinates),
the elliptic vortex with charge m=1, the step-index fiber of Table II
(V-number 5.46, DEC disk of radius 4 in units of the core radius), plus the
exact 1D fundamental soliton used as a closed-form check.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np
from scipy.spatial import Delaunay

# Table II of the paper, in normalized units (lengths / R0).
FIBER_V_NUMBER = 5.46                       # k0 R0 NA for n_core 1.450, n_clad 1.449
FIBER_V_CLAD = -(FIBER_V_NUMBER ** 2)       # V = (k0 R0)^2 (n^2 - n_core^2): 0 in core
FIBER_CHI_CLAD = 2.2 / 2.8                  # n2_clad / n2_core
# Townes critical power of i psi_z + lap psi + |psi|^2 psi = 0 (Weinstein 1983).
TOWNES_POWER = 11.7009


# --------------------------------------------------------------------------
# meshes
# --------------------------------------------------------------------------
@dataclass
class Mesh:
    coords: np.ndarray            # [N0, dim] float64
    cells: np.ndarray             # [Nc, dim+1] int32
    V_cell: np.ndarray            # [Nc] float64
    chi_cell: np.ndarray          # [Nc] float64
    sigma: np.ndarray             # [N0] float64 (absorber, >= 0)
    name: str = ""
    meta: dict = field(default_factory=dict)

    @property
    def dim(self) -> int:
        return int(self.coords.shape[1])

    @property
    def n_vertices(self) -> int:
        return int(self.coords.shape[0])


def mesh_1d_jittered(n: int = 1024, a: float = -20.0, b: float = 20.0,
                     jitter: float = 0.2, seed: int = 1) -> tuple[np.ndarray, np.ndarray]:
    """Nonuniform 1D mesh: uniform nodes on [a, b], interior nodes moved by
    U(-jitter, jitter) times the uniform spacing; end nodes fixed."""
    rng = np.random.default_rng(seed)
    h = (b - a) / (n - 1)
    x = a + h * np.arange(n, dtype=np.float64)
    x[1:-1] += rng.uniform(-jitter, jitter, n - 2) * h
    cells = np.stack([np.arange(n - 1), np.arange(1, n)], axis=1).astype(np.int32)
    return x.reshape(-1, 1), cells


def _orient_ccw(coords: np.ndarray, tris: np.ndarray) -> np.ndarray:
    p0, p1, p2 = coords[tris[:, 0]], coords[tris[:, 1]], coords[tris[:, 2]]
    cross = (p1[:, 0] - p0[:, 0]) * (p2[:, 1] - p0[:, 1]) - (p1[:, 1] - p0[:, 1]) * (p2[:, 0] - p0[:, 0])
    tris = tris.copy()
    flip = cross < 0
    tris[flip, 1], tris[flip, 2] = tris[flip, 2].copy(), tris[flip, 1].copy()
    return tris


def _triangulate(points: np.ndarray) -> np.ndarray:
    tri = Delaunay(points)
    tris = tri.simplices.astype(np.int32)
    if len(tri.coplanar):
        raise RuntimeError("triangulation dropped %d coincident points" % len(tri.coplanar))
    tris = _orient_ccw(points, tris)
    p0, p1, p2 = points[tris[:, 0]], points[tris[:, 1]], points[tris[:, 2]]
    area2 = (p1[:, 0] - p0[:, 0]) * (p2[:, 1] - p0[:, 1]) - (p1[:, 1] - p0[:, 1]) * (p2[:, 0] - p0[:, 0])
    # Qhull can leave zero-area slivers on exactly co-circular input; drop them.
    keep = area2 > 1e-14 * np.max(area2)
    return np.ascontiguousarray(tris[keep])


def _ring_radii(R: float, h_of_r, fixed: list[float]) -> np.ndarray:
    """Radii of concentric point rings on (0, R]; every radius in ``fixed``
    (material interfaces) and R itself are rings.  Between fixed radii the
    ring spacing follows the size function h(r)."""
    knots = [0.0] + sorted(fixed) + [R]
    radii = []
    for a, b in zip(knots[:-1], knots[1:]):
        rr = np.linspace(a, b, 4001)
        inv_h = 1.0 / h_of_r(rr)
        s = np.concatenate([[0.0], np.cumsum(0.5 * (inv_h[1:] + inv_h[:-1]) * np.diff(rr))])
        n = max(1, int(round(s[-1])))
        targets = np.arange(1, n + 1) * (s[-1] / n)
        r = np.interp(targets, s, rr)
        r[-1] = b
        radii.append(r)
    return np.concatenate(radii)


def _ring_points(R: float, h_of_r, fixed: list[float], rng, jitter: float = 0.12,
                 count_only: bool = False):
    radii = _ring_radii(R, h_of_r, fixed)
    exact = set(np.round(np.array(list(fixed) + [R]), 12).tolist())
    counts = np.maximum(6, np.round(2 * np.pi * radii / h_of_r(radii)).astype(np.int64))
    if count_only:
        return 1 + int(counts.sum())
    pts = [np.zeros((1, 2))]
    for r, n in zip(radii, counts):
        phase = rng.uniform(0.0, 2 * np.pi / n)
        ang = phase + 2 * np.pi * np.arange(n) / n
        rad = np.full(n, r)
        if round(float(r), 12) not in exact:
            h = float(h_of_r(np.array([r]))[0])
            rad = rad + rng.uniform(-jitter, jitter, n) * h
            ang = ang + rng.uniform(-jitter, jitter, n) * h / r
        pts.append(np.stack([rad * np.cos(ang), rad * np.sin(ang)], axis=1))
    return np.concatenate(pts)


def mesh_disk_graded(R: float, n_target: int, grading: float, interfaces=(), seed: int = 0,
                     grade_from: float = 0.0) -> tuple[np.ndarray, np.ndarray]:
    """Delaunay mesh of the disk r <= R from concentric rings of points.

    The size function is h(r) = h_c (1 + (grading-1) ((r-grade_from)_+/(R-grade_from))^2):
    finest at the centre (r <= grade_from) and ``grading`` times coarser at the rim.
    Every radius in ``interfaces`` is a ring of points, so material circles
    are followed by mesh edges.  h_c is found by bisection so that the vertex
    count is within 2% of ``n_target``.
    """
    rng = np.random.default_rng(seed)
    fixed = [float(r) for r in interfaces if 0 < r < R]

    def make_h(hc):
        def h(r):
            t = np.clip((np.asarray(r, dtype=np.float64) - grade_from) / (R - grade_from), 0.0, None)
            return hc * (1.0 + (grading - 1.0) * t * t)
        return h

    lo, hi = 1e-5 * R, 0.5 * R
    best, best_err = hi, float("inf")
    for _ in range(60):
        mid = math.sqrt(lo * hi)
        n = _ring_points(R, make_h(mid), fixed, rng, count_only=True)
        if abs(n - n_target) < best_err:
            best, best_err = mid, abs(n - n_target)
        if n > n_target:
            lo = mid
        else:
            hi = mid
        if best_err <= 0.005 * n_target:
            break
    h = make_h(best)
    pts = _ring_points(R, h, fixed, rng)
    tris = _triangulate(pts)
    return pts, tris


def mesh_pcf(n_target: int, pitch: float = 1.0, d_over_pitch: float = 0.5, rings: int = 4,
             R: float = 5.5, seed: int = 5) -> tuple[np.ndarray, np.ndarray, np.ndarray]:
    """Photonic-crystal-fiber-like cross-section: a triangular lattice of air
    holes (rings 1..``rings`` of the hexagonal lattice, the central hole
    missing: 6+12+18+24 = 60 holes for 4 rings) inside a disk of radius R.
    Points: a jittered triangular background lattice, cleared near every
    circle, plus rings of points on each hole circle and on the outer circle.
    Returns (coords, tris, hole_centres)."""
    rng = np.random.default_rng(seed)
    centres = []
    for i in range(-rings, rings + 1):
        for j in range(-rings, rings + 1):
            k = -i - j
            hexd = max(abs(i), abs(j), abs(k))
            if 1 <= hexd <= rings:
                centres.append((pitch * (i + 0.5 * j), pitch * (math.sqrt(3) / 2) * j))
    centres = np.array(centres)
    rh = 0.5 * d_over_pitch * pitch
    area = math.pi * R * R
    h = math.sqrt(area / n_target / (math.sqrt(3) / 2))
    for _ in range(3):
        pts = _pcf_points(centres, rh, R, h, rng)
        h *= math.sqrt(len(pts) / n_target)
    pts = _pcf_points(centres, rh, R, h, rng)
    tris = _triangulate(pts)
    return pts, tris, centres


def _pcf_points(centres, rh, R, h, rng):
    nx = int(math.ceil(R / h)) + 2
    ny = int(math.ceil(R / (h * math.sqrt(3) / 2))) + 2
    jj, ii = np.meshgrid(np.arange(-ny, ny + 1), np.arange(-nx, nx + 1), indexing="ij")
    x = h * (ii + 0.5 * (jj % 2))
    y = h * (math.sqrt(3) / 2) * jj
    bg = np.stack([x.ravel(), y.ravel()], axis=1)
    bg = bg + rng.uniform(-0.1, 0.1, bg.shape) * h
    r = np.hypot(bg[:, 0], bg[:, 1])
    keep = r < R - 0.6 * h
    for c in centres:
        d = np.abs(np.hypot(bg[:, 0] - c[0], bg[:, 1] - c[1]) - rh)
        keep &= d > 0.6 * h
    bg = bg[keep]
    out = [bg]
    n_h = max(8, int(round(2 * math.pi * rh / h)))
    for c in centres:
        a = rng.uniform(0, 2 * math.pi / n_h) + 2 * math.pi * np.arange(n_h) / n_h
        out.append(np.stack([c[0] + rh * np.cos(a), c[1] + rh * np.sin(a)], axis=1))
    n_o = int(round(2 * math.pi * R / h))
    a = rng.uniform(0, 2 * math.pi / n_o) + 2 * math.pi * np.arange(n_o) / n_o
    out.append(np.stack([R * np.cos(a), R * np.sin(a)], axis=1))
    return np.concatenate(out)


def centroids(coords: np.ndarray, cells: np.ndarray) -> np.ndarray:
    return coords[cells].mean(axis=1)


def absorber_profile(coords: np.ndarray, R: float, sigma_max: float, frac: float = 0.15) -> np.ndarray:
    """Absorber strength per vertex: sigma_max ((r - r_a)/(R - r_a))^2 on the
    outer ``frac`` of the radius, 0 inside (a complex-absorbing-potential
    style damping layer)."""
    r = np.hypot(coords[:, 0], coords[:, 1]) if coords.shape[1] == 2 else np.abs(coords[:, 0])
    ra = (1.0 - frac) * R
    t = np.clip((r - ra) / (R - ra), 0.0, None)
    return sigma_max * t * t


# --------------------------------------------------------------------------
# launch fields (Results section of the paper)
# --------------------------------------------------------------------------
def rotated_coords(coords, x0=0.0, y0=0.0, theta=math.pi / 4):
    """U, V of the paper's rotated, shifted transverse coordinates."""
    x = coords[:, 0] - x0
    y = coords[:, 1] - y0
    U = x * math.cos(theta) + y * math.sin(theta)
    V = -x * math.sin(theta) + y * math.cos(theta)
    return U, V


def elliptic_gaussian(coords, A=1.0, wx=1.2, wy=0.6, theta=math.pi / 4, x0=0.1, y0=-0.1):
    """Off-axis elliptic Gaussian launch (paper defaults: A=1, wx=1.2,
    wy=0.6, theta=pi/4, (x0, y0)=(0.1, -0.1))."""
    U, V = rotated_coords(coords, x0, y0, theta)
    return (A * np.exp(-U ** 2 / wx ** 2 - V ** 2 / wy ** 2)).astype(np.complex128)


def elliptic_vortex(coords, A=1.0, wx=1.0, wy=0.8, theta=math.pi / 4):
    """Elliptic vortex with charge m=1: A rho e^{i Phi} Gaussian, with
    rho e^{i Phi} = U/wx + i V/wy (paper defaults A=1, wx=1, wy=0.8)."""
    U, V = rotated_coords(coords, 0.0, 0.0, theta)
    return A * (U / wx + 1j * V / wy) * np.exp(-U ** 2 / wx ** 2 - V ** 2 / wy ** 2)


def vortex_charge1(coords, w=0.5, A=1.0):
    """Charge-1 vortex r e^{i theta} exp(-r^2/w^2)."""
    x, y = coords[:, 0], coords[:, 1]
    return A * (x + 1j * y) * np.exp(-(x * x + y * y) / w ** 2)


def gaussian(coords, w=0.7, A=1.0):
    x, y = coords[:, 0], coords[:, 1]
    return (A * np.exp(-(x * x + y * y) / w ** 2)).astype(np.complex128)


def sech_1d(coords):
    return (1.0 / np.cosh(coords[:, 0])).astype(np.complex128)


HG_ORDER = [(0, 0), (0, 1), (1, 0), (0, 2), (1, 1), (2, 0), (0, 3), (1, 2)]


def _hermite(n, u):
    h0, h1 = np.ones_like(u), 2 * u
    if n == 0:
        return h0
    for k in range(1, n):
        h0, h1 = h1, 2 * u * h1 - 2 * k * h0
    return h1


def hg_superpositions(coords, n_fields: int, rng, w: float = 0.5, power: float = 1.0) -> np.ndarray:
    """[N0, n_fields] complex: complex-normal superpositions of the 8 lowest
    Hermite-Gauss modes HG_mn (first 8 in (m+n, m) order), scaled so that
    the continuous power integral of each field equals ``power``."""
    x, y = coords[:, 0], coords[:, 1]
    g = np.exp(-(x * x + y * y) / w ** 2)
    modes, norms = [], []
    for m, n in HG_ORDER:
        modes.append(_hermite(m, math.sqrt(2) * x / w) * _hermite(n, math.sqrt(2) * y / w) * g)
        norms.append((math.pi * w * w / 2) * 2 ** (m + n) * math.factorial(m) * math.factorial(n))
    modes = np.stack(modes, axis=1)
    norms = np.array(norms)
    a = (rng.standard_normal((len(HG_ORDER), n_fields)) + 1j * rng.standard_normal((len(HG_ORDER), n_fields))) / math.sqrt(2)
    p = (np.abs(a) ** 2 * norms[:, None]).sum(axis=0)
    a = a * np.sqrt(power / p)[None, :]
    return np.ascontiguousarray(modes @ a)


# --------------------------------------------------------------------------
# the five workloads (sizes scale with n_target for test-sized versions)
# --------------------------------------------------------------------------
@dataclass
class Workload:
    name: str
    meshes: list            # list[Mesh]
    psi0: list              # list of [N0, B] complex128 arrays, one per mesh
    p: tuple = (1.0,)       # diffraction coefficients p_1..p_n
    dz: float = 5e-4
    n_steps: int = 100
    description: str = ""


def step_index_materials(coords, cells, core_radius=1.0, V_clad=FIBER_V_CLAD, chi_clad=FIBER_CHI_CLAD):
    c = centroids(coords, cells)
    r = np.hypot(c[:, 0], c[:, 1])
    core = r < core_radius
    V = np.where(core, 0.0, V_clad)
    chi = np.where(core, 1.0, chi_clad)
    return V.astype(np.float64), chi.astype(np.float64)


def soliton_1d(n: int = 1024, seed: int = 1, n_steps: int = 2000, dz: float = 1e-3) -> Workload:
    """1D NLSE i psi_z + psi_xx/2 + |psi|^2 psi = 0 (p1 = 1/2, chi = 1, V = 0)
    on [-20, 20]; the exact solution is sech(x) e^{iz/2}."""
    coords, cells = mesh_1d_jittered(n, seed=seed)
    m = Mesh(coords, cells, np.zeros(len(cells)), np.ones(len(cells)), np.zeros(n), name="soliton1d")
    return Workload("soliton_1d", [m], [sech_1d(coords)[:, None]], p=(0.5,), dz=dz, n_steps=n_steps,
                    description="1D fundamental soliton sech(x) on a jittered 1D mesh")


def gaussian_disk(n_target: int = 200_000, seed: int = 2, n_steps: int = 10_000, dz: float = 5e-4,
                  R: float = 30.0, sigma_max: float = 20.0) -> Workload:
    """2D Kerr NLSE (p1 = chi = 1, V = 0) on a graded disk of radius 30;
    off-axis elliptic Gaussian (wx:wy = 2:1) at half the collapse power;
    absorber on the outer 15% of the radius."""
    coords, tris = mesh_disk_graded(R, n_target, grading=8.0, seed=seed)
    nt = len(tris)
    sigma = absorber_profile(coords, R, sigma_max)
    m = Mesh(coords, tris, np.zeros(nt), np.ones(nt), sigma, name="gaussian_disk")
    wx, wy = 1.2, 0.6
    A = math.sqrt(2 * 0.5 * TOWNES_POWER / (math.pi * wx * wy))
    psi = elliptic_gaussian(coords, A=A, wx=wx, wy=wy)
    return Workload("gaussian_disk", [m], [psi[:, None]], p=(1.0,), dz=dz, n_steps=n_steps,
                    description="graded disk R=30, elliptic Gaussian at 0.5 P_cr, absorber r>25.5")


def vortex_multimode(n_target: int = 1_000_000, seed: int = 3, n_steps: int = 20_000, dz: float = 5e-4,
                     sigma_max: float = 20.0) -> Workload:
    """Large-core step-index guide (core radius 1 = 0.6 of the domain radius,
    index contrast 0.01 at 1.45 / 1.55 um / R0 = 25 um: V_clad = -296.9),
    charge-1 vortex launch, Kerr with n2 ratio 2.2/2.8 in the cladding."""
    R = 1.0 / 0.6
    coords, tris = mesh_disk_graded(R, n_target, grading=2.0, interfaces=(1.0,), seed=seed, grade_from=1.0)
    k0R0 = 2 * math.pi / 1.55 * 25.0
    V_clad = k0R0 ** 2 * (1.44 ** 2 - 1.45 ** 2)
    V, chi = step_index_materials(coords, tris, 1.0, V_clad, FIBER_CHI_CLAD)
    sigma = absorber_profile(coords, R, sigma_max)
    m = Mesh(coords, tris, V, chi, sigma, name="vortex_multimode")
    return Workload("vortex_multimode", [m], [vortex_charge1(coords, w=0.5)[:, None]], p=(1.0,), dz=dz,
                    n_steps=n_steps, description="large-core step-index guide, charge-1 vortex")


def batched_fibers(n_meshes: int = 16, fields_per_mesh: int = 16, n_min: int = 20_000, ratio: float = 25.0,
                   seed: int = 4, n_steps: int = 5000, dz: float = 5e-4, sigma_max: float = 20.0) -> Workload:
    """16 step-index fibers of the paper's Table II (core radius 1, DEC disk
    radius 4, V_clad = -V#^2) with vertex counts n_min * ratio^(i/15), each
    carrying 16 seeded Hermite-Gauss superposition launches of unit power."""
    rng = np.random.default_rng(seed)
    meshes, psis = [], []
    R = 4.0
    for i in range(n_meshes):
        n_i = int(round(n_min * ratio ** (i / max(1, n_meshes - 1))))
        coords, tris = mesh_disk_graded(R, n_i, grading=3.0, interfaces=(1.0,), seed=seed * 1000 + i,
                                        grade_from=1.0)
        V, chi = step_index_materials(coords, tris)
        sigma = absorber_profile(coords, R, sigma_max)
        meshes.append(Mesh(coords, tris, V, chi, sigma, name="fiber%02d" % i))
        psis.append(hg_superpositions(coords, fields_per_mesh, rng))
    return Workload("batched_fibers", meshes, psis, p=(1.0,), dz=dz, n_steps=n_steps,
                    description="16 step-index fibers (20k..500k vertices) x 16 HG-superposition launches")


def pcf(n_target: int = 300_000, seed: int = 5, n_steps: int = 2000, dz: float = 5e-4,
        sigma_max: float = 20.0) -> Workload:
    """PCF-like cross-section: 60 air holes (d/pitch = 0.5, pitch/lambda = 2)
    in silica, V_hole = (2 pi pitch/lambda)^2 (1 - 1.45^2), chi = 0 in air."""
    R = 5.5
    coords, tris, centres = mesh_pcf(n_target, R=R, seed=seed)
    c = centroids(coords, tris)
    d = np.full(len(c), np.inf)
    for cx, cy in centres:
        d = np.minimum(d, np.hypot(c[:, 0] - cx, c[:, 1] - cy))
    hole = d < 0.25
    V_hole = (4 * math.pi) ** 2 * (1.0 - 1.45 ** 2)
    V = np.where(hole, V_hole, 0.0)
    chi = np.where(hole, 0.0, 1.0)
    sigma = absorber_profile(coords, R, sigma_max)
    m = Mesh(coords, tris, V, chi, sigma, name="pcf", meta={"hole_centres": centres})
    return Workload("pcf", [m], [gaussian(coords, w=0.7)[:, None]], p=(1.0,), dz=dz, n_steps=n_steps,
                    description="PCF with 60 air holes, Gaussian launch")
