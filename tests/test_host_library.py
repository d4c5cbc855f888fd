"""Host-side checks of libdecbpm that need no GPU: the library loads and
exports every entry point its header declares, the FP64 host assembly equals
the oracle's operators, the Chebyshev/Bessel coefficients are right, and bad
input is rejected with the documented status codes."""
import ctypes
import math
import os
import re

import numpy as np
import pytest
import scipy.sparse as sp
import scipy.sparse.linalg as spla
from scipy.special import jv

from oracle import dec
from paper_2608_03587_b300 import _lib as L
from paper_2608_03587_b300 import api
from paper_2608_03587_b300 import workloads as W

HEADER = os.path.join(os.path.dirname(os.path.dirname(__file__)), "include", "decbpm.h")


def declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(decbpm_[a-z0-9_]+)\s*\(", text)))


def test_library_exports_every_declared_symbol(lib):
    names = declared_functions()
    assert len(names) >= 15
    for n in names:
        assert hasattr(lib, n), n
        assert n in L.SIGNATURES, "no ctypes signature for %s" % n
    assert lib.decbpm_version().decode().startswith("decbpm")


def test_bounds_checked_build_exports_the_same_entry_points():
    """libdecbpm_checked.so (-DDECBPM_BOUNDS_CHECK) is the same library with
    the march kernels' index checks compiled in: every declared entry point,
    and a version string that says so."""
    from paper_2608_03587_b300 import build as B
    B.build(checked=True)
    chk = ctypes.CDLL(B.CHECKED_LIB)
    for n in declared_functions():
        assert hasattr(chk, n), n
    chk.decbpm_version.restype = ctypes.c_char_p
    assert b"bounds-checked" in chk.decbpm_version()


@pytest.fixture(scope="module")
def fiber():
    coords, tris = W.mesh_disk_graded(4.0, 2500, 3.0, interfaces=(1.0,), seed=17, grade_from=1.0)
    V, chi = W.step_index_materials(coords, tris)
    sigma = W.absorber_profile(coords, 4.0, 10.0)
    return coords, tris, V, chi, sigma


def test_host_assembly_matches_oracle(fiber):
    coords, tris, V, chi, sigma = fiber
    a = api.assemble_host(coords, tris, V, chi, sigma)
    ops = dec.Operators(coords, tris, V, chi)
    assert np.allclose(a["m"], ops.H0, rtol=1e-13, atol=0)
    assert np.allclose(a["v"], ops.v, rtol=1e-12, atol=1e-12 * np.abs(ops.v).max())
    assert np.allclose(a["chib"], ops.chib, rtol=1e-12)
    n0 = len(coords)
    K = sp.csr_matrix((a["K_val"], a["K_col"], a["K_rowptr"]), shape=(n0, n0))
    assert abs(K - ops.K).max() <= 1e-12 * abs(ops.K).max()
    info = a["info"]
    assert info["n_vertices"] == n0 and info["n_cells"] == len(tris)
    assert info["nnz_offdiag"] == 2 * info["n_edges"]
    assert info["area"] == pytest.approx(ops.H0.sum(), rel=1e-13)
    # rho bounds the spectrum of A = *0^{-1} K from above (Gershgorin + margin)
    lam_max = spla.eigsh(ops.K, k=1, M=sp.diags(ops.H0), which="LA", return_eigenvectors=False)[0]
    assert lam_max <= info["rho"] <= 2.5 * lam_max
    # internal orders: permutations; RCM has a small bandwidth, the Hilbert
    # curve keeps most edges short (compact blocks of consecutive vertices)
    perm = a["perm"]
    assert np.array_equal(np.sort(perm), np.arange(n0))
    r = api.assemble_host(coords, tris, V, chi, sigma, ordering="rcm")
    assert np.array_equal(np.sort(r["perm"]), np.arange(n0))
    assert r["info"]["bandwidth"] < n0 / 8
    inv = np.empty(n0, dtype=np.int64)
    inv[perm] = np.arange(n0)
    E = dec.edges(tris)
    span = np.abs(inv[E[:, 0]] - inv[E[:, 1]])
    assert np.median(span) < 40
    assert np.mean(span < 256) > 0.8


@pytest.mark.parametrize("n", [300, 6000])
def test_spectral_bounds_contain_the_spectrum(n):
    """rho must bound lambda_max(*0^{-1} K) from above (the Chebyshev series
    diverges outside its interval): the Lanczos-certified default within 1%
    above it, the deterministic Gershgorin / element bound anywhere above."""
    coords, tris = W.mesh_disk_graded(4.0, n, 3.0, interfaces=(1.0,), seed=n, grade_from=1.0)
    ops = dec.Operators(coords, tris)
    lam = spla.eigsh(ops.K, k=1, M=sp.diags(ops.H0), which="LA", return_eigenvectors=False)[0]
    info = api.assemble_host(coords, tris)["info"]
    rho = info["rho"]
    rho_g = api.assemble_host(coords, tris, bound="gershgorin")["info"]["rho"]
    assert info["rho_kind"] == L.RHO_LANCZOS_CHECKED
    assert lam <= rho <= 1.0101 * lam
    assert lam <= rho_g
    assert rho_g == pytest.approx(min(rho_g, ops.rho * (1 + 1e-6)), rel=1e-12)   # never above Gershgorin
    # 1D: the element bound 4/L_min^2 and the exact spectrum
    x, cells = W.mesh_1d_jittered(200, seed=5)
    o1 = dec.Operators(x, cells)
    lam1 = np.linalg.eigvals(o1.A.toarray()).real.max()
    r1 = api.assemble_host(x, cells)["info"]["rho"]
    assert lam1 <= r1 <= 1.0101 * lam1


def test_lanczos_candidate_below_lambda_max_falls_back_to_the_rigorous_bound():
    """The per-mesh check of the Lanczos candidate 1.01 theta: with too few
    Lanczos steps theta falls short of lambda_max by more than 1%; the check
    must then reject the candidate (rho_kind = REJECTED) and rho must be the
    rigorous min(Gershgorin, element) bound, which contains the spectrum.  On
    the 60k-vertex mesh 10 steps leave the candidate only ~0.1% below
    lambda_max; 30 steps put it above, and it is accepted."""
    coords, tris = W.mesh_disk_graded(4.0, 60000, 3.0, interfaces=(1.0,), seed=60000, grade_from=1.0)
    ops = dec.Operators(coords, tris)
    lam = spla.eigsh(ops.K, k=1, M=sp.diags(ops.H0), which="LA", return_eigenvectors=False)[0]
    for steps in (3, 10):
        info = api.assemble_host(coords, tris, lanczos_steps=steps)["info"]
        assert 1.01 * info["rho_lanczos"] < lam            # the candidate is wrong
        assert info["rho_kind"] == L.RHO_LANCZOS_REJECTED
        assert info["rho"] == info["rho_rigorous"] and info["rho"] >= lam
    info = api.assemble_host(coords, tris, lanczos_steps=30)["info"]
    assert 1.01 * info["rho_lanczos"] >= lam
    assert info["rho_kind"] == L.RHO_LANCZOS_CHECKED and lam <= info["rho"] <= 1.0101 * lam
    g = api.assemble_host(coords, tris, bound="gershgorin")["info"]
    assert g["rho_kind"] == L.RHO_RIGOROUS and g["rho"] == info["rho_rigorous"]


def test_host_assembly_1d(fiber):
    x, cells = W.mesh_1d_jittered(300, seed=2)
    a = api.assemble_host(x, cells, p=(0.5,))
    ops = dec.Operators(x, cells)
    K = sp.csr_matrix((a["K_val"], a["K_col"], a["K_rowptr"]), shape=(300, 300))
    assert abs(K - ops.K).max() <= 1e-13 * abs(ops.K).max()
    assert np.allclose(a["m"], ops.H0, rtol=1e-14)
    assert a["info"]["bandwidth"] == 1


@pytest.mark.parametrize("a", [0.0, 1e-3, 0.7, 3.0, 17.5, 120.0])
def test_bessel_coefficients_match_scipy(a):
    J = api.bessel_coefficients(a, 1e-16)
    k = np.arange(len(J))
    ref = jv(k, a)
    assert np.max(np.abs(J - ref)) < 1e-14 * max(1.0, math.sqrt(a))
    # the truncated tail really is below the tolerance
    kk = np.arange(len(J), len(J) + 40)
    assert 2 * np.sum(np.abs(jv(kk, a))) <= 1.1e-16
    assert len(J) >= min(a, 1e9)


def test_chebyshev_sum_reproduces_exponential():
    """sum_k (2 - delta_k0) (-i)^k J_k(a) T_k(x) = exp(-i a x) on [-1, 1]."""
    a = 9.3
    J = api.bessel_coefficients(a, 1e-16)
    x = np.linspace(-1, 1, 101)
    T = np.cos(np.outer(np.arange(len(J)), np.arccos(x)))
    coef = J * (-1j) ** np.arange(len(J)) * np.where(np.arange(len(J)) == 0, 1.0, 2.0)
    assert np.max(np.abs(coef @ T - np.exp(-1j * a * x))) < 1e-14


def _rc(**kw):
    coords = np.array([[0.0, 0.0], [1.0, 0.0], [0.0, 1.0], [1.0, 1.0]])
    tris = np.array([[0, 1, 2], [1, 3, 2]], dtype=np.int32)
    args = dict(coords=coords, cells=tris)
    args.update(kw)
    try:
        api.assemble_host(**args)
        return 0
    except L.DecbpmError as e:
        return e.code


def test_rejects_bad_meshes():
    assert _rc() == 0
    assert _rc(cells=np.array([[0, 2, 1], [1, 3, 2]], dtype=np.int32)) == L.ERR_BAD_MESH       # clockwise
    assert _rc(cells=np.array([[0, 1, 2], [1, 3, 7]], dtype=np.int32)) == L.ERR_BAD_MESH       # index range
    bad = np.array([[0.0, 0.0], [1.0, 0.0], [0.0, np.nan], [1.0, 1.0]])
    assert _rc(coords=bad) == L.ERR_NONFINITE
    assert _rc(sigma=np.array([0.0, -1.0, 0.0, 0.0])) == L.ERR_INVALID_ARG
    # an edge shared by three triangles
    coords = np.array([[0.0, 0.0], [1.0, 0.0], [0.5, 1.0], [0.5, -1.0], [0.6, 2.0]])
    tris = np.array([[0, 1, 2], [1, 0, 3], [0, 1, 4]], dtype=np.int32)
    assert _rc(coords=coords, cells=tris) == L.ERR_BAD_MESH
    # an isolated vertex
    coords = np.array([[0.0, 0.0], [1.0, 0.0], [0.0, 1.0], [5.0, 5.0]])
    assert _rc(coords=coords, cells=np.array([[0, 1, 2]], dtype=np.int32)) == L.ERR_BAD_MESH
    assert "counter-clockwise" in _last_error_after(np.array([[0, 2, 1], [1, 3, 2]], dtype=np.int32))


def _last_error_after(cells):
    try:
        api.assemble_host(np.array([[0.0, 0.0], [1.0, 0.0], [0.0, 1.0], [1.0, 1.0]]), cells)
    except L.DecbpmError as e:
        return str(e)
    return ""


def test_element_kerr_operator_rows(fiber):
    """The element-averaged Kerr operator the library builds satisfies
    C 1 = chib (its rows reproduce the lumped coefficient for uniform |psi|)."""
    # exercised through the oracle identity Q^T D Q 1 = *0(chi) 1 on the same mesh
    coords, tris, V, chi, sigma = fiber
    ops = dec.Operators(coords, tris, V, chi)
    assert np.allclose(ops.QtDQ @ np.ones(ops.n0) / ops.H0, ops.chib, rtol=1e-12)


def test_null_arguments_are_rejected(lib):
    assert lib.decbpm_mesh_create(None, None) == L.ERR_INVALID_ARG
    assert lib.decbpm_propagate(None, None, None, 1, None, None) == L.ERR_INVALID_ARG
    h = ctypes.c_void_p()
    assert lib.decbpm_plan_create(None, 0, None, L.C64, ctypes.byref(h)) == L.ERR_INVALID_ARG
    assert lib.decbpm_mesh_destroy(None) == L.OK


def test_bessel_i_scaled_matches_scipy():
    """Coefficients of the Chebyshev series of e^{-a x} used by the soliton
    iteration: e^{-a} I_k(a) by Miller's recurrence, against scipy.special.ive."""
    from scipy.special import ive

    from paper_2608_03587_b300 import api
    assert list(api.bessel_i_scaled(0.0)) == [1.0]
    for a in (1e-3, 0.5, 3.0, 40.0, 700.0, 5000.0):
        s = api.bessel_i_scaled(a, 1e-17)
        k = np.arange(len(s))
        assert np.max(np.abs(s - ive(k, a))) < 1e-15 * max(1.0, ive(0, a))
        assert ive(len(s), a) < 1e-17 * ive(0, a) * 1.01          # truncated where the tail is negligible
        assert s[0] + 2 * s[1:].sum() == pytest.approx(1.0, abs=1e-13)
