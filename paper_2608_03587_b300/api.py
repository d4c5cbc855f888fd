"""Thin Python binding of the C ABI (include/decbpm.h).

Argument marshalling only: every step of the propagation runs in libdecbpm's
CUDA kernels.  Device fields are torch CUDA tensors (complex64 or complex128,
shape [N0] or [N0, B], contiguous, in the caller's vertex order); the current
torch stream is passed as the CUDA stream.
"""
from __future__ import annotations

import ctypes
from dataclasses import dataclass

import numpy as np

from . import _lib as L


def _lib():
    return L.load()


def _dptr(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double)) if a is not None else None


def _iptr(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)) if a is not None else None


_ORDERS = {"default": 0, "rcm": 1, "hilbert": 2}
_BOUNDS = {"default": 0, "lanczos": 1, "gershgorin": 2}


def _desc(coords, cells, V_cell=None, chi_cell=None, sigma=None, p=(1.0,), ordering="default", bound="default",
          lanczos_steps=0):
    coords = np.ascontiguousarray(coords, dtype=np.float64)
    if coords.ndim == 1:
        coords = coords.reshape(-1, 1)
    cells = np.ascontiguousarray(cells, dtype=np.int32)
    V_cell = None if V_cell is None else np.ascontiguousarray(V_cell, dtype=np.float64)
    chi_cell = None if chi_cell is None else np.ascontiguousarray(chi_cell, dtype=np.float64)
    sigma = None if sigma is None else np.ascontiguousarray(sigma, dtype=np.float64)
    p = np.ascontiguousarray(np.atleast_1d(np.asarray(p, dtype=np.float64)))
    keep = (coords, cells, V_cell, chi_cell, sigma, p)
    d = L.MeshDesc(dim=coords.shape[1], n_vertices=coords.shape[0], n_cells=cells.shape[0],
                   coords=_dptr(coords), cells=_iptr(cells), V_cell=_dptr(V_cell), chi_cell=_dptr(chi_cell),
                   sigma_vertex=_dptr(sigma), p_n=_dptr(p), n_p=len(p), ordering=_ORDERS[ordering],
                   spectral_bound=_BOUNDS[bound], lanczos_steps=int(lanczos_steps))
    return d, keep


def _params(dz, n_steps, precision, kerr="lumped", diag_every=0, variant="fused", cheb_tol=0.0):
    return L.Params(dz=float(dz), n_steps=int(n_steps), precision=precision,
                    kerr_mode=L.KERR_LUMPED if kerr == "lumped" else L.KERR_ELEMENT,
                    diag_every=int(diag_every), variant={"fused": L.VARIANT_FUSED, "plain": L.VARIANT_PLAIN,
                                                            "rows": L.VARIANT_ROWS, "pairs": L.VARIANT_PAIRS,
                                                            "flow": L.VARIANT_FLOW}[variant],
                    cheb_tol=float(cheb_tol))


def _n_diag(n_steps, diag_every):
    if n_steps == 0 or diag_every <= 0:
        return 1
    return n_steps // diag_every + (1 if n_steps % diag_every else 0)


def _diag_array(buf, n_points, n_fields):
    out = np.zeros((n_points, n_fields), dtype=[("z", "f8"), ("power", "f8"), ("hamiltonian", "f8"),
                                                ("max_intensity", "f8")])
    for i in range(n_points * n_fields):
        d = buf[i]
        out.flat[i] = (d.z, d.power, d.hamiltonian, d.max_intensity)
    return out


def _precision_of(t):
    import torch
    if t.dtype == torch.complex64:
        return L.C64
    if t.dtype == torch.complex128:
        return L.C128
    raise TypeError("field must be complex64 or complex128, got %s" % t.dtype)


def _stream_handle(stream):
    import torch
    s = torch.cuda.current_stream() if stream is None else stream
    return ctypes.c_void_p(s.cuda_stream)


# ---------------------------------------------------------------- host-only
def assemble_host(coords, cells, V_cell=None, chi_cell=None, sigma=None, p=(1.0,), ordering="default",
                  bound="default", lanczos_steps=0):
    """decbpm_assemble_host: FP64 operators in caller order (no GPU needed)."""
    lib = _lib()
    d, keep = _desc(coords, cells, V_cell, chi_cell, sigma, p, ordering, bound, lanczos_steps)
    info = L.MeshInfo()
    L.check(lib.decbpm_assemble_host(ctypes.byref(d), ctypes.byref(info), None, None, None, None, None, None, None))
    n0, nnz = info.n_vertices, info.nnz_offdiag + info.n_vertices
    m, v, chib = np.zeros(n0), np.zeros(n0), np.zeros(n0)
    rowptr = np.zeros(n0 + 1, dtype=np.int64)
    col = np.zeros(nnz, dtype=np.int32)
    val = np.zeros(nnz)
    perm = np.zeros(n0, dtype=np.int32)
    L.check(lib.decbpm_assemble_host(ctypes.byref(d), ctypes.byref(info), _dptr(m), _dptr(v), _dptr(chib),
                                     rowptr.ctypes.data_as(ctypes.POINTER(ctypes.c_int64)), _iptr(col), _dptr(val),
                                     _iptr(perm)))
    del keep
    return {"info": info.as_dict(), "m": m, "v": v, "chib": chib, "K_rowptr": rowptr, "K_col": col, "K_val": val,
            "perm": perm}


def bessel_coefficients(a, tol=1e-16):
    """decbpm_bessel_coefficients: J_0(a) .. J_{n-1}(a) with tail <= tol."""
    lib = _lib()
    n = ctypes.c_int32(0)
    lib.decbpm_bessel_coefficients(float(a), float(tol), 0, None, ctypes.byref(n))
    out = np.zeros(n.value)
    L.check(lib.decbpm_bessel_coefficients(float(a), float(tol), n.value, _dptr(out), ctypes.byref(n)))
    return out


# ---------------------------------------------------------------- meshes
class Mesh:
    """A mesh handle (decbpm_mesh_create): operators assembled in FP64 and
    uploaded to the current CUDA device."""

    def __init__(self, coords, cells, V_cell=None, chi_cell=None, sigma=None, p=(1.0,), ordering="default",
                 bound="default"):
        lib = _lib()
        d, keep = _desc(coords, cells, V_cell, chi_cell, sigma, p, ordering, bound)
        h = ctypes.c_void_p()
        L.check(lib.decbpm_mesh_create(ctypes.byref(d), ctypes.byref(h)))
        del keep
        self._h = h
        self.n_vertices = int(np.asarray(coords).shape[0])
        self._inputs = (coords, cells, V_cell, chi_cell, sigma, p)

    @classmethod
    def from_workload(cls, m, p=(1.0,), ordering="default", bound="default"):
        return cls(m.coords, m.cells, m.V_cell, m.chi_cell, m.sigma, p, ordering, bound)

    @property
    def handle(self):
        return self._h

    def info(self) -> dict:
        inf = L.MeshInfo()
        L.check(_lib().decbpm_mesh_info(self._h, ctypes.byref(inf)))
        return inf.as_dict()

    def close(self):
        if getattr(self, "_h", None) is not None and self._h.value:
            _lib().decbpm_mesh_destroy(self._h)
            self._h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:  # noqa: BLE001
            pass


def mesh_create(coords, cells, V_cell=None, chi_cell=None, sigma=None, p=(1.0,), ordering="default",
                bound="default") -> Mesh:
    return Mesh(coords, cells, V_cell, chi_cell, sigma, p, ordering, bound)


def _fields(psi):
    if not psi.is_cuda or not psi.is_contiguous():
        raise ValueError("field must be a contiguous CUDA tensor")
    return 1 if psi.dim() == 1 else int(psi.shape[1])


def propagate(mesh: Mesh, psi, dz, n_steps, diag_every=0, kerr="lumped", variant="fused", cheb_tol=0.0,
              stream=None):
    """decbpm_propagate: advance psi (torch CUDA [N0] or [N0, B]) in place.
    Returns the diagnostics as a structured numpy array [n_points, B]."""
    lib = _lib()
    B = _fields(psi)
    prm = _params(dz, n_steps, _precision_of(psi), kerr, diag_every, variant, cheb_tol)
    npts = _n_diag(n_steps, diag_every)
    buf = (L.Diag * (npts * B))()
    L.check(lib.decbpm_propagate(mesh.handle, ctypes.byref(prm), ctypes.c_void_p(psi.data_ptr()), B,
                                 _stream_handle(stream), buf))
    return _diag_array(buf, npts, B)


def propagate_noalloc(mesh: Mesh, psi, dz, n_steps, kerr="lumped", cheb_tol=0.0, stream=None):
    """decbpm_propagate_noalloc: like propagate(), for callers that cannot
    allocate device memory at call time; scratch comes from the library's
    static 32 MiB device array (size limits and sharing rules in decbpm.h).
    Returns nothing (no diagnostics)."""
    lib = _lib()
    B = _fields(psi)
    prm = _params(dz, n_steps, _precision_of(psi), kerr, 0, "fused", cheb_tol)
    L.check(lib.decbpm_propagate_noalloc(mesh.handle, ctypes.byref(prm), ctypes.c_void_p(psi.data_ptr()), B,
                                         _stream_handle(stream)))


def propagate_host(mesh: Mesh, psi_host, dz, n_steps, diag_every=0, kerr="lumped", variant="fused", cheb_tol=0.0,
                   stream=None):
    """decbpm_propagate_host: psi_host is a CPU torch tensor (pinned for speed), updated in place."""
    lib = _lib()
    B = 1 if psi_host.dim() == 1 else int(psi_host.shape[1])
    prm = _params(dz, n_steps, _precision_of(psi_host), kerr, diag_every, variant, cheb_tol)
    npts = _n_diag(n_steps, diag_every)
    buf = (L.Diag * (npts * B))()
    L.check(lib.decbpm_propagate_host(mesh.handle, ctypes.byref(prm), ctypes.c_void_p(psi_host.data_ptr()), B,
                                      _stream_handle(stream), buf))
    return _diag_array(buf, npts, B)


def diagnostics(mesh: Mesh, psi, stream=None):
    lib = _lib()
    B = _fields(psi)
    buf = (L.Diag * B)()
    L.check(lib.decbpm_diagnostics(mesh.handle, ctypes.c_void_p(psi.data_ptr()), B, _precision_of(psi),
                                   _stream_handle(stream), buf))
    return _diag_array(buf, 1, B)[0]


# ---------------------------------------------------------------- plans
class Plan:
    """decbpm_plan_create: many meshes x many fields in one persistent launch."""

    def __init__(self, meshes, fields_per_mesh, precision="c64"):
        lib = _lib()
        self.meshes = list(meshes)
        self.fields = [int(f) for f in fields_per_mesh]
        self.precision = L.C64 if precision in ("c64", L.C64) else L.C128
        arr = (ctypes.c_void_p * len(self.meshes))(*[m.handle.value for m in self.meshes])
        nf = (ctypes.c_int32 * len(self.fields))(*self.fields)
        h = ctypes.c_void_p()
        L.check(lib.decbpm_plan_create(arr, len(self.meshes), nf, self.precision, ctypes.byref(h)))
        self._h = h

    def degree(self, i, dz, cheb_tol=0.0):
        return int(_lib().decbpm_plan_degree(self._h, i, float(dz), self.precision, float(cheb_tol)))

    def propagate(self, psis, dz, n_steps, diag_every=0, kerr="lumped", cheb_tol=0.0, stream=None, variant="fused"):
        lib = _lib()
        prm = _params(dz, n_steps, self.precision, kerr, diag_every, variant, cheb_tol)
        npts = _n_diag(n_steps, diag_every)
        nrec = npts * sum(self.fields)
        buf = (L.Diag * nrec)()
        ptrs = (ctypes.c_void_p * len(psis))(*[p.data_ptr() for p in psis])
        L.check(lib.decbpm_plan_propagate(self._h, ctypes.byref(prm), ptrs, _stream_handle(stream), buf))
        return _diag_array(buf, npts, sum(self.fields))

    def propagate_host(self, psis_host, dz, n_steps, diag_every=0, kerr="lumped", cheb_tol=0.0, stream=None,
                       variant="fused"):
        lib = _lib()
        prm = _params(dz, n_steps, self.precision, kerr, diag_every, variant, cheb_tol)
        npts = _n_diag(n_steps, diag_every)
        buf = (L.Diag * (npts * sum(self.fields)))()
        ptrs = (ctypes.c_void_p * len(psis_host))(*[p.data_ptr() for p in psis_host])
        L.check(lib.decbpm_plan_propagate_host(self._h, ctypes.byref(prm), ptrs, _stream_handle(stream), buf))
        return _diag_array(buf, npts, sum(self.fields))

    def autotune(self, dz, trial_steps=3, kerr="lumped", stream=None) -> dict:
        """decbpm_plan_autotune: time the FUSED variant's launch shapes on
        trial marches and keep the fastest (cached per problem for the process)."""
        r = L.TuneResult()
        L.check(_lib().decbpm_plan_autotune(self._h, float(dz), L.KERR_LUMPED if kerr == "lumped" else L.KERR_ELEMENT,
                                            int(trial_steps), _stream_handle(stream), ctypes.byref(r)))
        return r.as_dict()

    def set_shape(self, kernel="rows", ctas_per_sm=1, tile_slots=0, forward_walk=0, values_per_thread=0,
                  walk_skip=0, no_meta_cache=0, flow_ranges=0):
        """decbpm_plan_set_shape: apply a launch shape without timing (kernel
        "pairs", "tile", "flow" or "rows"; e.g. the dict autotune() returned)."""
        var = {"pairs": L.VARIANT_PAIRS, "tile": L.VARIANT_FUSED, "flow": L.VARIANT_FLOW, "rows": L.VARIANT_ROWS}[kernel]
        r = L.TuneResult(variant=var, ctas_per_sm=int(ctas_per_sm), tile_slots=int(tile_slots),
                         forward_walk=int(forward_walk), values_per_thread=int(values_per_thread),
                         walk_skip=int(walk_skip), no_meta_cache=int(no_meta_cache), flow_ranges=int(flow_ranges))
        L.check(_lib().decbpm_plan_set_shape(self._h, ctypes.byref(r)))

    def config(self) -> dict:
        c = L.PlanConfig()
        L.check(_lib().decbpm_plan_get_config(self._h, ctypes.byref(c)))
        return c.as_dict()

    def last_march_ms(self) -> float:
        v = ctypes.c_double()
        L.check(_lib().decbpm_plan_last_march_ms(self._h, ctypes.byref(v)))
        return v.value

    def close(self):
        if getattr(self, "_h", None) is not None and self._h.value:
            _lib().decbpm_plan_destroy(self._h)
            self._h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:  # noqa: BLE001
            pass


def plan_create(meshes, fields_per_mesh, precision="c64") -> Plan:
    return Plan(meshes, fields_per_mesh, precision)


def selftest_barrier(missing_arrivals: int, timeout_ns: int, stream=None) -> int:
    """decbpm_selftest_barrier: returns the status code (no exception)."""
    return int(_lib().decbpm_selftest_barrier(int(missing_arrivals), int(timeout_ns), _stream_handle(stream)))


# ---------------------------------------------------------------- adjoint
def set_potential(mesh: Mesh, v_vertex=None):
    """decbpm_mesh_set_potential: per-vertex potential v_p (numpy, caller
    order) used by the diagonal flow; None restores the mesh's own."""
    v = None if v_vertex is None else np.ascontiguousarray(v_vertex, dtype=np.float64)
    L.check(_lib().decbpm_mesh_set_potential(mesh.handle, _dptr(v)))


def vjp(mesh: Mesh, psi0, gN, dz, n_steps, checkpoint_every=0, want_grad_v=True, stream=None):
    """decbpm_vjp: (psi_N, dJ/dpsi_0, dJ/dv) for a terminal cotangent gN
    (torch CUDA tensors like psi0; gradients in torch's complex convention)."""
    import torch
    lib = _lib()
    B = _fields(psi0)
    prm = _params(dz, n_steps, _precision_of(psi0))
    gN = gN.contiguous()
    psiN = torch.empty_like(psi0)
    g0 = torch.empty_like(psi0)
    gv = torch.zeros(psi0.shape[0], dtype=torch.float64, device=psi0.device) if want_grad_v else None
    L.check(lib.decbpm_vjp(mesh.handle, ctypes.byref(prm), ctypes.c_void_p(psi0.data_ptr()),
                           ctypes.c_void_p(gN.data_ptr()), ctypes.c_void_p(psiN.data_ptr()),
                           ctypes.c_void_p(g0.data_ptr()),
                           ctypes.c_void_p(gv.data_ptr()) if gv is not None else None, B,
                           int(checkpoint_every), _stream_handle(stream)))
    return psiN, g0, gv


def set_potential_offset(mesh: Mesh, dv=None, stream=None):
    """decbpm_mesh_set_potential_offset: v = base + dv on the device, dv a real
    CUDA tensor [N0] in caller order (None: v = base).  Stream-ordered, no host
    copy.  Returns the FP64 tensor handed to the library (keep it alive until
    the stream has run the offset kernel)."""
    import torch
    if dv is None:
        L.check(_lib().decbpm_mesh_set_potential_offset(mesh.handle, None, _stream_handle(stream)))
        return None
    if not dv.is_cuda or dv.dim() != 1 or dv.shape[0] != mesh.n_vertices:
        raise ValueError("dv must be a CUDA tensor of shape [n_vertices]")
    d64 = dv.detach().to(torch.float64).contiguous()
    L.check(_lib().decbpm_mesh_set_potential_offset(mesh.handle, ctypes.c_void_p(d64.data_ptr()),
                                                    _stream_handle(stream)))
    return d64


def adjoint(mesh: Mesh, psi0, target, dz, n_steps, checkpoint_every=0, want_grad_v=True, want_grad_psi0=True,
            stream=None):
    """decbpm_adjoint: J_f = |<target_f, psi_N,f>_{*0}|^2 (numpy [B]) and its
    gradients dJ/dv (FP64 CUDA [N0], summed over fields) and dJ/dpsi_0 (like
    psi0, torch's complex convention); None for a gradient not asked for."""
    import torch
    lib = _lib()
    B = _fields(psi0)
    if target.shape != psi0.shape or target.dtype != psi0.dtype:
        raise ValueError("target must have psi0's shape and dtype")
    prm = _params(dz, n_steps, _precision_of(psi0))
    target = target.contiguous()
    J = np.zeros(B)
    gv = torch.zeros(psi0.shape[0], dtype=torch.float64, device=psi0.device) if want_grad_v else None
    g0 = torch.empty_like(psi0) if want_grad_psi0 else None
    L.check(lib.decbpm_adjoint(mesh.handle, ctypes.byref(prm), ctypes.c_void_p(psi0.data_ptr()),
                               ctypes.c_void_p(target.data_ptr()), B, _dptr(J),
                               ctypes.c_void_p(gv.data_ptr()) if gv is not None else None,
                               ctypes.c_void_p(g0.data_ptr()) if g0 is not None else None,
                               int(checkpoint_every), _stream_handle(stream)))
    return J, gv, g0


def _march_function():
    import torch

    class MarchFunction(torch.autograd.Function):
        """psi_N = march(psi_0; v + dv): forward through decbpm_propagate,
        backward through the hand-written adjoint decbpm_vjp (checkpointed).
        dv reaches the library as a device array (decbpm_mesh_set_potential_offset):
        no host copy.  The mesh keeps v = base + dv afterwards."""

        @staticmethod
        def forward(ctx, psi0, dv, mesh, dz, n_steps, checkpoint_every):
            d64 = set_potential_offset(mesh, dv)
            out = psi0.detach().clone().contiguous()
            propagate(mesh, out, dz, n_steps)
            ctx.save_for_backward(psi0.detach(), d64)
            ctx.mesh, ctx.dz, ctx.n_steps, ctx.ck, ctx.dv_dtype = mesh, dz, n_steps, checkpoint_every, dv.dtype
            return out

        @staticmethod
        def backward(ctx, grad_out):
            psi0, d64 = ctx.saved_tensors
            mesh = ctx.mesh
            set_potential_offset(mesh, d64)
            _, g0, gv = vjp(mesh, psi0, grad_out.contiguous(), ctx.dz, ctx.n_steps, ctx.ck)
            return g0, gv.to(ctx.dv_dtype), None, None, None, None

    return MarchFunction


def march(mesh: Mesh, psi0, dv, dz, n_steps, checkpoint_every=0):
    """Differentiable march: gradients flow to psi0 (complex) and to the
    per-vertex potential offset dv (real CUDA tensor [N0]).  For a refractive-
    index perturbation write dv = (k0 L)^2 (n^2 - n_ref^2) in torch: autograd
    then returns dJ/dn."""
    return _march_function().apply(psi0, dv, mesh, dz, n_steps, checkpoint_every)


# ---------------------------------------------------------------- the paper's integrator
def rk45(mesh: Mesh, psi, z_end, rtol=1e-9, atol=1e-11, h0=0.0, kerr="lumped", max_steps=0, stream=None):
    """decbpm_rk45: adaptive Dormand-Prince integration of Eq. 10 in place on
    a complex128 CUDA field [N0]; returns the step statistics."""
    lib = _lib()
    if psi.dtype.__str__() != "torch.complex128" or psi.dim() != 1:
        raise TypeError("rk45 integrates one complex128 field [N0]")
    o = L.Rk45Opts(rtol=float(rtol), atol=float(atol), h0=float(h0), max_steps=int(max_steps))
    st = L.Rk45Stats()
    L.check(lib.decbpm_rk45(mesh.handle, float(z_end), L.KERR_LUMPED if kerr == "lumped" else L.KERR_ELEMENT,
                            ctypes.byref(o), ctypes.c_void_p(psi.data_ptr()), _stream_handle(stream), ctypes.byref(st)))
    return st.as_dict()


# ---------------------------------------------------------------- discrete soliton
def soliton(mesh: Mesh, psi, power, tau=0.05, tol=1e-11, max_iter=5000, kerr="lumped", mix=1.0, stream=None):
    """decbpm_soliton: the fundamental nonlinear mode of the given power, in
    place on a complex128 CUDA field [N0] (input: the start); returns
    {mu, residual, iterations, cheb_terms}."""
    lib = _lib()
    if psi.dtype.__str__() != "torch.complex128" or psi.dim() != 1:
        raise TypeError("soliton works on one complex128 field [N0]")
    o = L.SolitonOpts(power=float(power), tau=float(tau), tol=float(tol), mix=float(mix), max_iter=int(max_iter),
                      kerr_mode=L.KERR_LUMPED if kerr == "lumped" else L.KERR_ELEMENT)
    st = L.SolitonStats()
    L.check(lib.decbpm_soliton(mesh.handle, ctypes.byref(o), ctypes.c_void_p(psi.data_ptr()), _stream_handle(stream),
                               ctypes.byref(st)))
    return st.as_dict()


def bessel_i_scaled(a, tol=1e-17):
    """decbpm_bessel_i_scaled: e^{-a} I_k(a) for k = 0.. until below tol e^{-a} I_0(a)."""
    lib = _lib()
    n = ctypes.c_int32(0)
    L.check(lib.decbpm_bessel_i_scaled(float(a), float(tol), 0, None, ctypes.byref(n)))
    out = np.zeros(n.value)
    L.check(lib.decbpm_bessel_i_scaled(float(a), float(tol), n.value, out.ctypes.data_as(ctypes.POINTER(ctypes.c_double)),
                                       ctypes.byref(n)))
    return out


# ---------------------------------------------------------------- perfectly matched layer
def set_pml(mesh: Mesh, r_inner=None, r_outer=None, sigma_max=0.0, order=2, center=(0.0, 0.0)):
    """decbpm_mesh_set_pml: radial complex-stretching layer beyond r_inner
    (sigma_max = 0 or r_inner = None removes it).  A mesh with a layer runs
    with rk45 and with propagate / propagate_host (the split-step on the
    stretched operators, lumped Kerr, p_1)."""
    lib = _lib()
    if r_inner is None or sigma_max == 0.0:
        L.check(lib.decbpm_mesh_set_pml(mesh.handle, None))
        return
    o = L.Pml(x0=float(center[0]), y0=float(center[1]), r_inner=float(r_inner), r_outer=float(r_outer),
              sigma_max=float(sigma_max), order=int(order))
    L.check(lib.decbpm_mesh_set_pml(mesh.handle, ctypes.byref(o)))



def pml_degree(mesh: Mesh, dz, precision="c64", cheb_tol=0.0) -> int:
    """decbpm_mesh_pml_degree: Chebyshev degree of the march on the stretched
    operators for step dz (0 without a layer)."""
    prec = L.C64 if precision in ("c64", L.C64) else L.C128
    return int(_lib().decbpm_mesh_pml_degree(mesh.handle, float(dz), prec, float(cheb_tol)))
