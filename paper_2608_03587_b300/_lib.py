"""ctypes loader of libdecbpm.so: argument types of every C-ABI entry point.

The library is built in-tree (``paper_2608_03587_b300/libdecbpm.so``).  There
is no fallback: if it is missing and cannot be built, loading raises.  With
DECBPM_BOUNDS_CHECK=1 in the environment the bounds-check build
(``libdecbpm_checked.so``, same entry points) is loaded instead.
"""
from __future__ import annotations

import ctypes
import os
import threading

HERE = os.path.dirname(os.path.abspath(__file__))
CHECKED = os.environ.get("DECBPM_BOUNDS_CHECK", "0") not in ("", "0")
LIB_PATH = os.path.join(HERE, "libdecbpm_checked.so" if CHECKED else "libdecbpm.so")

# status codes (include/decbpm.h)
OK = 0
ERR_INVALID_ARG = -1
ERR_BAD_MESH = -2
ERR_NONFINITE = -3
ERR_TIMEOUT = -4
ERR_CUDA = -5
ERR_OOM = -6
ERR_UNSUPPORTED = -7
ERR_DEVICE_CHECK = -8
C64 = 1
C128 = 2
KERR_LUMPED = 0
KERR_ELEMENT = 1
VARIANT_FUSED = 0
VARIANT_PLAIN = 1
VARIANT_ROWS = 2
VARIANT_PAIRS = 3
VARIANT_FLOW = 4
ORDER_DEFAULT = 0
ORDER_RCM = 1
ORDER_HILBERT = 2
RHO_RIGOROUS = 0
RHO_LANCZOS_CHECKED = 1
RHO_LANCZOS_REJECTED = 2

_c_double_p = ctypes.POINTER(ctypes.c_double)
_c_int32_p = ctypes.POINTER(ctypes.c_int32)
_c_int64_p = ctypes.POINTER(ctypes.c_int64)


class MeshDesc(ctypes.Structure):
    _fields_ = [("dim", ctypes.c_int32), ("n_vertices", ctypes.c_int64), ("n_cells", ctypes.c_int64),
                ("coords", _c_double_p), ("cells", _c_int32_p), ("V_cell", _c_double_p),
                ("chi_cell", _c_double_p), ("sigma_vertex", _c_double_p), ("p_n", _c_double_p),
                ("n_p", ctypes.c_int32), ("ordering", ctypes.c_int32), ("spectral_bound", ctypes.c_int32),
                ("lanczos_steps", ctypes.c_int32)]


class MeshInfo(ctypes.Structure):
    _fields_ = [("n_vertices", ctypes.c_int64), ("n_edges", ctypes.c_int64), ("n_cells", ctypes.c_int64),
                ("nnz_offdiag", ctypes.c_int64), ("max_degree", ctypes.c_int32), ("n_p", ctypes.c_int32),
                ("bandwidth", ctypes.c_int64), ("rho", ctypes.c_double), ("area", ctypes.c_double),
                ("mean_degree", ctypes.c_double), ("sell_entries", ctypes.c_int64),
                ("device_bytes", ctypes.c_int64), ("rho_kind", ctypes.c_int32), ("pad_", ctypes.c_int32),
                ("rho_lanczos", ctypes.c_double), ("rho_rigorous", ctypes.c_double)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class Params(ctypes.Structure):
    _fields_ = [("dz", ctypes.c_double), ("n_steps", ctypes.c_int64), ("precision", ctypes.c_int32),
                ("kerr_mode", ctypes.c_int32), ("diag_every", ctypes.c_int32), ("variant", ctypes.c_int32),
                ("cheb_tol", ctypes.c_double)]


class PlanConfig(ctypes.Structure):
    _fields_ = [("grid", ctypes.c_int32), ("block", ctypes.c_int32), ("fields_padded", ctypes.c_int32),
                ("graphs", ctypes.c_int32), ("stages", ctypes.c_int32), ("n_meshes", ctypes.c_int32),
                ("tile_slots", ctypes.c_int32), ("tile_slot_bytes", ctypes.c_int32), ("tile_grid", ctypes.c_int32),
                ("tile_block", ctypes.c_int32), ("tuned", ctypes.c_int32), ("fused_kernel", ctypes.c_int32),
                ("tile_slots_used", ctypes.c_int32), ("forward_walk", ctypes.c_int32), ("pair_slots", ctypes.c_int32),
                ("pair_slot_bytes", ctypes.c_int32), ("pair_grid", ctypes.c_int32), ("passes", ctypes.c_int32),
                ("values_per_thread", ctypes.c_int32), ("rows_per_item", ctypes.c_int32),
                ("flow_grid", ctypes.c_int32), ("flow_skip", ctypes.c_int32), ("flow_ranges", ctypes.c_int32),
                ("tile_rows", ctypes.c_int32),
                ("meta_items", ctypes.c_int32), ("field_groups", ctypes.c_int32)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class TuneResult(ctypes.Structure):
    _fields_ = [("variant", ctypes.c_int32), ("ctas_per_sm", ctypes.c_int32), ("tile_slots", ctypes.c_int32),
                ("forward_walk", ctypes.c_int32), ("ms_per_step", ctypes.c_double), ("candidates", ctypes.c_int32),
                ("from_cache", ctypes.c_int32), ("values_per_thread", ctypes.c_int32), ("walk_skip", ctypes.c_int32),
                ("no_meta_cache", ctypes.c_int32), ("flow_ranges", ctypes.c_int32)]

    def as_dict(self):
        d = {k: getattr(self, k) for k, _ in self._fields_}
        d["kernel"] = {VARIANT_FUSED: "tile", VARIANT_PAIRS: "pairs", VARIANT_FLOW: "flow"}.get(self.variant, "rows")
        return d


class Pml(ctypes.Structure):
    _fields_ = [("x0", ctypes.c_double), ("y0", ctypes.c_double), ("r_inner", ctypes.c_double),
                ("r_outer", ctypes.c_double), ("sigma_max", ctypes.c_double), ("order", ctypes.c_int32)]


class Rk45Opts(ctypes.Structure):
    _fields_ = [("rtol", ctypes.c_double), ("atol", ctypes.c_double), ("h0", ctypes.c_double),
                ("max_steps", ctypes.c_int64)]


class Rk45Stats(ctypes.Structure):
    _fields_ = [("n_accepted", ctypes.c_int64), ("n_rejected", ctypes.c_int64), ("n_rhs", ctypes.c_int64),
                ("h_last", ctypes.c_double), ("z", ctypes.c_double)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class SolitonOpts(ctypes.Structure):
    _fields_ = [("power", ctypes.c_double), ("tau", ctypes.c_double), ("tol", ctypes.c_double),
                ("mix", ctypes.c_double), ("max_iter", ctypes.c_int64), ("kerr_mode", ctypes.c_int32)]


class SolitonStats(ctypes.Structure):
    _fields_ = [("mu", ctypes.c_double), ("residual", ctypes.c_double), ("iterations", ctypes.c_int64),
                ("cheb_terms", ctypes.c_int64)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class Diag(ctypes.Structure):
    _fields_ = [("z", ctypes.c_double), ("power", ctypes.c_double), ("hamiltonian", ctypes.c_double),
                ("max_intensity", ctypes.c_double)]


_vp = ctypes.c_void_p
_i32 = ctypes.c_int32
_i64 = ctypes.c_int64
_dbl = ctypes.c_double

# name -> (restype, argtypes)
SIGNATURES = {
    "decbpm_version": (ctypes.c_char_p, []),
    "decbpm_last_error": (ctypes.c_char_p, []),
    "decbpm_mesh_create": (_i32, [ctypes.POINTER(MeshDesc), ctypes.POINTER(_vp)]),
    "decbpm_mesh_destroy": (_i32, [_vp]),
    "decbpm_mesh_info": (_i32, [_vp, ctypes.POINTER(MeshInfo)]),
    "decbpm_assemble_host": (_i32, [ctypes.POINTER(MeshDesc), ctypes.POINTER(MeshInfo), _c_double_p, _c_double_p,
                                    _c_double_p, _c_int64_p, _c_int32_p, _c_double_p, _c_int32_p]),
    "decbpm_bessel_coefficients": (_i32, [_dbl, _dbl, _i32, _c_double_p, _c_int32_p]),
    "decbpm_propagate": (_i32, [_vp, ctypes.POINTER(Params), _vp, _i64, _vp, ctypes.POINTER(Diag)]),
    "decbpm_propagate_host": (_i32, [_vp, ctypes.POINTER(Params), _vp, _i64, _vp, ctypes.POINTER(Diag)]),
    "decbpm_diagnostics": (_i32, [_vp, _vp, _i64, _i32, _vp, ctypes.POINTER(Diag)]),
    "decbpm_plan_create": (_i32, [ctypes.POINTER(_vp), _i32, _c_int32_p, _i32, ctypes.POINTER(_vp)]),
    "decbpm_plan_destroy": (_i32, [_vp]),
    "decbpm_plan_propagate": (_i32, [_vp, ctypes.POINTER(Params), ctypes.POINTER(_vp), _vp, ctypes.POINTER(Diag)]),
    "decbpm_plan_propagate_host": (_i32, [_vp, ctypes.POINTER(Params), ctypes.POINTER(_vp), _vp,
                                          ctypes.POINTER(Diag)]),
    "decbpm_plan_degree": (_i32, [_vp, _i32, _dbl, _i32, _dbl]),
    "decbpm_plan_get_config": (_i32, [_vp, ctypes.POINTER(PlanConfig)]),
    "decbpm_plan_autotune": (_i32, [_vp, _dbl, _i32, _i32, _vp, ctypes.POINTER(TuneResult)]),
    "decbpm_plan_set_shape": (_i32, [_vp, ctypes.POINTER(TuneResult)]),
    "decbpm_plan_last_march_ms": (_i32, [_vp, ctypes.POINTER(ctypes.c_double)]),
    "decbpm_selftest_barrier": (_i32, [_i32, _i64, _vp]),
    "decbpm_selftest_bounds_check": (_i32, [_vp]),
    "decbpm_mesh_set_potential": (_i32, [_vp, _c_double_p]),
    "decbpm_vjp": (_i32, [_vp, ctypes.POINTER(Params), _vp, _vp, _vp, _vp, _vp, _i64, _i32, _vp]),
    "decbpm_mesh_set_potential_offset": (_i32, [_vp, _vp, _vp]),
    "decbpm_adjoint": (_i32, [_vp, ctypes.POINTER(Params), _vp, _vp, _i64, _c_double_p, _vp, _vp, _i32, _vp]),
    "decbpm_soliton": (_i32, [_vp, ctypes.POINTER(SolitonOpts), _vp, _vp, ctypes.POINTER(SolitonStats)]),
    "decbpm_bessel_i_scaled": (_i32, [_dbl, _dbl, _i32, ctypes.POINTER(ctypes.c_double), ctypes.POINTER(_i32)]),
    "decbpm_mesh_set_pml": (_i32, [_vp, ctypes.POINTER(Pml)]),
    "decbpm_mesh_pml_degree": (_i32, [_vp, _dbl, _i32, _dbl]),
    "decbpm_rk45": (_i32, [_vp, _dbl, _i32, ctypes.POINTER(Rk45Opts), _vp, _vp, ctypes.POINTER(Rk45Stats)]),
    "decbpm_propagate_noalloc": (_i32, [_vp, ctypes.POINTER(Params), _vp, _i64, _vp]),
    "decbpm_propagate_batch": (_i32, [ctypes.POINTER(_vp), _i32, _c_int32_p, ctypes.POINTER(Params),
                                      ctypes.POINTER(_vp), _vp, ctypes.POINTER(Diag)]),
}

_lib = None
_lock = threading.Lock()


class DecbpmError(RuntimeError):
    def __init__(self, code: int, message: str):
        super().__init__("decbpm error %d: %s" % (code, message))
        self.code = code


def load(build_if_missing: bool = True) -> ctypes.CDLL:
    """Load (building first if needed) the CUDA library.  Raises if it
    cannot be loaded: there is no non-CUDA implementation of the product path."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        if build_if_missing:
            from . import build as _build
            if not os.path.exists(LIB_PATH) or not _build.up_to_date(CHECKED):
                try:
                    _build.build(checked=CHECKED)
                except Exception as exc:  # noqa: BLE001
                    if not os.path.exists(LIB_PATH):
                        raise RuntimeError("%s is missing and could not be built: %s"
                                           % (os.path.basename(LIB_PATH), exc)) from exc
        if not os.path.exists(LIB_PATH):
            raise RuntimeError("%s not found (run python -m paper_2608_03587_b300.build --all)" % LIB_PATH)
        lib = ctypes.CDLL(LIB_PATH)
        for name, (res, args) in SIGNATURES.items():
            fn = getattr(lib, name)
            fn.restype = res
            fn.argtypes = args
        _lib = lib
        return lib


def check(rc: int) -> None:
    if rc != OK:
        msg = _lib.decbpm_last_error().decode() if _lib is not None else ""
        raise DecbpmError(rc, msg)
