"""B300-native (sm_103a) DEC beam propagation: the split-step z-march of a
complex transverse field on an unstructured mesh (linear DEC diffraction
propagator, Kerr phase, absorber) behind the C ABI of include/decbpm.h.

The compute path is libdecbpm.so (hand-written CUDA); this package only
marshals arguments.  ``workloads`` makes seeded synthetic inputs and can be
imported without the library.
"""
_API = ("Mesh", "Plan", "mesh_create", "plan_create", "propagate", "propagate_host", "diagnostics",
        "assemble_host", "bessel_coefficients", "vjp", "adjoint", "march", "set_potential", "set_potential_offset",
        "propagate_noalloc", "rk45",
        "soliton", "bessel_i_scaled", "set_pml")


def __getattr__(name):
    if name in _API:
        from . import api
        return getattr(api, name)
    raise AttributeError(name)


__all__ = list(_API)
