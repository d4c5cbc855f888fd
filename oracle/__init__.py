"""CPU FP64 oracle for the DEC beam propagation method.

TEST INFRASTRUCTURE ONLY.  Nothing in the product path imports this package:
only the tests, the smoke check in ``__graft_entry__`` and the CPU-baseline leg
of ``bench.py`` may call it.  It shares no code with the CUDA library; it takes
the same seeded input arrays (coordinates, cells, per-cell materials, per-vertex
absorber, launch fields) and computes everything else itself.

Modules
-------
``dec``   discrete exterior calculus operators assembled as the paper defines
          them: incidence matrices d0/d1, barycentric Hodge star *0, the
          material stars *0(V) and *0(chi|psi~|^2), the Galerkin Hodge star *1
          built from Whitney 1-forms (Eqs. 8-9), the projection Q (Eq. 13).
``bpm``   the z-march: exact-action linear propagator (Taylor series with
          substeps), exact diagonal phase/absorber flow, Strang composition,
          power / Hamiltonian / error diagnostics, the paper's own adaptive
          RK45 integration of Eq. 10 (cross-check), and the exact discrete
          adjoint of the split-step march.

Parity status: every function here is pinned by a ``-m "not gpu"`` test
(closed forms, exactness identities, dense brute force, conservation laws,
convergence orders) except where its docstring says "parity unpinned".
"""
from . import dec, bpm  # noqa: F401
