"""Plain FP64 CPU oracle for the immersed-FSI hot path.

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` may import, call or
link anything in this package.  The product library never touches it, and it
shares no code, header, table or helper with the CUDA path; the only thing
the two sides have in common is the seeded input generator module, which
holds none of the method's arithmetic.

Contents and the passages they follow:

* ``core``      -- ctypes wrappers over ``fsi_oracle.c``: Q1 shape functions,
  tau_m / tau_c (Sec. 2.1), the VMS residual and its consistent Jacobian-vector
  product (Eq. fluid_weak_form + the VMS terms Sec. 2.1 refers to; reduced
  system of Sec. 2.4), point location, interpolation (Eq. nodal_solid_velo)
  and spreading (Eq. fsi_constraint_matrix).
* ``tet``       -- the same operators on unstructured meshes of linear
  tetrahedra (the element family of the paper's valve mesh, Sec. 4).
* ``timeint``   -- generalized-alpha constants and stage values (Sec. 2.4).
* ``newton``    -- the Newton step of Sec. 2.4 on the reduced 2x2 block system
  with direct sparse solves (small grids), and the point-mass solid stand-in.
* ``mlp``       -- the FP64 reference of the learned initial-guess network
  (forward, backward, Adam), and its stencil features.

Parity status of every function is listed in its module docstring.
"""
from . import core, timeint  # noqa: F401
