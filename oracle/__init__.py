"""FP64 CPU oracle for the corotational hinge-based thin plate / shell time step.

TEST INFRASTRUCTURE ONLY. This package is a plain, slow, independent restatement of the method of
"Corotational Hinge-based Thin Plates/Shells" (Liang, arXiv 2502.10872) in numpy/scipy float64. It
exists to check the CUDA library. Only the test suite, ``__graft_entry__.smoke()`` and the CPU-baseline
leg of ``bench.py`` may import or run it; the library itself never does and has no CPU fallback.

It shares no code with the CUDA path: its only shared dependency is :mod:`shellgen`, which generates
seeded meshes and holds no mechanics.

Layout:

* :mod:`oracle.topology`  -- edge-based and triangle-centred stencils from a triangle list (Section 4.2,
  Figure "boundary_shell_patch" for virtual nodes).
* :mod:`oracle.operators` -- rest-state curvature operators L_m (Eq. 9-10, Eq. 31), L_p (App. C,
  Eq. 76-78), R (Eq. 38), C_p and L_g (Eq. 49-50), the boundary folds (Eq. 59, Eq. 61) and the
  material matrices.
* :mod:`oracle.energies`  -- per-stencil bending energies and exact gradients for the six models
  (Eq. 16-26, Eq. 39-45, Eq. 52-57, App. B) and the corotated constant-strain membrane.
* :mod:`oracle.appendix_d` -- App. D's world-frame edge-hinge models QTP and QTS and the Quadratic/Cubic
  shell energy (Eq. 79-89), written from App. D's printed operator.
* :mod:`oracle.system`    -- lumped mass, the constant matrix M + dt^2 (K_b + K_m), the linearised
  backward-Euler step (Section 5, Eq. 62-63), the exact backward-Euler step by chord iteration with its
  residual and incremental potential, and energy totals.

Readings of points the paper leaves open are listed in the docstrings where they are used; the same
readings are implemented (independently) by the CUDA library.

Parity status per function: every function here is pinned by a CPU test against closed forms,
invariants, finite differences or values printed in the paper, except the multi-step trajectories
of the benchmark scenarios (parity unpinned: only self-consistency and oracle-vs-GPU agreement).
"""
from .system import Model, build_model, step, forces, energy, stiffness_matrices  # noqa: F401
