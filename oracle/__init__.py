"""Plain, slow FP64 CPU oracle for the multiscale-multigrid (MMG) heat solve.

TEST INFRASTRUCTURE ONLY.  Nothing in the product path may import, call, link
or execute this package; only the test-suite, ``__graft_entry__.smoke()`` and
``bench.py``'s CPU-baseline / reference arm use it.  It shares no code with the
CUDA library (no kernels, headers, tables or pre/post-processing); the only
common dependency is the seeded input generator module ``workloads``.

Modules
  fem     Q1 trilinear discretisation of the steady heat equation with SIMP
          conductivity (Sec. 2.1 Eq. (1), Sec. 2.2 Eq. (5)), load vector,
          compliance (Eq. (6)) and adjoint sensitivity (Sec. 2.3 Eq. (7)).
  mmg     Multiscale multigrid: local spectral problems (Sec. 3 Eqs. (8), (9)),
          Galerkin coarse operators, smoothed V-cycle (Algorithm 1).
  krylov  CG / preconditioned CG / flexible CG (Sec. 4, PETSc CG).
  topopt  Density filter and optimality-criteria update (textbook SIMP
          harness; the paper uses MMA instead, Sec. 2.3).

Parity status of every function is stated in its docstring; a function with
no independent pin says "parity unpinned".
"""
