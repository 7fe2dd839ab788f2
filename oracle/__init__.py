"""CPU FP64 oracle of the matrix-free FMG Stokes solver.

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and
the ``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` may import
or run anything in this package.  The CUDA library never links, imports or
calls it, and it never calls the CUDA library.

Modules:
  * fe         -- exact element matrices (barycentric monomial integration)
  * mesh       -- Kuhn lattices of refined Kuhn-box macro meshes, Bey's rule
  * stokes     -- assembly, rhs, multicolour Gauss-Seidel, inexact Uzawa,
                  transfers, bordered coarse solve, V-cycle, FMG, errors,
                  power iteration for omega^{-1}
  * workmodel  -- the paper's work-unit model
  * unstructured -- the operator blocks on Bey-refined unstructured macro
                  meshes (the paper's 24-tetrahedron cube), assembled
                  element by element without a lattice
  * sampled    -- single rows of the operator at any level
  * mlp        -- the learned coarse correction's network (reference)

Every function here is pinned by a test in tests/test_oracle_pins.py against
values the paper prints, closed forms, invariants, dense linear algebra or
brute force (e.g. the error norms by exact L2 norms of polynomials, the
omega^{-1} power iteration by the dense eigenvalue, the Uzawa step by dense
splitting matrices).
"""
