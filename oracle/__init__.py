"""Plain FP64 CPU oracle for the adaptive volume-potential box FMM.

TEST INFRASTRUCTURE ONLY. This package restates, slowly and in plain numpy, what
the box code of Section 3 computes: the volume integral
V[f](x) = -(1/2 pi) int_B log|x - y| f(y) dy (Eq. volumeint3, Section 3) and its
gradient (Eq. volumeint3x, Section 3.2) at the collocation nodes of the leaves of
a level-restricted quadtree (Section 3.1).

Only ``tests/``, ``__graft_entry__.smoke()`` and the ``cpu_baseline`` /
``--impl reference`` legs of ``bench.py`` may import it. The CUDA library never
imports, links or calls anything here, and nothing here calls the CUDA library.

Modules:
  cheb    - nodes, Fejer weights, Lagrange basis, values->coefficients (Section 3.1)
  source  - evaluation of the synthetic right-hand sides
  tree    - adaptive refinement, level restriction, U/V/W/X lists (Section 3.1, Fig. 1)
  quad    - box integrals of the kernel against the Lagrange basis (Section 3.1: the
            near-field tables; Section 3.2 for the gradient kernels)
  tables  - unit-scale operators: near tables, S2M, S2L, M2T, L2T, M2M, M2L, L2L
  fmm     - the FMM passes (Section 3.1) producing u, u_x, u_y at leaf nodes
  brute   - direct quadrature of V[f~] without FMM or tables, for small trees
  interp  - the leaf interpolant v~ of computed values at arbitrary points (Section 3.1)
  offnode - V f~ at arbitrary points from the stored expansions plus per-point near-field
            quadrature (Sections 3.1 and 5.3)

Parity status: every function is pinned by tests/test_oracle_*.py except where
its docstring says "parity unpinned".
"""
