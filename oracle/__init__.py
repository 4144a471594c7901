"""Plain, slow, FP64 CPU oracle of the ORAS-FGMRES Maxwell solve (test infrastructure).

This package is TEST INFRASTRUCTURE.  Only `tests/`, `__graft_entry__.smoke()` and the
CPU-baseline leg of `bench.py` may import it.  The CUDA library never calls it and
shares no code, tables or constants with it: the two sides agree on conventions
(stated in each function's docstring), not on code.

What it computes (paper: Bonazzoli, Dolean, Rapetti, Tournier, arXiv:1605.04521):

* `topology`  -- sorted-vertex tetrahedra, edges, faces, global numbering of the
  degree-r Nedelec degrees of freedom (Sec. 3).
* `basis`     -- the generators w^{k,e} = lambda^k w^e of Sec. 3 and the selected
  linearly independent subset; point evaluation of values and curls.
* `elements`  -- element matrices of the weak form of Sec. 2 (curl-curl, mass,
  impedance boundary term) from their definition: conical-product quadrature,
  exact for the degree-2r integrands, of the directly evaluated generators and
  curls.
* `quadrature`-- Gauss-Jacobi rules (Golub-Welsch) and conical-product rules on
  triangles and tetrahedra; used for the element matrices and the loads.
* `assemble`  -- global sparse matrix of Sec. 4 (A u_j = b_j) and right-hand sides.
* `dd`        -- recursive coordinate bisection, overlapping subdomains, restriction
  R_s, partition of unity D_s, local impedance matrices A_s, and the ORAS
  preconditioner M^{-1} = sum_s R_s^T D_s A_s^{-1} R_s (Sec. 4).
* `fgmres`    -- right-preconditioned flexible GMRES(m) with modified Gram-Schmidt
  and Givens rotations (Sec. 5, first paragraph).
* `problem`   -- convenience driver that runs the whole chain on one workload.

Parity pins live in tests/test_oracle_*.py; see each test's docstring for what
independent fact it checks.
"""
