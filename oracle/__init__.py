"""CPU FP64 oracle for the staggered space-time DG scheme (arXiv:1802.04516).

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / reference leg of ``bench.py`` may import or run anything in this
package; the library's compute path never does.  It shares no code with the CUDA
library: it has its own bases, quadrature, mesh connectivity, operator blocks,
explicitly assembled sparse velocity system and direct (SuperLU) solve.

Modules
  basis      nodal P_p basis on the reference simplex, Taylor-monomial dual basis,
             Lagrange time basis on Gauss-Legendre points (Sec. 3, "Space-time basis
             functions")
  quadrature collapsed-coordinate Gauss-Legendre rules on simplices
  mesh       faces Gamma_j, l(j)/r(j), normals n_j, dual cells R_j = T_{l,j} u T_{r,j}
             (Sec. 3, "Two space dimensions" / "Three space dimensions")
  operators  M_j, Mbar_i, D_{i,j}, Q_{i,j}, time matrices (Eqs. MD_2 - SD_1), the
             Schur velocity system (Eq. velocity.sys, Eq. velocity.sys.cn); the dual
             basis is the Taylor space or, in 2D, the paper's (p+1)^2 tensor space on the
             bilinearly mapped dual quadrilateral (dual="quad")
  precond    Appendix A preconditioners on the assembled system: block Jacobi (Eq. pre1)
             and the stencil-local inverse (Eqs. APPRE1 / APPRE2)
  adjoint    receiver misfit and its exact discrete gradient w.r.t. per-element lambda, mu,
             rho (not in the paper: the adjoint of the oracle's own forward map)
  stepper    one time slab: right-hand side, direct solve, stress back-substitution
             (Eq. NM26 / NM26.cn), traces, energy (Eq. SP3F), receivers, Ricker point
             sources (Sec. 6.3)

Parity status of every function is pinned by ``tests/test_oracle_*.py`` against
closed forms, theorems of the paper and brute-force checks, and by the values the paper
prints (``tests/golden/``: its convergence table, reproduced in rate by
``tests/test_oracle_table1.py``); see each module header.
"""
from . import adjoint, basis, quadrature, mesh, operators, precond, stepper  # noqa: F401
