"""FP64 CPU oracle for the spectral two-level preconditioned CG of NeuraLSP.

TEST INFRASTRUCTURE ONLY.  Nothing on the product path may import, call or
execute this package: only the test suite, the smoke check of the CUDA path and
the benchmark's CPU-baseline leg use it.  It shares no code with the CUDA
library; both sides read the same seeded inputs from
`paper_2601_20174_gb300.inputs`, which holds no solver arithmetic.

Every function follows a passage of the paper (arXiv 2601.20174) in plain
numpy/scipy FP64, without blocking, fusion or reordering:

  operator.py  sparse SPD operator A of the stencil PDE families (Sec. 3,
               Eq. discretized_pde; the PDE families of the Appendix).
  setup.py     Algorithm 1 setup: D = diag(A), S = (I - w D^-1 A)^s1 S0
               (Sec. 3 "Near-Nullspace Vectors"), P = leading k left singular
               vectors of S (Sec. 3 "SVD-Centric Construction"), rank
               truncation, A_c = P^T A P and its Cholesky factor.
  prec.py      Algorithm 1 apply: nu1 Jacobi sweeps from z = 0, residual,
               restriction, coarse solve, prolongation, nu2 sweeps.
  pcg.py       preconditioned CG (Sec. 4 "Two-grid Solver Evaluation").
  losses.py    subspace energy / loss (Eq. subspace_energy and its residual
               form in the Appendix optimality proof), NLSS (Eq. nlss_loss),
               Energy(r) (Sec. 4), the T-step unrolled PCG residual loss.

Parity status of each function is listed in its docstring; functions without
an independent pin say "parity unpinned".
"""
from . import operator, setup, prec, pcg, losses  # noqa: F401
