"""Oracle: one application z = B b of the two-level preconditioner
(Algorithm 1, "Apply preconditioner to residual b"), FP64.

Test infrastructure only (see the package docstring).

  z <- 0
  nu1 weighted-Jacobi sweeps on A z = b
  rho <- b - A z
  solve A_c e_c = P^T rho            (dense Cholesky, A_c = L L^T)
  z <- z + P e_c
  nu2 weighted-Jacobi sweeps on A z = b, from the current z

Works column-wise when b is n x m.

Pins (tests/test_oracle_prec.py): the coarse correction annihilates range(P)
(Appendix, Two-Level Subspace Correction: E_c P y = 0); after it the residual
is orthogonal to range(P) and the error is the A-norm best approximation from
range(P); B is symmetric and positive definite for nu1 = nu2 >= 1; k = n gives
B = A^-1; for the Poisson operator with P = the k lowest sine modes, B acts on
each mode by the closed-form factor (1 - (1 - w mu)^(2 nu)) / lambda outside
range(P) and 1/lambda inside.
"""
from __future__ import annotations

import numpy as np
import scipy.linalg as sla


def coarse_solve(L: np.ndarray, c: np.ndarray) -> np.ndarray:
    """e_c = (L L^T)^-1 c by two triangular solves."""
    y = sla.solve_triangular(L, c, lower=True)
    return sla.solve_triangular(L.T, y, lower=False)


def apply(A, P: np.ndarray, L: np.ndarray, b: np.ndarray, omega: float, nu1: int, nu2: int) -> np.ndarray:
    b = np.asarray(b, dtype=np.float64)
    dinv = 1.0 / A.diagonal()
    d = dinv if b.ndim == 1 else dinv[:, None]
    z = np.zeros_like(b)
    for _ in range(nu1):
        z = z + omega * d * (b - A @ z)
    rho = b - A @ z
    ec = coarse_solve(L, P.T @ rho)
    z = z + P @ ec
    for _ in range(nu2):
        z = z + omega * d * (b - A @ z)
    return z


def coarse_error_propagator(A, P: np.ndarray) -> np.ndarray:
    """Dense E_c = I - P A_c^-1 P^T A (small n only)."""
    Ad = A.toarray() if hasattr(A, "toarray") else np.asarray(A)
    Ac = P.T @ Ad @ P
    return np.eye(Ad.shape[0]) - P @ np.linalg.solve(Ac, P.T @ Ad)
