"""Oracle: Algorithm 1 setup (FP64, plain numpy).

Test infrastructure only (see the package docstring).

  diag_inv        D^-1, D = diag(A)                        (Algorithm 1, setup)
  smooth_samples  S = (I - w D^-1 A)^s1 S0, s1 explicit sweeps
                                                           (Sec. 3, Near-Nullspace Vectors)
  prolongation    P = U_k, the leading k left singular vectors of S, with the
                  singular values (Sec. 3, SVD-Centric Construction; the
                  Eckart-Young optimum that the neural map f_theta imitates)
  truncate        P_r = P[:, :r]                           (Algorithm 1, setup)
  galerkin        A_c = P^T A P                            (Algorithm 1, setup; Appendix,
                                                            Two-Level Subspace Correction)
  coarse_factor   lower Cholesky factor L, A_c = L L^T     (coarse solve of Algorithm 1,
                                                            read as a dense Cholesky)

Pins (tests/test_oracle_setup.py): sine modes of the Poisson operator are
damped by (1 - w mu)^s1 (closed form); P^T P = I; the captured energy of U_k
equals sum_{i<=k} sigma_i^2 / sum sigma_i^2 (Eckart-Young); a matrix built with
a known SVD returns its own left factor; an independent eigen route (S^T S)
gives the same projector; P = I gives A_c = A; A_c is SPD.
"""
from __future__ import annotations

import numpy as np


def diag_inv(A) -> np.ndarray:
    return 1.0 / A.diagonal()


def jacobi_sweep(A, dinv: np.ndarray, z: np.ndarray, b: np.ndarray, omega: float) -> np.ndarray:
    """One weighted-Jacobi sweep z + w D^-1 (b - A z), column-wise for blocks."""
    d = dinv if z.ndim == 1 else dinv[:, None]
    return z + omega * d * (b - A @ z)


def smooth_samples(A, S0: np.ndarray, omega: float, s1: int) -> np.ndarray:
    """S = (I - w D^-1 A)^s1 S0: s1 Jacobi sweeps on A S = 0 from S0."""
    dinv = diag_inv(A)[:, None]
    S = np.array(S0, dtype=np.float64, copy=True)
    for _ in range(s1):
        S = S - omega * dinv * (A @ S)
    return S


def prolongation(S: np.ndarray, k: int):
    """Leading k left singular vectors of S (thin SVD) and all singular values,
    in descending order.  Only span(P) is determined (Sec. 3)."""
    U, sig, _ = np.linalg.svd(S, full_matrices=False)
    return U[:, :k].copy(), sig


def truncate(P: np.ndarray, r: int) -> np.ndarray:
    return P[:, :r].copy()


def galerkin(A, P: np.ndarray) -> np.ndarray:
    return P.T @ (A @ P)


def coarse_factor(Ac: np.ndarray) -> np.ndarray:
    """Lower Cholesky factor of A_c; raises numpy.linalg.LinAlgError if A_c
    is not SPD."""
    return np.linalg.cholesky(0.5 * (Ac + Ac.T))


def build(A, S0: np.ndarray, k: int, omega: float, s1: int, r: int | None = None):
    """Full setup: returns dict(S, P, sigma, Ac, L)."""
    S = smooth_samples(A, S0, omega, s1)
    P, sig = prolongation(S, k)
    if r is not None:
        P = truncate(P, r)
    Ac = galerkin(A, P)
    L = coarse_factor(Ac)
    return {"S": S, "P": P, "sigma": sig, "Ac": Ac, "L": L}
