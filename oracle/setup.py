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
  prolongation_a_weighted
                  the A-weighted spectral basis: range(A^{1/2} P) = the top-k
                  left singular subspace of A^{1/2} S, the minimiser of the
                  post-correction smooth-energy error (Appendix, Galerkin
                  Convergence theorem); the paper does not use it for its own
                  experiments
  post_correction_energy
                  J(P) = ||A^{1/2} (I - Pi_A(P)) S||_F^2, Pi_A(P) = P (P^T A P)^-1 P^T A
                                                           (Appendix, Galerkin Convergence)
  prolongation_randomized
                  randomised range finder with q power iterations and the SVD
                  of the small projected matrix (Halko, Martinsson, Tropp 2011,
                  Algorithms 4.4 and 5.1); the paper's RandomSVD baseline

Pins (tests/test_oracle_setup.py): sine modes of the Poisson operator are
damped by (1 - w mu)^s1 (closed form); P^T P = I; the captured energy of U_k
equals sum_{i<=k} sigma_i^2 / sum sigma_i^2 (Eckart-Young); a matrix built with
a known SVD returns its own left factor; an independent eigen route (S^T S)
gives the same projector; P = I gives A_c = A; A_c is SPD.  A-weighted basis:
P^T A P = I; J(P) equals the Eckart-Young tail of A^{1/2} S computed with a
dense square root of A and a library SVD; no Euclidean SVD basis or perturbed
basis does better; its A^{1/2}-image spans the dense route's singular
subspace.  Randomised basis: exact when rank(S) <= k + oversampling; with
power iterations it converges to the SVD projector.
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


def prolongation_a_weighted(A, S: np.ndarray, k: int):
    """A-weighted spectral basis (Appendix, Galerkin Convergence): with
    Z = A^{1/2} S = U Sigma V^T, take P = S V_k Sigma_k^-1, so that
    A^{1/2} P = U_k spans the top-k left singular subspace of Z and
    P^T A P = I.  V and Sigma come from the eigen-decomposition of
    Z^T Z = S^T A S, so no square root of A is formed.  Returns P and the
    singular values of Z in descending order."""
    G = S.T @ (A @ S)
    lam, V = np.linalg.eigh(0.5 * (G + G.T))
    order = np.argsort(lam)[::-1]
    lam, V = lam[order], V[:, order]
    sig = np.sqrt(np.maximum(lam, 0.0))
    return S @ V[:, :k] / sig[:k][None, :], sig


def post_correction_energy(A, P: np.ndarray, S: np.ndarray) -> float:
    """J(P) = ||A^{1/2} (I - Pi_A(P)) S||_F^2 with the Galerkin projector
    Pi_A(P) = P (P^T A P)^-1 P^T A (Appendix, Galerkin Convergence),
    evaluated as tr(E^T A E), E = (I - Pi_A(P)) S."""
    Ac = P.T @ (A @ P)
    E = S - P @ np.linalg.solve(Ac, P.T @ (A @ S))
    return float(np.sum(E * (A @ E)))


def prolongation_randomized(S: np.ndarray, k: int, oversample: int, power_iters: int,
                            Omega: np.ndarray, return_sigma: bool = False):
    """Randomised SVD basis (Halko, Martinsson, Tropp 2011): Y = S Omega with
    a Gaussian test matrix Omega (K x (k + oversample), passed in), q power
    iterations Y <- S (S^T Y) with re-orthonormalisation (their Algorithm
    4.4), Q = qr(Y), then the SVD of the small matrix B = Q^T S (their
    Algorithm 5.1): P = Q U_B[:, :k].  With return_sigma, also the singular
    values of B."""
    assert Omega.shape == (S.shape[1], k + oversample)
    Q, _ = np.linalg.qr(S @ Omega)
    for _ in range(power_iters):
        W, _ = np.linalg.qr(S.T @ Q)
        Q, _ = np.linalg.qr(S @ W)
    UB, sB, _ = np.linalg.svd(Q.T @ S, full_matrices=False)
    P = Q @ UB[:, :k]
    return (P, sB) if return_sigma else P
