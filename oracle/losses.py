"""Oracle: subspace objectives and the unrolled-PCG loss, FP64.

Test infrastructure only (see the package docstring).

  qf              thin-Q factor of a QR decomposition (Sec. 3: P = qf(P_hat))
  subspace_energy J(P) = ||P P^T S||_F^2 = tr(P^T S S^T P)   (Eq. subspace_energy)
  subspace_loss   ||(I - Q Q^T) B||_F^2, Q = qf(P_hat): the residual energy whose
                  minimisation is equivalent to maximising J (Appendix,
                  optimality of smooth error reduction)
  nlss_loss       (1/k) sum_l (1 - ||Q_{1:l}^T S||^2 / ||S||^2) (Eq. nlss_loss)
  energy          Energy(r) = ||Q_r^T S||^2 / ||S||^2   (Sec. 4, subspace-ordering
                  diagnostic)
  unrolled_pcg_loss  ||r_T||_2 after T PCG steps with the two-level
                  preconditioner built from a full-rank P (A_c = P^T A P),
                  x0 = 0.  The differentiation workload's loss; the paper
                  itself trains only subspace objectives (reading recorded in
                  the design notes).

Reference gradients are taken by PyTorch CPU FP64 autograd of these same
definitions restated with torch.linalg routines (grad_* below); they are
pinned in the tests by central finite differences, by the invariance
P_hat^T grad = 0 of range-only losses, and by stationarity at P_hat = U_k.

Pins (tests/test_oracle_losses.py): subspace loss at U_k equals
sum_{i>k} sigma_i^2; NLSS at U_k equals the closed-form minimum of Thm 1 /
Cor. 2, (1/k) sum_l (1 - sum_{i<=l} sigma_i^2 / ||S||^2); the weighted Ky-Fan
identity; Energy(r) of U_k equals the Eckart-Young fraction.
"""
from __future__ import annotations

import numpy as np


def qf(P_hat: np.ndarray) -> np.ndarray:
    Q, _ = np.linalg.qr(P_hat, mode="reduced")
    return Q


def subspace_energy(P: np.ndarray, S: np.ndarray) -> float:
    return float(np.linalg.norm(P @ (P.T @ S)) ** 2)


def subspace_loss(P_hat: np.ndarray, B: np.ndarray) -> float:
    Q = qf(P_hat)
    R = B - Q @ (Q.T @ B)
    return float(np.sum(R * R))


def nlss_loss(P_hat: np.ndarray, S: np.ndarray) -> float:
    Q = qf(P_hat)
    k = Q.shape[1]
    s2 = float(np.sum(S * S))
    C = Q.T @ S
    cap = np.cumsum(np.sum(C * C, axis=1))  # ||Q_{1:l}^T S||^2 for l = 1..k
    return float(np.sum(1.0 - cap / s2) / k)


def energy(Q: np.ndarray, S: np.ndarray, r: int) -> float:
    C = Q[:, :r].T @ S
    return float(np.sum(C * C) / np.sum(S * S))


def unrolled_pcg_loss(A, P: np.ndarray, b: np.ndarray, T: int, omega: float, nu: int) -> float:
    """||r_T|| after exactly T PCG iterations (standard beta), x0 = 0."""
    from . import prec as _prec
    Ac = P.T @ (A @ P)
    L = np.linalg.cholesky(0.5 * (Ac + Ac.T))
    r = np.array(b, dtype=np.float64, copy=True)
    z = _prec.apply(A, P, L, r, omega, nu, nu)
    p = z.copy()
    rz = float(r @ z)
    for t in range(T):
        q = A @ p
        alpha = rz / float(p @ q)
        r = r - alpha * q
        if t == T - 1:
            break
        z = _prec.apply(A, P, L, r, omega, nu, nu)
        rzn = float(r @ z)
        p = z + (rzn / rz) * p
        rz = rzn
    return float(np.linalg.norm(r))


# ---------------------------------------------------------------------------
# Reference gradients: torch CPU FP64 autograd of the same definitions.
# ---------------------------------------------------------------------------

def _torch():
    import torch
    return torch


def grad_subspace_loss(P_hat: np.ndarray, B: np.ndarray) -> np.ndarray:
    torch = _torch()
    Ph = torch.tensor(P_hat, dtype=torch.float64, requires_grad=True)
    Bt = torch.tensor(B, dtype=torch.float64)
    Q, _ = torch.linalg.qr(Ph, mode="reduced")
    R = Bt - Q @ (Q.T @ Bt)
    (R * R).sum().backward()
    return Ph.grad.numpy().copy()


def grad_nlss_loss(P_hat: np.ndarray, S: np.ndarray) -> np.ndarray:
    torch = _torch()
    Ph = torch.tensor(P_hat, dtype=torch.float64, requires_grad=True)
    St = torch.tensor(S, dtype=torch.float64)
    Q, _ = torch.linalg.qr(Ph, mode="reduced")
    k = Q.shape[1]
    C = Q.T @ St
    cap = torch.cumsum((C * C).sum(dim=1), dim=0)
    loss = (1.0 - cap / (St * St).sum()).sum() / k
    loss.backward()
    return Ph.grad.numpy().copy()


def grad_unrolled_pcg_loss(A, P: np.ndarray, b: np.ndarray, T: int, omega: float, nu: int) -> np.ndarray:
    """Autograd through a dense restatement of unrolled_pcg_loss (small n)."""
    torch = _torch()
    Ad = torch.tensor(A.toarray(), dtype=torch.float64)
    dinv = 1.0 / torch.diagonal(Ad)
    Pt = torch.tensor(P, dtype=torch.float64, requires_grad=True)
    Ac = Pt.T @ Ad @ Pt
    L = torch.linalg.cholesky(0.5 * (Ac + Ac.T))

    def apply_B(bv):
        z = torch.zeros_like(bv)
        for _ in range(nu):
            z = z + omega * dinv * (bv - Ad @ z)
        rho = bv - Ad @ z
        ec = torch.cholesky_solve((Pt.T @ rho)[:, None], L)[:, 0]
        z = z + Pt @ ec
        for _ in range(nu):
            z = z + omega * dinv * (bv - Ad @ z)
        return z

    r = torch.tensor(b, dtype=torch.float64)
    z = apply_B(r)
    p = z
    rz = r @ z
    for t in range(T):
        q = Ad @ p
        alpha = rz / (p @ q)
        r = r - alpha * q
        if t == T - 1:
            break
        z = apply_B(r)
        rzn = r @ z
        p = z + (rzn / rz) * p
        rz = rzn
    torch.linalg.norm(r).backward()
    return Pt.grad.numpy().copy()
