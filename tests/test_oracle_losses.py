"""Pins for oracle.losses: Eq. subspace_energy, Eq. nlss_loss, Thm 1 / Cor. 2,
the weighted Ky-Fan identity, Energy(r), and the reference gradients."""
import math

import numpy as np
import pytest

from oracle import losses, operator as op, setup as su
from paper_2601_20174_gb300 import inputs as gen


@pytest.fixture(scope="module")
def smoothed():
    p = gen.iid_diffusion_2d(N=10, k=6, K=16, seed=11)
    A = op.assemble(p)
    S = su.smooth_samples(A, p.S0, p.omega, p.s1)
    U, sig, _ = np.linalg.svd(S, full_matrices=False)
    return p, A, S, U, sig


def test_subspace_loss_minimum_is_tail_energy(smoothed):
    p, _, S, U, sig = smoothed
    k = p.k
    assert math.isclose(losses.subspace_loss(U[:, :k], S), float(np.sum(sig[k:] ** 2)), rel_tol=1e-10)
    # invariant under P_hat -> P_hat R for any invertible R (range-only)
    R = np.random.default_rng(0).standard_normal((k, k)) + 3 * np.eye(k)
    assert math.isclose(losses.subspace_loss(U[:, :k] @ R, S), float(np.sum(sig[k:] ** 2)), rel_tol=1e-9)
    # J(P) + loss = ||S||^2 for orthonormal P (Appendix optimality proof)
    Q = losses.qf(np.random.default_rng(1).standard_normal((p.n, k)))
    assert math.isclose(losses.subspace_energy(Q, S) + losses.subspace_loss(Q, S), float(np.sum(S * S)),
                        rel_tol=1e-12)


def test_nlss_minimum_closed_form_thm1_cor2(smoothed):
    p, _, S, U, sig = smoothed
    k = p.k
    s2 = np.sum(sig ** 2)
    want = np.mean([1 - np.sum(sig[:l] ** 2) / s2 for l in range(1, k + 1)])
    assert math.isclose(losses.nlss_loss(U[:, :k], S), want, rel_tol=1e-12)
    # a rotation inside the optimal subspace keeps the subspace loss but raises NLSS
    Qr, _ = np.linalg.qr(np.random.default_rng(2).standard_normal((k, k)))
    assert losses.nlss_loss(U[:, :k] @ Qr, S) > want + 1e-6
    # sign flips of columns leave it unchanged (Cor. 2: U_k D)
    D = np.diag([1, -1, 1, -1, -1, 1][:k])
    assert math.isclose(losses.nlss_loss(U[:, :k] @ D, S), want, rel_tol=1e-12)


def test_weighted_kyfan_identity(smoothed):
    p, _, S, _, _ = smoothed
    k = p.k
    Q = losses.qf(np.random.default_rng(3).standard_normal((p.n, k)))
    s2 = np.sum(S * S)
    kyfan = sum((k - j) * float(Q[:, j] @ S @ (S.T @ Q[:, j])) for j in range(k))  # weight k-j+1, 1-based
    assert math.isclose(losses.nlss_loss(Q, S), 1 - kyfan / (k * s2), rel_tol=1e-12)


def test_energy_eckart_young(smoothed):
    _, _, S, U, sig = smoothed
    for r in (1, 3, 6):
        assert math.isclose(losses.energy(U, S, r), np.sum(sig[:r] ** 2) / np.sum(sig ** 2), rel_tol=1e-12)


def _fd_errors(f, X, G, rng, t=1e-5, ndir=3):
    """Relative errors of <G, V> against the central difference of f at one
    fixed step t, along ndir seeded random directions V."""
    errs = []
    for _ in range(ndir):
        V = rng.standard_normal(X.shape)
        ref = float(np.sum(G * V))
        fd = (f(X + t * V) - f(X - t * V)) / (2 * t)
        errs.append(abs(fd - ref) / abs(ref))
    return errs


def test_subspace_loss_gradient(smoothed):
    p, _, S, U, _ = smoothed
    rng = np.random.default_rng(4)
    Ph = U[:, :p.k] + 0.1 * rng.standard_normal((p.n, p.k))
    G = losses.grad_subspace_loss(Ph, S)
    assert max(_fd_errors(lambda X: losses.subspace_loss(X, S), Ph, G, rng)) <= 1e-6
    assert np.linalg.norm(Ph.T @ G) <= 1e-10 * np.linalg.norm(Ph) * np.linalg.norm(G)
    # stationary at the exact basis
    assert np.linalg.norm(losses.grad_subspace_loss(U[:, :p.k], S)) <= 1e-9 * np.sum(S * S)


def test_nlss_gradient(smoothed):
    p, _, S, U, _ = smoothed
    rng = np.random.default_rng(5)
    Ph = U[:, :p.k] + 0.1 * rng.standard_normal((p.n, p.k))
    G = losses.grad_nlss_loss(Ph, S)
    assert max(_fd_errors(lambda X: losses.nlss_loss(X, S), Ph, G, rng)) <= 1e-6
    # invariant under P_hat -> P_hat R, R upper triangular (every prefix span kept)
    M = Ph.T @ G
    assert np.linalg.norm(np.triu(M)) <= 1e-10 * np.linalg.norm(M) + 1e-14


def test_unrolled_pcg_loss_gradient():
    p = gen.iid_diffusion_2d(N=6, k=5, K=10, seed=12)
    A = op.assemble(p)
    S = su.smooth_samples(A, p.S0, p.omega, p.s1)
    P, _ = su.prolongation(S, p.k)
    rng = np.random.default_rng(6)
    P = P + 0.05 * rng.standard_normal(P.shape)
    b = p.f[:, 0]
    G = losses.grad_unrolled_pcg_loss(A, P, b, 3, p.omega, 2)
    assert max(_fd_errors(lambda X: losses.unrolled_pcg_loss(A, X, b, 3, p.omega, 2), P, G, rng)) <= 1e-6
    # the loss depends on range(P) only
    assert np.linalg.norm(P.T @ G) <= 1e-8 * np.linalg.norm(P) * np.linalg.norm(G)


@pytest.mark.parametrize("T", [1, 3, 10])
def test_unrolled_pcg_loss_is_pcg_residual_history(T):
    """The unrolled loss is ||r_T|| of the PCG of Sec. 4 with the two-level
    preconditioner of Algorithm 1: it must equal ||b|| times the recursive
    relative residual that oracle.pcg (pinned by exact solves and the CG bound)
    records after its T-th iteration when no tolerance stops it earlier."""
    from oracle import pcg as opcg
    p = gen.iid_diffusion_2d(N=9, k=6, K=12, seed=21)
    A = op.assemble(p)
    S = su.smooth_samples(A, p.S0, p.omega, p.s1)
    P, _ = su.prolongation(S, p.k)
    P = P + 0.05 * np.random.default_rng(7).standard_normal(P.shape)  # full rank, not orthonormal
    Ac = P.T @ (A @ P)
    L = np.linalg.cholesky(0.5 * (Ac + Ac.T))
    b = p.f[:, 0]
    res = opcg.pcg(A, opcg.two_level_solver(A, P, L, p.omega, 2, 2), b, tol=0.0, maxit=T)
    assert res["iters"] == T and len(res["history"]) == T
    want = np.linalg.norm(b) * res["history"][T - 1]
    assert math.isclose(losses.unrolled_pcg_loss(A, P, b, T, p.omega, 2), want, rel_tol=1e-12)


def test_unrolled_pcg_loss_vanishes_with_exact_coarse_space():
    """k = n makes the coarse correction exact (B = A^-1, Appendix, Two-Level
    Subspace Correction), so one PCG step solves the system: r_1 = 0."""
    p = gen.poisson_2d(N=5, k=25, K=25, seed=3)
    A = op.assemble(p)
    P = np.linalg.qr(np.random.default_rng(8).standard_normal((p.n, p.n)))[0]
    b = p.f[:, 0]
    assert losses.unrolled_pcg_loss(A, P, b, 1, p.omega, 2) <= 1e-10 * np.linalg.norm(b)
