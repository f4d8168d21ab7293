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


def _fd(f, X, V, ts=(1e-4, 1e-5, 1e-6)):
    return [(f(X + t * V) - f(X - t * V)) / (2 * t) for t in ts]


def test_subspace_loss_gradient(smoothed):
    p, _, S, U, _ = smoothed
    rng = np.random.default_rng(4)
    Ph = U[:, :p.k] + 0.1 * rng.standard_normal((p.n, p.k))
    G = losses.grad_subspace_loss(Ph, S)
    V = rng.standard_normal(Ph.shape)
    ref = float(np.sum(G * V))
    assert min(abs(d - ref) for d in _fd(lambda X: losses.subspace_loss(X, S), Ph, V)) <= 1e-6 * abs(ref)
    assert np.linalg.norm(Ph.T @ G) <= 1e-10 * np.linalg.norm(Ph) * np.linalg.norm(G)
    # stationary at the exact basis
    assert np.linalg.norm(losses.grad_subspace_loss(U[:, :p.k], S)) <= 1e-9 * np.sum(S * S)


def test_nlss_gradient(smoothed):
    p, _, S, U, _ = smoothed
    rng = np.random.default_rng(5)
    Ph = U[:, :p.k] + 0.1 * rng.standard_normal((p.n, p.k))
    G = losses.grad_nlss_loss(Ph, S)
    V = rng.standard_normal(Ph.shape)
    ref = float(np.sum(G * V))
    assert min(abs(d - ref) for d in _fd(lambda X: losses.nlss_loss(X, S), Ph, V)) <= 1e-6 * abs(ref)
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
    V = rng.standard_normal(P.shape)
    ref = float(np.sum(G * V))
    fds = _fd(lambda X: losses.unrolled_pcg_loss(A, X, b, 3, p.omega, 2), P, V)
    assert min(abs(d - ref) for d in fds) <= 1e-6 * abs(ref)
    # the loss depends on range(P) only
    assert np.linalg.norm(P.T @ G) <= 1e-8 * np.linalg.norm(P) * np.linalg.norm(G)
