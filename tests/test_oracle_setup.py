"""Pins for oracle.setup (Algorithm 1 setup; Sec. 3)."""
import math

import numpy as np
import pytest

from oracle import operator as op, setup as su
from paper_2601_20174_gb300 import inputs as gen


def _projector_dist(P, Q):
    return float(np.linalg.norm(P @ P.T - Q @ Q.T, 2))


def test_smoothing_damps_sine_modes_by_closed_form():
    # For the Poisson operator D = 4/h^2 I, so (I - w D^-1 A) multiplies the
    # sine mode (p, q) by 1 - w mu, mu = lambda h^2 / 4.
    N, w, s1 = 9, 2.0 / 3.0, 20
    h = 1.0 / (N + 1)
    A = op.diffusion_5pt(N, np.ones((N + 1, N + 1)))
    x = (np.arange(N) + 1) * h
    cols, factors = [], []
    for p, q in [(1, 1), (3, 2), (9, 9)]:
        cols.append(np.outer(np.sin(q * math.pi * x), np.sin(p * math.pi * x)).ravel())
        mu = math.sin(p * math.pi * h / 2) ** 2 + math.sin(q * math.pi * h / 2) ** 2
        factors.append((1 - w * mu) ** s1)
    S0 = np.stack(cols, axis=1)
    S = su.smooth_samples(A, S0, w, s1)
    assert np.allclose(S, S0 * np.array(factors)[None, :], rtol=0, atol=1e-12)


def test_prolongation_recovers_known_left_factor():
    rng = np.random.default_rng(2)
    n, K, k = 60, 12, 5
    U0, _ = np.linalg.qr(rng.standard_normal((n, K)))
    V0, _ = np.linalg.qr(rng.standard_normal((K, K)))
    sig = np.geomspace(10.0, 0.1, K)
    S = U0 @ np.diag(sig) @ V0.T
    P, s = su.prolongation(S, k)
    assert np.allclose(s, sig, rtol=1e-12)
    assert _projector_dist(P, U0[:, :k]) < 1e-12


def test_prolongation_orthonormal_and_eckart_young():
    p = gen.iid_diffusion_2d(N=12, k=8, K=24, seed=1)
    A = op.assemble(p)
    S = su.smooth_samples(A, p.S0, p.omega, p.s1)
    P, sig = su.prolongation(S, p.k)
    assert np.allclose(P.T @ P, np.eye(p.k), atol=1e-13)
    frac = np.linalg.norm(P.T @ S) ** 2 / np.linalg.norm(S) ** 2
    assert math.isclose(frac, np.sum(sig[:p.k] ** 2) / np.sum(sig ** 2), rel_tol=1e-12)
    # and no other rank-k orthonormal basis captures more energy
    rng = np.random.default_rng(0)
    for _ in range(5):
        Q, _ = np.linalg.qr(P + 0.1 * rng.standard_normal(P.shape))
        assert np.linalg.norm(Q.T @ S) ** 2 < np.linalg.norm(P.T @ S) ** 2


def test_prolongation_matches_independent_gram_eigen_route():
    p = gen.grf_diffusion_2d(N=16, k=8, K=32, seed=4)
    A = op.assemble(p)
    S = su.smooth_samples(A, p.S0, p.omega, p.s1)
    P, sig = su.prolongation(S, p.k)
    w, V = np.linalg.eigh(S.T @ S)
    order = np.argsort(w)[::-1][:p.k]
    U = S @ V[:, order] / np.sqrt(w[order])[None, :]
    assert sig[p.k - 1] > 1.01 * sig[p.k]
    assert _projector_dist(P, U) < 1e-8


def test_galerkin_identity_and_spd():
    p = gen.iid_diffusion_2d(N=6, k=36, K=36, seed=2)
    A = op.assemble(p)
    Ac = su.galerkin(A, np.eye(p.n))
    assert np.allclose(Ac, A.toarray(), rtol=0, atol=1e-12 * abs(A).max())
    S = su.smooth_samples(A, p.S0, p.omega, p.s1)
    P, _ = su.prolongation(S, 10)
    Ac = su.galerkin(A, P)
    assert np.allclose(Ac, Ac.T, atol=1e-10 * abs(Ac).max())
    L = su.coarse_factor(Ac)
    assert np.allclose(L @ L.T, Ac, rtol=1e-12, atol=1e-12 * abs(Ac).max())
    with pytest.raises(np.linalg.LinAlgError):
        su.coarse_factor(-Ac)


def test_truncation_is_prefix():
    rng = np.random.default_rng(3)
    P, _ = np.linalg.qr(rng.standard_normal((30, 6)))
    assert np.array_equal(su.truncate(P, 4), P[:, :4])


def _dense_sqrt(A):
    w, V = np.linalg.eigh(A.toarray())
    return (V * np.sqrt(w)) @ V.T


def test_a_weighted_basis_minimises_post_correction_energy():
    # Galerkin Convergence theorem (Appendix): J(P) is smallest when
    # range(A^{1/2} P) is the top-k left singular subspace of A^{1/2} S, where
    # it equals the Eckart-Young tail of A^{1/2} S
    p = gen.grf_diffusion_2d(N=14, k=8, K=24, seed=3)
    A = op.assemble(p)
    S = su.smooth_samples(A, p.S0, p.omega, p.s1)
    P, sig = su.prolongation_a_weighted(A, S, p.k)
    assert np.allclose(P.T @ (A @ P), np.eye(p.k), atol=1e-10)
    Z = _dense_sqrt(A) @ S                       # independent route: dense A^{1/2}, library SVD
    Uz, sz, _ = np.linalg.svd(Z, full_matrices=False)
    assert np.allclose(sig[: len(sz)], sz, rtol=1e-8, atol=1e-10 * sz[0])
    J = su.post_correction_energy(A, P, S)
    assert math.isclose(J, float(np.sum(sz[p.k:] ** 2)), rel_tol=1e-8)
    Q = _dense_sqrt(A) @ P                        # A^{1/2} P spans the top-k subspace of Z
    assert _projector_dist(Q, Uz[:, : p.k]) < 1e-7
    # neither the Euclidean SVD basis nor perturbations of the A-weighted one do better
    Pe, _ = su.prolongation(S, p.k)
    assert su.post_correction_energy(A, Pe, S) > J
    rng = np.random.default_rng(1)
    for _ in range(4):
        assert su.post_correction_energy(A, P + 0.05 * rng.standard_normal(P.shape), S) > J


def test_randomized_basis_exact_for_low_rank_and_converges_with_power_iterations():
    rng = np.random.default_rng(5)
    n, K, k, over = 300, 40, 6, 4
    # rank k + over: the range finder captures range(S) exactly, so the basis
    # is the SVD basis
    S = rng.standard_normal((n, k + over)) @ rng.standard_normal((k + over, K))
    P = su.prolongation_randomized(S, k, over, 0, rng.standard_normal((K, k + over)))
    U, _ = su.prolongation(S, k)
    assert np.allclose(P.T @ P, np.eye(k), atol=1e-12)
    assert _projector_dist(P, U) < 1e-8
    # full-rank samples with a gap after k: power iterations approach the SVD
    p = gen.iid_diffusion_2d(N=16, k=8, K=32, seed=2)
    A = op.assemble(p)
    S = su.smooth_samples(A, p.S0, p.omega, p.s1)
    U, sig = su.prolongation(S, p.k)
    Om = rng.standard_normal((p.K, p.k + 4))
    d = [_projector_dist(su.prolongation_randomized(S, p.k, 4, q, Om), U) for q in (0, 1, 3, 6, 10)]
    assert all(b < a for a, b in zip(d, d[1:]))
    assert d[-1] < 1e-8
