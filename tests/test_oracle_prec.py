"""Pins for oracle.prec (Algorithm 1 apply; Appendix, Two-Level Subspace
Correction)."""
import math

import numpy as np
import pytest

from oracle import operator as op, prec, setup as su
from paper_2601_20174_gb300 import inputs as gen


def _setup(N=8, k=10, K=32, seed=0, kind="iid"):
    p = gen.iid_diffusion_2d(N=N, k=k, K=K, seed=seed) if kind == "iid" else gen.poisson_2d(N, k, K, seed)
    A = op.assemble(p)
    st = su.build(A, p.S0, k, p.omega, p.s1)
    return p, A, st


def test_coarse_correction_annihilates_range_P():
    p, A, st = _setup()
    Ec = prec.coarse_error_propagator(A, st["P"])
    y = np.random.default_rng(0).standard_normal(p.k)
    assert np.linalg.norm(Ec @ (st["P"] @ y)) < 1e-10 * np.linalg.norm(y)


def test_coarse_correction_is_A_norm_best_approximation():
    p, A, st = _setup(seed=1)
    P = st["P"]
    Ad = A.toarray()
    Ec = prec.coarse_error_propagator(A, P)
    e = np.random.default_rng(1).standard_normal(p.n)
    # independent route: least squares in the A^(1/2)-transformed space
    w, V = np.linalg.eigh(Ad)
    Ah = V @ np.diag(np.sqrt(w)) @ V.T
    y, *_ = np.linalg.lstsq(Ah @ P, Ah @ e, rcond=None)
    best = np.linalg.norm(Ah @ (e - P @ y))
    got = math.sqrt((Ec @ e) @ Ad @ (Ec @ e))
    assert math.isclose(got, best, rel_tol=1e-9)


def test_residual_orthogonal_to_range_P_after_coarse_correction():
    p, A, st = _setup(seed=2)
    b = p.f[:, 0]
    z = prec.apply(A, st["P"], st["L"], b, p.omega, 2, 0)  # stop right after z += P e_c
    res = st["P"].T @ (b - A @ z)
    assert np.linalg.norm(res) < 1e-10 * np.linalg.norm(st["P"].T @ b)


def test_B_symmetric_positive_definite():
    p, A, st = _setup(N=7, seed=3)
    B = prec.apply(A, st["P"], st["L"], np.eye(p.n), p.omega, 2, 2)
    assert np.linalg.norm(B - B.T) < 1e-12 * np.linalg.norm(B)
    assert np.linalg.eigvalsh(0.5 * (B + B.T)).min() > 0
    Bn = prec.apply(A, st["P"], st["L"], np.eye(p.n), p.omega, 2, 1)
    assert np.linalg.norm(Bn - Bn.T) > 1e-6 * np.linalg.norm(Bn)  # nu1 != nu2 is not symmetric


def test_full_rank_coarse_space_gives_inverse():
    p, A, _ = _setup(N=6, k=36, K=36)
    P = np.eye(p.n)
    L = su.coarse_factor(su.galerkin(A, P))
    b = p.f[:, 0]
    z = prec.apply(A, P, L, b, p.omega, 2, 2)
    assert np.allclose(z, np.linalg.solve(A.toarray(), b), rtol=1e-10, atol=1e-14)


def test_poisson_sine_basis_closed_form_action():
    # P = a set of normalised sine modes of the Poisson operator: then
    # I - BA = S^nu E_c S^nu is diagonal in the sine basis, with factor 0 on
    # range(P) and (1 - w mu)^(2 nu) elsewhere, so B v = beta v with
    # beta = 1/lambda (in P) or (1 - (1 - w mu)^(2nu))/lambda (outside).
    N, w, nu = 10, 2.0 / 3.0, 2
    h = 1.0 / (N + 1)
    A = op.diffusion_5pt(N, np.ones((N + 1, N + 1)))
    x = (np.arange(N) + 1) * h
    modes = {}
    for p in range(1, N + 1):
        for q in range(1, N + 1):
            v = np.outer(np.sin(q * math.pi * x), np.sin(p * math.pi * x)).ravel()
            mu = math.sin(p * math.pi * h / 2) ** 2 + math.sin(q * math.pi * h / 2) ** 2
            modes[(p, q)] = (v / np.linalg.norm(v), mu, 4 * mu / h ** 2)
    chosen = [(1, 1), (1, 2), (2, 1), (3, 5), (7, 2)]
    P = np.stack([modes[c][0] for c in chosen], axis=1)
    L = su.coarse_factor(su.galerkin(A, P))
    for key in [(1, 1), (3, 5), (2, 2), (4, 6), (10, 10)]:
        v, mu, lam = modes[key]
        beta = 1 / lam if key in chosen else (1 - (1 - w * mu) ** (2 * nu)) / lam
        z = prec.apply(A, P, L, v, w, nu, nu)
        assert np.allclose(z, beta * v, rtol=0, atol=1e-12 * abs(beta))


def test_block_apply_equals_columnwise():
    p, A, st = _setup(seed=4)
    Bm = np.random.default_rng(4).standard_normal((p.n, 3))
    Z = prec.apply(A, st["P"], st["L"], Bm, p.omega, 2, 2)
    for j in range(3):
        assert np.allclose(Z[:, j], prec.apply(A, st["P"], st["L"], Bm[:, j], p.omega, 2, 2), atol=1e-14)
