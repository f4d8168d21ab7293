"""Pins for oracle.pcg (Sec. 4 two-grid PCG)."""
import math

import numpy as np
import pytest

from oracle import operator as op, pcg, prec, setup as su
from paper_2601_20174_gb300 import inputs as gen


@pytest.mark.parametrize("N", [3, 4, 5])
def test_tiny_grids_exact_solution(N):
    p = gen.iid_diffusion_2d(N=N, k=min(4, N * N), K=8, seed=N, tol=1e-14)
    out = pcg.solve_problem(p)
    x_ref = np.linalg.solve(out["A"].toarray(), p.f[:, 0])
    assert out["results"][0]["status"] == "converged"
    assert np.linalg.norm(out["X"][:, 0] - x_ref) <= 1e-12 * np.linalg.norm(x_ref)


def test_full_rank_coarse_space_converges_in_one_iteration():
    p = gen.iid_diffusion_2d(N=6, k=36, K=36, seed=1, tol=1e-12)
    A = op.assemble(p)
    P = np.eye(p.n)
    L = su.coarse_factor(su.galerkin(A, P))
    res = pcg.pcg(A, pcg.two_level_solver(A, P, L, p.omega, 2, 2), p.f[:, 0], 1e-12)
    assert res["iters"] == 1 and res["status"] == "converged"


def test_iterations_within_cg_bound():
    # CG bound: ||e_m||_A <= 2 ((sqrt(kappa)-1)/(sqrt(kappa)+1))^m ||e_0||_A, so
    # m <= ceil(sqrt(kappa)/2 ln(2/eps)) iterations reduce the A-norm error by eps;
    # the residual 2-norm differs by at most sqrt(kappa(A)), folded into eps.
    p = gen.poisson_2d(16, 8, 32, tol=1e-8)
    A = op.assemble(p)
    st = su.build(A, p.S0, p.k, p.omega, p.s1)
    B = prec.apply(A, st["P"], st["L"], np.eye(p.n), p.omega, 2, 2)
    lam = np.sort(np.linalg.eigvals(B @ A.toarray()).real)
    kap_BA = lam[-1] / lam[0]
    kap_A = np.linalg.cond(A.toarray())
    eps = p.tol / math.sqrt(kap_A)
    bound = math.ceil(math.sqrt(kap_BA) / 2 * math.log(2 / eps))
    res = pcg.pcg(A, pcg.two_level_solver(A, st["P"], st["L"], p.omega, 2, 2), p.f[:, 0], p.tol)
    assert res["status"] == "converged" and res["iters"] <= bound


def test_iterations_bounded_at_fixed_n_over_k():
    # kappa(BA) ~ n / (2 nu w pi k) for Poisson with the smooth coarse space,
    # so a fixed n/k keeps iteration counts flat under refinement ...
    its = []
    for N in (16, 32, 64):
        k = N * N // 16
        p = gen.poisson_2d(N, k, 2 * k, tol=1e-8)
        its.append(pcg.solve_problem(p)["results"][0]["iters"])
    assert max(its) - min(its) <= 2, its


def test_iterations_grow_like_sqrt_n_at_fixed_k():
    # ... while a fixed k lets them grow like sqrt(n): x2 per halving of h.
    its = []
    for N in (32, 64):
        p = gen.poisson_2d(N, 8, 16, tol=1e-8)
        its.append(pcg.solve_problem(p)["results"][0]["iters"])
    ratio = its[1] / its[0]
    assert 1.6 <= ratio <= 2.6, its


def test_flexible_equals_standard_for_exact_preconditioner():
    p = gen.iid_diffusion_2d(N=12, k=8, K=16, seed=7, tol=1e-9)
    a = pcg.solve_problem(p)
    b = pcg.solve_problem(p, A=a["A"], setup=a["setup"], flexible=True)
    assert abs(a["results"][0]["iters"] - b["results"][0]["iters"]) <= 1
    assert np.linalg.norm(a["X"] - b["X"]) <= 1e-7 * np.linalg.norm(a["X"])


def test_multi_rhs_columns_independent_and_zero_rhs():
    p = gen.iid_diffusion_2d(N=10, k=6, K=12, seed=8, tol=1e-9)
    A = op.assemble(p)
    st = su.build(A, p.S0, p.k, p.omega, p.s1)
    Bm = np.stack([p.f[:, 0], np.zeros(p.n), 2.0 * p.f[:, 0]], axis=1)
    X, res = pcg.pcg_multi(A, pcg.two_level_solver(A, st["P"], st["L"], p.omega, 2, 2), Bm, p.tol)
    assert res[1]["iters"] == 0 and np.all(X[:, 1] == 0)
    assert res[0]["iters"] == res[2]["iters"]
    assert np.allclose(X[:, 2], 2 * X[:, 0], rtol=1e-12, atol=1e-15)


def test_breakdown_on_indefinite_operator():
    p = gen.iid_diffusion_2d(N=6, k=4, K=8, seed=9)
    A = op.assemble(p)
    st = su.build(A, p.S0, p.k, p.omega, p.s1)
    res = pcg.pcg(-A, pcg.two_level_solver(A, st["P"], st["L"], p.omega, 2, 2), p.f[:, 0], 1e-8)
    assert res["status"] == "breakdown"


def _grf_setup():
    from oracle import operator as op, setup as su
    p = gen.grf_diffusion_2d(N=24, k=8, K=20, seed=31)
    A = op.assemble(p)
    st = su.build(A, p.S0, p.k, p.omega, p.s1)
    return p, A, pcg.two_level_solver(A, st["P"], st["L"], p.omega, p.nu, p.nu)


def test_block_cg_one_column_is_pcg():
    p, A, apply_B = _grf_setup()
    b = p.f[:, 0]
    o = pcg.pcg(A, apply_B, b, 1e-10)
    X, its, true = pcg.block_cg(A, apply_B, b[:, None], 1e-10)
    assert its[0] == o["iters"]
    assert np.linalg.norm(X[:, 0] - o["x"]) <= 1e-10 * np.linalg.norm(o["x"])


def test_block_cg_needs_no_more_iterations_than_each_column():
    p, A, apply_B = _grf_setup()
    Bm = gen.rhs_uniform(p.n, 6, seed=5)
    X, its, true = pcg.block_cg(A, apply_B, Bm, 1e-8)
    single = [pcg.pcg(A, apply_B, Bm[:, c], 1e-8)["iters"] for c in range(6)]
    assert np.all(true <= 1e-8 * 1.01)
    assert max(its) <= max(single) and np.all(its <= np.array(single))
    assert max(its) < max(single)  # the shared space helps on this problem


def test_block_cg_deflates_dependent_and_zero_columns():
    p, A, apply_B = _grf_setup()
    b, b2 = p.f[:, 0], gen.rhs_uniform(p.n, 1, seed=7)[:, 0]
    Bm = np.stack([b, 2.0 * b, np.zeros(p.n), b2], axis=1)
    X, its, true = pcg.block_cg(A, apply_B, Bm, 1e-9)
    assert its[2] == 0 and np.all(X[:, 2] == 0)
    assert np.linalg.norm(X[:, 1] - 2.0 * X[:, 0]) <= 1e-9 * np.linalg.norm(X[:, 1])
    assert np.all(true[[0, 1, 3]] <= 1e-9 * 1.01)


def test_block_cg_exact_on_tiny_grid():
    from oracle import operator as op
    p = gen.poisson_2d(4, 4, 8, seed=2)
    A = op.assemble(p)
    Bm = gen.rhs_uniform(p.n, 3, seed=3)
    ident = lambda R: R.copy()  # no preconditioner: plain block CG
    X, its, true = pcg.block_cg(A, ident, Bm, 1e-12, maxit=50)
    ref = np.linalg.solve(A.toarray(), Bm)
    assert np.max(np.abs(X - ref)) <= 1e-10 * np.max(np.abs(ref))
    assert max(its) <= p.n // 3 + 2  # block Krylov: about n / m steps in exact arithmetic
