"""GPU tests of the block PCG (nlsp_solve_block): m <= 32 right-hand sides
advanced together with one preconditioner application per iteration for all
columns.

Each column runs its own PCG recurrence, so it must reproduce what a
single-column solve gives: for the FP64 path the oracle's iterations (+-1,
the block sums are added in another order) and its solution (1e-8); for
both paths the FP64 true relative residual (oracle operator) below the
tolerance and the iteration count of the library's single-column solve
(+-1 FP64, +-2 mixed).  Edge cases: a zero column, a scaled column, maxit,
more than 32 columns rejected."""
import numpy as np
import pytest
import torch

from helpers import rel, to_dev, to_np
from oracle import operator as op, pcg as opcg
from paper_2601_20174_gb300 import inputs as gen

pytestmark = pytest.mark.gpu

FP64, MIXED = 0, 1


@pytest.fixture(scope="module")
def ctx():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2601_20174_gb300 import api
    return api.Context(0)


def _api():
    from paper_2601_20174_gb300 import api
    return api


CASES = {
    "poisson5": lambda: gen.poisson_2d(37, 8, 24, seed=1),
    "grf5": lambda: gen.grf_diffusion_2d(N=45, k=12, K=32, seed=2),
    "aniso9": lambda: gen.aniso_9pt_2d(N=29, k=10, K=24, m=1, seed=3),
    "iid3d": lambda: gen.iid_diffusion_3d(N=11, k=10, K=24, seed=4),
}


@pytest.mark.parametrize("name", list(CASES))
def test_block_matches_oracle_and_single_column(ctx, name):
    api = _api()
    p = CASES[name]()
    p.tol = 1e-8
    A = op.assemble(p)
    B = gen.rhs_uniform(p.n, 5, seed=11)
    Aop = api.Operator.from_problem(ctx, p)
    for precision in (FP64, MIXED):
        M = api.Preconditioner.build(Aop, to_dev(p.S0), p.k, p.s1, p.nu, p.omega, precision)
        X, res = M.solve_block(to_dev(B), tol=p.tol)
        X = to_np(X)
        X1, res1 = M.solve(to_dev(B), tol=p.tol, graph_mode=1)
        X1 = to_np(X1)
        for c in range(B.shape[1]):
            true = np.linalg.norm(B[:, c] - A @ X[:, c]) / np.linalg.norm(B[:, c])
            assert res[c].status == 0 and true <= p.tol * 1.01, (precision, c, res[c], true)
            assert abs(res[c].true_relres - true) <= 1e-3 * true
            assert abs(res[c].iterations - res1[c].iterations) <= (1 if precision == FP64 else 2)
            assert rel(X[:, c], X1[:, c]) <= 1e-6
        if precision == FP64:
            P = to_np(M.basis())
            import scipy.linalg as sla
            Lc = sla.cholesky(P.T @ (A @ P), lower=True)
            apply_B = opcg.two_level_solver(A, P, Lc, p.omega, p.nu, p.nu)
            for c in range(B.shape[1]):
                o = opcg.pcg(A, apply_B, B[:, c], p.tol)
                assert abs(res[c].iterations - o["iters"]) <= 1
                assert rel(X[:, c], o["x"]) <= 1e-8


def test_block_32_columns_zero_and_scaled(ctx):
    api = _api()
    p = CASES["grf5"]()
    A = op.assemble(p)
    B = gen.rhs_uniform(p.n, 32, seed=12)
    B[:, 3] = 0.0
    B[:, 7] = 4.0 * B[:, 5]
    Aop = api.Operator.from_problem(ctx, p)
    M = api.Preconditioner.build(Aop, to_dev(p.S0), p.k, p.s1, p.nu, p.omega, FP64)
    X, res = M.solve_block(to_dev(B), tol=1e-9)
    X = to_np(X)
    assert res[3].iterations == 0 and res[3].status == 0 and np.all(X[:, 3] == 0)
    assert res[7].iterations == res[5].iterations
    assert rel(X[:, 7], 4.0 * X[:, 5]) <= 1e-10
    for c in range(32):
        if c == 3:
            continue
        true = np.linalg.norm(B[:, c] - A @ X[:, c]) / np.linalg.norm(B[:, c])
        assert res[c].status == 0 and true <= 1e-9 * 1.01


def test_block_maxit_and_too_many_columns(ctx):
    api = _api()
    p = CASES["grf5"]()
    Aop = api.Operator.from_problem(ctx, p)
    M = api.Preconditioner.build(Aop, to_dev(p.S0), 2, p.s1, p.nu, p.omega, FP64)
    B = gen.rhs_uniform(p.n, 3, seed=13)
    X, res = M.solve_block(to_dev(B), tol=1e-14, maxit=3)
    assert all(r.status == 1 and r.iterations == 3 for r in res)
    with pytest.raises(api.L.NlspError):
        M.solve_block(to_dev(gen.rhs_uniform(p.n, 33, seed=14)))


@pytest.mark.parametrize("tc_mode", ["0", "2"])
def test_block_tensor_core_modes_agree(ctx, tc_mode, monkeypatch):
    # CUDA-core contractions (0) and both contractions on tensor cores (2)
    # against the default (tensor-core restriction): same iterations to +-1
    api = _api()
    p = CASES["aniso9"]()
    A = op.assemble(p)
    B = gen.rhs_uniform(p.n, 8, seed=21)
    Aop = api.Operator.from_problem(ctx, p)
    M = api.Preconditioner.build(Aop, to_dev(p.S0), p.k, p.s1, p.nu, p.omega, MIXED)
    X0, r0 = M.solve_block(to_dev(B), tol=1e-8)
    monkeypatch.setenv("NLSP_BLOCK_TC", tc_mode)
    X1, r1 = M.solve_block(to_dev(B), tol=1e-8)
    for c in range(B.shape[1]):
        true = np.linalg.norm(B[:, c] - A @ to_np(X1)[:, c]) / np.linalg.norm(B[:, c])
        assert r1[c].status == 0 and true <= 1e-8 * 1.01
        assert abs(r1[c].iterations - r0[c].iterations) <= 1


def test_block_anisotropic_256_mixed(ctx):
    # 9-point rotated anisotropy (eps = 1e-3), k = 64, 32 right-hand sides
    api = _api()
    p = gen.aniso_9pt_2d(N=256, k=64, K=128, m=32, seed=5, tol=1e-8)
    A = op.assemble(p)
    Aop = api.Operator.from_problem(ctx, p)
    M = api.Preconditioner.build(Aop, to_dev(p.S0), p.k, p.s1, p.nu, p.omega, MIXED)
    X, res = M.solve_block(to_dev(p.f), tol=p.tol, maxit=5000)
    X = to_np(X)
    for c in range(p.f.shape[1]):
        true = np.linalg.norm(p.f[:, c] - A @ X[:, c]) / np.linalg.norm(p.f[:, c])
        assert res[c].status == 0 and true <= 1e-8 * 1.01, (c, res[c], true)


BF16, TF32 = 2, 3


@pytest.mark.parametrize("name", list(CASES))
@pytest.mark.parametrize("precision", [BF16, TF32])
def test_block_reduced_precision_contractions(ctx, name, precision):
    # BF16 / TF32 tensor-core restriction and prolongation (FP32 accumulate):
    # after one iteration the iterate equals the FP32 path's to the operand
    # precision (a wrong operand layout would give O(1) errors), and every
    # column still reaches the FP64 true residual 1e-8 (flexible CG) within a
    # few more iterations than the FP32 preconditioner
    api = _api()
    p = CASES[name]()
    A = op.assemble(p)
    B = gen.rhs_uniform(p.n, 6, seed=31)
    Aop = api.Operator.from_problem(ctx, p)
    M32 = api.Preconditioner.build(Aop, to_dev(p.S0), p.k, p.s1, p.nu, p.omega, MIXED)
    Mlp = api.Preconditioner.build(Aop, to_dev(p.S0), p.k, p.s1, p.nu, p.omega, precision)
    X1, _ = M32.solve_block(to_dev(B), tol=1e-8, maxit=1)
    Y1, _ = Mlp.solve_block(to_dev(B), tol=1e-8, maxit=1)
    assert rel(to_np(Y1), to_np(X1)) <= (3e-2 if precision == BF16 else 4e-3)
    X, r32 = M32.solve_block(to_dev(B), tol=1e-8)
    Y, rlp = Mlp.solve_block(to_dev(B), tol=1e-8)
    Y = to_np(Y)
    for c in range(B.shape[1]):
        true = np.linalg.norm(B[:, c] - A @ Y[:, c]) / np.linalg.norm(B[:, c])
        assert rlp[c].status == 0 and true <= 1e-8 * 1.01, (c, rlp[c], true)
        assert rlp[c].iterations <= 1.5 * r32[c].iterations + 3, (rlp[c].iterations, r32[c].iterations)


@pytest.mark.parametrize("precision", [BF16, TF32])
def test_block_reduced_precision_anisotropic_256(ctx, precision):
    # several tiles per block, k = 64: every column of 32 converges
    api = _api()
    p = gen.aniso_9pt_2d(N=256, k=64, K=128, m=32, seed=5, tol=1e-8)
    A = op.assemble(p)
    Aop = api.Operator.from_problem(ctx, p)
    M = api.Preconditioner.build(Aop, to_dev(p.S0), p.k, p.s1, p.nu, p.omega, precision)
    X, res = M.solve_block(to_dev(p.f), tol=p.tol, maxit=5000)
    X = to_np(X)
    for c in range(p.f.shape[1]):
        true = np.linalg.norm(p.f[:, c] - A @ X[:, c]) / np.linalg.norm(p.f[:, c])
        assert res[c].status == 0 and true <= 1e-8 * 1.01, (c, res[c], true)


@pytest.mark.parametrize("name", list(CASES))
def test_block_cg_matches_oracle_block_cg(ctx, name):
    # breakdown-free block CG (shared search space): FP64 with the oracle's
    # basis reproduces the oracle's block CG (iterations per column +-1,
    # solution 1e-7); mixed precision reaches the FP64 true residual
    from oracle import setup as osetup
    api = _api()
    p = CASES[name]()
    A = op.assemble(p)
    ref = osetup.build(A, p.S0, p.k, p.omega, p.s1)
    B = gen.rhs_uniform(p.n, 6, seed=41)
    apply_B = opcg.two_level_solver(A, ref["P"], ref["L"], p.omega, p.nu, p.nu)
    Xo, its_o, true_o = opcg.block_cg(A, apply_B, B, 1e-8)
    Aop = api.Operator.from_problem(ctx, p)
    M = api.Preconditioner.from_basis(Aop, to_dev(ref["P"]), p.nu, p.omega, FP64)
    X, res = M.solve_block_cg(to_dev(B), tol=1e-8)
    X = to_np(X)
    for c in range(B.shape[1]):
        true = np.linalg.norm(B[:, c] - A @ X[:, c]) / np.linalg.norm(B[:, c])
        assert res[c].status == 0 and true <= 1e-8 * 1.01, (c, res[c], true)
        assert abs(res[c].iterations - its_o[c]) <= 1, (c, res[c].iterations, its_o[c])
        assert abs(res[c].true_relres - true) <= 1e-3 * true + 1e-14
    assert rel(X, Xo) <= 1e-7
    Mm = api.Preconditioner.build(Aop, to_dev(p.S0), p.k, p.s1, p.nu, p.omega, MIXED)
    Y, rm = Mm.solve_block_cg(to_dev(B), tol=1e-8)
    Y = to_np(Y)
    for c in range(B.shape[1]):
        true = np.linalg.norm(B[:, c] - A @ Y[:, c]) / np.linalg.norm(B[:, c])
        assert rm[c].status == 0 and true <= 1e-8 * 1.01


def test_block_cg_deflation_and_maxit(ctx):
    api = _api()
    p = CASES["grf5"]()
    A = op.assemble(p)
    Aop = api.Operator.from_problem(ctx, p)
    M = api.Preconditioner.build(Aop, to_dev(p.S0), p.k, p.s1, p.nu, p.omega, FP64)
    b, b2 = p.f[:, 0], gen.rhs_uniform(p.n, 1, seed=7)[:, 0]
    B = np.stack([b, 2.0 * b, np.zeros(p.n), b2], axis=1)
    X, res = M.solve_block_cg(to_dev(B), tol=1e-9)
    X = to_np(X)
    assert res[2].iterations == 0 and res[2].status == 0 and np.all(X[:, 2] == 0)
    assert rel(X[:, 1], 2.0 * X[:, 0]) <= 1e-8
    for c in (0, 1, 3):
        assert res[c].status == 0
        assert np.linalg.norm(B[:, c] - A @ X[:, c]) / np.linalg.norm(B[:, c]) <= 1e-9 * 1.01
    _, r3 = M.solve_block_cg(to_dev(B[:, [0, 3]]), tol=1e-14, maxit=3)
    assert all(r.status == 1 for r in r3)


def test_block_cg_fewer_iterations_than_independent_columns(ctx):
    # the shared block space: no column needs more block iterations than its
    # own PCG, on the 256^2 anisotropic 9-point problem with 16 columns
    api = _api()
    p = gen.aniso_9pt_2d(N=128, k=32, K=64, m=16, seed=5, tol=1e-8)
    A = op.assemble(p)
    Aop = api.Operator.from_problem(ctx, p)
    M = api.Preconditioner.build(Aop, to_dev(p.S0), p.k, p.s1, p.nu, p.omega, FP64)
    X, res = M.solve_block_cg(to_dev(p.f), tol=1e-8, maxit=5000)
    _, res1 = M.solve_block(to_dev(p.f), tol=1e-8, maxit=5000)
    X = to_np(X)
    for c in range(p.f.shape[1]):
        true = np.linalg.norm(p.f[:, c] - A @ X[:, c]) / np.linalg.norm(p.f[:, c])
        assert res[c].status == 0 and true <= 1e-8 * 1.01
        assert res[c].iterations <= res1[c].iterations + 1
    assert max(r.iterations for r in res) < max(r.iterations for r in res1)
