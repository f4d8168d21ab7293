"""GPU parity of the general sparse operator (nlsp_assemble_csr) against the
FP64 oracle.

The operator of Sec. 3 (Eq. discretized_pde) is any SPD matrix; the paper's
own are finite-element matrices handed over in compressed sparse rows.  Every
stencil problem of the other parity tests is exported from the oracle's
explicit CSR and solved through the sparse path: results must equal the
oracle's (same tolerances as the stencil tests) and the stencil path's.
Inputs that are not a plain sorted CSR (shuffled rows, repeated entries) and a
symmetric permutation (a sparsity pattern no stencil has) must give the same
results, and malformed inputs must be rejected on the host.
"""
import numpy as np
import pytest
import scipy.sparse as sp
import torch

from helpers import projector_dist, rel, to_dev, to_np
from oracle import operator as op, pcg as opcg, prec as oprec, setup as osetup
from paper_2601_20174_gb300 import inputs as gen

pytestmark = pytest.mark.gpu

FP64, MIXED = 0, 1


@pytest.fixture(scope="module")
def ctx():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2601_20174_gb300 import api
    c = api.Context(0)
    yield c
    torch.cuda.synchronize()


def _api():
    from paper_2601_20174_gb300 import api
    return api


PROBLEMS = {
    "poisson5": lambda: gen.poisson_2d(37, 8, 24, seed=1),
    "grf5": lambda: gen.grf_diffusion_2d(N=45, k=12, K=32, seed=2),
    "aniso9": lambda: gen.aniso_9pt_2d(N=29, k=10, K=24, m=1, seed=3),
    "iid7": lambda: gen.iid_diffusion_3d(N=11, k=10, K=24, seed=4),
}


def _csr_op(ctx, A):
    A = sp.csr_matrix(A)
    return _api().Operator.from_csr(ctx, torch.as_tensor(A.indptr.astype(np.int64)),
                                    torch.as_tensor(A.indices.astype(np.int32)), torch.as_tensor(A.data))


def _scrambled(A, seed):
    """The same matrix as an unsorted CSR with repeated entries: every row's
    entries shuffled and every third entry split into two halves."""
    A = sp.csr_matrix(A)
    rng = np.random.default_rng(seed)
    rows, cols, vals = [], [], []
    for i in range(A.shape[0]):
        c = A.indices[A.indptr[i]:A.indptr[i + 1]]
        v = A.data[A.indptr[i]:A.indptr[i + 1]]
        cc, vv = [], []
        for q, (cj, vj) in enumerate(zip(c, v)):
            if q % 3 == 0:
                cc += [cj, cj]
                vv += [0.5 * vj, vj - 0.5 * vj]
            else:
                cc.append(cj)
                vv.append(vj)
        perm = rng.permutation(len(cc))
        rows.append(len(cc))
        cols += [cc[t] for t in perm]
        vals += [vv[t] for t in perm]
    indptr = np.concatenate([[0], np.cumsum(rows)]).astype(np.int64)
    return indptr, np.asarray(cols, dtype=np.int32), np.asarray(vals, dtype=np.float64)


@pytest.mark.parametrize("name", list(PROBLEMS))
def test_csr_apply_and_diagonal(ctx, name):
    p = PROBLEMS[name]()
    A = op.assemble(p)
    Aop = _csr_op(ctx, A)
    assert Aop.n == p.n
    X = np.random.default_rng(0).standard_normal((p.n, 3))
    ref = A @ X
    assert np.max(np.abs(to_np(Aop.apply(to_dev(X))) - ref)) <= 1e-13 * np.max(np.abs(ref))
    assert np.max(np.abs(to_np(Aop.diagonal()) - A.diagonal())) <= 1e-15 * A.diagonal().max()
    # an unsorted CSR with repeated entries describes the same operator
    ip, ci, va = _scrambled(A, 1)
    As = _api().Operator.from_csr(ctx, torch.as_tensor(ip), torch.as_tensor(ci), torch.as_tensor(va))
    assert np.max(np.abs(to_np(As.apply(to_dev(X))) - ref)) <= 1e-13 * np.max(np.abs(ref))


@pytest.mark.parametrize("name", list(PROBLEMS))
@pytest.mark.parametrize("precision", [FP64, MIXED])
def test_csr_smoothing_and_apply_match_oracle(ctx, name, precision):
    p = PROBLEMS[name]()
    A = op.assemble(p)
    Aop = _csr_op(ctx, A)
    S = to_np(Aop.smooth_samples(to_dev(p.S0), p.s1, p.omega, precision))
    tol = 1e-12 if precision == FP64 else 2e-5
    assert rel(S, osetup.smooth_samples(A, p.S0, p.omega, p.s1)) <= tol
    ref = osetup.build(A, p.S0, p.k, p.omega, p.s1)
    M = _api().Preconditioner.from_basis(Aop, to_dev(ref["P"]), p.nu, p.omega, precision)
    R = np.random.default_rng(5).standard_normal((p.n, 2))
    Zref = oprec.apply(A, ref["P"], ref["L"], R, p.omega, p.nu, p.nu)
    assert rel(to_np(M.apply(to_dev(R))), Zref) <= (1e-12 if precision == FP64 else 1e-4)


@pytest.mark.parametrize("name", list(PROBLEMS))
def test_csr_setup_fp64_matches_oracle(ctx, name):
    p = PROBLEMS[name]()
    A = op.assemble(p)
    ref = osetup.build(A, p.S0, p.k, p.omega, p.s1)
    M = _api().Preconditioner.build(_csr_op(ctx, A), to_dev(p.S0), p.k, p.s1, p.nu, p.omega, FP64)
    P, sig = to_np(M.basis()), to_np(M.sigma())
    s_ref = ref["sigma"][: p.k + 1]
    assert np.all(np.abs(sig[: p.k + 1] - s_ref) <= 1e-9 * s_ref + 1e-13 * s_ref[0] ** 2 / s_ref)
    gap = (s_ref[p.k - 1] ** 2 - s_ref[p.k] ** 2) / s_ref[0] ** 2
    assert projector_dist(P, ref["P"]) <= max(1e-8, 1e-13 / gap)
    Ac, _ = (to_np(t) for t in M.coarse())
    Ac_ref = osetup.galerkin(A, P)
    assert np.max(np.abs(Ac - Ac_ref)) <= 1e-12 * np.max(np.abs(Ac_ref))


@pytest.mark.parametrize("name", list(PROBLEMS))
@pytest.mark.parametrize("graph_mode", [0, 1, 2])
def test_csr_pcg_fp64_matches_oracle_and_stencil(ctx, name, graph_mode):
    p = PROBLEMS[name]()
    A = op.assemble(p)
    ref = osetup.build(A, p.S0, p.k, p.omega, p.s1)
    b = p.f[:, 0]
    o = opcg.pcg(A, opcg.two_level_solver(A, ref["P"], ref["L"], p.omega, p.nu, p.nu), b, p.tol)
    M = _api().Preconditioner.from_basis(_csr_op(ctx, A), to_dev(ref["P"]), p.nu, p.omega, FP64)
    x, res = M.solve(to_dev(b), tol=p.tol, graph_mode=graph_mode)
    assert res[0].status == 0
    assert abs(res[0].iterations - o["iters"]) <= 1
    assert rel(to_np(x), o["x"]) <= 1e-8
    Ms = _api().Preconditioner.from_basis(_api().Operator.from_problem(ctx, p), to_dev(ref["P"]), p.nu, p.omega,
                                          FP64)
    xs, rs = Ms.solve(to_dev(b), tol=p.tol, graph_mode=graph_mode)
    assert abs(res[0].iterations - rs[0].iterations) <= 1
    assert rel(to_np(x), to_np(xs)) <= 1e-8


@pytest.mark.parametrize("name", list(PROBLEMS))
@pytest.mark.parametrize("graph_mode", [1, 2])
def test_csr_pcg_end_to_end_both_precisions(ctx, name, graph_mode):
    p = PROBLEMS[name]()
    A = op.assemble(p)
    o = opcg.solve_problem(p, A=A)
    Aop = _csr_op(ctx, A)
    b = p.f[:, 0]
    for precision in (FP64, MIXED):
        M = _api().Preconditioner.build(Aop, to_dev(p.S0), p.k, p.s1, p.nu, p.omega, precision)
        x, res = M.solve(to_dev(b), tol=1e-8, graph_mode=graph_mode)
        true = np.linalg.norm(b - A @ to_np(x)) / np.linalg.norm(b)
        assert res[0].status == 0 and true <= 1e-8 * 1.01
        if precision == FP64 and p.tol == 1e-8:
            assert abs(res[0].iterations - o["results"][0]["iters"]) <= 1


def test_csr_symmetric_permutation(ctx):
    # a symmetric permutation scatters every row's neighbours across the
    # whole index range: P^T A P solved with the permuted basis must give the
    # permuted solution of the oracle (FP64), and reach 1e-8 mixed
    p = gen.grf_diffusion_2d(N=60, k=16, K=32, seed=8, tol=1e-8)
    A = op.assemble(p)
    perm = np.random.default_rng(3).permutation(p.n)
    Ap = sp.csr_matrix(A[perm][:, perm])
    ref = osetup.build(A, p.S0, p.k, p.omega, p.s1)
    b = p.f[:, 0]
    o = opcg.pcg(A, opcg.two_level_solver(A, ref["P"], ref["L"], p.omega, p.nu, p.nu), b, p.tol)
    Aop = _csr_op(ctx, Ap)
    M = _api().Preconditioner.from_basis(Aop, to_dev(ref["P"][perm]), p.nu, p.omega, FP64)
    for graph_mode in (1, 2):
        x, res = M.solve(to_dev(b[perm]), tol=p.tol, graph_mode=graph_mode)
        assert res[0].status == 0 and abs(res[0].iterations - o["iters"]) <= 1
        assert rel(to_np(x), o["x"][perm]) <= 1e-8
    Mm = _api().Preconditioner.build(Aop, to_dev(p.S0[perm]), p.k, p.s1, p.nu, p.omega, MIXED)
    x, res = Mm.solve(to_dev(b[perm]), tol=1e-8, graph_mode=2)
    assert res[0].status == 0
    assert np.linalg.norm(b[perm] - Ap @ to_np(x)) / np.linalg.norm(b) <= 1e-8 * 1.01


def test_csr_block_batched_and_unrolled(ctx):
    from oracle import losses as olosses
    api = _api()
    p = PROBLEMS["grf5"]()
    A = op.assemble(p)
    ref = osetup.build(A, p.S0, p.k, p.omega, p.s1)
    Aop = _csr_op(ctx, A)
    # block PCG, FP64, oracle basis: each column reproduces the oracle's PCG
    B = p.f[:, 0][:, None] * np.array([1.0, -2.0]) + np.random.default_rng(4).standard_normal((p.n, 2))
    M = api.Preconditioner.from_basis(Aop, to_dev(ref["P"]), p.nu, p.omega, FP64)
    X, res = M.solve_block(to_dev(B), tol=1e-8)
    for j in range(2):
        o = opcg.pcg(A, opcg.two_level_solver(A, ref["P"], ref["L"], p.omega, p.nu, p.nu), B[:, j], 1e-8)
        assert res[j].status == 0 and abs(res[j].iterations - o["iters"]) <= 1
        assert rel(to_np(X)[:, j], o["x"]) <= 1e-8
    # batched: two sparse instances in one launch, FP64 with oracle bases
    q = gen.iid_diffusion_2d(30, 8, 16, seed=9, tol=1e-8)
    Aq = op.assemble(q)
    refq = osetup.build(Aq, q.S0, q.k, q.omega, q.s1)
    Mp = api.Preconditioner.from_basis(_csr_op(ctx, A), to_dev(ref["P"]), p.nu, p.omega, FP64)
    Mq = api.Preconditioner.from_basis(_csr_op(ctx, Aq), to_dev(refq["P"]), q.nu, q.omega, FP64)
    xs, rs = api.solve_batched([Mp, Mq], [to_dev(p.f[:, 0]), to_dev(q.f[:, 0])], tol=1e-8, tiles_per_cta=2)
    for (AA, su, f), x, r in zip([(A, ref, p.f[:, 0]), (Aq, refq, q.f[:, 0])], xs, rs):
        o = opcg.pcg(AA, opcg.two_level_solver(AA, su["P"], su["L"], p.omega, p.nu, p.nu), f, 1e-8)
        assert r.status == 0 and abs(r.iterations - o["iters"]) <= 1
        assert rel(to_np(x), o["x"]) <= 1e-8
    # unrolled PCG loss and gradient through the sparse operator
    P = ref["P"] + 0.05 * np.random.default_rng(6).standard_normal(ref["P"].shape)
    b = p.f[:, 0]
    L64, g64 = api.unrolled_pcg(Aop, to_dev(P), to_dev(b), 10, p.nu, p.omega, FP64)
    assert abs(L64 - olosses.unrolled_pcg_loss(A, P, b, 10, p.omega, p.nu)) <= 1e-10 * L64
    assert rel(to_np(g64), olosses.grad_unrolled_pcg_loss(A, P, b, 10, p.omega, p.nu)) <= 1e-7


def test_csr_rejects_malformed_input(ctx):
    api = _api()
    A = sp.csr_matrix(op.assemble(gen.poisson_2d(6, 2, 4, seed=0)))
    ip, ci, va = A.indptr.astype(np.int64), A.indices.astype(np.int32), A.data.copy()

    def build(ip_, ci_, va_):
        return api.Operator.from_csr(ctx, torch.as_tensor(ip_), torch.as_tensor(ci_), torch.as_tensor(va_))

    bad_col = ci.copy()
    bad_col[5] = A.shape[0]  # column out of range
    no_diag = va.copy()
    no_diag[A.indptr[3] + list(A.indices[A.indptr[3]:A.indptr[4]]).index(3)] = 0.0  # zero diagonal
    bad_ptr = ip.copy()
    bad_ptr[4], bad_ptr[5] = bad_ptr[5], bad_ptr[4]  # not monotone
    nan_val = va.copy()
    nan_val[7] = np.nan
    for args, word in (((ip, bad_col, va), "column"), ((ip, ci, no_diag), "diagonal"), ((bad_ptr, ci, va), "row"),
                       ((ip, ci, nan_val), "non-finite")):
        with pytest.raises(api.L.NlspError):
            build(*args)
        assert word in ctx._lib.nlsp_last_error().decode()
    build(ip, ci, va)  # the unmodified matrix is accepted
