"""GPU tests of the differentiation entry points against the oracle.

Subspace loss (Sec. 3 "P = qf(P_hat)", Appendix optimality): loss and
gradient against oracle.losses (FP64 autograd of the definition).  Unrolled
PCG loss ||r_T||: loss and gradient dL/dP against the oracle's dense
autograd restatement on small grids.  At larger sizes, where the oracle's
dense autograd is out of reach, by what holds at any size: central finite
differences of the GPU's own FP64 loss along random directions, and the
invariance P^T grad = 0 of losses that depend on range(P) only.

Tolerances: FP64 loss to 1e-10 relative, gradients to 1e-8 (subspace; a
handful of k x k solves) and 1e-7 (ten unrolled iterations with their
reverse sweep); the FP32 production arithmetic against the FP64 result to
the FP32 level of the products (1e-3).
"""
import numpy as np
import pytest
import torch

from helpers import rel, to_dev, to_np
from oracle import losses as olosses, operator as op, setup as osetup
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


def _noisy_basis(p, A, scale=0.1):
    """The problem's SVD basis U_k plus seeded N(0, scale^2) noise."""
    S = osetup.smooth_samples(A, p.S0, p.omega, p.s1)
    U = np.linalg.svd(S, full_matrices=False)[0][:, : p.k]
    noise = gen.normal(p.seed, gen.STREAM_NOISE, p.n * p.k).reshape(p.k, p.n).T
    return S, U, U + scale * noise


SUB_CASES = {
    "grf45_k12": lambda: gen.grf_diffusion_2d(N=45, k=12, K=32, seed=2),
    "iid3d_k10": lambda: gen.iid_diffusion_3d(N=11, k=10, K=24, seed=4),
}


@pytest.mark.parametrize("name", list(SUB_CASES))
def test_subspace_loss_and_gradient_match_oracle(ctx, name):
    api = _api()
    p = SUB_CASES[name]()
    A = op.assemble(p)
    S, U, Ph = _noisy_basis(p, A)
    L_ref = olosses.subspace_loss(Ph, S)
    g_ref = olosses.grad_subspace_loss(Ph, S)
    L64, g64 = api.subspace_loss(ctx, to_dev(Ph), to_dev(S), FP64)
    assert abs(L64 - L_ref) <= 1e-10 * abs(L_ref)
    g64 = to_np(g64)
    assert rel(g64, g_ref) <= 1e-8
    # depends on range(P_hat) only
    assert np.linalg.norm(Ph.T @ g64) <= 1e-9 * np.linalg.norm(Ph) * np.linalg.norm(g64)
    L32, g32 = api.subspace_loss(ctx, to_dev(Ph), to_dev(S), MIXED)
    assert abs(L32 - L_ref) <= 1e-3 * abs(L_ref)
    assert rel(to_np(g32), g_ref) <= 1e-3
    # stationary at the SVD basis: the gradient vanishes to rounding
    L0, g0 = api.subspace_loss(ctx, to_dev(U), to_dev(S), FP64)
    sig = np.linalg.svd(S, compute_uv=False)
    assert abs(L0 - np.sum(sig[p.k:] ** 2)) <= 1e-9 * np.sum(sig ** 2)
    assert np.linalg.norm(to_np(g0)) <= 1e-8 * np.linalg.norm(g64)


@pytest.mark.parametrize("name", list(SUB_CASES))
def test_nlss_loss_and_gradient_match_oracle(ctx, name):
    api = _api()
    p = SUB_CASES[name]()
    A = op.assemble(p)
    S, U, Ph = _noisy_basis(p, A)
    L_ref = olosses.nlss_loss(Ph, S)
    g_ref = olosses.grad_nlss_loss(Ph, S)
    L64, g64 = api.nlss_loss(ctx, to_dev(Ph), to_dev(S), FP64)
    assert abs(L64 - L_ref) <= 1e-10 * abs(L_ref)
    g64 = to_np(g64)
    assert rel(g64, g_ref) <= 1e-8
    # not range-only: reordering the columns of P_hat changes the loss
    L_rev, _ = api.nlss_loss(ctx, to_dev(Ph[:, ::-1].copy()), to_dev(S), FP64, grad=False)
    assert abs(L_rev - olosses.nlss_loss(Ph[:, ::-1], S)) <= 1e-10 * abs(L_rev)
    assert abs(L_rev - L64) > 1e-6 * abs(L64)
    L32, g32 = api.nlss_loss(ctx, to_dev(Ph), to_dev(S), MIXED)
    assert abs(L32 - L_ref) <= 1e-3 * abs(L_ref)
    assert rel(to_np(g32), g_ref) <= 1e-3
    # the ordered SVD basis attains the closed-form minimum (Thm. 1 / Cor. 2),
    # where the gradient vanishes to rounding
    L0, g0 = api.nlss_loss(ctx, to_dev(U), to_dev(S), FP64)
    sig2 = np.linalg.svd(S, compute_uv=False) ** 2
    L_min = np.mean(1.0 - np.cumsum(sig2[: p.k]) / np.sum(sig2))
    assert abs(L0 - L_min) <= 1e-10
    assert np.linalg.norm(to_np(g0)) <= 1e-7 * np.linalg.norm(g64)


UNROLL_CASES = {
    "poisson16": lambda: gen.poisson_2d(16, 6, 16, seed=1),
    "grf20": lambda: gen.grf_diffusion_2d(N=20, k=8, K=20, seed=3),
    "aniso9_15": lambda: gen.aniso_9pt_2d(N=15, k=6, K=16, m=1, seed=5),
    "iid3d_8": lambda: gen.iid_diffusion_3d(N=8, k=6, K=16, seed=6),
}


@pytest.mark.parametrize("name", list(UNROLL_CASES))
def test_unrolled_pcg_loss_and_gradient_match_oracle(ctx, name):
    api = _api()
    p = UNROLL_CASES[name]()
    A = op.assemble(p)
    _, _, P = _noisy_basis(p, A, scale=0.05)
    b = p.f[:, 0]
    T = 10
    L_ref = olosses.unrolled_pcg_loss(A, P, b, T, p.omega, p.nu)
    g_ref = olosses.grad_unrolled_pcg_loss(A, P, b, T, p.omega, p.nu)
    Aop = api.Operator.from_problem(ctx, p)
    L64, g64 = api.unrolled_pcg(Aop, to_dev(P), to_dev(b), T, p.nu, p.omega, FP64)
    assert abs(L64 - L_ref) <= 1e-10 * abs(L_ref), (L64, L_ref)
    g64 = to_np(g64)
    assert rel(g64, g_ref) <= 1e-7
    assert np.linalg.norm(P.T @ g64) <= 1e-7 * np.linalg.norm(P) * np.linalg.norm(g64)
    L32, g32 = api.unrolled_pcg(Aop, to_dev(P), to_dev(b), T, p.nu, p.omega, MIXED)
    assert abs(L32 - L64) <= 1e-3 * L64
    assert rel(to_np(g32), g64) <= 1e-2
    # forward only
    L_only, g_none = api.unrolled_pcg(Aop, to_dev(P), to_dev(b), T, p.nu, p.omega, FP64, grad=False)
    assert g_none is None and L_only == L64


def _fd_check(loss_fn, P, g, seed, t=1e-3, ndir=3):
    """Largest relative disagreement of <g, V> with the fourth-order central
    difference (f(-2t) - 8 f(-t) + 8 f(t) - f(2t)) / (12 t) of the loss at one
    fixed step t, over ndir seeded unit-norm random directions V.  The
    fourth-order stencil keeps the truncation error (O(t^4)) and the rounding
    error (O(eps L / t)) both far below the 1e-6 gate at this step."""
    worst = 0.0
    for j in range(ndir):
        V = gen.normal(seed + 1000 * j, gen.STREAM_DIRECTION, P.size).reshape(P.shape[1], P.shape[0]).T
        V /= np.linalg.norm(V)
        d = float(np.sum(g * V))
        fd = (loss_fn(P - 2 * t * V) - 8 * loss_fn(P - t * V) + 8 * loss_fn(P + t * V) - loss_fn(P + 2 * t * V)) \
            / (12 * t)
        worst = max(worst, abs(fd - d) / max(abs(d), 1e-300))
    return worst


def test_unrolled_pcg_gradient_finite_differences_3d(ctx):
    # 3D 7-point, n = 24^3, beyond the oracle's dense autograd
    api = _api()
    p = gen.iid_diffusion_3d(N=24, k=16, K=32, seed=7, with_samples=False)
    Aop = api.Operator.from_problem(ctx, p)
    Q = np.linalg.qr(gen.normal(11, gen.STREAM_NOISE, p.n * p.k).reshape(p.k, p.n).T)[0]
    b = to_dev(p.f[:, 0])
    loss = lambda X: api.unrolled_pcg(Aop, to_dev(X), b, 10, 2, p.omega, FP64, grad=False)[0]
    L, g = api.unrolled_pcg(Aop, to_dev(Q), b, 10, 2, p.omega, FP64)
    g = to_np(g)
    assert _fd_check(loss, Q, g, seed=1) <= 1e-6
    assert np.linalg.norm(Q.T @ g) <= 1e-7 * np.linalg.norm(g)


def test_subspace_gradient_finite_differences_large(ctx):
    api = _api()
    p = gen.grf_diffusion_2d(N=128, k=32, K=64, seed=9)
    A = op.assemble(p)
    S = osetup.smooth_samples(A, p.S0, p.omega, p.s1)
    Ph = np.linalg.qr(S[:, : p.k])[0] + 0.1 * gen.normal(3, gen.STREAM_NOISE, p.n * p.k).reshape(p.k, p.n).T
    Sd = to_dev(S)
    loss = lambda X: api.subspace_loss(ctx, to_dev(X), Sd, FP64, grad=False)[0]
    L, g = api.subspace_loss(ctx, to_dev(Ph), Sd, FP64)
    g = to_np(g)
    assert abs(L - olosses.subspace_loss(Ph, S)) <= 1e-10 * L
    assert _fd_check(loss, Ph, g, seed=2) <= 1e-6


def test_autograd_functions(ctx):
    from paper_2601_20174_gb300.autograd import NlssLoss, SubspaceLoss, UnrolledPCG
    api = _api()
    p = UNROLL_CASES["grf20"]()
    A = op.assemble(p)
    S, _, Ph = _noisy_basis(p, A)
    Pt = to_dev(Ph).requires_grad_(True)
    loss = SubspaceLoss.apply(Pt, to_dev(S), ctx, FP64)
    (3.0 * loss).backward()
    assert rel(to_np(Pt.grad), 3.0 * olosses.grad_subspace_loss(Ph, S)) <= 1e-8
    Pn = to_dev(Ph).requires_grad_(True)
    ln = NlssLoss.apply(Pn, to_dev(S), ctx, FP64)
    (2.0 * ln).backward()
    assert rel(to_np(Pn.grad), 2.0 * olosses.grad_nlss_loss(Ph, S)) <= 1e-8
    Aop = api.Operator.from_problem(ctx, p)
    P2 = to_dev(Ph).requires_grad_(True)
    l2 = UnrolledPCG.apply(P2, Aop, to_dev(p.f[:, 0]), 10, p.nu, p.omega, FP64)
    l2.backward()
    g_ref = olosses.grad_unrolled_pcg_loss(A, Ph, p.f[:, 0], 10, p.omega, p.nu)
    assert rel(to_np(P2.grad), g_ref) <= 1e-7


def test_differentiation_rejects_bad_arguments(ctx):
    api = _api()
    p = UNROLL_CASES["poisson16"]()
    Aop = api.Operator.from_problem(ctx, p)
    P = to_dev(np.zeros((p.n, 3)))  # rank deficient: A_c singular
    with pytest.raises(api.L.NlspError):
        api.unrolled_pcg(Aop, P, to_dev(p.f[:, 0]), 10, 2, p.omega, FP64)
    with pytest.raises(api.L.NlspError):
        api.subspace_loss(ctx, P, to_dev(p.S0), FP64)
    with pytest.raises(api.L.NlspError):
        api.nlss_loss(ctx, P, to_dev(p.S0), FP64)
