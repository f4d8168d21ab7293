"""GPU tests of the batched persistent solver (nlsp_solve_batched) and of the
device-side sample generator.

Each instance of a batch must reach what a solve of that instance alone
reaches with the same preconditioner: the FP64 true relative residual below
the tolerance (checked with the oracle's assembled operator), the iteration
count of the single-instance persistent solve within one (the team's partial
sums are added in another order), and the same iterate to the accuracy the
tolerance leaves.  In FP64 every instance is given the oracle's basis and
must reproduce the oracle's PCG (iterations +-1, solution to 1e-8)."""
import numpy as np
import pytest
import torch

from helpers import rel, to_dev, to_np
from oracle import operator as op, pcg as opcg, setup as osetup
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


def _build(ctx, problems, precision):
    api = _api()
    ops = [api.Operator.from_problem(ctx, p) for p in problems]
    precs = [api.Preconditioner.build(A, to_dev(p.S0), p.k, p.s1, p.nu, p.omega, precision)
             for A, p in zip(ops, problems)]
    return ops, precs


def _check_batch(ctx, problems, precision, tiles_per_cta, tol=1e-8):
    api = _api()
    ops, precs = _build(ctx, problems, precision)
    bs = [to_dev(p.f[:, 0]) for p in problems]
    xs, res = api.solve_batched(precs, bs, tol=tol, maxit=3000, tiles_per_cta=tiles_per_cta)
    for p, M, b, x, r in zip(problems, precs, bs, xs, res):
        A = op.assemble(p)
        f = p.f[:, 0]
        xb = to_np(x)
        true = np.linalg.norm(f - A @ xb) / np.linalg.norm(f)
        assert r.status == 0 and true <= tol * 1.01, (p.name, p.N, r, true)
        assert abs(r.true_relres - true) <= 1e-3 * true
        x1, r1 = M.solve(b, tol=tol, maxit=3000, graph_mode=2)
        assert abs(r.iterations - r1[0].iterations) <= 1, (p.N, p.k, r.iterations, r1[0].iterations)
        assert rel(xb, to_np(x1)) <= 1e-5
    return res


def test_batched_uneven_instances_mixed(ctx):
    # uneven sizes and ranks; tiles_per_cta = 4 gives teams of 1 .. 18 CTAs
    sides = [16, 24, 33, 48, 64, 96, 40, 20, 72, 56]
    ranks = [4, 8, 16, 24, 32, 16, 12, 6, 64, 40]
    probs = [gen.iid_diffusion_2d(N, k, 2 * k, seed=100 + i, tol=1e-8) for i, (N, k) in enumerate(zip(sides, ranks))]
    _check_batch(ctx, probs, MIXED, tiles_per_cta=4)


def test_batched_more_instances_than_ctas_fp64(ctx):
    # 170 single-CTA teams on 152 SMs: CTAs run several instances one after
    # another (ring barriers re-initialised, tensor memory not used in FP64,
    # most of each P streamed through the ring).  Every instance gets the
    # oracle's basis and must reproduce the oracle's PCG: iterations +-1,
    # solution to 1e-8.
    api = _api()
    rng = np.random.default_rng(5)
    probs = [gen.iid_diffusion_2d(int(N), 16, 24, seed=200 + i, tol=1e-8)
             for i, N in enumerate(rng.integers(36, 45, size=170))]
    refs, precs, bs = [], [], []
    for p in probs:
        A = op.assemble(p)
        su = osetup.build(A, p.S0, p.k, p.omega, p.s1)
        o = opcg.pcg(A, opcg.two_level_solver(A, su["P"], su["L"], p.omega, p.nu, p.nu), p.f[:, 0], p.tol)
        refs.append((A, o))
        precs.append(api.Preconditioner.from_basis(api.Operator.from_problem(ctx, p), to_dev(su["P"]), p.nu,
                                                   p.omega, FP64))
        bs.append(to_dev(p.f[:, 0]))
    xs, res = api.solve_batched(precs, bs, tol=1e-8, maxit=3000, tiles_per_cta=1000)
    for p, (A, o), x, r in zip(probs, refs, xs, res):
        xb = to_np(x)
        assert r.status == 0 and o["status"] == "converged"
        assert abs(r.iterations - o["iters"]) <= 1, (p.N, r.iterations, o["iters"])
        assert rel(xb, o["x"]) <= 1e-8
        true = np.linalg.norm(p.f[:, 0] - A @ xb) / np.linalg.norm(p.f[:, 0])
        assert true <= 1e-8 * 1.01 and abs(r.true_relres - true) <= 1e-3 * true


def test_batched_grf_and_team_of_all_ctas(ctx):
    # one large instance spread over every CTA beside small ones
    probs = [gen.grf_diffusion_2d(N=160, k=32, K=64, seed=7, tol=1e-8),
             gen.poisson_2d(37, 8, 24, seed=1), gen.iid_diffusion_2d(30, 10, 20, seed=3, tol=1e-8)]
    _check_batch(ctx, probs, MIXED, tiles_per_cta=1)


def test_batched_rejects_mixed_kinds_and_duplicates(ctx):
    api = _api()
    p5 = gen.iid_diffusion_2d(20, 4, 8, seed=1)
    p9 = gen.aniso_9pt_2d(N=20, k=4, K=8, m=1, seed=2)
    _, (M5,) = _build(ctx, [p5], MIXED)
    _, (M9,) = _build(ctx, [p9], MIXED)
    b5, b9 = to_dev(p5.f[:, 0]), to_dev(p9.f[:, 0])
    with pytest.raises(api.L.NlspError):
        api.solve_batched([M5, M9], [b5, b9])
    with pytest.raises(api.L.NlspError):
        api.solve_batched([M5, M5], [b5, b5.clone()])
    assert api.solve_batched([], []) == ([], [])


def test_device_normals_match_counter_generator(ctx):
    # nlsp_random_normal draws the same SplitMix64 / Box-Muller stream as the
    # shared host generator (both are written from the published definitions)
    import ctypes as C
    api = _api()
    seed, stream, count, offset = 1234, gen.STREAM_S0, 10007, 3
    out = torch.empty(count, dtype=torch.float64, device="cuda")
    api.L.check(ctx._lib.nlsp_random_normal(ctx.h, seed, stream, offset, count, C.c_void_p(out.data_ptr())),
                "nlsp_random_normal")
    ref = gen.normal(seed, stream, count + offset)[offset:]
    got = to_np(out)
    assert np.max(np.abs(got - ref) / (1.0 + np.abs(ref))) <= 1e-12


def test_build_with_device_samples_matches_uploaded_samples(ctx):
    api = _api()
    p = gen.grf_diffusion_2d(N=45, k=12, K=32, seed=2)
    A = api.Operator.from_problem(ctx, p)
    for precision in (FP64, MIXED):
        M_host = api.Preconditioner.build(A, to_dev(p.S0), p.k, p.s1, p.nu, p.omega, precision)
        M_dev = api.Preconditioner.build(A, None, p.k, p.s1, p.nu, p.omega, precision, K=p.K, seed=p.seed)
        tol = 1e-12 if precision == FP64 else 1e-5
        assert rel(to_np(M_dev.sigma()), to_np(M_host.sigma())) <= tol
        P1, P2 = to_np(M_host.basis()), to_np(M_dev.basis())
        # same subspace: the projectors agree
        assert np.linalg.norm(P1 @ (P1.T @ P2) - P2, 2) <= (1e-9 if precision == FP64 else 1e-3)


def test_tuner_remembers_the_fastest_team_size(ctx):
    # nlsp_tune_batched times the candidates and the context then uses the
    # fastest for batches of the same sizes when tiles_per_cta = 0: the
    # result is the one an explicit call with that value gives, bit for bit
    # (the team plan, and so every partial sum's order, is the same)
    api = _api()
    probs = [gen.iid_diffusion_2d(N, k, 2 * k, seed=300 + i, tol=1e-8)
             for i, (N, k) in enumerate(zip([24, 40, 64, 33], [8, 16, 32, 12]))]
    _, precs = _build(ctx, probs, MIXED)
    bs = [to_dev(p.f[:, 0]) for p in probs]
    best, ms = api.tune_batched(precs, bs, candidates=(1, 4, 1000))
    assert best in (1, 4, 1000) and set(ms) == {1, 4, 1000} and all(v > 0 for v in ms.values())
    xa, ra = api.solve_batched(precs, bs, tiles_per_cta=0)
    xb, rb = api.solve_batched(precs, bs, tiles_per_cta=best)
    for a, b, r1, r2 in zip(xa, xb, ra, rb):
        assert r1.iterations == r2.iterations and torch.equal(a, b)
