"""GPU parity of the CUDA path (through the C ABI) against the FP64 oracle.

Tolerances: FP64 kernels agree with the oracle to rounding (1e-12 relative on
operator and preconditioner applications, which sum a handful of terms per
entry; subspace agreement to 1e-8 given the singular-value gap).  The FP32
preconditioner is checked against what the method fixes: the solve reaches the FP64
true relative residual 1e-8 and the preconditioner error stays at FP32 level.
"""
import numpy as np
import pytest
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


@pytest.mark.parametrize("name", list(PROBLEMS))
def test_operator_apply_and_diagonal(ctx, name):
    p = PROBLEMS[name]()
    A = op.assemble(p)
    Aop = _api().Operator.from_problem(ctx, p)
    X = np.random.default_rng(0).standard_normal((p.n, 3))
    Y = to_np(Aop.apply(to_dev(X)))
    ref = A @ X
    assert np.max(np.abs(Y - ref)) <= 1e-13 * np.max(np.abs(ref))
    assert np.array_equal(to_np(Aop.diagonal()), A.diagonal()) or \
        np.max(np.abs(to_np(Aop.diagonal()) - A.diagonal())) <= 1e-15 * A.diagonal().max()


@pytest.mark.parametrize("name", list(PROBLEMS))
@pytest.mark.parametrize("precision", [FP64, MIXED])
def test_smooth_samples(ctx, name, precision):
    p = PROBLEMS[name]()
    A = op.assemble(p)
    Aop = _api().Operator.from_problem(ctx, p)
    S = to_np(Aop.smooth_samples(to_dev(p.S0), p.s1, p.omega, precision))
    ref = osetup.smooth_samples(A, p.S0, p.omega, p.s1)
    tol = 1e-12 if precision == FP64 else 2e-5
    assert rel(S, ref) <= tol


@pytest.mark.parametrize("N,K,s1", [(37, 6, 1), (37, 6, 3), (29, 5, 7), (700, 3, 3), (300, 13, 2)])
@pytest.mark.parametrize("kind", ["5pt", "9pt"])
@pytest.mark.parametrize("precision", [FP64, MIXED])
def test_smooth_samples_sweep_counts_and_shapes(ctx, N, K, s1, kind, precision):
    # odd and even sweep counts, sample counts that are not a multiple of the
    # kernels' four or eight columns per thread, grid rows that span node
    # tiles, and grids of 65536 nodes and more (700^2: n = 490000 with a
    # ragged last tile; 300^2 with K = 13: two column groups, the second
    # ragged), which the FP32 path sweeps by streaming along grid rows with a
    # partial block of grid columns at the edge, for both 2D stencils
    p = gen.poisson_2d(N, 2, K, seed=5) if kind == "5pt" else gen.aniso_9pt_2d(N=N, k=2, K=K, m=1, seed=6)
    A = op.assemble(p)
    Aop = _api().Operator.from_problem(ctx, p)
    S = to_np(Aop.smooth_samples(to_dev(p.S0), s1, p.omega, precision))
    ref = osetup.smooth_samples(A, p.S0, p.omega, s1)
    tol = 1e-12 if precision == FP64 else 2e-5
    assert rel(S, ref) <= tol


@pytest.mark.parametrize("name", ["grf5", "aniso9"])
@pytest.mark.parametrize("precision", [FP64, MIXED])
def test_a_weighted_setup_matches_oracle_and_solves(ctx, name, precision):
    # the A-weighted basis (Appendix, Galerkin Convergence): the device's
    # S^T A S Gram route against the oracle's, then a PCG solve with it
    p = PROBLEMS[name]()
    A = op.assemble(p)
    S = osetup.smooth_samples(A, p.S0, p.omega, p.s1)
    P_ref, sig_ref = osetup.prolongation_a_weighted(A, S, p.k)
    Aop = _api().Operator.from_problem(ctx, p)
    M = _api().Preconditioner.build(Aop, to_dev(p.S0), p.k, p.s1, p.nu, p.omega, precision, a_weighted=True)
    P, sig = to_np(M.basis()), to_np(M.sigma())
    fp64 = precision == FP64
    assert rel(sig[: p.k], sig_ref[: p.k]) <= (1e-10 if fp64 else 1e-4)
    assert np.max(np.abs(P.T @ (A @ P) - np.eye(p.k))) <= (1e-9 if fp64 else 1e-4)
    gap = sig_ref[p.k - 1] / sig_ref[p.k] - 1.0
    Qg, Qr = np.linalg.qr(P)[0], np.linalg.qr(P_ref)[0]
    assert projector_dist(Qg, Qr) <= (max(1e-8, 1e-13 / gap) if fp64 else max(1e-3, 1e-6 / gap))
    # the coarse space never does worse on J than the Euclidean SVD basis
    Pe, _ = osetup.prolongation(S, p.k)
    assert osetup.post_correction_energy(A, P, S) <= osetup.post_correction_energy(A, Pe, S) * (1 + 1e-6)
    b = p.f[:, 0]
    x, res = M.solve(to_dev(b), tol=1e-8)
    true = np.linalg.norm(b - A @ to_np(x)) / np.linalg.norm(b)
    assert res[0].status == 0 and true <= 1e-8 * 1.01
    if fp64:
        L_ref = osetup.coarse_factor(osetup.galerkin(A, P_ref))
        o = opcg.pcg(A, opcg.two_level_solver(A, P_ref, L_ref, p.omega, p.nu, p.nu), b, 1e-8)
        assert abs(res[0].iterations - o["iters"]) <= 1


@pytest.mark.parametrize("name", ["grf5", "aniso9", "iid7"])
@pytest.mark.parametrize("oversample,power_iters", [(0, 0), (6, 1), (8, 2)])
def test_randomized_setup_matches_oracle(ctx, name, oversample, power_iters):
    # the randomised SVD basis (Halko, Martinsson, Tropp: range finder with
    # power iterations, SVD of the projected matrix) given the same sketch
    p = PROBLEMS[name]()
    A = op.assemble(p)
    S = osetup.smooth_samples(A, p.S0, p.omega, p.s1)
    l = p.k + oversample
    sk = gen.sketch_normal(p.K, l, seed=5)
    P_ref, sB = osetup.prolongation_randomized(S, p.k, oversample, power_iters, sk, return_sigma=True)
    Aop = _api().Operator.from_problem(ctx, p)
    gap = (sB[p.k - 1] ** 2 - (sB[p.k] ** 2 if l > p.k else 0.0)) / sB[0] ** 2
    for precision in (FP64, MIXED):
        M = _api().Preconditioner.build_randomized(Aop, to_dev(p.S0), p.k, oversample, power_iters, to_dev(sk),
                                                   p.s1, p.nu, p.omega, precision)
        P, sig = to_np(M.basis()), to_np(M.sigma())
        fp64 = precision == FP64
        assert rel(sig[:l], sB) <= (1e-9 if fp64 else 1e-4), (sig[:l], sB)
        assert np.all(sig[l:] == 0.0)
        Q = np.linalg.qr(P)[0]
        assert projector_dist(Q, P_ref) <= (max(1e-8, 1e-12 / gap) if fp64 else max(2e-3, 1e-6 / gap))
        if fp64:
            assert np.max(np.abs(P.T @ P - np.eye(p.k))) <= 1e-12
    # a sketch drawn on the device is the counter-based stream the host draws
    Md = _api().Preconditioner.build_randomized(Aop, to_dev(p.S0), p.k, oversample, power_iters, None, p.s1, p.nu,
                                                p.omega, FP64, seed=5)
    assert projector_dist(to_np(Md.basis()), P_ref) <= max(1e-8, 1e-12 / gap)


def test_randomized_setup_solves_and_rejects_bad_arguments(ctx):
    p = PROBLEMS["grf5"]()
    A = op.assemble(p)
    S = osetup.smooth_samples(A, p.S0, p.omega, p.s1)
    sk = gen.sketch_normal(p.K, p.k + 8, seed=2)
    P_ref = osetup.prolongation_randomized(S, p.k, 8, 2, sk)
    L_ref = osetup.coarse_factor(osetup.galerkin(A, P_ref))
    b = p.f[:, 0]
    o = opcg.pcg(A, opcg.two_level_solver(A, P_ref, L_ref, p.omega, p.nu, p.nu), b, 1e-8)
    Aop = _api().Operator.from_problem(ctx, p)
    for precision in (FP64, MIXED):
        M = _api().Preconditioner.build_randomized(Aop, to_dev(p.S0), p.k, 8, 2, to_dev(sk), p.s1, p.nu, p.omega,
                                                   precision)
        x, res = M.solve(to_dev(b), tol=1e-8, graph_mode=2)
        true = np.linalg.norm(b - A @ to_np(x)) / np.linalg.norm(b)
        assert res[0].status == 0 and true <= 1e-8 * 1.01
        assert abs(res[0].iterations - o["iters"]) <= (1 if precision == FP64 else 2)
    with pytest.raises(_api().L.NlspError):  # k + oversample > K
        _api().Preconditioner.build_randomized(Aop, to_dev(p.S0), p.k, p.K - p.k + 1, 1, None, p.s1, p.nu, p.omega,
                                               FP64)


@pytest.mark.parametrize("name", list(PROBLEMS))
def test_setup_fp64_subspace_sigma_and_galerkin(ctx, name):
    p = PROBLEMS[name]()
    A = op.assemble(p)
    ref = osetup.build(A, p.S0, p.k, p.omega, p.s1)
    M = _api().Preconditioner.build(_api().Operator.from_problem(ctx, p), to_dev(p.S0), p.k, p.s1, p.nu, p.omega, FP64)
    P = to_np(M.basis())
    sig = to_np(M.sigma())
    # The SVD goes through the Gram matrix S^T S, which resolves sigma_i only to
    # ~eps sigma_1^2 / sigma_i; the leading k+1 values are the ones that matter.
    s_ref = ref["sigma"][: p.k + 1]
    tol_s = 1e-9 * s_ref + 1e-13 * s_ref[0] ** 2 / s_ref
    assert np.all(np.abs(sig[: p.k + 1] - s_ref) <= tol_s), (sig[: p.k + 1] - s_ref) / s_ref
    gap = (s_ref[p.k - 1] ** 2 - s_ref[p.k] ** 2) / s_ref[0] ** 2
    dist = projector_dist(P, ref["P"])
    assert dist <= max(1e-8, 1e-13 / gap), (dist, gap)
    assert np.max(np.abs(P.T @ P - np.eye(p.k))) <= 1e-12, np.max(np.abs(P.T @ P - np.eye(p.k)))
    Ac, Lf = (to_np(t) for t in M.coarse())
    Ac_ref = osetup.galerkin(A, P)  # Galerkin product of the GPU's own basis
    assert np.max(np.abs(Ac - Ac_ref)) <= 1e-12 * np.max(np.abs(Ac_ref))
    assert np.max(np.abs(Lf @ Lf.T - Ac)) <= 1e-12 * np.max(np.abs(Ac))


@pytest.mark.parametrize("K", [160, 256])
@pytest.mark.parametrize("precision", [FP64, MIXED])
def test_setup_wide_sample_blocks(ctx, K, precision):
    # 128 < K <= 256: the Gram matrix in 128-column quadrants and its
    # eigenvectors by one-sided Jacobi on a cluster of two CTAs (then the
    # FP64 refinement in the FP64 path); sigma, span(P) and A_c against the
    # oracle's SVD of the same smoothed samples
    p = gen.grf_diffusion_2d(N=40, k=64, K=K, seed=31, tol=1e-8)
    A = op.assemble(p)
    ref = osetup.build(A, p.S0, p.k, p.omega, p.s1)
    M = _api().Preconditioner.build(_api().Operator.from_problem(ctx, p), to_dev(p.S0), p.k, p.s1, p.nu, p.omega,
                                    precision)
    P, sig = to_np(M.basis()), to_np(M.sigma())
    s_ref = ref["sigma"][: p.k + 1]
    gap = (s_ref[p.k - 1] ** 2 - s_ref[p.k] ** 2) / s_ref[0] ** 2
    if precision == FP64:
        tol_s = 1e-9 * s_ref + 1e-13 * s_ref[0] ** 2 / s_ref
        assert np.all(np.abs(sig[: p.k + 1] - s_ref) <= tol_s), (sig[: p.k + 1] - s_ref) / s_ref
        assert projector_dist(P, ref["P"]) <= max(1e-8, 1e-13 / gap)
        assert np.max(np.abs(P.T @ P - np.eye(p.k))) <= 1e-12
        Ac, _ = (to_np(t) for t in M.coarse())
        Ac_ref = osetup.galerkin(A, P)
        assert np.max(np.abs(Ac - Ac_ref)) <= 1e-12 * np.max(np.abs(Ac_ref))
    else:
        assert np.all(np.abs(sig[: p.k + 1] - s_ref) <= 1e-4 * s_ref[0]), (sig[: p.k + 1] - s_ref)
        Q = np.linalg.qr(P)[0]
        assert projector_dist(Q, ref["P"]) <= max(1e-3, 1e-6 / gap)
    b = p.f[:, 0]
    x, res = M.solve(to_dev(b), tol=1e-8)
    assert res[0].status == 0
    assert np.linalg.norm(b - A @ to_np(x)) / np.linalg.norm(b) <= 1e-8 * 1.01


def test_setup_wide_sample_blocks_limits(ctx):
    # K <= 256 for the exact-SVD basis; the A-weighted and randomised bases
    # keep K <= 128
    api = _api()
    p = gen.grf_diffusion_2d(N=24, k=8, K=160, seed=3, tol=1e-8)
    Aop = api.Operator.from_problem(ctx, p)
    with pytest.raises(api.L.NlspError):
        api.Preconditioner.build(Aop, to_dev(p.S0), p.k, p.s1, p.nu, p.omega, FP64, a_weighted=True)
    with pytest.raises(api.L.NlspError):
        api.Preconditioner.build_randomized(Aop, to_dev(p.S0), p.k, 8, 1, None, p.s1, p.nu, p.omega, FP64)
    q = gen.grf_diffusion_2d(N=24, k=8, K=257, seed=3, tol=1e-8)
    with pytest.raises(api.L.NlspError):
        api.Preconditioner.build(api.Operator.from_problem(ctx, q), to_dev(q.S0), q.k, q.s1, q.nu, q.omega, FP64)


@pytest.mark.parametrize("name", list(PROBLEMS))
def test_setup_mixed_sigma_and_subspace(ctx, name):
    # FP32 preconditioner: the Gram matrix is decomposed in FP32 (pivoted
    # Cholesky, then one-sided Jacobi on the factor); sigma and span(P)
    # against the oracle's SVD to FP32 accuracy
    p = PROBLEMS[name]()
    A = op.assemble(p)
    ref = osetup.build(A, p.S0, p.k, p.omega, p.s1)
    M = _api().Preconditioner.build(_api().Operator.from_problem(ctx, p), to_dev(p.S0), p.k, p.s1, p.nu, p.omega,
                                    MIXED)
    sig = to_np(M.sigma())
    s_ref = ref["sigma"]
    assert np.all(np.abs(sig[: p.k + 1] - s_ref[: p.k + 1]) <= 1e-4 * s_ref[0]), (sig[: p.k + 1] - s_ref[: p.k + 1])
    gap = (s_ref[p.k - 1] ** 2 - s_ref[p.k] ** 2) / s_ref[0] ** 2
    Q = np.linalg.qr(to_np(M.basis()))[0]
    assert projector_dist(Q, ref["P"]) <= max(1e-3, 1e-6 / gap)


@pytest.mark.parametrize("K,k", [(7, 3), (3, 3), (1, 1)])
def test_setup_mixed_odd_and_tiny_sample_counts(ctx, K, k):
    p = gen.grf_diffusion_2d(N=30, k=k, K=K, seed=21, tol=1e-8)
    A = op.assemble(p)
    ref = osetup.build(A, p.S0, p.k, p.omega, p.s1)
    Aop = _api().Operator.from_problem(ctx, p)
    M = _api().Preconditioner.build(Aop, to_dev(p.S0), p.k, p.s1, p.nu, p.omega, MIXED)
    sig = to_np(M.sigma())
    assert np.all(np.abs(sig[:K] - ref["sigma"][:K]) <= 1e-4 * ref["sigma"][0])
    x, res = M.solve(to_dev(p.f[:, 0]), tol=1e-8)
    assert res[0].status == 0


@pytest.mark.parametrize("precision", [FP64, MIXED])
def test_setup_rank_deficient_samples(ctx, precision):
    # K = 2k samples whose second half repeats the first: G = S^T S has rank k,
    # the factorisation stops at the numerical rank and the top k eigenpairs
    # are those of the distinct half
    p = PROBLEMS["grf5"]()
    A = op.assemble(p)
    half = p.S0[:, : p.K // 2]
    S0 = np.concatenate([half, half], axis=1)
    k = min(p.k, p.K // 2)
    ref = osetup.build(A, half, k, p.omega, p.s1)
    Aop = _api().Operator.from_problem(ctx, p)
    M = _api().Preconditioner.build(Aop, to_dev(np.ascontiguousarray(S0)), k, p.s1, p.nu, p.omega, precision)
    sig = to_np(M.sigma())
    s_ref = np.sqrt(2.0) * ref["sigma"][:k]  # every direction counted twice
    tol = 1e-9 * s_ref + 1e-13 * s_ref[0] ** 2 / s_ref if precision == FP64 else 1e-4 * s_ref[0]
    assert np.all(np.abs(sig[:k] - s_ref) <= tol), (sig[:k], s_ref)
    assert np.all(sig[p.K // 2:] <= (1e-6 if precision == FP64 else 1e-2) * s_ref[0])
    b = p.f[:, 0]
    x, res = M.solve(to_dev(b), tol=1e-8)
    assert res[0].status == 0
    assert np.linalg.norm(b - A @ to_np(x)) / np.linalg.norm(b) <= 1e-8 * 1.01


@pytest.mark.parametrize("precision", [FP64, MIXED])
def test_setup_zero_sample_column(ctx, precision):
    # a zero sample column makes G singular with an exactly zero pivot: the
    # FP32 factorisation stops one short of K and the basis is completed by
    # the complement before the FP64 refinement; the leading k pairs are
    # those of the remaining samples
    p = PROBLEMS["grf5"]()
    A = op.assemble(p)
    S0 = p.S0.copy()
    S0[:, -1] = 0.0
    ref = osetup.build(A, S0[:, :-1], p.k, p.omega, p.s1)
    Aop = _api().Operator.from_problem(ctx, p)
    M = _api().Preconditioner.build(Aop, to_dev(S0), p.k, p.s1, p.nu, p.omega, precision)
    sig, P = to_np(M.sigma()), to_np(M.basis())
    s_ref = ref["sigma"][: p.k]
    fp64 = precision == FP64
    assert np.all(np.abs(sig[: p.k] - s_ref) <= (1e-9 * s_ref + 1e-13 * s_ref[0] ** 2 / s_ref if fp64
                                                  else 1e-4 * s_ref[0])), (sig[: p.k] - s_ref) / s_ref
    assert abs(sig[-1]) <= (1e-6 if fp64 else 1e-2) * s_ref[0]
    if fp64:
        assert np.max(np.abs(P.T @ P - np.eye(p.k))) <= 1e-12
    gap = (s_ref[p.k - 1] ** 2 - ref["sigma"][p.k] ** 2) / s_ref[0] ** 2
    Q = np.linalg.qr(P)[0]
    assert projector_dist(Q, ref["P"]) <= (max(1e-8, 1e-13 / gap) if fp64 else max(1e-3, 1e-6 / gap))
    b = p.f[:, 0]
    x, res = M.solve(to_dev(b), tol=1e-8)
    assert res[0].status == 0
    assert np.linalg.norm(b - A @ to_np(x)) / np.linalg.norm(b) <= 1e-8 * 1.01


@pytest.mark.parametrize("name", list(PROBLEMS))
@pytest.mark.parametrize("precision", [FP64, MIXED])
def test_apply_matches_algorithm1(ctx, name, precision):
    # The oracle's basis is handed to the GPU so both apply the same B.
    p = PROBLEMS[name]()
    A = op.assemble(p)
    ref = osetup.build(A, p.S0, p.k, p.omega, p.s1)
    M = _api().Preconditioner.from_basis(_api().Operator.from_problem(ctx, p), to_dev(ref["P"]), p.nu, p.omega,
                                         precision)
    R = np.random.default_rng(5).standard_normal((p.n, 2))
    Z = to_np(M.apply(to_dev(R)))
    Zref = oprec.apply(A, ref["P"], ref["L"], R, p.omega, p.nu, p.nu)
    tol = 1e-12 if precision == FP64 else 1e-4
    assert rel(Z, Zref) <= tol


def test_rank_truncation(ctx):
    p = PROBLEMS["grf5"]()
    A = op.assemble(p)
    ref = osetup.build(A, p.S0, p.k, p.omega, p.s1)
    M = _api().Preconditioner.from_basis(_api().Operator.from_problem(ctx, p), to_dev(ref["P"]), p.nu, p.omega, FP64)
    r = 5
    M.factor(r)
    Pr = osetup.truncate(ref["P"], r)
    Ac, _ = (to_np(t) for t in M.coarse())
    assert np.max(np.abs(Ac - osetup.galerkin(A, Pr))) <= 1e-12 * np.max(np.abs(Ac))
    R = np.random.default_rng(6).standard_normal(p.n)
    Z = to_np(M.apply(to_dev(R)))
    Zref = oprec.apply(A, Pr, osetup.coarse_factor(osetup.galerkin(A, Pr)), R, p.omega, p.nu, p.nu)
    assert rel(Z, Zref) <= 1e-12


@pytest.mark.parametrize("name", list(PROBLEMS))
@pytest.mark.parametrize("graph_mode", [0, 1, 2])
def test_pcg_fp64_matches_oracle_iterates(ctx, name, graph_mode):
    p = PROBLEMS[name]()
    A = op.assemble(p)
    ref = osetup.build(A, p.S0, p.k, p.omega, p.s1)
    M = _api().Preconditioner.from_basis(_api().Operator.from_problem(ctx, p), to_dev(ref["P"]), p.nu, p.omega, FP64)
    b = p.f[:, 0]
    o = opcg.pcg(A, opcg.two_level_solver(A, ref["P"], ref["L"], p.omega, p.nu, p.nu), b, p.tol)
    x, res = M.solve(to_dev(b), tol=p.tol, graph_mode=graph_mode)
    assert res[0].status == 0
    assert abs(res[0].iterations - o["iters"]) <= 1
    assert rel(to_np(x), o["x"]) <= 1e-8
    true = np.linalg.norm(b - A @ to_np(x)) / np.linalg.norm(b)
    assert true <= p.tol * 1.01 and abs(res[0].true_relres - true) <= 1e-3 * true


@pytest.mark.parametrize("name", list(PROBLEMS))
@pytest.mark.parametrize("cluster", ["1", "0"])
def test_single_launch_solvers_match_oracle(ctx, name, cluster, monkeypatch):
    # graph_mode 2 runs small systems on the cluster-resident solver (one
    # thread-block cluster, vectors in distributed shared memory) and the
    # rest on the grid-wide persistent solver; NLSP_CLUSTER=0 forces the
    # latter.  Both must reproduce the oracle's iterates (FP64, the oracle's
    # basis) and reach the FP64 true residual in mixed precision.
    monkeypatch.setenv("NLSP_CLUSTER", cluster)
    p = PROBLEMS[name]()
    A = op.assemble(p)
    ref = osetup.build(A, p.S0, p.k, p.omega, p.s1)
    b = p.f[:, 0]
    o = opcg.pcg(A, opcg.two_level_solver(A, ref["P"], ref["L"], p.omega, p.nu, p.nu), b, p.tol)
    Aop = _api().Operator.from_problem(ctx, p)
    M = _api().Preconditioner.from_basis(Aop, to_dev(ref["P"]), p.nu, p.omega, FP64)
    x, res = M.solve(to_dev(b), tol=p.tol, graph_mode=2)
    assert res[0].status == 0 and abs(res[0].iterations - o["iters"]) <= 1
    assert rel(to_np(x), o["x"]) <= 1e-8
    true = np.linalg.norm(b - A @ to_np(x)) / np.linalg.norm(b)
    assert abs(res[0].true_relres - true) <= 1e-3 * true
    Mm = _api().Preconditioner.from_basis(Aop, to_dev(ref["P"]), p.nu, p.omega, MIXED)
    x, res = Mm.solve(to_dev(b), tol=1e-8, graph_mode=2)
    true = np.linalg.norm(b - A @ to_np(x)) / np.linalg.norm(b)
    assert res[0].status == 0 and true <= 1e-8 * 1.01
    # zero right-hand side and maxit through the same launch
    x0, r0 = M.solve(to_dev(np.zeros(p.n)), tol=p.tol, graph_mode=2)
    assert r0[0].iterations == 0 and r0[0].status == 0 and np.all(to_np(x0) == 0)
    _, r3 = M.solve(to_dev(b), tol=1e-14, maxit=3, graph_mode=2)
    assert r3[0].status == 1 and r3[0].iterations == 3


@pytest.mark.parametrize("name", list(PROBLEMS))
@pytest.mark.parametrize("graph_mode", [1, 2])
def test_pcg_end_to_end_both_precisions(ctx, name, graph_mode):
    p = PROBLEMS[name]()
    p.tol = 1e-8
    A = op.assemble(p)
    o = opcg.solve_problem(p, A=A)
    Aop = _api().Operator.from_problem(ctx, p)
    for precision in (FP64, MIXED):
        M = _api().Preconditioner.build(Aop, to_dev(p.S0), p.k, p.s1, p.nu, p.omega, precision)
        x, res = M.solve(to_dev(p.f[:, 0]), tol=p.tol, graph_mode=graph_mode)
        true = np.linalg.norm(p.f[:, 0] - A @ to_np(x)) / np.linalg.norm(p.f[:, 0])
        assert res[0].status == 0 and true <= 1e-8 * 1.01
        if precision == FP64:
            assert abs(res[0].iterations - o["results"][0]["iters"]) <= 1
        else:
            assert abs(res[0].iterations - o["results"][0]["iters"]) <= 2


@pytest.mark.parametrize("graph_mode", [1, 2])
def test_multi_rhs_zero_and_scaled_columns(ctx, graph_mode):
    p = PROBLEMS["grf5"]()
    A = op.assemble(p)
    M = _api().Preconditioner.build(_api().Operator.from_problem(ctx, p), to_dev(p.S0), p.k, p.s1, p.nu, p.omega,
                                    FP64)
    b = p.f[:, 0]
    B = np.stack([b, np.zeros(p.n), 3.0 * b], axis=1)
    X, res = M.solve(to_dev(B), tol=1e-9, graph_mode=graph_mode)
    X = to_np(X)
    assert res[1].iterations == 0 and res[1].status == 0 and np.all(X[:, 1] == 0)
    assert res[0].iterations == res[2].iterations
    assert rel(X[:, 2], 3.0 * X[:, 0]) <= 1e-10


@pytest.mark.parametrize("graph_mode", [1, 2])
def test_full_rank_basis_one_iteration(ctx, graph_mode):
    p = gen.iid_diffusion_2d(N=7, k=4, K=8, seed=9)
    M = _api().Preconditioner.from_basis(_api().Operator.from_problem(ctx, p), to_dev(np.eye(p.n)), 2, p.omega, FP64)
    x, res = M.solve(to_dev(p.f[:, 0]), tol=1e-10, graph_mode=graph_mode)
    assert res[0].iterations == 1 and res[0].true_relres <= 1e-10


@pytest.mark.parametrize("graph_mode", [1, 2])
def test_maxit_and_nonfinite_rhs(ctx, graph_mode):
    p = PROBLEMS["grf5"]()
    M = _api().Preconditioner.build(_api().Operator.from_problem(ctx, p), to_dev(p.S0), 2, p.s1, p.nu, p.omega, FP64)
    x, res = M.solve(to_dev(p.f[:, 0]), tol=1e-14, maxit=3, graph_mode=graph_mode)
    assert res[0].status == 1 and res[0].iterations == 3
    bad = p.f[:, 0].copy()
    bad[5] = np.nan
    x, res = M.solve(to_dev(bad), tol=1e-8, graph_mode=graph_mode)
    assert res[0].status == -4


def test_invalid_arguments_rejected(ctx):
    api = _api()
    p = PROBLEMS["poisson5"]()
    Aop = api.Operator.from_problem(ctx, p)
    with pytest.raises(api.L.NlspError):
        api.Preconditioner.build(Aop, to_dev(p.S0), p.k, p.s1, 0, p.omega, FP64)  # nu = 0
    with pytest.raises(api.L.NlspError):
        api.Preconditioner.build(Aop, to_dev(p.S0), p.K + 1, p.s1, 2, p.omega, FP64)  # k > K
    with pytest.raises(api.L.NlspError):
        api.Operator(ctx, 2, 8, 5, -torch.ones(81, dtype=torch.float64).cuda(), 0)  # kappa < 0


@pytest.mark.parametrize("case", ["bench512_k64", "iid1024_k32"])
def test_persistent_solver_large_grids(ctx, case):
    # Full-size grids: the persistent solver keeps P in tensor memory, shared
    # memory and a streamed remainder (all three tiers at n = 1024^2, k = 32).
    # Checked by what holds at any size: the FP64 true residual computed by
    # the oracle's own operator, and agreement with the graph-driven solver.
    if case == "bench512_k64":
        p = gen.grf_diffusion_2d(512, 64, 128, seed=0, tol=1e-8)
    else:
        p = gen.iid_diffusion_2d(1024, 32, 64, seed=3, tol=1e-8)
    A = op.assemble(p)
    Aop = _api().Operator.from_problem(ctx, p)
    M = _api().Preconditioner.build(Aop, to_dev(p.S0), p.k, p.s1, p.nu, p.omega, MIXED)
    b = p.f[:, 0]
    x2, r2 = M.solve(to_dev(b), tol=p.tol, maxit=5000, graph_mode=2)
    x1, r1 = M.solve(to_dev(b), tol=p.tol, maxit=5000, graph_mode=1)
    true2 = np.linalg.norm(b - A @ to_np(x2)) / np.linalg.norm(b)
    assert r2[0].status == 0 and true2 <= 1e-8 * 1.01, (r2[0], true2)
    assert abs(r2[0].iterations - r1[0].iterations) <= max(2, r1[0].iterations // 100)
    assert abs(r2[0].true_relres - true2) <= 1e-3 * true2
    if case == "bench512_k64":
        import json, os
        golden = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "bench_workloads.json")))
        it_oracle = golden["grf_diffusion2d_N512_k64_K128_seed0"]["iters"]
        assert abs(r2[0].iterations - it_oracle) <= 8


LARGE_FP64 = {
    # several 128-node tiles per CTA (152 CTAs), and an FP64 P of 64 columns
    # (64 KB per tile) that overflows shared memory into the streamed ring
    "grf2d_N256_k64": lambda: gen.grf_diffusion_2d(N=256, k=64, K=128, seed=12, tol=1e-8),
    "aniso9_N192_k64": lambda: gen.aniso_9pt_2d(N=192, k=64, K=128, m=1, seed=13, tol=1e-8),
    "iid3d_N40_k64": lambda: gen.iid_diffusion_3d(N=40, k=64, K=128, seed=14, tol=1e-8),
}


@pytest.mark.parametrize("name", list(LARGE_FP64))
def test_persistent_fp64_matches_oracle_iterates_multi_tile(ctx, name):
    # FP64 persistent solver against the oracle's own iterates (same basis,
    # the oracle's) where each CTA owns several node tiles and part of P is
    # streamed every phase: iterations +-1, solution to 1e-8
    p = LARGE_FP64[name]()
    A = op.assemble(p)
    ref = osetup.build(A, p.S0, p.k, p.omega, p.s1)
    b = p.f[:, 0]
    o = opcg.pcg(A, opcg.two_level_solver(A, ref["P"], ref["L"], p.omega, p.nu, p.nu), b, p.tol, maxit=5000)
    assert o["status"] == "converged"
    M = _api().Preconditioner.from_basis(_api().Operator.from_problem(ctx, p), to_dev(ref["P"]), p.nu, p.omega, FP64)
    x, res = M.solve(to_dev(b), tol=p.tol, maxit=5000, graph_mode=2)
    assert res[0].status == 0
    assert abs(res[0].iterations - o["iters"]) <= 1, (res[0].iterations, o["iters"])
    assert rel(to_np(x), o["x"]) <= 1e-8
    true = np.linalg.norm(b - A @ to_np(x)) / np.linalg.norm(b)
    assert true <= p.tol * 1.01


def test_bench_workload_fp64_iterations_match_oracle(ctx):
    # the 512^2 GRF workload, plain FP64 end to end (device setup from the same
    # samples): the oracle's stored iteration count +-1 and its true residual
    import json, os
    golden = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "bench_workloads.json")))
    want = golden["grf_diffusion2d_N512_k64_K128_seed0"]
    p = gen.grf_diffusion_2d(512, 64, 128, seed=0, tol=1e-8)
    A = op.assemble(p)
    Aop = _api().Operator.from_problem(ctx, p)
    M = _api().Preconditioner.build(Aop, to_dev(p.S0), p.k, p.s1, p.nu, p.omega, FP64)
    b = p.f[:, 0]
    x, res = M.solve(to_dev(b), tol=p.tol, maxit=5000, graph_mode=2)
    true = np.linalg.norm(b - A @ to_np(x)) / np.linalg.norm(b)
    assert res[0].status == 0 and true <= 1e-8 * 1.01
    assert abs(res[0].iterations - want["iters"]) <= 1, (res[0].iterations, want["iters"])


@pytest.mark.parametrize("name", ["poisson5", "grf5", "aniso9"])
def test_persistent_merged_update_matches_separate_phase(ctx, name, monkeypatch):
    # the CG update inside the staged restriction (default on 2D FP32) and
    # the separate update phase (NLSP_MERGE_PRE=0) take the same iterations
    # (+-1) and both reach the FP64 true residual
    p = PROBLEMS[name]()
    A = op.assemble(p)
    Aop = _api().Operator.from_problem(ctx, p)
    M = _api().Preconditioner.build(Aop, to_dev(p.S0), p.k, p.s1, p.nu, p.omega, MIXED)
    b = p.f[:, 0]
    x_m, r_m = M.solve(to_dev(b), tol=1e-8, graph_mode=2)
    monkeypatch.setenv("NLSP_MERGE_PRE", "0")
    x_s, r_s = M.solve(to_dev(b), tol=1e-8, graph_mode=2)
    for x, r in ((x_m, r_m), (x_s, r_s)):
        true = np.linalg.norm(b - A @ to_np(x)) / np.linalg.norm(b)
        assert r[0].status == 0 and true <= 1e-8 * 1.01
    assert abs(r_m[0].iterations - r_s[0].iterations) <= 1


def _conversion_patterns():
    """64-bit patterns covering every exponent of both formats, the FP32
    rounding halfway cases (odd and even), the edges of the FP32 normal range
    and the special values; the low 32 bits double as FP32 inputs."""
    rng = np.random.default_rng(11)
    pats = [rng.integers(0, 2**63, size=200_000, dtype=np.int64).astype(np.uint64) * np.uint64(2)
            + rng.integers(0, 2, size=200_000, dtype=np.int64).astype(np.uint64)]
    # FP64 values with exponents across the FP32 normal range and just past
    # it, mantissa bits below FP32 precision set to exactly half (ties), just
    # above / below half, or random
    e = rng.integers(1023 - 128, 1023 + 130, size=50_000).astype(np.uint64)
    m23 = rng.integers(0, 2**23, size=50_000).astype(np.uint64)
    sign = rng.integers(0, 2, size=50_000).astype(np.uint64) << np.uint64(63)
    for low in (np.uint64(1 << 28), np.uint64((1 << 28) + 1), np.uint64((1 << 28) - 1), np.uint64(0),
                rng.integers(0, 2**29, size=50_000).astype(np.uint64)):
        pats.append(sign | (e << np.uint64(52)) | (m23 << np.uint64(29)) | low)
    specials = np.array([0.0, -0.0, np.inf, -np.inf, np.nan, 1.0, -1.0, 3.4028234663852886e38,
                         3.4028235677973366e38, 3.4028236e38, 1.1754943508222875e-38, 1.1754942e-38,
                         1.401298464324817e-45, 7e-46, 1e-300, 1e300, 2.0 ** -126, 2.0 ** -149, 2.0 ** 128],
                        dtype=np.float64)
    pats.append(specials.view(np.uint64))
    f32 = np.array([0.0, -0.0, np.inf, np.nan, 1e-40, -1e-45, 3.4e38, 1.0], dtype=np.float32).view(np.uint32)
    pats.append(f32.astype(np.uint64))
    return np.concatenate(pats)


def test_integer_pipe_conversions_match_hardware(ctx):
    # the solver converts FP64 <-> FP32 with bit operations (GB300 runs F2F at
    # the FP64 rate); both directions must equal the hardware conversions
    import ctypes as C
    pats = _conversion_patterns()
    dev = torch.as_tensor(pats.view(np.int64)).cuda()
    bad = C.c_ulonglong(0)
    st = ctx._lib.nlsp_check_conversions(ctx.h, C.c_void_p(dev.data_ptr()), dev.numel(), C.byref(bad))
    assert st == 0
    assert bad.value == 0
