"""Pins for the finite-element workload generator (Appendix, "FEM Dataset
Generation"): the mesher returns a Delaunay triangulation of the jittered
point cloud, and the P1 matrices have the properties that fix them (textbook
facts about linear finite elements), so that the sparse-operator parity tests
run on the matrices the paper describes."""
import numpy as np
import pytest
import scipy.sparse as sp

from paper_2601_20174_gb300 import fem


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_mesh_is_a_delaunay_triangulation(seed):
    N = 7
    p, tri = fem.mesh(N, seed)
    n = p.shape[0]
    # counter-clockwise, non-degenerate, covering the unit square exactly
    area2 = fem.orient(p, tri[:, 0], tri[:, 1], tri[:, 2])
    assert np.all(area2 > 0)
    assert abs(0.5 * area2.sum() - 1.0) <= 1e-12
    # a triangulation of a convex polygon with 4N hull vertices has 2n - 4N - 2 triangles
    assert tri.shape[0] == 2 * n - 4 * N - 2
    # every edge is shared by at most two triangles, hull edges by one
    e = np.sort(np.concatenate([tri[:, [0, 1]], tri[:, [1, 2]], tri[:, [2, 0]]]), axis=1)
    _, cnt = np.unique(e[:, 0] * n + e[:, 1], return_counts=True)
    assert cnt.max() == 2 and np.sum(cnt == 1) == 4 * N
    # empty circumcircles, by brute force over all points
    for t in tri:
        others = np.setdiff1d(np.arange(n), t)
        v = fem.incircle(p, np.full(others.size, t[0]), np.full(others.size, t[1]), np.full(others.size, t[2]),
                         others)
        assert np.all(v <= 1e-14)


def test_mesh_matches_library_delaunay():
    spatial = pytest.importorskip("scipy.spatial")
    p, tri = fem.mesh(12, 5)
    ref = spatial.Delaunay(p).simplices
    key = lambda T: set(map(tuple, np.sort(T, axis=1)))
    assert key(tri) == key(ref)


def test_jitter_bounds():
    N = 16
    p = fem.jittered_points(N, 4)
    g = fem.jittered_points(N, 4, jitter=0.0)
    h = 1.0 / N
    d = np.minimum(np.minimum(g[:, 0], 1 - g[:, 0]), np.minimum(g[:, 1], 1 - g[:, 1]))
    lim = np.minimum(0.35 * h, 0.49 * d)
    assert np.all(np.abs(p - g) <= lim[:, None] + 1e-15)
    assert np.all(p[d == 0] == g[d == 0])
    assert np.abs(p - g).max() > 0.3 * h  # the draws reach the bound


def _assembled(N, seed, jitter=0.35, kappa=None, tensor=None):
    p, tri = fem.mesh(N, seed, jitter)
    if kappa is None and tensor is None:
        kappa = np.ones(tri.shape[0])
    r, c, kv, mv = fem.stiffness_mass(p, tri, kappa=kappa, tensor=tensor)
    n = p.shape[0]
    K = sp.csr_matrix((kv, (r, c)), shape=(n, n))
    M = sp.csr_matrix((mv, (r, c)), shape=(n, n))
    return p, tri, K, M


def test_p1_stiffness_patch_test_and_kernel():
    p, tri, K, _ = _assembled(10, 3)
    Kd = K.toarray()
    assert np.allclose(Kd, Kd.T, atol=1e-13)
    assert np.max(np.abs(Kd.sum(axis=1))) <= 1e-12          # constants are in the kernel
    assert np.linalg.eigvalsh(Kd).min() >= -1e-12           # positive semidefinite
    interior = ~fem.boundary_mask(10)
    for u in (p[:, 0], p[:, 1], 2 * p[:, 0] - 3 * p[:, 1]):  # linear functions: zero at interior rows
        assert np.max(np.abs((Kd @ u)[interior])) <= 1e-12
    # energy of a linear function = area x |grad|^2
    u = 2 * p[:, 0] - 3 * p[:, 1]
    assert abs(u @ Kd @ u - 13.0) <= 1e-11


def test_p1_on_the_plain_grid_is_the_five_point_stencil():
    N = 8
    _, _, K, _ = _assembled(N, 0, jitter=0.0)
    Kd = K.toarray()
    M = N + 1
    for j in range(1, N):
        for i in range(1, N):
            r = j * M + i
            row = np.zeros(M * M)
            row[r] = 4.0
            row[[r - 1, r + 1, r - M, r + M]] = -1.0
            assert np.allclose(Kd[r], row, atol=1e-12)


def test_p1_mass_matrix():
    p, tri, _, M = _assembled(9, 2)
    Md = M.toarray()
    assert abs(Md.sum() - 1.0) <= 1e-12                       # integral of 1 over the square
    x = p[:, 0]
    assert abs(x @ Md @ np.ones(p.shape[0]) - 0.5) <= 1e-12   # integral of x
    assert abs(x @ Md @ x - 1.0 / 3.0) <= 1e-12               # integral of x^2 (exact for P1 x)
    assert np.linalg.eigvalsh(Md).min() > 0


def test_tensor_coefficient_reduces_to_scalar():
    p, tri = fem.mesh(6, 1)
    kap = np.exp(np.random.default_rng(0).standard_normal(tri.shape[0]))
    r, c, k1, _ = fem.stiffness_mass(p, tri, kappa=kap)
    _, _, k2, _ = fem.stiffness_mass(p, tri, tensor=kap[:, None, None] * np.eye(2)[None])
    assert np.allclose(k1, k2, rtol=1e-13, atol=1e-13)


@pytest.mark.parametrize("family", fem.FAMILIES)
def test_family_matrices_are_spd_with_dirichlet_rows(family):
    N = 10
    pr = fem.fem_problem(family, N=N, k=8, K=16, seed=3)
    A = sp.csr_matrix((pr.data, pr.indices, pr.indptr), shape=(pr.n, pr.n)).toarray()
    assert pr.n == (N + 1) ** 2
    assert np.max(np.abs(A - A.T)) <= 1e-12 * np.max(np.abs(A))
    assert np.linalg.eigvalsh(A).min() > 0
    b = fem.boundary_mask(N)
    assert np.all(A[b][:, b] == np.eye(b.sum())) and np.all(A[b][:, ~b] == 0)
    assert np.all(pr.f[b] == 0)
    # sampled scalars inside the paper's ranges
    if family == "screened_poisson":
        assert 1.0 <= pr.params["alpha"] <= 100.0
    if family == "heat":
        assert 1e-2 <= pr.params["dt"] <= 1.0
    if family == "wave":
        assert 100.0 <= pr.params["c"] <= 1000.0 and 1.0 / N <= pr.params["dt"] <= 2.0 / N
