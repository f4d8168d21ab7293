"""Finite-element workloads for the general sparse operator (host side, numpy).

The paper's own test matrices are P1 finite-element matrices on jittered
Delaunay meshes of the unit square (Appendix, "FEM Dataset Generation"): an
(N+1) x (N+1) point cloud with spacing h = 1/N whose interior vertices move by
U([-eps_i, eps_i]^2), eps_i = min(0.35 h, 0.49 d_i) (d_i the distance to the
boundary), a Delaunay triangulation with near-degenerate triangles removed,
P1 stiffness and mass matrices assembled triangle by triangle, and homogeneous
Dirichlet conditions imposed by zeroing the boundary rows and columns and
putting one on their diagonal (n = (N+1)^2).  Five families (Appendix,
Diffusion ... Wave equation):

  diffusion   K(kappa), kappa_T = exp(N(0, 1.5^2)) per triangle
  anisotropic K(K_T), K_T = R(theta_T) diag(10^3, 1) R(theta_T)^T, theta_T ~ U(0, pi)
  screened    K(kappa) + alpha M, kappa_T = exp(N(0, 1)), alpha = 10^U(0, 2)
  heat        M + dt K(kappa), kappa_T = exp(N(0, 1)), dt = 10^U[-2, 0]
  wave        M + (c dt)^2 K(kappa), kappa_T = exp(N(0, 1.5^2)), c = 10^U[2, 3],
              dt ~ U[h, 2h]

This module generates problems (meshes, coefficients, matrices as CSR, right-
hand sides, random test vectors); it holds none of the method's arithmetic
(Algorithm 1, PCG).  Random draws come from the counter-based streams of
`inputs` (SplitMix64 + Box-Muller).  Everything is vectorised so that meshes of
millions of vertices build in seconds.

The Delaunay triangulation is computed here: start from the grid's cells, each
split along the diagonal that the empty-circumcircle test prefers (the other
one when only one keeps both triangles positively oriented), then flip every
interior edge whose opposite vertex lies inside the neighbouring circumcircle
(Lawson's algorithm), in rounds of non-conflicting flips, until no such edge
is left.  Lawson's flips end at the Delaunay triangulation for points in
general position (de Berg, Cheong, van Kreveld, Overmars, "Computational
Geometry", Thm. 9.8 and Sec. 9.1).
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np

from . import inputs as gen

STREAM_MESH = 8      # vertex jitter (two uniforms per vertex)
STREAM_TRI = 9       # per-triangle coefficient draws
STREAM_FAMILY = 10   # per-instance scalars (alpha, dt, c)

FAMILIES = ("diffusion", "anisotropic", "screened_poisson", "heat", "wave")


# ----------------------------------------------------------------------------
# mesh
# ----------------------------------------------------------------------------
def jittered_points(N: int, seed: int, jitter: float = 0.35) -> np.ndarray:
    """The (N+1)^2 vertices, index j*(N+1) + i for grid point (i/N, j/N);
    boundary vertices fixed, interior ones jittered by U([-eps, eps]^2) with
    eps = min(jitter h, 0.49 d) (d = distance to the boundary; the paper's
    jitter is 0.35, and 0 gives the plain grid)."""
    h = 1.0 / N
    j, i = np.meshgrid(np.arange(N + 1), np.arange(N + 1), indexing="ij")
    x = (i * h).ravel()
    y = (j * h).ravel()
    d = np.minimum(np.minimum(x, 1.0 - x), np.minimum(y, 1.0 - y))
    eps = np.minimum(jitter * h, 0.49 * d)
    u = gen.uniform(seed, STREAM_MESH, 2 * x.size, -1.0, 1.0).reshape(x.size, 2)
    interior = d > 0
    pts = np.stack([x, y], axis=1)
    pts[interior] += eps[interior, None] * u[interior]
    return pts


def orient(p: np.ndarray, a, b, c) -> np.ndarray:
    """Twice the signed area of triangles (a, b, c) (positive: counter-clockwise)."""
    return ((p[b, 0] - p[a, 0]) * (p[c, 1] - p[a, 1]) - (p[b, 1] - p[a, 1]) * (p[c, 0] - p[a, 0]))


def incircle(p: np.ndarray, a, b, c, d) -> np.ndarray:
    """Positive when d lies inside the circumcircle of the counter-clockwise
    triangle (a, b, c) (the classical 3 x 3 lifted determinant)."""
    ax, ay = p[a, 0] - p[d, 0], p[a, 1] - p[d, 1]
    bx, by = p[b, 0] - p[d, 0], p[b, 1] - p[d, 1]
    cx, cy = p[c, 0] - p[d, 0], p[c, 1] - p[d, 1]
    return ((ax * ax + ay * ay) * (bx * cy - by * cx) - (bx * bx + by * by) * (ax * cy - ay * cx)
            + (cx * cx + cy * cy) * (ax * by - ay * bx))


def _grid_triangles(p: np.ndarray, N: int) -> np.ndarray:
    """Each cell split into two counter-clockwise triangles along one diagonal."""
    M = N + 1
    j, i = np.meshgrid(np.arange(N), np.arange(N), indexing="ij")
    v00 = (j * M + i).ravel()
    v10 = v00 + 1
    v01 = v00 + M
    v11 = v01 + 1
    # diagonal v00-v11: (v00, v10, v11), (v00, v11, v01); diagonal v10-v01:
    # (v00, v10, v01), (v10, v11, v01)
    okA = (orient(p, v00, v10, v11) > 0) & (orient(p, v00, v11, v01) > 0)
    okB = (orient(p, v00, v10, v01) > 0) & (orient(p, v10, v11, v01) > 0)
    preferA = incircle(p, v00, v10, v11, v01) <= 0  # v01 outside circle(v00, v10, v11)
    useA = okA & (preferA | ~okB)
    t1 = np.where(useA[:, None], np.stack([v00, v10, v11], 1), np.stack([v00, v10, v01], 1))
    t2 = np.where(useA[:, None], np.stack([v00, v11, v01], 1), np.stack([v10, v11, v01], 1))
    return np.concatenate([t1, t2], axis=0)


def _interior_edges(tri: np.ndarray, n: int):
    """Edges shared by two triangles: (t1, t2, local edge index in t1, in t2).
    Local edge e of a triangle joins its vertices e and (e+1) % 3."""
    T = tri.shape[0]
    a = tri
    b = np.roll(tri, -1, axis=1)
    lo = np.minimum(a, b).ravel().astype(np.int64)
    hi = np.maximum(a, b).ravel().astype(np.int64)
    key = lo * n + hi
    order = np.argsort(key, kind="stable")
    ks = key[order]
    same = np.nonzero(ks[1:] == ks[:-1])[0]
    e1, e2 = order[same], order[same + 1]
    return e1 // 3, e2 // 3, e1 % 3, e2 % 3


def delaunay_grid(p: np.ndarray, N: int, max_rounds: int = 200) -> np.ndarray:
    """Delaunay triangulation of the jittered grid points by Lawson flips
    (counter-clockwise triangles, int64 (T, 3))."""
    n = p.shape[0]
    tri = _grid_triangles(p, N).astype(np.int64)
    for _ in range(max_rounds):
        t1, t2, l1, l2 = _interior_edges(tri, n)
        a = tri[t1, l1]
        b = tri[t1, (l1 + 1) % 3]
        c = tri[t1, (l1 + 2) % 3]          # opposite vertex in t1
        d = tri[t2, (l2 + 2) % 3]          # opposite vertex in t2
        bad = incircle(p, a, b, c, d) > 0
        if not bad.any():
            return tri
        idx = np.nonzero(bad)[0]
        # one flip per triangle per round: an edge is taken when it is the
        # lowest-numbered bad edge of both its triangles
        claim = np.full(tri.shape[0], np.iinfo(np.int64).max, dtype=np.int64)
        np.minimum.at(claim, t1[idx], idx)
        np.minimum.at(claim, t2[idx], idx)
        take = idx[(claim[t1[idx]] == idx) & (claim[t2[idx]] == idx)]
        # t1 = (a, b, c), t2 = (b, a, d); the quad a, d, b, c is convex when d
        # is inside circle(a, b, c), and the flipped pair is (a, d, c), (d, b, c)
        tri[t1[take]] = np.stack([a[take], d[take], c[take]], 1)
        tri[t2[take]] = np.stack([d[take], b[take], c[take]], 1)
    raise RuntimeError("Lawson flips did not finish")


def mesh(N: int, seed: int, jitter: float = 0.35):
    """(points, triangles) of one instance; triangles whose area is below
    1e-12 h^2 are dropped."""
    p = jittered_points(N, seed, jitter)
    tri = delaunay_grid(p, N)
    area2 = orient(p, tri[:, 0], tri[:, 1], tri[:, 2])
    keep = area2 > 2e-12 / (N * N)
    return p, tri[keep]


# ----------------------------------------------------------------------------
# P1 assembly
# ----------------------------------------------------------------------------
def _gradients(p: np.ndarray, tri: np.ndarray):
    """Areas |T| and the constant gradients of the three P1 basis functions of
    every triangle, shape (T, 3, 2): grad phi_a = perp(x_c - x_b) / (2|T|)
    rotated so that it points from the opposite edge towards vertex a."""
    x = p[tri]                                   # (T, 3, 2)
    area2 = orient(p, tri[:, 0], tri[:, 1], tri[:, 2])
    g = np.empty_like(x)
    for a in range(3):
        b, c = (a + 1) % 3, (a + 2) % 3
        e = x[:, c] - x[:, b]                    # edge opposite vertex a
        g[:, a, 0] = -e[:, 1] / area2
        g[:, a, 1] = e[:, 0] / area2
    return 0.5 * area2, g


def _csr_from_triplets(n: int, rows, cols, vals):
    """Sums repeated (row, col) pairs; rows sorted by column."""
    key = rows.astype(np.int64) * n + cols.astype(np.int64)
    order = np.argsort(key, kind="stable")
    key, vals = key[order], vals[order]
    start = np.concatenate([[True], key[1:] != key[:-1]])
    uk = key[start]
    uv = np.add.reduceat(vals, np.nonzero(start)[0])
    r = uk // n
    c = uk % n
    indptr = np.zeros(n + 1, dtype=np.int64)
    np.add.at(indptr, r + 1, 1)
    return np.cumsum(indptr), c.astype(np.int32), uv


def stiffness_mass(p: np.ndarray, tri: np.ndarray, kappa=None, tensor=None):
    """Element contributions (rows, cols, stiffness values, mass values) of
    K(kappa) or K(tensor) (|T| g_a^T K_T g_b) and of M (|T|/12 (1 + [a = b]))."""
    area, g = _gradients(p, tri)
    if tensor is not None:
        Kg = np.einsum("tij,tbj->tbi", tensor, g)             # K_T g_b
        loc = area[:, None, None] * np.einsum("tai,tbi->tab", g, Kg)
    else:
        loc = (area * kappa)[:, None, None] * np.einsum("tai,tbi->tab", g, g)
    mloc = (area / 12.0)[:, None, None] * (np.ones((3, 3)) + np.eye(3))[None]
    rows = np.repeat(tri, 3, axis=1).ravel()
    cols = np.tile(tri, (1, 3)).ravel()
    return rows, cols, loc.ravel(), mloc.ravel()


def dirichlet(n: int, rows, cols, vals, boundary: np.ndarray):
    """Zeroes the boundary rows and columns and puts one on their diagonal."""
    keep = ~(boundary[rows] | boundary[cols])
    b = np.nonzero(boundary)[0]
    return (np.concatenate([rows[keep], b]), np.concatenate([cols[keep], b]),
            np.concatenate([vals[keep], np.ones(b.size)]))


@dataclasses.dataclass
class FemProblem:
    """One FEM system A u = f (CSR) with its setup parameters."""
    name: str
    N: int
    points: np.ndarray
    triangles: np.ndarray
    indptr: np.ndarray
    indices: np.ndarray
    data: np.ndarray
    params: dict
    k: int
    K: int
    s1: int = 20
    omega: float = 2.0 / 3.0
    nu: int = 2
    tol: float = 1e-8
    m: int = 1
    seed: int = 0
    f: np.ndarray | None = None
    S0: np.ndarray | None = None

    @property
    def n(self) -> int:
        return self.points.shape[0]

    @property
    def nnz(self) -> int:
        return int(self.indices.size)


def boundary_mask(N: int) -> np.ndarray:
    j, i = np.meshgrid(np.arange(N + 1), np.arange(N + 1), indexing="ij")
    return ((i == 0) | (i == N) | (j == 0) | (j == N)).ravel()


def family_matrix(family: str, p: np.ndarray, tri: np.ndarray, N: int, seed: int):
    """CSR (indptr, indices, data) of one family's matrix and its sampled
    parameters (Appendix, the five equations)."""
    T = tri.shape[0]
    h = 1.0 / N
    sc = gen.uniform(seed, STREAM_FAMILY, 2)
    params: dict = {}
    if family == "anisotropic":
        theta = gen.uniform(seed, STREAM_TRI, T, 0.0, math.pi)
        c, s = np.cos(theta), np.sin(theta)
        R = np.stack([np.stack([c, -s], 1), np.stack([s, c], 1)], 1)      # (T, 2, 2)
        D = np.diag([1.0e3, 1.0])
        tensor = np.einsum("tij,jk,tlk->til", R, D, R)
        rows, cols, kv, mv = stiffness_mass(p, tri, tensor=tensor)
        vals = kv
    else:
        sigma = 1.5 if family in ("diffusion", "wave") else 1.0
        kappa = np.exp(sigma * gen.normal(seed, STREAM_TRI, T))
        rows, cols, kv, mv = stiffness_mass(p, tri, kappa=kappa)
        if family == "diffusion":
            vals = kv
        elif family == "screened_poisson":
            alpha = 10.0 ** (2.0 * sc[0])
            params["alpha"] = alpha
            vals = kv + alpha * mv
        elif family == "heat":
            dt = 10.0 ** (-2.0 + 2.0 * sc[0])
            params["dt"] = dt
            vals = mv + dt * kv
        elif family == "wave":
            cw = 10.0 ** (2.0 + sc[0])
            dt = h * (1.0 + sc[1])
            params.update(c=cw, dt=dt)
            vals = mv + (cw * dt) ** 2 * kv
        else:
            raise ValueError(f"unknown family {family}")
    n = p.shape[0]
    rows, cols, vals = dirichlet(n, rows, cols, vals, boundary_mask(N))
    indptr, indices, data = _csr_from_triplets(n, rows, cols, vals)
    return indptr, indices, data, params


def fem_problem(family: str, N: int = 64, k: int = 48, K: int = 72, seed: int = 0, tol: float = 1e-6,
                nu: int = 5, omega: float = 0.66, s1: int = 20, m: int = 1, with_samples: bool = True) -> FemProblem:
    """One instance of a family on an N x N jittered Delaunay mesh.  The
    defaults are the paper's two-grid evaluation (Sec. 4: N = 64, K = 72,
    coarse dimension 48, tolerance 1e-6, nu1 = nu2 = 5, omega = 0.66); the
    number of test-vector sweeps s1 is not stated there and is 20 here.
    f ~ U[-1, 1] at the interior vertices and 0 on the boundary."""
    p, tri = mesh(N, seed)
    indptr, indices, data, params = family_matrix(family, p, tri, N, seed)
    prob = FemProblem(f"fem_{family}", N, p, tri, indptr, indices, data, params, k, K, s1=s1, omega=omega, nu=nu,
                      tol=tol, m=m, seed=seed)
    n = prob.n
    f = gen.rhs_uniform(n, m, seed)
    f[boundary_mask(N)] = 0.0
    prob.f = f
    if with_samples:
        prob.S0 = gen.samples_normal(n, K, seed)
    return prob
