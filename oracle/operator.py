"""Oracle: the SPD system matrix A of the stencil PDE families, as explicit CSR.

Test infrastructure only (see the package docstring).

A is assembled entry by entry from the finite-difference definitions below,
never through the CUDA path's matrix-free indexing.  Boundary (Dirichlet,
Eq. generalized_pde) nodes are eliminated: an edge or stencil arm that reaches
the boundary contributes to the diagonal only (5/7-point) or is dropped
(9-point off-diagonal arms).

Pins (tests/test_oracle_operator.py): sine-mode eigenpairs of the constant
5-point Laplacian (closed form); kappa = 1 reduces the variable form to the
constant one; symmetry; positive definiteness by dense Cholesky; the 9-point
stencil applied to quadratics reproduces -div(K grad u) exactly.
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp


def _csr(n, rows, cols, vals):
    return sp.csr_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))),
                         shape=(n, n))


def _edge_terms(a, ia, ib, rows, cols, vals):
    """Adds a (e_a - e_b)(e_a - e_b)^T for each edge; ia/ib = -1 marks a
    boundary endpoint (its row and column are eliminated)."""
    ka = ia >= 0
    kb = ib >= 0
    rows += [ia[ka], ib[kb]]
    cols += [ia[ka], ib[kb]]
    vals += [a[ka], a[kb]]
    both = ka & kb
    rows += [ia[both], ib[both]]
    cols += [ib[both], ia[both]]
    vals += [-a[both], -a[both]]


def diffusion_5pt(N: int, kappa: np.ndarray) -> sp.csr_matrix:
    """2D -div(kappa grad u), 5-point, cell kappa of shape (N+1, N+1) [cj, ci].

    The x-edge between node columns i-1 and i (i = 0..N) of node row j lies in
    cell column i between cell rows j and j+1: weight 1/2 (kappa[j,i] +
    kappa[j+1,i]).  The y-edge between node rows j-1 and j of node column i
    lies in cell row j between cell columns i and i+1: weight 1/2
    (kappa[j,i] + kappa[j,i+1]).  A = h^-2 sum_e a_e (e_a - e_b)(e_a - e_b)^T.
    """
    h2 = float(N + 1) ** 2
    n = N * N
    rows, cols, vals = [], [], []
    j, i = np.meshgrid(np.arange(N), np.arange(N + 1), indexing="ij")  # x-edges
    a = 0.5 * (kappa[j, i] + kappa[j + 1, i]) * h2
    ia = np.where(i - 1 >= 0, j * N + (i - 1), -1)
    ib = np.where(i <= N - 1, j * N + i, -1)
    _edge_terms(a.ravel(), ia.ravel(), ib.ravel(), rows, cols, vals)
    j, i = np.meshgrid(np.arange(N + 1), np.arange(N), indexing="ij")  # y-edges
    a = 0.5 * (kappa[j, i] + kappa[j, i + 1]) * h2
    ia = np.where(j - 1 >= 0, (j - 1) * N + i, -1)
    ib = np.where(j <= N - 1, j * N + i, -1)
    _edge_terms(a.ravel(), ia.ravel(), ib.ravel(), rows, cols, vals)
    return _csr(n, rows, cols, vals)


def diffusion_7pt(N: int, kappa: np.ndarray) -> sp.csr_matrix:
    """3D -div(kappa grad u), 7-point, cell kappa of shape (N+1,)*3 [cl, cj, ci].

    Each edge's weight is the mean of the four cells around it; e.g. the
    x-edge between node columns i-1 and i at node (j, l) uses cells
    (ci=i, cj in {j, j+1}, cl in {l, l+1}).
    """
    h2 = float(N + 1) ** 2
    n = N ** 3
    rows, cols, vals = [], [], []
    k = kappa
    # x-edges: index grid (l, j, i), i = 0..N
    l, j, i = np.meshgrid(np.arange(N), np.arange(N), np.arange(N + 1), indexing="ij")
    a = 0.25 * (k[l, j, i] + k[l, j + 1, i] + k[l + 1, j, i] + k[l + 1, j + 1, i]) * h2
    base = (l * N + j) * N
    ia = np.where(i - 1 >= 0, base + i - 1, -1)
    ib = np.where(i <= N - 1, base + i, -1)
    _edge_terms(a.ravel(), ia.ravel(), ib.ravel(), rows, cols, vals)
    # y-edges: (l, j, i), j = 0..N
    l, j, i = np.meshgrid(np.arange(N), np.arange(N + 1), np.arange(N), indexing="ij")
    a = 0.25 * (k[l, j, i] + k[l, j, i + 1] + k[l + 1, j, i] + k[l + 1, j, i + 1]) * h2
    ia = np.where(j - 1 >= 0, (l * N + j - 1) * N + i, -1)
    ib = np.where(j <= N - 1, (l * N + j) * N + i, -1)
    _edge_terms(a.ravel(), ia.ravel(), ib.ravel(), rows, cols, vals)
    # z-edges: (l, j, i), l = 0..N
    l, j, i = np.meshgrid(np.arange(N + 1), np.arange(N), np.arange(N), indexing="ij")
    a = 0.25 * (k[l, j, i] + k[l, j, i + 1] + k[l, j + 1, i] + k[l, j + 1, i + 1]) * h2
    ia = np.where(l - 1 >= 0, ((l - 1) * N + j) * N + i, -1)
    ib = np.where(l <= N - 1, (l * N + j) * N + i, -1)
    _edge_terms(a.ravel(), ia.ravel(), ib.ravel(), rows, cols, vals)
    return _csr(n, rows, cols, vals)


def aniso_9pt(N: int, tensor: np.ndarray) -> sp.csr_matrix:
    """2D -(a_xx u_xx + 2 a_xy u_xy + a_yy u_yy), constant tensor, 9-point.

    Second differences for u_xx, u_yy and the centred cross difference
    u_xy ~ (u[i+1,j+1] - u[i+1,j-1] - u[i-1,j+1] + u[i-1,j-1]) / (4h^2):
    centre 2(a_xx + a_yy)/h^2, E/W -a_xx/h^2, N/S -a_yy/h^2,
    NE/SW -a_xy/(2h^2), NW/SE +a_xy/(2h^2).  Arms reaching the boundary drop.
    """
    axx, ayy, axy = (float(t) for t in tensor)
    h2 = float(N + 1) ** 2
    n = N * N
    arms = [((0, 0), 2.0 * (axx + ayy)),
            ((1, 0), -axx), ((-1, 0), -axx),
            ((0, 1), -ayy), ((0, -1), -ayy),
            ((1, 1), -0.5 * axy), ((-1, -1), -0.5 * axy),
            ((-1, 1), 0.5 * axy), ((1, -1), 0.5 * axy)]
    j, i = np.meshgrid(np.arange(N), np.arange(N), indexing="ij")
    rows, cols, vals = [], [], []
    for (di, dj), w in arms:
        ii, jj = i + di, j + dj
        ok = (ii >= 0) & (ii < N) & (jj >= 0) & (jj < N)
        rows.append((j * N + i)[ok])
        cols.append((jj * N + ii)[ok])
        vals.append(np.full(int(ok.sum()), w * h2))
    return _csr(n, rows, cols, vals)


def assemble(problem) -> sp.csr_matrix:
    """A for an `inputs.Problem` (dispatch on dimension, points and layout)."""
    if problem.dim == 2 and problem.points == 5 and problem.layout == 0:
        return diffusion_5pt(problem.N, np.asarray(problem.coeffs, dtype=np.float64))
    if problem.dim == 2 and problem.points == 9 and problem.layout == 1:
        return aniso_9pt(problem.N, np.asarray(problem.coeffs, dtype=np.float64))
    if problem.dim == 3 and problem.points == 7 and problem.layout == 0:
        return diffusion_7pt(problem.N, np.asarray(problem.coeffs, dtype=np.float64))
    raise ValueError(f"unsupported stencil: dim={problem.dim} points={problem.points} "
                     f"layout={problem.layout}")
