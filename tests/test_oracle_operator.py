"""Pins for oracle.operator: closed-form spectra, brute-force quadratic forms
and exactness on polynomials (PDE discretisation of Eq. discretized_pde)."""
import itertools
import math

import numpy as np
import pytest

from oracle import operator as op
from paper_2601_20174_gb300 import inputs as gen


def _sine_mode_2d(N, p, q):
    h = 1.0 / (N + 1)
    x = (np.arange(N) + 1) * h
    return np.outer(np.sin(q * math.pi * x), np.sin(p * math.pi * x)).ravel()  # [j, i]


@pytest.mark.parametrize("N", [5, 8])
def test_poisson_sine_eigenpairs(N):
    # Textbook: the 5-point Dirichlet Laplacian has eigenvectors
    # sin(p pi x_i) sin(q pi y_j), eigenvalues (4/h^2)(sin^2(p pi h/2) + sin^2(q pi h/2)).
    A = op.diffusion_5pt(N, np.ones((N + 1, N + 1)))
    h = 1.0 / (N + 1)
    for p, q in [(1, 1), (2, 3), (N, 1), (N, N)]:
        v = _sine_mode_2d(N, p, q)
        lam = 4.0 / h ** 2 * (math.sin(p * math.pi * h / 2) ** 2 + math.sin(q * math.pi * h / 2) ** 2)
        assert np.allclose(A @ v, lam * v, rtol=0, atol=1e-10 * lam)


def test_poisson_entries():
    N = 4
    A = op.diffusion_5pt(N, np.ones((N + 1, N + 1))).toarray()
    h2 = (N + 1) ** 2
    ref = np.zeros((N * N, N * N))
    for j, i in itertools.product(range(N), range(N)):
        ref[j * N + i, j * N + i] = 4 * h2
        for di, dj in [(1, 0), (-1, 0), (0, 1), (0, -1)]:
            if 0 <= i + di < N and 0 <= j + dj < N:
                ref[j * N + i, (j + dj) * N + i + di] = -h2
    assert np.array_equal(A, ref)


def _brute_quadratic_form_2d(N, kappa, u):
    # u^T A u = h^-2 sum over grid edges of a_e (u_a - u_b)^2 with u = 0 on the
    # boundary, a_e the mean kappa of the two cells that share the edge,
    # found from the edge midpoint's coordinates (independent of the index
    # bookkeeping in the oracle).
    h = 1.0 / (N + 1)
    U = np.zeros((N + 2, N + 2))  # full grid incl. boundary, [y, x] node indices 0..N+1
    U[1:-1, 1:-1] = u.reshape(N, N)
    total = 0.0
    for y in range(N + 2):
        for x in range(N + 2):
            for dx, dy in [(1, 0), (0, 1)]:
                x2, y2 = x + dx, y + dy
                if x2 > N + 1 or y2 > N + 1:
                    continue
                if (x in (0, N + 1) and x2 in (0, N + 1) and dx == 0) or (y in (0, N + 1) and y2 in (0, N + 1) and dy == 0):
                    continue  # edge on the boundary itself: both ends zero
                mx, my = (x + x2) / 2 * h, (y + y2) / 2 * h
                cells = []
                for ox, oy in ([(0, 0.5 * h), (0, -0.5 * h)] if dx else [(0.5 * h, 0), (-0.5 * h, 0)]):
                    cx, cy = mx + ox, my + oy
                    if 0 < cx < 1 and 0 < cy < 1:
                        cells.append(kappa[int(cy / h), int(cx / h)])
                a = sum(cells) / 2.0
                total += a * (U[y, x] - U[y2, x2]) ** 2
    return total / h ** 2


def test_variable_kappa_quadratic_form():
    N = 5
    kap = np.exp(gen.iid_log_kappa((N + 1, N + 1), seed=3))
    A = op.diffusion_5pt(N, kap)
    rng = np.random.default_rng(0)
    for _ in range(3):
        u = rng.standard_normal(N * N)
        assert math.isclose(u @ (A @ u), _brute_quadratic_form_2d(N, kap, u), rel_tol=1e-12)
    assert abs(A - A.T).max() == 0.0


def test_kappa_scaling_reduces_to_poisson():
    N = 6
    A1 = op.diffusion_5pt(N, np.ones((N + 1, N + 1)))
    A3 = op.diffusion_5pt(N, 3.0 * np.ones((N + 1, N + 1)))
    assert abs(A3 - 3.0 * A1).max() < 1e-9


def test_9pt_exact_on_quadratics():
    # -(axx u_xx + 2 axy u_xy + ayy u_yy) is exact for quadratics at nodes whose
    # whole 3x3 neighbourhood is interior.
    N = 9
    t = gen.rotated_aniso_tensor(0.7, 1e-3)
    A = op.aniso_9pt(N, t)
    h = 1.0 / (N + 1)
    X, Y = np.meshgrid((np.arange(N) + 1) * h, (np.arange(N) + 1) * h)  # [j, i]
    inner = np.zeros((N, N), bool)
    inner[1:-1, 1:-1] = True
    for u, want in [(X ** 2, -2 * t[0]), (Y ** 2, -2 * t[1]), (X * Y, -2 * t[2])]:
        got = (A @ u.ravel()).reshape(N, N)[inner]
        assert np.allclose(got, want, rtol=1e-9, atol=1e-9)


@pytest.mark.parametrize("theta", [0.1, 1.2, 2.9])
def test_9pt_spd(theta):
    A = op.aniso_9pt(12, gen.rotated_aniso_tensor(theta, 1e-3)).toarray()
    assert np.array_equal(A, A.T)
    np.linalg.cholesky(A)


def test_7pt_sine_eigenpairs_and_quadratic_form():
    N = 4
    A1 = op.diffusion_7pt(N, np.ones((N + 1,) * 3))
    h = 1.0 / (N + 1)
    x = (np.arange(N) + 1) * h
    for p, q, s in [(1, 1, 1), (2, 1, 3), (4, 4, 2)]:
        v = np.einsum("l,j,i->lji", np.sin(s * math.pi * x), np.sin(q * math.pi * x),
                      np.sin(p * math.pi * x)).ravel()
        lam = 4 / h ** 2 * sum(math.sin(t * math.pi * h / 2) ** 2 for t in (p, q, s))
        assert np.allclose(A1 @ v, lam * v, atol=1e-9 * lam)
    # variable kappa: quadratic form by brute force over the 3 edge directions
    kap = np.exp(gen.iid_log_kappa((N + 1,) * 3, seed=5))
    A = op.diffusion_7pt(N, kap)
    u = np.random.default_rng(1).standard_normal(N ** 3)
    U = np.zeros((N + 2,) * 3)
    U[1:-1, 1:-1, 1:-1] = u.reshape(N, N, N)
    tot = 0.0
    for l, j, i in itertools.product(range(N + 2), repeat=3):
        for d in range(3):
            o = [0, 0, 0]
            o[d] = 1
            l2, j2, i2 = l + o[0], j + o[1], i + o[2]
            if max(l2, j2, i2) > N + 1:
                continue
            # the four cells around the edge: along the edge direction the cell
            # index is the lower node index; across it, both neighbours
            ranges = []
            for dd, c in zip(range(3), (l, j, i)):
                ranges.append([c] if dd == d else [c - 1, c])
            cells = [kap[a, b, cc] for a in ranges[0] for b in ranges[1] for cc in ranges[2]
                     if 0 <= a <= N and 0 <= b <= N and 0 <= cc <= N]
            if len(cells) < 4:
                continue  # an edge lying in the boundary surface: both ends zero
            tot += np.mean(cells) * (U[l, j, i] - U[l2, j2, i2]) ** 2
    assert math.isclose(u @ (A @ u), tot / h ** 2, rel_tol=1e-12)
