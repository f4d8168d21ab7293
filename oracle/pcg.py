"""Oracle: preconditioned conjugate gradient with the two-level preconditioner
(Sec. 4, "Two-grid Solver Evaluation"; Hestenes-Stiefel CG), FP64.

Test infrastructure only (see the package docstring).

Readings of the paper (it gives only "PCG, relative residual tolerance,
maximum iteration cap"):
  * x0 = 0; relative residual ||r||_2 / ||b||_2 of the recursively updated
    residual decides the stop; the true residual ||b - A x|| / ||b|| is
    recomputed at exit and reported.
  * the iteration count is the number of products A p taken until the stop
    test passes (0 for b = 0).
  * standard beta = r_new^T z_new / r_old^T z_old; the flexible variant
    (used for preconditioners applied in reduced precision, which are not
    exactly fixed linear SPD maps) uses Polak-Ribiere
    beta = r_new^T (z_new - z_old) / r_old^T z_old.
  * several right-hand sides run independent recurrences; a converged column
    is frozen.
  * breakdown (p^T A p <= 0, r^T z <= 0 or a non-finite scalar) stops the
    column with status "breakdown".

Pins (tests/test_oracle_pcg.py): exact solutions of tiny grids against a
dense solve; one iteration when k = n (B = A^-1); iteration counts within the
CG bound ceil(sqrt(kappa(BA))/2 ln(2/tol)) with kappa(BA) from the closed-form
Poisson spectrum; A-orthogonality of successive search directions.  Block CG:
one column reproduces pcg's iterates; the block space contains every
column's Krylov space, so no column needs more iterations than its own PCG
(A-norm error minimised over a larger space); dependent and zero columns are
deflated (x of 2b is 2x of b); exact solutions of tiny grids.
"""
from __future__ import annotations

import numpy as np

from . import prec as _prec


def pcg(A, apply_B, b: np.ndarray, tol: float, maxit: int = 2000, flexible: bool = False):
    """Single right-hand side. apply_B(r) -> z.  Returns dict with x, iters,
    relres (recursive), true_relres, status ('converged' | 'maxit' |
    'breakdown'), history (recursive relres after each iteration)."""
    b = np.asarray(b, dtype=np.float64)
    n = b.shape[0]
    x = np.zeros(n)
    bn = float(np.linalg.norm(b))
    if bn == 0.0:
        return {"x": x, "iters": 0, "relres": 0.0, "true_relres": 0.0, "status": "converged",
                "history": []}
    r = b.copy()
    z = apply_B(r)
    p = z.copy()
    rz = float(r @ z)
    hist = []
    status = "maxit"
    it = 0
    while it < maxit:
        if not np.isfinite(rz) or rz <= 0.0:
            status = "breakdown"
            break
        q = A @ p
        pq = float(p @ q)
        it += 1
        if not np.isfinite(pq) or pq <= 0.0:
            status = "breakdown"
            break
        alpha = rz / pq
        x = x + alpha * p
        r = r - alpha * q
        rel = float(np.linalg.norm(r)) / bn
        hist.append(rel)
        if rel <= tol:
            status = "converged"
            break
        zn = apply_B(r)
        if flexible:
            beta = float(r @ (zn - z)) / rz
        else:
            beta = float(r @ zn) / rz
        rz = float(r @ zn)
        p = zn + beta * p
        z = zn
    true_rel = float(np.linalg.norm(b - A @ x)) / bn
    return {"x": x, "iters": it, "relres": hist[-1] if hist else 1.0, "true_relres": true_rel,
            "status": status, "history": hist}


def pcg_multi(A, apply_B, B: np.ndarray, tol: float, maxit: int = 2000, flexible: bool = False):
    """Independent recurrences per column of the n x m block B."""
    B = np.asarray(B, dtype=np.float64)
    if B.ndim == 1:
        B = B[:, None]
    res = [pcg(A, apply_B, B[:, j], tol, maxit, flexible) for j in range(B.shape[1])]
    X = np.stack([r["x"] for r in res], axis=1)
    return X, res


def two_level_solver(A, P, L, omega: float, nu1: int, nu2: int):
    """Returns apply_B for the two-level preconditioner of Algorithm 1."""
    return lambda r: _prec.apply(A, P, L, r, omega, nu1, nu2)


def solve_problem(problem, A=None, setup=None, maxit: int = 2000, flexible: bool = False):
    """Setup + PCG for an `inputs.Problem` (all columns of its f)."""
    from . import operator as _op, setup as _setup
    if A is None:
        A = _op.assemble(problem)
    if setup is None:
        setup = _setup.build(A, problem.S0, problem.k, problem.omega, problem.s1)
    apply_B = two_level_solver(A, setup["P"], setup["L"], problem.omega, problem.nu, problem.nu)
    X, res = pcg_multi(A, apply_B, problem.f, problem.tol, maxit, flexible)
    return {"A": A, "setup": setup, "X": X, "results": res}


def _orth_pivoted(W: np.ndarray, drop: float) -> np.ndarray:
    """Orthonormal basis of range(W) by a Cholesky factorisation of W^T W with
    diagonal pivoting (largest remaining diagonal first), stopping when the
    largest remaining pivot is below `drop` times the largest diagonal; the
    kept columns, in pivot order, times L^-T."""
    G = W.T @ W
    m = G.shape[0]
    perm = list(range(m))
    L = np.zeros((m, m))
    G = G.copy()
    dmax0 = max(float(np.max(np.diag(G))) if m else 0.0, 0.0)
    s = 0
    for j in range(m):
        q = j + int(np.argmax(np.diag(G)[j:]))
        d = G[q, q]
        if not (d > drop * dmax0) or not np.isfinite(d):
            break
        if q != j:
            G[[j, q], :] = G[[q, j], :]
            G[:, [j, q]] = G[:, [q, j]]
            L[[j, q], :j] = L[[q, j], :j]
            perm[j], perm[q] = perm[q], perm[j]
        L[j, j] = np.sqrt(G[j, j])
        L[j + 1:, j] = G[j + 1:, j] / L[j, j]
        G[j + 1:, j + 1:] -= np.outer(L[j + 1:, j], L[j + 1:, j])
        s = j + 1
    if s == 0:
        return np.zeros((W.shape[0], 0))
    Ls = L[:s, :s]
    return W[:, perm[:s]] @ np.linalg.inv(Ls).T


def block_cg(A, apply_B, B: np.ndarray, tol: float, maxit: int = 2000, drop: float = 1e-14):
    """Breakdown-free block conjugate gradient (Ji & Li 2017, after O'Leary
    1980): the m columns share one search space; every iteration the search
    block is re-orthonormalised and rank-deflated (_orth_pivoted).  Not part
    of the paper (its PCG is per right-hand side); the block-Krylov variant.
    Returns (X, iterations per column (the iteration at which the column
    first met ||r_c|| <= tol ||b_c||, maxit + 1 if never), true relative
    residual per column)."""
    B = np.asarray(B, dtype=np.float64)
    n, m = B.shape
    X = np.zeros((n, m))
    R = B.copy()
    bn = np.linalg.norm(B, axis=0)
    done = bn == 0.0
    iters = np.where(done, 0, maxit + 1)
    P = _orth_pivoted(apply_B(R), drop)
    for t in range(1, maxit + 1):
        if done.all() or P.shape[1] == 0:
            break
        Q = A @ P
        D = P.T @ Q
        Lc = np.linalg.cholesky(0.5 * (D + D.T))
        alpha = np.linalg.solve(Lc.T, np.linalg.solve(Lc, P.T @ R))
        X = X + P @ alpha
        R = R - Q @ alpha
        rn = np.linalg.norm(R, axis=0)
        newly = (~done) & (rn <= tol * bn)
        iters[newly] = t
        done = done | newly
        if done.all():
            break
        Z = apply_B(R)
        beta = -np.linalg.solve(Lc.T, np.linalg.solve(Lc, Q.T @ Z))
        P = _orth_pivoted(Z + P @ beta, drop)
    true = np.linalg.norm(B - A @ X, axis=0) / np.where(bn > 0, bn, 1.0)
    return X, iters, true
