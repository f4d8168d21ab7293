"""Python interface over the nlsp C ABI, taking and returning torch CUDA
tensors.  PyTorch provides device memory and the stream; every computation is
a call into libnlsp.so.

Vectors are float64 tensors of shape (n,) or blocks of shape (n, m); they are
handed to the library as column-major storage (a block is stored as its
transpose, contiguous).
"""
from __future__ import annotations

import ctypes as C
from dataclasses import dataclass

import torch

from . import _lib as L


def _ptr(t: torch.Tensor) -> C.c_void_p:
    return C.c_void_p(t.data_ptr())


def _colmajor(X: torch.Tensor, n: int) -> tuple[torch.Tensor, int]:
    """Returns (storage tensor of shape (m, n) contiguous, m)."""
    if X.dtype != torch.float64 or not X.is_cuda:
        raise TypeError("expected a CUDA float64 tensor")
    if X.dim() == 1:
        if X.shape[0] != n:
            raise ValueError(f"length {X.shape[0]} != n = {n}")
        return X.contiguous().view(1, n), 1
    if X.dim() != 2 or X.shape[0] != n:
        raise ValueError(f"expected shape (n, m) with n = {n}, got {tuple(X.shape)}")
    return X.t().contiguous(), X.shape[1]


def _out_like(store: torch.Tensor, one_d: bool) -> torch.Tensor:
    return store.view(-1) if one_d else store.t()


class Context:
    """A library context on one CUDA device, enqueueing on a torch stream."""

    def __init__(self, device: int = 0, stream: torch.cuda.Stream | None = None):
        self._lib = L.load()
        self.device = device
        self.stream = stream or torch.cuda.current_stream(device)
        h = C.c_void_p()
        L.check(self._lib.nlsp_create(C.byref(h), device, C.c_void_p(self.stream.cuda_stream)), "nlsp_create")
        self.h = h

    def set_stream(self, stream: torch.cuda.Stream):
        self.stream = stream
        L.check(self._lib.nlsp_set_stream(self.h, C.c_void_p(stream.cuda_stream)), "nlsp_set_stream")

    def close(self):
        if getattr(self, "h", None):
            self._lib.nlsp_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Operator:
    """SPD operator A: a structured-grid stencil (nlsp_assemble_stencil) or a
    general sparse matrix (Operator.from_csr, nlsp_assemble_csr)."""

    def __init__(self, ctx: Context, dim: int, N: int, points: int, coeffs: torch.Tensor, layout: int):
        self.ctx = ctx
        self.dim, self.N, self.points, self.layout = dim, N, points, layout
        coeffs = coeffs.to(device=f"cuda:{ctx.device}", dtype=torch.float64).contiguous()
        grid = (C.c_int64 * 3)(N, N, N if dim == 3 else 1)
        h = C.c_void_p()
        L.check(ctx._lib.nlsp_assemble_stencil(ctx.h, dim, grid, points, _ptr(coeffs), layout, C.byref(h)),
                "nlsp_assemble_stencil")
        self.h = h
        self.n = int(ctx._lib.nlsp_op_size(h))

    @classmethod
    def from_csr(cls, ctx: Context, rowptr: torch.Tensor, col: torch.Tensor, val: torch.Tensor) -> "Operator":
        """From compressed sparse rows: rowptr (n + 1) int64, col (nnz) int32,
        val (nnz) float64; copied to the context's device if needed."""
        dev = f"cuda:{ctx.device}"
        rp = rowptr.to(device=dev, dtype=torch.int64).contiguous()
        cc = col.to(device=dev, dtype=torch.int32).contiguous()
        vv = val.to(device=dev, dtype=torch.float64).contiguous()
        n, nnz = rp.numel() - 1, cc.numel()
        if vv.numel() != nnz:
            raise ValueError("col and val must have the same length")
        h = C.c_void_p()
        L.check(ctx._lib.nlsp_assemble_csr(ctx.h, n, nnz, _ptr(rp), _ptr(cc), _ptr(vv), C.byref(h)),
                "nlsp_assemble_csr")
        self = cls.__new__(cls)
        self.ctx = ctx
        self.dim, self.N, self.points, self.layout = 0, 0, 0, -1
        self.h = h
        self.n = int(ctx._lib.nlsp_op_size(h))
        return self

    @classmethod
    def from_problem(cls, ctx: Context, problem) -> "Operator":
        """From an inputs.Problem (its coefficients are uploaded)."""
        coeffs = torch.as_tensor(problem.coeffs, dtype=torch.float64).reshape(-1)
        return cls(ctx, problem.dim, problem.N, problem.points, coeffs.cuda(ctx.device), problem.layout)

    def apply(self, X: torch.Tensor) -> torch.Tensor:
        store, m = _colmajor(X, self.n)
        out = torch.empty_like(store)
        L.check(self.ctx._lib.nlsp_op_apply(self.ctx.h, self.h, m, _ptr(store), self.n, _ptr(out), self.n),
                "nlsp_op_apply")
        return _out_like(out, X.dim() == 1)

    def diagonal(self) -> torch.Tensor:
        d = torch.empty(self.n, dtype=torch.float64, device=f"cuda:{self.ctx.device}")
        L.check(self.ctx._lib.nlsp_op_diagonal(self.ctx.h, self.h, _ptr(d)), "nlsp_op_diagonal")
        return d

    def smooth_samples(self, S0: torch.Tensor, s1: int, omega: float, precision: int = L.NLSP_FP64) -> torch.Tensor:
        store, K = _colmajor(S0, self.n)
        out = torch.empty_like(store)
        L.check(self.ctx._lib.nlsp_smooth_samples(self.ctx.h, self.h, K, s1, omega, precision, _ptr(store),
                                                   _ptr(out)), "nlsp_smooth_samples")
        return out.t()

    def close(self):
        if getattr(self, "h", None):
            self.ctx._lib.nlsp_free_op(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


@dataclass
class SolveResult:
    iterations: int
    status: int
    relres: float
    true_relres: float


class Preconditioner:
    """Two-level preconditioner (nlsp_build_prolongation / nlsp_prec_from_basis)."""

    def __init__(self, op: Operator, handle: C.c_void_p):
        self.op = op
        self.ctx = op.ctx
        self.h = handle
        n, k, r, K, prec = C.c_int64(), C.c_int(), C.c_int(), C.c_int(), C.c_int()
        L.check(self.ctx._lib.nlsp_prec_dims(handle, C.byref(n), C.byref(k), C.byref(r), C.byref(K),
                                             C.byref(prec)), "nlsp_prec_dims")
        self.n, self.k, self.K, self.precision = n.value, k.value, K.value, prec.value
        self.r = r.value

    @staticmethod
    def _params(k, K, s1, nu, omega, precision, seed=0):
        return L.SetupParams(K=K, k=k, s1=s1, nu1=nu, nu2=nu, omega=omega, precision=precision, seed=seed)

    @classmethod
    def build(cls, op: Operator, S0: torch.Tensor | None, k: int, s1: int = 20, nu: int = 2,
              omega: float = 2.0 / 3.0, precision: int = L.NLSP_FP64, K: int | None = None,
              seed: int = 0, a_weighted: bool = False) -> "Preconditioner":
        """S0: n x K random test vectors, or None to draw them on the device
        (K columns, counter-based generator under `seed`).  a_weighted: the
        A-orthonormal basis of nlsp_build_prolongation_a_weighted."""
        if S0 is None:
            if K is None:
                raise ValueError("K is required when S0 is drawn on the device")
            store, ptr = None, C.c_void_p(0)
        else:
            store, K = _colmajor(S0, op.n)
            ptr = _ptr(store)
        p = cls._params(k, K, s1, nu, omega, precision, seed)
        h = C.c_void_p()
        name = "nlsp_build_prolongation_a_weighted" if a_weighted else "nlsp_build_prolongation"
        L.check(getattr(op.ctx._lib, name)(op.ctx.h, op.h, C.byref(p), ptr, C.byref(h)), name)
        return cls(op, h)

    @classmethod
    def build_randomized(cls, op: Operator, S0: torch.Tensor | None, k: int, oversample: int = 10,
                         power_iters: int = 2, sketch: torch.Tensor | None = None, s1: int = 20, nu: int = 2,
                         omega: float = 2.0 / 3.0, precision: int = L.NLSP_FP64, K: int | None = None,
                         seed: int = 0) -> "Preconditioner":
        """Randomised-SVD basis (nlsp_build_prolongation_randomized).  sketch:
        the K x (k + oversample) Gaussian test matrix, or None to draw it on
        the device from `seed`."""
        if S0 is None:
            if K is None:
                raise ValueError("K is required when S0 is drawn on the device")
            ptr = C.c_void_p(0)
        else:
            store, K = _colmajor(S0, op.n)
            ptr = _ptr(store)
        sk = C.c_void_p(0)
        if sketch is not None:
            sks, _ = _colmajor(sketch, K)
            sk = _ptr(sks)
        p = cls._params(k, K, s1, nu, omega, precision, seed)
        h = C.c_void_p()
        L.check(op.ctx._lib.nlsp_build_prolongation_randomized(op.ctx.h, op.h, C.byref(p), ptr, oversample,
                                                                power_iters, sk, C.byref(h)),
                "nlsp_build_prolongation_randomized")
        return cls(op, h)

    @classmethod
    def from_basis(cls, op: Operator, P: torch.Tensor, nu: int = 2, omega: float = 2.0 / 3.0,
                   precision: int = L.NLSP_FP64) -> "Preconditioner":
        store, k = _colmajor(P, op.n)
        p = cls._params(k, 0, 0, nu, omega, precision)
        h = C.c_void_p()
        L.check(op.ctx._lib.nlsp_prec_from_basis(op.ctx.h, op.h, C.byref(p), _ptr(store), k, C.byref(h)),
                "nlsp_prec_from_basis")
        return cls(op, h)

    def factor(self, r: int):
        L.check(self.ctx._lib.nlsp_factor_coarse(self.ctx.h, self.op.h, self.h, r), "nlsp_factor_coarse")
        self.r = r

    def basis(self) -> torch.Tensor:
        out = torch.empty(self.k, self.n, dtype=torch.float64, device=f"cuda:{self.ctx.device}")
        L.check(self.ctx._lib.nlsp_prec_copy_basis(self.ctx.h, self.h, _ptr(out)), "nlsp_prec_copy_basis")
        return out.t()

    def sigma(self) -> torch.Tensor:
        out = torch.zeros(max(self.K, 1), dtype=torch.float64, device=f"cuda:{self.ctx.device}")
        L.check(self.ctx._lib.nlsp_prec_copy_sigma(self.ctx.h, self.h, _ptr(out)), "nlsp_prec_copy_sigma")
        return out[: self.K]

    def coarse(self) -> tuple[torch.Tensor, torch.Tensor]:
        r = self.r
        Ac = torch.empty(r, r, dtype=torch.float64, device=f"cuda:{self.ctx.device}")
        Lf = torch.empty(r, r, dtype=torch.float64, device=f"cuda:{self.ctx.device}")
        L.check(self.ctx._lib.nlsp_prec_copy_coarse(self.ctx.h, self.h, _ptr(Ac), _ptr(Lf)), "nlsp_prec_copy_coarse")
        return Ac.t(), Lf.t()  # stored column-major

    def apply(self, R: torch.Tensor) -> torch.Tensor:
        store, m = _colmajor(R, self.n)
        out = torch.empty_like(store)
        L.check(self.ctx._lib.nlsp_apply_prec(self.ctx.h, self.h, m, _ptr(store), self.n, _ptr(out), self.n),
                "nlsp_apply_prec")
        return _out_like(out, R.dim() == 1)

    def solve(self, B: torch.Tensor, tol: float = 1e-8, maxit: int = 2000, flexible: int = -1,
              graph_mode: int = 1):
        """PCG for A X = B (x0 = 0).  Returns (X, [SolveResult per column])."""
        store, m = _colmajor(B, self.n)
        out = torch.empty_like(store)
        infos = (L.SolveInfo * m)()
        prm = L.SolveParams(tol=tol, maxit=maxit, flexible=flexible, graph_mode=graph_mode)
        st = self.ctx._lib.nlsp_solve(self.ctx.h, self.op.h, self.h, m, _ptr(store), self.n, _ptr(out), self.n,
                                      C.byref(prm), infos)
        L.check(st, "nlsp_solve", allow=(L.NLSP_OK, L.NLSP_NOT_CONVERGED, L.NLSP_ERR_BREAKDOWN))
        res = [SolveResult(i.iterations, i.status, i.relres, i.true_relres) for i in infos]
        return _out_like(out, B.dim() == 1), res

    def solve_block(self, B: torch.Tensor, tol: float = 1e-8, maxit: int = 2000, flexible: int = -1):
        """Block PCG for A X = B with up to 32 columns advanced together
        (nlsp_solve_block).  Returns (X, [SolveResult per column])."""
        store, m = _colmajor(B, self.n)
        out = torch.empty_like(store)
        infos = (L.SolveInfo * m)()
        prm = L.SolveParams(tol=tol, maxit=maxit, flexible=flexible, graph_mode=0)
        st = self.ctx._lib.nlsp_solve_block(self.ctx.h, self.op.h, self.h, m, _ptr(store), self.n, _ptr(out),
                                            self.n, C.byref(prm), infos)
        L.check(st, "nlsp_solve_block", allow=(L.NLSP_OK, L.NLSP_NOT_CONVERGED, L.NLSP_ERR_BREAKDOWN))
        res = [SolveResult(i.iterations, i.status, i.relres, i.true_relres) for i in infos]
        return _out_like(out, B.dim() == 1), res

    def solve_block_cg(self, B: torch.Tensor, tol: float = 1e-8, maxit: int = 2000):
        """Breakdown-free block CG for A X = B, up to 32 columns sharing one
        search space (nlsp_solve_block_cg).  Returns (X, [SolveResult per column])."""
        store, m = _colmajor(B, self.n)
        out = torch.empty_like(store)
        infos = (L.SolveInfo * m)()
        prm = L.SolveParams(tol=tol, maxit=maxit, flexible=0, graph_mode=0)
        st = self.ctx._lib.nlsp_solve_block_cg(self.ctx.h, self.op.h, self.h, m, _ptr(store), self.n, _ptr(out),
                                               self.n, C.byref(prm), infos)
        L.check(st, "nlsp_solve_block_cg", allow=(L.NLSP_OK, L.NLSP_NOT_CONVERGED, L.NLSP_ERR_BREAKDOWN))
        res = [SolveResult(i.iterations, i.status, i.relres, i.true_relres) for i in infos]
        return _out_like(out, B.dim() == 1), res

    def close(self):
        if getattr(self, "h", None):
            self.ctx._lib.nlsp_free_prec(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def solve_batched(precs: list[Preconditioner], bs: list[torch.Tensor], tol: float = 1e-8, maxit: int = 2000,
                  flexible: int = -1, tiles_per_cta: int = 0):
    """Solves A_i x_i = b_i for every instance in one launch of the persistent
    solver (nlsp_solve_batched).  precs: distinct preconditioners of one
    context, one stencil kind and one precision; bs: float64 CUDA vectors of
    length n_i.  Returns ([x_i], [SolveResult per instance])."""
    count = len(precs)
    if len(bs) != count:
        raise ValueError("one right-hand side per preconditioner")
    if count == 0:
        return [], []
    ctx = precs[0].ctx
    bvec = [b.contiguous() for b in bs]
    for M, b in zip(precs, bvec):
        if b.dtype != torch.float64 or not b.is_cuda or b.dim() != 1 or b.shape[0] != M.n:
            raise ValueError("each b_i must be a float64 CUDA vector of length n_i")
    xs = [torch.empty_like(b) for b in bvec]
    hp = (C.c_void_p * count)(*[M.h.value for M in precs])
    hb = (C.c_void_p * count)(*[b.data_ptr() for b in bvec])
    hx = (C.c_void_p * count)(*[x.data_ptr() for x in xs])
    infos = (L.SolveInfo * count)()
    prm = L.SolveParams(tol=tol, maxit=maxit, flexible=flexible, graph_mode=2)
    st = ctx._lib.nlsp_solve_batched(ctx.h, count, hp, hb, hx, C.byref(prm), tiles_per_cta, infos)
    L.check(st, "nlsp_solve_batched", allow=(L.NLSP_OK, L.NLSP_NOT_CONVERGED, L.NLSP_ERR_BREAKDOWN))
    return xs, [SolveResult(i.iterations, i.status, i.relres, i.true_relres) for i in infos]


def tune_batched(precs: list[Preconditioner], bs: list[torch.Tensor], candidates=(2, 4, 8, 16, 32, 64),
                 tol: float = 1e-8, maxit: int = 2000, flexible: int = -1):
    """Measures nlsp_solve_batched for each candidate tiles_per_cta and lets
    the context remember the fastest for batches of these sizes
    (nlsp_tune_batched; later solve_batched(..., tiles_per_cta=0) uses it).
    Returns (best, {candidate: ms})."""
    count = len(precs)
    ctx = precs[0].ctx
    bvec = [b.contiguous() for b in bs]
    xs = [torch.empty_like(b) for b in bvec]
    hp = (C.c_void_p * count)(*[M.h.value for M in precs])
    hb = (C.c_void_p * count)(*[b.data_ptr() for b in bvec])
    hx = (C.c_void_p * count)(*[x.data_ptr() for x in xs])
    cand = (C.c_int * len(candidates))(*candidates)
    ms = (C.c_double * len(candidates))()
    best = C.c_int()
    prm = L.SolveParams(tol=tol, maxit=maxit, flexible=flexible, graph_mode=2)
    L.check(ctx._lib.nlsp_tune_batched(ctx.h, count, hp, hb, hx, C.byref(prm), cand, len(candidates),
                                       C.byref(best), ms), "nlsp_tune_batched")
    return best.value, {c: m for c, m in zip(candidates, ms)}


def plan_teams(n: list[int], num_ctas: int, tiles_per_cta: int = 0):
    """The batched solver's team plan for instances of n[i] nodes
    (nlsp_plan_teams; host computation).  Returns (first_cta, team_size,
    start) lists."""
    lib = L.load()
    count = len(n)
    hn = (C.c_int64 * count)(*n)
    first = (C.c_int * count)()
    size = (C.c_int * count)()
    start = (C.c_double * count)()
    L.check(lib.nlsp_plan_teams(count, hn, num_ctas, tiles_per_cta, first, size, start), "nlsp_plan_teams")
    return list(first), list(size), list(start)


def subspace_loss(ctx: Context, P_hat: torch.Tensor, B: torch.Tensor, precision: int = L.NLSP_FP64,
                  grad: bool = True):
    """L = ||(I - Q Q^T) B||_F^2 with Q = qf(P_hat) and dL/dP_hat
    (nlsp_subspace_loss).  P_hat (n, k), B (n, K) float64 CUDA.  Returns
    (loss as a Python float, gradient (n, k) or None)."""
    n = P_hat.shape[0]
    ps, k = _colmajor(P_hat, n)
    bs, K = _colmajor(B, n)
    g = torch.empty_like(ps) if grad else None
    out = C.c_double()
    L.check(ctx._lib.nlsp_subspace_loss(ctx.h, n, k, K, precision, _ptr(ps), _ptr(bs), C.byref(out),
                                        _ptr(g) if grad else None), "nlsp_subspace_loss")
    return out.value, (g.t() if grad else None)


def nlss_loss(ctx: Context, P_hat: torch.Tensor, S: torch.Tensor, precision: int = L.NLSP_FP64,
              grad: bool = True):
    """Nested subspace loss (1/k) sum_l (1 - ||Q_{1:l}^T S||^2 / ||S||^2) with
    Q = qf(P_hat) and dL/dP_hat (nlsp_nlss_loss).  P_hat (n, k), S (n, K)
    float64 CUDA.  Returns (loss as a Python float, gradient (n, k) or None)."""
    n = P_hat.shape[0]
    ps, k = _colmajor(P_hat, n)
    ss, K = _colmajor(S, n)
    g = torch.empty_like(ps) if grad else None
    out = C.c_double()
    L.check(ctx._lib.nlsp_nlss_loss(ctx.h, n, k, K, precision, _ptr(ps), _ptr(ss), C.byref(out),
                                    _ptr(g) if grad else None), "nlsp_nlss_loss")
    return out.value, (g.t() if grad else None)


def unrolled_pcg(op: Operator, P: torch.Tensor, b: torch.Tensor, T: int = 10, nu: int = 2,
                 omega: float = 2.0 / 3.0, precision: int = L.NLSP_FP64, grad: bool = True):
    """||r_T|| after T PCG iterations with the two-level preconditioner
    built from P, and its gradient dL/dP (nlsp_unrolled_pcg).  P (n, k),
    b (n,) float64 CUDA.  Returns (loss, gradient (n, k) or None)."""
    ps, k = _colmajor(P, op.n)
    bs, _ = _colmajor(b, op.n)
    g = torch.empty_like(ps) if grad else None
    out = C.c_double()
    L.check(op.ctx._lib.nlsp_unrolled_pcg(op.ctx.h, op.h, _ptr(ps), k, nu, omega, precision, _ptr(bs), T,
                                          C.byref(out), _ptr(g) if grad else None), "nlsp_unrolled_pcg")
    return out.value, (g.t() if grad else None)
