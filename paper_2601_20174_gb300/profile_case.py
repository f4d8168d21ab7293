"""A short run of the benchmark workload for profilers.

Builds the 512 x 512 GRF diffusion system (k = 64 from K = 128 smoothed
samples, nu = 2, omega = 2/3), sets up the preconditioner and runs a few PCG
iterations.  With --mode 0 (default) the iterations use the host-relaunched
iteration graph, so that a profiler sees every kernel as a separate launch;
with --mode 2 and NLSP_PHASE_TIMERS=1 in the environment the persistent
solver's per-phase times are printed (microseconds per iteration).

    python -m paper_2601_20174_gb300.profile_case [--precision mixed|fp64] [--iters 4] [--N 512] [--mode 0|1|2]

With --fem FAMILY a P1 finite-element system of the paper's Appendix (CSR
input) replaces it.

With --block the 2D rotated anisotropic 9-point workload (N^2 nodes, k from K
device-drawn samples, 32 right-hand sides) runs --iters iterations of the
block PCG instead (--precision bf16 / tf32: reduced-precision tensor-core
restriction and prolongation).
"""
from __future__ import annotations

import argparse
import os

import numpy as np
import torch

from . import _lib as L, api, inputs as gen


def main() -> int:
    ap = argparse.ArgumentParser()
    ap.add_argument("--precision", default="mixed", choices=["mixed", "fp64", "bf16", "tf32"])
    ap.add_argument("--iters", type=int, default=4)
    ap.add_argument("--N", type=int, default=512)
    ap.add_argument("--k", type=int, default=64)
    ap.add_argument("--K", type=int, default=128)
    ap.add_argument("--mode", type=int, default=0, choices=[0, 1, 2])
    ap.add_argument("--block", action="store_true", help="block PCG on the anisotropic 9-point workload")
    ap.add_argument("--csr-spmv", action="store_true",
                    help="sparse SpMV (nlsp_op_apply) on the FEM diffusion matrix of an N x N jittered mesh")
    ap.add_argument("--fem", default=None, choices=["diffusion", "anisotropic", "screened_poisson", "heat", "wave"],
                    help="P1 finite-element family on an N x N jittered mesh (k = 48 from K = 72, nu = 5, "
                         "omega = 0.66, tol 1e-6), CSR input, solved with --mode")
    ap.add_argument("--adjoint", action="store_true",
                    help="subspace loss and T=10 unrolled-PCG loss with gradients on the 3D 7-point N^3 workload")
    args = ap.parse_args()
    if args.csr_spmv:
        import ctypes as C
        from . import fem
        pts, tri = fem.mesh(args.N, 0)
        ip, ix, dv, _ = fem.family_matrix("diffusion", pts, tri, args.N, 0)
        ctx = api.Context(0)
        A = api.Operator.from_csr(ctx, torch.as_tensor(ip), torch.as_tensor(ix), torch.as_tensor(dv))
        n = A.n
        x = torch.randn(n, dtype=torch.float64, device="cuda")
        y = torch.empty_like(x)
        for _ in range(args.iters):
            L.check(ctx._lib.nlsp_op_apply(ctx.h, A.h, 1, C.c_void_p(x.data_ptr()), n, C.c_void_p(y.data_ptr()), n),
                    "nlsp_op_apply")
        torch.cuda.synchronize()
        print(f"profile case (csr spmv): n={n} nnz={ix.size} launches={args.iters}")
        A.close()
        ctx.close()
        return 0
    if args.adjoint:
        import ctypes as C
        p = gen.iid_diffusion_3d(args.N, args.k, args.K, seed=0, with_samples=False)
        ctx = api.Context(0)
        A = api.Operator.from_problem(ctx, p)
        prec = L.NLSP_MIXED_FP32 if args.precision == "mixed" else L.NLSP_FP64
        M = api.Preconditioner.build(A, None, args.k, p.s1, p.nu, p.omega, L.NLSP_FP64, K=args.K, seed=p.seed)
        U = M.basis().contiguous()
        S0 = torch.empty(args.K, p.n, dtype=torch.float64, device="cuda")
        L.check(ctx._lib.nlsp_random_normal(ctx.h, p.seed, gen.STREAM_S0, 0, p.n * args.K,
                                            C.c_void_p(S0.data_ptr())), "nlsp_random_normal")
        B = torch.empty_like(S0)
        L.check(ctx._lib.nlsp_smooth_samples(ctx.h, A.h, args.K, p.s1, p.omega, L.NLSP_FP64,
                                             C.c_void_p(S0.data_ptr()), C.c_void_p(B.data_ptr())), "smooth")
        b = torch.as_tensor(p.f[:, 0].copy()).cuda()
        l1, _ = api.subspace_loss(ctx, U, B.t(), prec)
        l2, _ = api.unrolled_pcg(A, U, b, 10, p.nu, p.omega, prec)
        torch.cuda.synchronize()
        print(f"profile case (adjoint): n={p.n} k={args.k} K={args.K} subspace loss={l1:.6e} unrolled loss={l2:.6e}")
        M.close()
        A.close()
        ctx.close()
        return 0
    if args.block:
        p = gen.aniso_9pt_2d(args.N, args.k, args.K, m=32, seed=0, tol=1e-8, with_samples=False)
        ctx = api.Context(0)
        A = api.Operator.from_problem(ctx, p)
        prec = {"mixed": L.NLSP_MIXED_FP32, "fp64": L.NLSP_FP64, "bf16": L.NLSP_MIXED_BF16,
                "tf32": L.NLSP_MIXED_TF32}[args.precision]
        M = api.Preconditioner.build(A, None, args.k, p.s1, p.nu, p.omega, prec, K=args.K, seed=p.seed)
        F = torch.as_tensor(p.f).cuda()
        _, res = M.solve_block(F, tol=1e-8, maxit=args.iters)
        torch.cuda.synchronize()
        print(f"profile case (block): n={p.n} k={args.k} rhs=32 iterations={res[0].iterations} status={res[0].status}")
        M.close()
        A.close()
        ctx.close()
        return 0
    ctx = api.Context(0)
    prec = L.NLSP_MIXED_FP32 if args.precision == "mixed" else L.NLSP_FP64
    if args.fem:
        from . import fem
        p = fem.fem_problem(args.fem, N=args.N, seed=0)
        A = api.Operator.from_csr(ctx, torch.as_tensor(p.indptr), torch.as_tensor(p.indices), torch.as_tensor(p.data))
        tol = p.tol
    else:
        p = gen.grf_diffusion_2d(args.N, args.k, args.K, seed=0)
        A = api.Operator.from_problem(ctx, p)
        tol = 1e-8
    S0 = torch.as_tensor(np.ascontiguousarray(p.S0.T)).cuda()
    M = api.Preconditioner.build(A, S0.t(), p.k, p.s1, p.nu, p.omega, prec)
    f = torch.as_tensor(p.f[:, 0].copy()).cuda()
    _, res = M.solve(f, tol=tol, maxit=args.iters, graph_mode=args.mode)
    torch.cuda.synchronize()
    print(f"profile case: n={p.n} k={p.k} iterations={res[0].iterations} status={res[0].status}")
    if args.mode == 2:
        import ctypes as C
        out = (C.c_double * 31)()
        L.check(ctx._lib.nlsp_prec_phase_times(ctx.h, M.h, out, 31), "nlsp_prec_phase_times")
        if os.environ.get("NLSP_CLUSTER", "1") != "0" and p.n <= 16 * 4096:
            cmarks = ["S1 wait", "update", "S2 wait", "pre sweeps", "rho wait", "rho", "restrict", "c wait",
                      "coarse", "prolong", "post sweeps", "rz wait", "direction"]
            it = max(1, res[0].iterations)
            print("  cluster solver marks (rank 0, us per iteration):")
            for i, name in enumerate(cmarks):
                print(f"  {name:18s} {out[14 + i] / 1e3 / it:8.2f}")
        names = ["spmv", "pre", "stored sweeps", "restrict", "prolong", "post", "other"]
        marks = ["spmv totals", "spmv nodes", "pre totals", "pre nodes", "restrict rho", "restrict resident",
                 "restrict streamed", "restrict reduce", "prolong coarse", "prolong resident", "prolong streamed",
                 "post nodes", "spmv issue", "spmv finish", "restrict stage A", "restrict stage B", "post stage"]
        it = max(1, res[0].iterations)
        for i, name in enumerate(names):
            print(f"  {name:18s} work {out[2 * i] / 1e3 / it:8.2f} us/it   barrier wait {out[2 * i + 1] / 1e3 / it:8.2f} us/it")
        for i, name in enumerate(marks):
            print(f"  mark {name:18s} {out[14 + i] / 1e3 / it:8.2f} us/it")
    M.close()
    A.close()
    ctx.close()
    return 0


if __name__ == "__main__":
    raise SystemExit(main())
