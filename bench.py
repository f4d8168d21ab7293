#!/usr/bin/env python3
"""Benchmark: PCG solves/s to relative residual 1e-8 with the spectral
two-level preconditioner, on one GB300 (or N replicas).

Workload: 2D variable-coefficient diffusion, 5-point, 512 x 512 interior
grid (n = 262144), log kappa a squared-exponential Gaussian random field
(length 0.1, sigma 1), k = 64 from K = 128 Jacobi-smoothed N(0,1) samples
(s1 = 20, omega = 2/3), nu1 = nu2 = 2, one right-hand side f ~ U[-1, 1],
tolerance 1e-8.  Seeded synthetic inputs (no dataset exists for it).

One step = assemble A + build P (smoothing, SVD, Galerkin, Cholesky) + PCG
solve, through the library's public API, with the inputs already resident in
HBM; L2 is flushed (256 MiB write) between timed steps.  The headline runs the
mixed path (FP32 preconditioner, FP64 recurrences); the plain FP64 path and
the solve-only throughput are reported beside it.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "PCG solves/s to rel-res 1e-8 (mixed/batched vs plain FP64); % HBM roofline"
UNIT = "solves/s"
WL = dict(N=512, k=64, K=128, s1=20, nu=2, omega=2.0 / 3.0, tol=1e-8, seed=0)
WORKLOAD_NAME = "grf_diffusion2d_N512_k64_K128_seed0"
WORKLOAD_DESC = ("2D diffusion 5-point 512x512 (n=262144), GRF log-kappa (l=0.1, sigma=1), "
                 "k=64 from K=128 smoothed samples (s1=20, omega=2/3), nu1=nu2=2, 1 RHS U[-1,1], tol 1e-8")
FLUSH_BYTES = 256 << 20


def _profiled_traffic(k: int, iterations: int):
    """DRAM bytes (read + write) of one persistent-solver launch from the
    committed two-point ncu fit (fixed + per-iteration bytes) -- only while
    the kernel source is unchanged since that capture (else None)."""
    import hashlib
    try:
        with open(os.path.join(ROOT, "profiles", "k_pcg_persistent_grf512_k64.json")) as f:
            prof = json.load(f)
        src = open(os.path.join(ROOT, "paper_2601_20174_gb300", "csrc", "pcg_impl.cuh"), "rb").read()
        if hashlib.sha256(src).hexdigest() != prof.get("pcg_impl_sha256") or prof["k"] != k:
            return None
        return prof["dram_bytes_fixed"] + prof["dram_bytes_per_iteration"] * iterations
    except Exception:
        return None


def _peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


# ----------------------------------------------------------------------------
# clocks during the timed region
# ----------------------------------------------------------------------------
class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int | None):
        self.gpu_index = gpu_index
        self.proc = None
        self.path = None

    def start(self):
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            cmd = ["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits", "-lms", "100"]
            if self.gpu_index is not None:
                cmd += ["-i", str(self.gpu_index)]
            self.proc = subprocess.Popen(cmd, stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if not self.proc:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        rows = []
        for line in open(self.path):
            parts = [x.strip() for x in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                rows.append((float(parts[1]), float(parts[2]), parts[5:9]))
            except ValueError:
                continue
        os.unlink(self.path)
        if not rows:
            return None
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for _, _, fl in rows for i, v in enumerate(fl) if v.lower() == "active"})
        return {"sm_mhz": statistics.median(r[0] for r in rows), "sm_max_mhz": max(r[1] for r in rows),
                "reasons": reasons, "samples": len(rows)}


def _gpu_index(torch, dev):
    try:
        uuid = str(torch.cuda.get_device_properties(dev).uuid)
        out = subprocess.run(["nvidia-smi", "--query-gpu=index,uuid", "--format=csv,noheader"], capture_output=True,
                             text=True, timeout=20).stdout
        for line in out.strip().splitlines():
            idx, u = [x.strip() for x in line.split(",")]
            if uuid.replace("GPU-", "") in u:
                return int(idx)
    except Exception:
        pass
    return None


# ----------------------------------------------------------------------------
# CPU baseline: the FP64 oracle on the same workload
# ----------------------------------------------------------------------------
def blas_threads():
    """Threads of the OpenBLAS that numpy loaded (its get_num_threads, found
    through the process's mapped libraries), or None when it cannot be read.
    scipy's sparse products run on one thread whatever this says."""
    import ctypes
    try:
        import numpy  # noqa: F401  (maps the BLAS)
        paths = set()
        for line in open("/proc/self/maps"):
            parts = line.split()
            if len(parts) >= 6 and "blas" in os.path.basename(parts[-1]).lower():
                paths.add(parts[-1])
        for path in sorted(paths):
            lib = ctypes.CDLL(path)
            for name in ("scipy_openblas_get_num_threads64_", "scipy_openblas_get_num_threads",
                         "openblas_get_num_threads64_", "openblas_get_num_threads"):
                fn = getattr(lib, name, None)
                if fn is not None:
                    fn.restype = ctypes.c_int
                    return int(fn())
    except Exception:
        pass
    return None


def oracle_problem(seed: int = 0):
    from paper_2601_20174_gb300 import inputs as gen
    return gen.grf_diffusion_2d(WL["N"], WL["k"], WL["K"], seed=seed, tol=WL["tol"])


def oracle_full_solve(p):
    """Times one complete oracle solve of the workload: assemble A, setup
    (smoothing, SVD, Galerkin, Cholesky) and PCG to the tolerance.  Returns
    (seconds, detail dict)."""
    from oracle import operator as op, pcg, setup as su
    t0 = time.perf_counter()
    A = op.assemble(p)
    st = su.build(A, p.S0, p.k, p.omega, p.s1)
    t1 = time.perf_counter()
    r = pcg.pcg(A, pcg.two_level_solver(A, st["P"], st["L"], p.omega, p.nu, p.nu), p.f[:, 0], p.tol)
    t2 = time.perf_counter()
    return t2 - t0, {"setup_s": round(t1 - t0, 3), "pcg_s": round(t2 - t1, 3), "iterations": r["iters"],
                     "true_relres": r["true_relres"], "status": r["status"]}


def oracle_sample(p, pcg_iters_sample: int = 64):
    """Times the oracle's assemble + setup plus `pcg_iters_sample` PCG
    iterations (a bounded sample of one solve) and scales it to a full solve
    with the oracle's own iteration count for this workload
    (tests/golden/bench_workloads.json, written by an oracle-only script).
    Returns (measured sample seconds, scaled solves/s, detail dict)."""
    from oracle import operator as op, pcg, setup as su
    with open(os.path.join(ROOT, "tests", "golden", "bench_workloads.json")) as f:
        iters_full = json.load(f)[WORKLOAD_NAME]["iters"]
    t0 = time.perf_counter()
    A = op.assemble(p)
    st = su.build(A, p.S0, p.k, p.omega, p.s1)
    t1 = time.perf_counter()
    pcg.pcg(A, pcg.two_level_solver(A, st["P"], st["L"], p.omega, p.nu, p.nu), p.f[:, 0], 0.0,
            maxit=pcg_iters_sample)
    t2 = time.perf_counter()
    per_it = (t2 - t1) / pcg_iters_sample
    total = (t1 - t0) + per_it * iters_full
    return t2 - t0, 1.0 / total, {"setup_s": round(t1 - t0, 3), "pcg_s_per_iter": per_it,
                                  "iters_full": iters_full, "sample_s": round(t2 - t0, 3),
                                  "scaled_solve_s": round(total, 3)}


def run_reference(args):
    """The reference arm: the FP64 oracle, as it stands, on the host cores.
    Each step is a bounded sample (assemble + setup + 64 PCG iterations of
    the workload), timed; `value` scales the measured samples to solves/s with
    the oracle's iteration count, and `ms_per_step` is the measured wall time
    of one sample step.  Rank 0 only."""
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return 0
    p = oracle_problem()
    for _ in range(args.warmup):
        oracle_sample(p, pcg_iters_sample=4)
    walls, totals, det = [], [], None
    t0 = time.perf_counter()
    for _ in range(args.steps):
        w, v, det = oracle_sample(p)
        walls.append(w)
        totals.append(1.0 / v)
    wall = time.perf_counter() - t0
    value = 1.0 / statistics.median(totals)
    threads = blas_threads()
    sample = (f"per step: oracle assemble + setup (smoothing, numpy SVD, Galerkin, Cholesky) + 64 of the "
              f"oracle's {det['iters_full']} PCG iterations, timed; value = 1 / (setup + 64-iteration time x "
              f"{det['iters_full']}/64), median over steps; ms_per_step = measured sample wall time")
    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": 1000.0 * statistics.mean(walls), "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic", "impl": "reference",
            "config": {"workload": WORKLOAD_DESC, "impl": "FP64 CPU oracle (numpy/scipy)"},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": threads or os.cpu_count(), "kind": "oracle",
                             "sample": sample, "blas_threads": threads, "sparse_threads": 1,
                             "host_cpus": os.cpu_count(), "detail": det},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
            "wall_s": round(wall, 1)}
    print(json.dumps(line))
    return 0


# ----------------------------------------------------------------------------
# replicas (N > 1): each rank solves its own seeded instance; the only
# collective is the max of the ranks' timed totals
# ----------------------------------------------------------------------------
def replica_seed(base_seed: int, rank: int) -> int:
    """Instance seed of a rank: independent problems, no data-path exchange."""
    return base_seed + rank


def max_over_ranks(total_ms: float, world: int, device) -> float:
    """The slowest rank's timed total (all-reduce MAX; identity for one rank)."""
    if world <= 1:
        return total_ms
    import torch
    import torch.distributed as dist
    t = torch.tensor([total_ms], device=device, dtype=torch.float64)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def whole_job_rate(world: int, steps: int, total_ms: float) -> float:
    """Units processed by all ranks per second of the slowest rank."""
    return world * steps / (total_ms / 1000.0)


# ----------------------------------------------------------------------------
# our arm
# ----------------------------------------------------------------------------
BATCH = dict(count=256, seed=0, tol=1e-8, tiles_per_cta=(2, 4, 8, 16, 32, 64))
BATCH_DESC = ("256 2D diffusion 5-point instances, sides drawn from {64,128,192,256,384,512}, log-kappa i.i.d. "
              "N(0,1) per cell, ranks k from {16,32,64}, K = 2k device-drawn samples (s1=20, omega=2/3), nu=2, "
              "1 RHS U[-1,1] each, tol 1e-8, FP32 preconditioner / FP64 PCG")


DIFF = dict(N=64, k=64, K=128, s1=20, nu=2, omega=2.0 / 3.0, T=10, seed=0, noise=0.1)
DIFF_DESC = ("3D diffusion 7-point 64^3 (n=262144), log-kappa i.i.d. N(0,1) per cell, k=64, K=128 smoothed "
             "device-drawn samples; subspace loss ||(I-QQ^T)B||^2 and nested loss (1/k) sum_l (1 - "
             "||Q_1:l^T B||^2/||B||^2) at P_hat = SVD basis + N(0,0.1^2) noise, and "
             "||r_T|| after T=10 unrolled PCG steps (nu=2, omega=2/3) at the SVD basis; FP32 arithmetic, "
             "gradients by the library's reverse sweep")


def run_differentiation(ctx, dev, timed):
    """Loss + gradient of both objectives on the 64^3 problem (FP32), with
    the FP64 results beside them for the error of the FP32 production path."""
    import statistics as st
    import ctypes as C

    import torch

    from paper_2601_20174_gb300 import _lib as L, api, inputs as gen

    p = gen.iid_diffusion_3d(DIFF["N"], DIFF["k"], DIFF["K"], seed=DIFF["seed"], with_samples=False)
    n, k, K = p.n, DIFF["k"], DIFF["K"]
    A = api.Operator(ctx, 3, p.N, 7, torch.as_tensor(p.coeffs.reshape(-1)).to(dev), L.NLSP_COEF_CELL_KAPPA)
    S0 = torch.empty(K, n, dtype=torch.float64, device=dev)
    L.check(ctx._lib.nlsp_random_normal(ctx.h, p.seed, gen.STREAM_S0, 0, n * K, C.c_void_p(S0.data_ptr())),
            "nlsp_random_normal")
    B = torch.empty_like(S0)
    L.check(ctx._lib.nlsp_smooth_samples(ctx.h, A.h, K, DIFF["s1"], DIFF["omega"], L.NLSP_FP64,
                                         C.c_void_p(S0.data_ptr()), C.c_void_p(B.data_ptr())), "smooth")
    M = api.Preconditioner.build(A, None, k, DIFF["s1"], DIFF["nu"], DIFF["omega"], L.NLSP_FP64, K=K, seed=p.seed)
    U = M.basis().contiguous()
    noise = torch.empty(k, n, dtype=torch.float64, device=dev)
    L.check(ctx._lib.nlsp_random_normal(ctx.h, p.seed, gen.STREAM_NOISE, 0, n * k, C.c_void_p(noise.data_ptr())),
            "nlsp_random_normal")
    Ph = U + DIFF["noise"] * noise.t()
    Bt = B.t()
    b = torch.as_tensor(p.f[:, 0].copy()).to(dev)
    out = {"workload": DIFF_DESC}
    for name, fn in (("subspace", lambda prec: api.subspace_loss(ctx, Ph, Bt, prec)),
                     ("nlss", lambda prec: api.nlss_loss(ctx, Ph, Bt, prec)),
                     ("unrolled_pcg", lambda prec: api.unrolled_pcg(A, U, b, DIFF["T"], DIFF["nu"], DIFF["omega"],
                                                                     prec))):
        fn(L.NLSP_MIXED_FP32)  # warm
        ms, (l32, g32) = timed(lambda: fn(L.NLSP_MIXED_FP32), 3)
        l64, g64 = fn(L.NLSP_FP64)
        out[name] = {"ms_loss_and_grad": st.median(ms), "loss_fp32": l32, "loss_fp64": l64,
                     "grad_rel_err_fp32_vs_fp64": float(torch.linalg.norm(g32 - g64) / torch.linalg.norm(g64))}
        if name != "nlss":  # NLSS depends on the order of Q's columns, not on the range alone
            out[name]["range_invariance"] = float(torch.linalg.norm(Ph.t() @ g64 if name == "subspace" else U.t() @ g64)
                                                  / torch.linalg.norm(g64))
    # algorithmic bytes of the subspace pass: FP64 inputs read, FP32 tiled
    # copies written and read by the two products and the gradient pass,
    # gradient written (FP64)
    sub_bytes = n * (k + K) * 8 + n * (k + K) * 4 * 3 + n * k * 8
    out["subspace"]["algorithmic_bytes"] = sub_bytes
    out["subspace"]["achieved_gbs"] = sub_bytes / (out["subspace"]["ms_loss_and_grad"] / 1e3) / 1e9
    M.close()
    A.close()
    return out


SMALL = dict(N=32, k=16, K=64, s1=20, nu=2, omega=2.0 / 3.0, tol=1e-10, seed=0, reps=20)
SMALL_DESC = ("2D Poisson 5-point 32x32 interior (n=1024), k=16 from K=64 N(0,1) samples smoothed 20x "
              "(omega=2/3), nu=2, 1 RHS U[-1,1], plain FP64 to tol 1e-10")


def run_small(ctx, dev, timed):
    """The plain-FP64 32 x 32 Poisson configuration: microseconds per solve
    (assemble + build P + factor + PCG, and the PCG alone).  Its whole
    working set (~0.6 MB) stays on chip, so no HBM fraction is stated."""
    import statistics as st

    import numpy as np
    import torch

    from paper_2601_20174_gb300 import _lib as L, api, inputs as gen

    p = gen.poisson_2d(SMALL["N"], SMALL["k"], SMALL["K"], seed=SMALL["seed"], tol=SMALL["tol"])
    kap = torch.as_tensor(np.asarray(p.coeffs, dtype=np.float64).reshape(-1)).to(dev)
    S0 = torch.as_tensor(np.ascontiguousarray(p.S0.T)).to(dev)
    f = torch.as_tensor(p.f[:, 0].copy()).to(dev)

    def step():
        A = api.Operator(ctx, p.dim, p.N, p.points, kap, p.layout)
        M = api.Preconditioner.build(A, S0.t(), SMALL["k"], SMALL["s1"], SMALL["nu"], SMALL["omega"], L.NLSP_FP64)
        x, res = M.solve(f, tol=SMALL["tol"], graph_mode=2)
        return A, M, x, res[0]

    for _ in range(3):
        step()
    ms, (A, M, x, info) = timed(step, SMALL["reps"])
    M.solve(f, tol=SMALL["tol"], graph_mode=2)
    ms_s, _ = timed(lambda: M.solve(f, tol=SMALL["tol"], graph_mode=2), SMALL["reps"])
    out = {"workload": SMALL_DESC, "value": 1e3 / st.mean(ms), "unit": "solves/s",
           "us_per_solve": 1e3 * st.mean(ms), "solve_only_us": 1e3 * st.mean(ms_s),
           "iterations": info.iterations, "true_relres": info.true_relres, "converged": info.status == 0,
           "hbm": "not stated: A, P (1024 x 16) and the vectors (~0.6 MB) stay in L2 / shared memory"}
    M.close()
    A.close()
    return out


FEM_SPMV_N = 1448
FEM_DESC = ("P1 finite elements on jittered Delaunay meshes of the unit square (Appendix, FEM Dataset Generation), "
            "five families, N=64 (n=4225), k=48 from K=72 smoothed samples (s1=20), nu1=nu2=5, omega=0.66, "
            "tol 1e-6, f ~ U[-1,1] on the interior vertices; CSR input (nlsp_assemble_csr)")
PAPER_SVD_ITERS = {"diffusion": 64, "anisotropic": 55, "screened_poisson": 46, "heat": 45, "wave": 64}


def run_fem(ctx, dev, timed):
    """The paper's own workload type through the general sparse operator:
    (1) the sliced-ELLPACK SpMV (nlsp_op_apply) on a large FEM diffusion matrix,
    against the HBM roofline; (2) each of the five FEM families at the paper's
    two-grid settings: CSR assembly + build P + PCG (mixed precision) per
    step, with the FP64 iteration count beside the paper's SVD column (Table
    iter_counts; other machine, same method)."""
    import ctypes as C
    import statistics as st

    import torch

    from paper_2601_20174_gb300 import _lib as L, api, fem

    out = {"workload": FEM_DESC}
    # ---- SpMV ---------------------------------------------------------------
    pts, tri = fem.mesh(FEM_SPMV_N, 0)
    ip, ix, dv, _ = fem.family_matrix("diffusion", pts, tri, FEM_SPMV_N, 0)
    n, nnz = ip.size - 1, ix.size
    rp_d = torch.as_tensor(ip).to(dev)
    ci_d = torch.as_tensor(ix).to(dev)
    va_d = torch.as_tensor(dv).to(dev)
    A = api.Operator.from_csr(ctx, rp_d, ci_d, va_d)
    x = torch.randn(n, dtype=torch.float64, device=dev)
    y = torch.empty_like(x)
    call = lambda: L.check(ctx._lib.nlsp_op_apply(ctx.h, A.h, 1, C.c_void_p(x.data_ptr()), n,
                                                   C.c_void_p(y.data_ptr()), n), "nlsp_op_apply")
    for _ in range(3):
        call()
    ms, _ = timed(call, 20, read_flush=True)
    avg = st.mean(ms) / 1000.0
    offdiag = nnz - n
    alg = offdiag * 12 + n * 24  # off-diagonal value + column, diagonal, x, y (FP64)
    peak, kind = _peaks()
    ncu_tr = _fem_spmv_traffic()
    out["csr_spmv"] = {"n": n, "nnz": nnz, "mesh": f"N={FEM_SPMV_N} jittered Delaunay, diffusion family",
                       "avg_us_cold_l2": avg * 1e6, "algorithmic_bytes": alg, "achieved_gbs": alg / avg / 1e9,
                       "frac_of_hbm": alg / avg / 1e9 / peak, "peak_gbs": peak, "peak_kind": kind,
                       "traffic": ncu_tr,
                       "bytes_note": "algorithmic = off-diagonal entries x (8-byte value + 4-byte column) + n x "
                                     "(diagonal + x + y, 8 bytes each); the sliced storage adds the padding of each "
                                     "32-row slice to its longest row"}
    A.close()
    del rp_d, ci_d, va_d, x, y
    # ---- the five families at the paper's settings --------------------------
    fam_out = {}
    for family in fem.FAMILIES:
        pr = fem.fem_problem(family, N=64, seed=0)
        rp = torch.as_tensor(pr.indptr).to(dev)
        ci = torch.as_tensor(pr.indices).to(dev)
        va = torch.as_tensor(pr.data).to(dev)
        S0 = torch.as_tensor(pr.S0.T.copy()).to(dev)
        f = torch.as_tensor(pr.f[:, 0].copy()).to(dev)

        def step(precision):
            Aop = api.Operator.from_csr(ctx, rp, ci, va)
            M = api.Preconditioner.build(Aop, S0.t(), pr.k, pr.s1, pr.nu, pr.omega, precision)
            xs, res = M.solve(f, tol=pr.tol, graph_mode=2)
            return Aop, M, xs, res[0]

        for _ in range(2):
            step(L.NLSP_MIXED_FP32)
        ms_m, (_, M, _, info_m) = timed(lambda: step(L.NLSP_MIXED_FP32), 5)
        ms_so, _ = timed(lambda: M.solve(f, tol=pr.tol, graph_mode=2), 5)
        step(L.NLSP_FP64)
        ms_d, (_, _, _, info_d) = timed(lambda: step(L.NLSP_FP64), 3)
        fam_out[family] = {"solves_per_s": 1e3 / st.median(ms_m), "ms_per_step": st.median(ms_m),
                           "solve_only_ms": st.median(ms_so), "iterations_mixed": info_m.iterations,
                           "iterations_fp64": info_d.iterations, "fp64_ms_per_step": st.median(ms_d),
                           "converged": info_m.status == 0 and info_d.status == 0,
                           "paper_svd_median_iterations": PAPER_SVD_ITERS[family], "params": pr.params}
    out["families"] = fam_out
    out["paper_context"] = ("Table iter_counts of the paper: median PCG iterations with the SVD basis at coarse "
                            "dimension 48 (Apple M1 CPU; the iteration count is machine-independent)")
    return out


def _fem_spmv_traffic():
    """DRAM bytes per launch of the sparse SpMV from the committed ncu
    summary, while op.cu is unchanged since that capture (else None)."""
    import hashlib
    try:
        with open(os.path.join(ROOT, "profiles", "csr_spmv_fem1448.json")) as f:
            prof = json.load(f)
        src = open(os.path.join(ROOT, "paper_2601_20174_gb300", "csrc", "op.cu"), "rb").read()
        if hashlib.sha256(src).hexdigest() != prof["op_cu_sha256"]:
            return None
        return prof["dram_bytes_per_launch"]
    except Exception:
        return None


BLOCK = dict(N=1024, k=128, K=256, m=32, s1=20, nu=2, omega=2.0 / 3.0, tol=1e-8, seed=0, seq_cols=4)
BLOCK_DESC = ("2D rotated anisotropic diffusion, 9-point, 1024^2 (n=1046529), theta ~ U[0,pi), eps=1e-3, k=128 "
              "from K=2k=256 device-drawn smoothed samples (s1=20, omega=2/3), nu=2; 32 RHS U[-1,1] by block PCG "
              "(BF16 tensor-core restriction/prolongation with FP32 accumulation, FP32 smoothing, FP64 "
              "recurrences), tol 1e-8")


def run_block(ctx, dev, timed):
    """32 right-hand sides advanced together (nlsp_solve_block).  The
    configuration's precision: BF16 tensor-core restriction and prolongation
    with FP32 accumulation, FP64 recurrences; TF32 operands and the FP32
    (split-TF32 restriction, CUDA-core prolongation) preconditioner are
    reported beside it, and the persistent single-column solver on a bounded
    sample of the columns (scaled to 32)."""
    import statistics as st

    import torch

    from paper_2601_20174_gb300 import _lib as L, api, inputs as gen

    p = gen.aniso_9pt_2d(BLOCK["N"], BLOCK["k"], BLOCK["K"], m=BLOCK["m"], seed=BLOCK["seed"], tol=BLOCK["tol"],
                         with_samples=False)
    A = api.Operator.from_problem(ctx, p)
    F = torch.as_tensor(p.f).to(dev)

    def leg(prec, K=BLOCK["K"]):
        api.Preconditioner.build(A, None, BLOCK["k"], BLOCK["s1"], BLOCK["nu"], BLOCK["omega"], prec, K=K,
                                 seed=p.seed).close()  # untimed: grows the setup scratch
        setup_ms, (M,) = timed(lambda: (api.Preconditioner.build(A, None, BLOCK["k"], BLOCK["s1"], BLOCK["nu"],
                                                                BLOCK["omega"], prec, K=K, seed=p.seed),), 1)
        M.solve_block(F, tol=BLOCK["tol"], maxit=16)  # warm (repacking, graph build)
        ms, (X, res) = timed(lambda: M.solve_block(F, tol=BLOCK["tol"], maxit=20000), 1)
        its = [r.iterations for r in res]
        out = {"ms": ms[0], "value": BLOCK["m"] / (ms[0] / 1e3), "unit": "solves/s", "K": K,
               "setup_ms": setup_ms[0],
               "iterations": {"min": min(its), "max": max(its)}, "ms_per_iteration": ms[0] / max(its),
               "all_converged": all(r.status == 0 for r in res),
               "max_true_relres": max(r.true_relres for r in res)}
        return M, out

    M, out = leg(L.NLSP_MIXED_BF16)
    out = {"workload": BLOCK_DESC, "rhs": BLOCK["m"], "precision": "BF16 tensor-core P^T R and P E, FP32 accum",
           **out}
    cols = BLOCK["seq_cols"]
    ms1, (X1, res1) = timed(lambda: M.solve(F[:, :cols], tol=BLOCK["tol"], maxit=20000, graph_mode=2), 1)
    out["single_column_solver"] = {"columns_timed": cols, "ms": ms1[0], "value": cols / (ms1[0] / 1e3),
                                   "unit": "solves/s", "iterations": [r.iterations for r in res1]}
    M.close()
    out["other_precisions"] = {}
    for name, prec in (("tf32", L.NLSP_MIXED_TF32), ("fp32_split_tf32", L.NLSP_MIXED_FP32)):
        Ml, o = leg(prec)
        out["other_precisions"][name] = o
        Ml.close()
    # the same BF16 leg with k = K = 128 samples (a basis of the whole sample span)
    Ml, o = leg(L.NLSP_MIXED_BF16, K=BLOCK["k"])
    out["bf16_from_K_eq_k"] = o
    Ml.close()
    A.close()
    return out


BCG = dict(N=512, k=64, K=128, m=32, s1=20, nu=2, omega=2.0 / 3.0, tol=1e-8, seed=1)
BCG_DESC = ("2D rotated anisotropic diffusion, 9-point, 512^2 (n=261121), eps=1e-3, k=64 from K=128 device-drawn "
            "smoothed samples, nu=2, 32 RHS U[-1,1], tol 1e-8: breakdown-free block CG (shared search space, FP64 "
            "block algebra) against the 32 independent recurrences of the block PCG, same BF16 preconditioner")


def run_block_cg(ctx, dev, timed):
    """Block Krylov (nlsp_solve_block_cg) against independent columns
    (nlsp_solve_block) on one workload: iterations and time to 1e-8."""
    import torch

    from paper_2601_20174_gb300 import _lib as L, api, inputs as gen

    p = gen.aniso_9pt_2d(BCG["N"], BCG["k"], BCG["K"], m=BCG["m"], seed=BCG["seed"], tol=BCG["tol"],
                         with_samples=False)
    A = api.Operator.from_problem(ctx, p)
    M = api.Preconditioner.build(A, None, BCG["k"], BCG["s1"], BCG["nu"], BCG["omega"], L.NLSP_MIXED_BF16,
                                 K=BCG["K"], seed=p.seed)
    F = torch.as_tensor(p.f).to(dev)
    M.solve_block_cg(F, tol=BCG["tol"], maxit=4)  # warm
    M.solve_block(F, tol=BCG["tol"], maxit=4)
    ms_cg, (_, res_cg) = timed(lambda: M.solve_block_cg(F, tol=BCG["tol"], maxit=20000), 1)
    ms_ind, (_, res_ind) = timed(lambda: M.solve_block(F, tol=BCG["tol"], maxit=20000), 1)
    its_cg = [r.iterations for r in res_cg]
    its_ind = [r.iterations for r in res_ind]
    out = {"workload": BCG_DESC, "rhs": BCG["m"],
           "block_cg": {"ms": ms_cg[0], "value": BCG["m"] / (ms_cg[0] / 1e3), "unit": "solves/s",
                        "iterations_max": max(its_cg), "ms_per_iteration": ms_cg[0] / max(1, max(its_cg)),
                        "all_converged": all(r.status == 0 for r in res_cg),
                        "max_true_relres": max(r.true_relres for r in res_cg)},
           "independent_columns": {"ms": ms_ind[0], "value": BCG["m"] / (ms_ind[0] / 1e3), "unit": "solves/s",
                                   "iterations_max": max(its_ind),
                                   "ms_per_iteration": ms_ind[0] / max(1, max(its_ind)),
                                   "all_converged": all(r.status == 0 for r in res_ind)}}
    M.close()
    A.close()
    return out


def run_batched(ctx, dev, timed, rank):
    """The batched leg: builds every instance's operator and preconditioner,
    then solves all of them in one launch of the persistent solver.  The team
    size target (tiles per CTA) is tuned on the solve alone first."""
    import statistics as st

    import torch

    from paper_2601_20174_gb300 import _lib as L, api, inputs as gen

    probs = gen.batch_instances(BATCH["count"], seed=BATCH["seed"] + 7919 * rank, tol=BATCH["tol"],
                                with_samples=False)
    kap_h = [torch.as_tensor(p.coeffs.reshape(-1)) for p in probs]
    f_h = [torch.as_tensor(p.f[:, 0].copy()) for p in probs]
    kaps = [k.to(dev) for k in kap_h]
    fs = [f.to(dev) for f in f_h]

    def build_all():
        ops = [api.Operator(ctx, 2, p.N, 5, kd, L.NLSP_COEF_CELL_KAPPA) for p, kd in zip(probs, kaps)]
        precs = [api.Preconditioner.build(A, None, p.k, p.s1, p.nu, p.omega, L.NLSP_MIXED_FP32, K=p.K, seed=p.seed)
                 for A, p in zip(ops, probs)]
        return ops, precs

    ops, precs = build_all()
    # the library's autotuner picks the team size and the context remembers it
    # for batches of these sizes; the solves below pass tiles_per_cta = 0
    best, tune = api.tune_batched(precs, fs, candidates=BATCH["tiles_per_cta"], tol=BATCH["tol"])
    so_ms, (xs, res) = timed(lambda: api.solve_batched(precs, fs, tol=BATCH["tol"], tiles_per_cta=0), 3)
    # one by one with the single-instance persistent solver, for comparison
    def one_by_one():
        return [M.solve(f, tol=BATCH["tol"], graph_mode=2)[1][0] for M, f in zip(precs, fs)]
    seq_ms, seq_res = timed(one_by_one, 1)
    for M in precs:
        M.close()
    for A in ops:
        A.close()
    del ops, precs

    # the full step: setup of every instance + the batched solve
    def full_step():
        o, m = build_all()
        x, r = api.solve_batched(m, fs, tol=BATCH["tol"], tiles_per_cta=0)
        return o, m, r
    full_ms, (o2, m2, res2) = timed(full_step, 2)
    for M in m2:
        M.close()
    for A in o2:
        A.close()
    its = [r.iterations for r in res]
    true_max = max(r.true_relres for r in res)
    cnt = BATCH["count"]
    return {"workload": BATCH_DESC, "instances": cnt,
            "value": cnt / (st.median(full_ms) / 1000.0), "unit": "solves/s",
            "ms_per_step": st.median(full_ms), "step": "assemble + setup (device-drawn samples) of all 256 instances, "
                                                       "then one batched persistent solve",
            "solve_only": {"value": cnt / (st.median(so_ms) / 1000.0), "unit": "solves/s", "ms": st.median(so_ms),
                           "tiles_per_cta": best, "autotune_ms": {str(k): v for k, v in tune.items()},
                           "autotune": "nlsp_tune_batched (library), remembered per context; solves pass 0"},
            "one_by_one_solve_only": {"value": cnt / (seq_ms[0] / 1000.0), "unit": "solves/s", "ms": seq_ms[0],
                                      "iterations_total": sum(r.iterations for r in seq_res)},
            "iterations": {"min": min(its), "median": int(st.median(its)), "max": max(its), "total": sum(its)},
            "all_converged": all(r.status == 0 for r in res) and all(r.status == 0 for r in res2),
            "max_true_relres": true_max,
            "l2": "not flushed: the batch's data (GBs) exceeds L2"}


def run_ours(args):
    import numpy as np
    import torch
    import torch.distributed as dist

    from paper_2601_20174_gb300 import _lib as L, api, inputs as gen

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    if world > 1:
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    dev = torch.device("cuda", local)
    p = gen.grf_diffusion_2d(WL["N"], WL["k"], WL["K"], seed=replica_seed(WL["seed"], rank), tol=WL["tol"])
    n = p.n
    kap_h = torch.as_tensor(p.coeffs.reshape(-1)).pin_memory()
    S0_h = torch.as_tensor(np.ascontiguousarray(p.S0.T)).pin_memory()  # (K, n): column-major n x K
    f_h = torch.as_tensor(p.f[:, 0].copy()).pin_memory()
    kap, S0s, f = kap_h.to(dev), S0_h.to(dev), f_h.to(dev)
    x_h = torch.empty(n, dtype=torch.float64).pin_memory()
    flush = torch.empty(FLUSH_BYTES // 4, dtype=torch.float32, device=dev)
    flush_src = torch.ones(FLUSH_BYTES // 4, dtype=torch.float32, device=dev)
    ctx = api.Context(local)
    stream = ctx.stream
    mixed, fp64 = L.NLSP_MIXED_FP32, L.NLSP_FP64

    def step(precision, kap_d, S0_d, f_d):
        A = api.Operator(ctx, 2, WL["N"], 5, kap_d, L.NLSP_COEF_CELL_KAPPA)
        M = api.Preconditioner.build(A, S0_d.t(), WL["k"], WL["s1"], WL["nu"], WL["omega"], precision)
        x, res = M.solve(f_d, tol=WL["tol"], graph_mode=args.graph_mode)
        return A, M, x, res[0]

    def timed(fn, reps, flush_between=True, read_flush=False):
        ms = []
        out = None
        for _ in range(reps):
            out = None  # the previous step's objects are freed outside the timed region
            if flush_between and read_flush:
                flush_src.sum()  # evicts L2 with clean lines (no write-backs charged to the next kernel)
            elif flush_between:
                flush.zero_()
            torch.cuda.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            out = fn()
            e1.record(stream)
            torch.cuda.synchronize()
            ms.append(e0.elapsed_time(e1))
        return ms, out

    # warm-up (also builds the solver graphs and grows the scratch slots)
    for _ in range(args.warmup):
        step(mixed, kap, S0s, f)
    torch.cuda.synchronize()

    # ---- headline: mixed path, full step --------------------------------
    sampler = ClockSampler(_gpu_index(torch, local))
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    sampler.start()
    l0 = ctx._lib.nlsp_launch_count(ctx.h)
    ms, (A_m, M_m, x_m, res_m) = timed(lambda: step(mixed, kap, S0s, f), args.steps)
    launches = int(ctx._lib.nlsp_launch_count(ctx.h) - l0)
    clocks = sampler.stop()
    total_ms = max_over_ranks(sum(ms), world, dev)
    if world > 1:
        dist.barrier()
    value = whole_job_rate(world, args.steps, total_ms)
    true_m = float(torch.linalg.norm(f - A_m.apply(x_m)) / torch.linalg.norm(f))

    # ---- solve only (preconditioner prebuilt) ---------------------------
    so_ms, (x_s, res_s) = timed(lambda: M_m.solve(f, tol=WL["tol"], graph_mode=args.graph_mode), max(2, args.steps))
    # ---- roofline ---------------------------------------------------------
    # Dominant kernel: the persistent solver (one launch per solve).  Its
    # algorithmic bytes per PCG iteration are the minimum HBM traffic of the
    # iteration when every pass reads and writes its vectors once and P is read
    # twice (restriction, prolongation): n (188 + 8 k) bytes for the FP32
    # preconditioner with FP64 recurrences (spmv 56, CG update 52, restriction
    # 24 + 4k, prolongation 8 + 4k, post-smoothing 48 bytes per node).
    peak, peak_kind = _peaks()
    it_s = res_s[0].iterations
    alg_iter = n * (188 + 8 * WL["k"])
    solve_s = statistics.median(so_ms) / 1000.0
    achieved = it_s * alg_iter / solve_s / 1e9
    traffic = _profiled_traffic(WL["k"], it_s)
    roof = {"kernel": "k_pcg_persistent", "bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
            "frac": achieved / peak, "traffic": traffic,
            "traffic_note": "DRAM read+write bytes per launch from the committed two-point ncu fit "
                            "(profiles/k_pcg_persistent_grf512_k64.json): a fixed ~83 MB (loading the resident P "
                            "tiles and vectors) and ~0 per iteration, since the iteration runs out of tensor "
                            "memory, shared memory and L2; the kernel is bound by on-chip latency and grid "
                            "synchronisation rather than HBM",
            "peak_kind": f"{peak_kind} (copy, burst)",
            "algorithmic_bytes_per_iteration": alg_iter, "iterations": it_s,
            "timing": "solve-only launches (one persistent kernel per solve), CUDA events on the library stream, "
                      "L2 flushed before each"}
    # What binds the persistent kernel instead of HBM: its FP64 arithmetic on
    # GB300's 1/64-rate FP64 pipe and its team barriers.  Per node and
    # iteration the FP64 operations are: spmv 8 (5-point A z 5, the q / p
    # updates 2, p^T q 1), CG update 4 (x, r, r^T r, the FP32 copy of r),
    # post-smoothing 3 (z stored in FP64, r^T z, r^T z_old); the rate is the
    # measured FP64 FMA rate counted per lane-operation (1.20 TFLOP/s = 0.60 T
    # operations/s) and each of the 4 barriers per iteration costs the measured
    # 1.22 us of a 152-CTA bounded grid barrier (both microbenchmarks on this
    # pool's GB300).
    fp64_ops = 15 * n
    floor_us = fp64_ops / 0.60e12 * 1e6 + 4 * 1.22
    us_it = 1000.0 * statistics.median(so_ms) / max(1, it_s)
    roof["binding_floor"] = {"bound": "fp64 pipe + grid barriers", "fp64_ops_per_iteration": fp64_ops,
                             "fp64_ops_per_s": 0.60e12, "barriers_per_iteration": 4, "barrier_us": 1.22,
                             "floor_us_per_iteration": floor_us, "achieved_us_per_iteration": us_it,
                             "frac": floor_us / us_it}
    # the multi-kernel path's two P-streaming kernels, replayed alone
    kern = {}
    alg_bytes = {"restrict": n * (4 * WL["k"] + 8 + 4 + 12), "prolong": n * (4 * WL["k"] + 8)}
    for which, name in ((0, "restrict"), (1, "prolong")):
        kms, _ = timed(lambda: L.check(ctx._lib.nlsp_bench_kernel(ctx.h, M_m.h, which, 1), "bench"), 20,
                       read_flush=True)
        wms, _ = timed(lambda: L.check(ctx._lib.nlsp_bench_kernel(ctx.h, M_m.h, which, 20), "bench"), 3,
                       flush_between=False)
        avg = statistics.mean(kms) / 1000.0
        kern[name] = {"avg_us_cold_l2": avg * 1e6, "avg_us_warm": min(wms) / 20 * 1000.0,
                      "algorithmic_bytes": alg_bytes[name], "achieved_gbs": alg_bytes[name] / avg / 1e9}

    # ---- plain FP64 path, same step (one untimed warm-up step first, like
    # the mixed path's: it sizes the FP64 scratch and builds its graphs) ----
    step(fp64, kap, S0s, f)
    torch.cuda.synchronize()
    f64_ms, (_, _, x_d, res_d) = timed(lambda: step(fp64, kap, S0s, f), max(1, min(args.steps, 3)))

    # ---- end to end from host buffers -----------------------------------
    def e2e_step():
        kap_d = kap_h.to(dev, non_blocking=True)
        S0_d = S0_h.to(dev, non_blocking=True)
        f_d = f_h.to(dev, non_blocking=True)
        A, M, x, _ = step(mixed, kap_d, S0_d, f_d)
        x_h.copy_(x, non_blocking=True)
        return A, M, x_h

    e2e_step()  # untimed warm-up: the caching allocator's first device buffers for the copies
    torch.cuda.synchronize()
    e2e_ms, _ = timed(e2e_step, max(2, args.steps))
    e2e_total = max_over_ranks(sum(e2e_ms), world, dev)
    e2e_val = whole_job_rate(world, len(e2e_ms), e2e_total)
    h2d = kap_h.numel() * 8 + S0_h.numel() * 8 + f_h.numel() * 8

    # ---- batched: 256 uneven instances in one persistent launch ----------
    batched = None if args.no_batched else run_batched(ctx, dev, timed, rank)
    differentiation = None if args.no_differentiation else run_differentiation(ctx, dev, timed)
    block = None if args.no_block else run_block(ctx, dev, timed)
    small = run_small(ctx, dev, timed)
    fem_leg = None if args.no_fem else run_fem(ctx, dev, timed)
    bcg_leg = None if args.no_block else run_block_cg(ctx, dev, timed)

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        secs, det = oracle_full_solve(oracle_problem())
        threads = blas_threads()
        cpu = {"value": 1.0 / secs, "unit": UNIT, "cores": threads or os.cpu_count(), "kind": "oracle",
               "sample": "one complete oracle solve of the same workload, timed (assemble + setup + "
                         f"{det['iterations']} PCG iterations to 1e-8, {secs:.1f} s); numpy BLAS on "
                         f"{threads} threads, scipy sparse products single-threaded",
               "blas_threads": threads, "sparse_threads": 1, "host_cpus": os.cpu_count(), "detail": det}

    if rank == 0:
        line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": total_ms / args.steps, "higher_is_better": True,
                "scaling": "weak", "vs_baseline": None, "dtype": "f32-prec/f64-outer", "data": "synthetic",
                "config": {"workload": WORKLOAD_DESC, "precision": "mixed (FP32 preconditioner, FP64 PCG)",
                           "step": "assemble A + build P + factor A_c + PCG to 1e-8 through the C ABI",
                           "l2": "flushed between timed steps (256 MiB write)",
                           "graph_mode": args.graph_mode,
                           "parallelism": f"replicas x{world} (independent instances, no collective)"},
                "iterations": res_m.iterations, "true_relres": true_m,
                "solve_only": {"value": 1000.0 / statistics.median(so_ms), "unit": UNIT,
                               "ms": statistics.median(so_ms), "iterations": res_s[0].iterations,
                               "us_per_iteration": 1000.0 * statistics.median(so_ms) / max(1, res_s[0].iterations)},
                "fp64_plain": {"value": 1000.0 / statistics.median(f64_ms), "unit": UNIT,
                               "ms_per_step": statistics.median(f64_ms), "iterations": res_d.iterations,
                               "true_relres": res_d.true_relres},
                "roofline": roof, "kernels": kern,
                "e2e": {"value": e2e_val, "unit": UNIT, "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": n * 8},
                "gpu_launches": launches, "clocks": clocks, "cpu_baseline": cpu, "batched": batched,
                "differentiation": differentiation, "block": block, "small": small, "fem": fem_leg, "block_krylov": bcg_leg}
        print(json.dumps(line))
    if world > 1:
        dist.barrier()
        dist.destroy_process_group()
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-batched", action="store_true", help="skip the 256-instance batched leg")
    ap.add_argument("--no-differentiation", action="store_true", help="skip the differentiation leg")
    ap.add_argument("--no-block", action="store_true", help="skip the 32-RHS block PCG leg")
    ap.add_argument("--no-fem", action="store_true", help="skip the finite-element (CSR) leg")
    ap.add_argument("--graph-mode", type=int, default=2, choices=[0, 1, 2],
                    help="2: one persistent cooperative kernel per solve (default); 1: PCG loop as one graph "
                         "with a device-side while node; 0: one-iteration graph relaunched by the host "
                         "(profilers see each kernel)")
    args = ap.parse_args()
    if args.warmup < 3 and args.impl == "ours":
        args.warmup = 3
    if args.impl == "reference":
        return run_reference(args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
