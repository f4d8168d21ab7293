"""Writes the stored expected values by running ONLY the FP64 oracle on seeded
synthetic inputs:

  bench_workloads.json  iteration counts of the benchmark workloads (the CPU
                        baseline times a bounded sample and scales it);
  fem_iterations.json   PCG iteration counts with the exact SVD basis on the
                        five finite-element families at the paper's two-grid
                        settings (Sec. 4: N = 64, K = 72, coarse dimension 48,
                        tolerance 1e-6, nu1 = nu2 = 5, omega = 0.66), ten
                        instances each, with their medians.

    python tests/golden/make_golden.py [--fem-only]
"""
import json
import os
import sys
import time

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

from oracle import operator as op, pcg, setup as su  # noqa: E402
from paper_2601_20174_gb300 import fem, inputs as gen  # noqa: E402

WORKLOADS = {
    # 2D variable-coefficient diffusion, 5-point, 512 x 512, GRF log kappa
    # (squared-exponential, length 0.1, sigma 1), k = 64 from K = 128 samples,
    # s1 = 20, nu = 2, omega = 2/3, one RHS f ~ U[-1, 1], tol 1e-8.
    "grf_diffusion2d_N512_k64_K128_seed0": lambda: gen.grf_diffusion_2d(512, 64, 128, seed=0, tol=1e-8),
    # 2D Poisson, 32 x 32, k = 16 from K = 64, tol 1e-10.
    "poisson2d_N32_k16_K64_seed0": lambda: gen.poisson_2d(32, 16, 64, seed=0, tol=1e-10),
}


FEM_INSTANCES = 10


def fem_iterations():
    import numpy as np
    import scipy.sparse as sparse
    out = {}
    for family in fem.FAMILIES:
        its = []
        for seed in range(FEM_INSTANCES):
            p = fem.fem_problem(family, N=64, seed=seed)
            A = sparse.csr_matrix((p.data, p.indices, p.indptr), shape=(p.n, p.n))
            st = su.build(A, p.S0, p.k, p.omega, p.s1)
            res = pcg.pcg(A, pcg.two_level_solver(A, st["P"], st["L"], p.omega, p.nu, p.nu), p.f[:, 0], p.tol)
            assert res["status"] == "converged"
            its.append(res["iters"])
        out[family] = {"iters": its, "median": float(np.median(its)), "N": 64, "k": 48, "K": 72, "tol": 1e-6,
                       "nu": 5, "omega": 0.66, "s1": 20}
        print(family, out[family], flush=True)
    with open(os.path.join(os.path.dirname(os.path.abspath(__file__)), "fem_iterations.json"), "w") as f:
        json.dump(out, f, indent=1, sort_keys=True)


def main():
    fem_iterations()
    if "--fem-only" in sys.argv:
        return
    out = {}
    for name, make in WORKLOADS.items():
        p = make()
        t0 = time.time()
        A = op.assemble(p)
        st = su.build(A, p.S0, p.k, p.omega, p.s1)
        t1 = time.time()
        res = pcg.pcg(A, pcg.two_level_solver(A, st["P"], st["L"], p.omega, p.nu, p.nu), p.f[:, 0], p.tol)
        t2 = time.time()
        sig = st["sigma"]
        out[name] = {"iters": res["iters"], "status": res["status"], "true_relres": res["true_relres"],
                     "sigma_k_over_sigma_k1": float(sig[p.k - 1] / sig[p.k]),
                     "sigma_1_over_sigma_k": float(sig[0] / sig[p.k - 1]),
                     "oracle_setup_s_here": round(t1 - t0, 2), "oracle_pcg_s_here": round(t2 - t1, 2)}
        print(name, out[name], flush=True)
    with open(os.path.join(os.path.dirname(os.path.abspath(__file__)), "bench_workloads.json"), "w") as f:
        json.dump(out, f, indent=1, sort_keys=True)


if __name__ == "__main__":
    main()
