"""Writes tests/golden/bench_workloads.json by running ONLY the FP64 oracle on
the benchmark workloads (seeded synthetic inputs).  The stored iteration
counts let the CPU baseline time a bounded sample (setup plus a fixed number
of PCG iterations) and extrapolate to a full solve.

    python tests/golden/make_golden.py
"""
import json
import os
import sys
import time

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

from oracle import operator as op, pcg, setup as su  # noqa: E402
from paper_2601_20174_gb300 import inputs as gen  # noqa: E402

WORKLOADS = {
    # 2D variable-coefficient diffusion, 5-point, 512 x 512, GRF log kappa
    # (squared-exponential, length 0.1, sigma 1), k = 64 from K = 128 samples,
    # s1 = 20, nu = 2, omega = 2/3, one RHS f ~ U[-1, 1], tol 1e-8.
    "grf_diffusion2d_N512_k64_K128_seed0": lambda: gen.grf_diffusion_2d(512, 64, 128, seed=0, tol=1e-8),
    # 2D Poisson, 32 x 32, k = 16 from K = 64, tol 1e-10.
    "poisson2d_N32_k16_K64_seed0": lambda: gen.poisson_2d(32, 16, 64, seed=0, tol=1e-10),
}


def main():
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
