"""Write tests/golden/oracle_iterations.json: PCG iteration counts of the CPU
oracle on the benchmark workloads (FP64, Jacobi seed, L Lanczos steps from
the shared start vector, xi = clip(10 alpha/beta, 1e-6, 1e-2), rtol 1e-8),
keyed "<workload>/k<degree>/L<steps>".

Calls only oracle/ and the seeded input generators.  The reference arm of
bench.py multiplies its timed per-iteration oracle work by these counts.
Run from the repository root:  python tests/golden/make_oracle_iterations.py
(about ten minutes on one core: the 192^3 solves are done in full).
"""
import json
import os
import sys
import time

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
sys.path.insert(0, ROOT)

import oracle as O  # noqa: E402
from paper_2208_01339_gb300 import inputs as I  # noqa: E402

CASES = [("poisson32", 20, 10), ("diffusion192", 5, 10), ("diffusion192", 20, 10), ("diffusion192", 5, 60),
         ("diffusion192", 20, 60)]


def problem(name):
    if name == "poisson32":
        A = I.poisson3d(32)
        return A, I.rhs_ones_plus_noise(A, 0)
    A = I.diffusion3d(192, 2.0, seed=1)
    return A, I.rhs_normal(A.n, 1)


def main():
    out_path = os.path.join(HERE, "oracle_iterations.json")
    res = {}
    if os.path.exists(out_path):
        with open(out_path) as fh:
            res = json.load(fh)
    for name, k, steps in CASES:
        key = f"{name}/k{k}/L{steps}"
        if key in res:
            continue
        A, b = problem(name)
        t0 = time.perf_counter()
        _, st = O.pcg_csr(A, b, v0=I.lanczos_start(A.n, 0), k=k, lanczos_steps=steps, rtol=1e-8)
        res[key] = st["iterations"]
        print(key, st["iterations"], st["status"], f"{time.perf_counter() - t0:.1f}s", flush=True)
        with open(out_path, "w") as fh:
            json.dump(res, fh, indent=1, sort_keys=True)


if __name__ == "__main__":
    main()
