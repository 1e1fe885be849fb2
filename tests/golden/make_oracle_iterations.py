"""Writes tests/golden/oracle_iterations.json: outer-iteration counts of the FP64 oracle's own
R-ChFSI solves (Algorithm 1 with Algorithm 3), used by bench.py to turn the oracle's measured
per-iteration time on the full-size finite-element workload into a time-to-tolerance.

The full 16^3-cell problem (262,144 dofs, block 600) takes hours per solve in the oracle (its
sparse products run on one core), so the count comes from the same construction on 8^3 cells with
the wanted count scaled to the same energy window: the number of eigenvalues below a given energy
grows with the volume, 1/8 of it here, so nev = 500/8 -> 63 and block = ceil(1.2 nev / 4) * 4 = 76.

Run from the repository root:  python tests/golden/make_oracle_iterations.py
Only oracle/ and workloads/ are used (no GPU code).
"""
import json
import os
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

import workloads as wl  # noqa: E402
from oracle import fe as ofe, lanczos, solver  # noqa: E402


def fe_solve(n, nev, block, degree=25, tol=1e-8, max_iter=200):
    p = wl.fe_config3(n=n)
    A = ofe.assemble(p["cell_dofs"], p["A_cells"], p["m"])
    B = ofe.assemble(p["cell_dofs"], p["B_cell"], p["m"])
    d = p["Dinv"]
    X0 = wl.gaussian_block(p["m"], block, seed=2)
    Af = lambda v: A @ v  # noqa: E731
    Bf = lambda v: B @ v  # noqa: E731
    lmax = lanczos.upper_bound(Af, d, X0[:, 0], 10)
    normA = lanczos.norm_estimate(Af, X0[:, 0], 10)
    t0 = time.perf_counter()
    r = solver.solve(Af, Bf, X0, nev, degree, tol, max_iter, lmax, normA, method="rchfsi",
                     Dinv=lambda R: d[:, None] * R)
    return {"cells_per_dim": n, "dofs": int(p["m"]), "nev": nev, "block": block, "degree": degree, "tol": tol,
            "iterations": int(r["iters"]), "max_rel_residual": float(r["history_rel"][-1]),
            "oracle_seconds": round(time.perf_counter() - t0, 1)}


def main():
    out = {"_source": "written by tests/golden/make_oracle_iterations.py (oracle.solver.solve, R-ChFSI, FP64; "
                      "X0 = gaussian_block(seed=2); lmax and ||A|| from 10 Lanczos steps on the first column)",
           "fe_8cubed_energy_matched": fe_solve(8, 63, 76)}
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "oracle_iterations.json")
    with open(path, "w") as f:
        json.dump(out, f, indent=1)
    print(json.dumps(out))


if __name__ == "__main__":
    main()
