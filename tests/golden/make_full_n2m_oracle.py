"""Write the FP64 oracle's eight lowest eigenvalues of the n = 2,000,000
workload (``full_n2m``: ~400 stored entries per row, float32 values, k = 16,
nev = 8) to ``full_n2m_oracle_evals.json`` beside this script.

Calls only ``oracle/`` and ``synth/``: the matrix and X0 come from the seeded
generators, the eigenpairs from the FP64 block LOBPCG of Algorithm 1
(``oracle.lobpcg.lobpcg``) with the diagonal preconditioner, run to a
relative residual of 1e-10 on the same float32-valued matrix the GPU stores
(its values promoted exactly to float64), with HX and HP formed by explicit
SpMMs each iteration (the recurrences drift once columns reach rounding
level).  X0 is the solver's initial guess
(unit vectors at the 16 smallest diagonal entries plus 1e-5 seeded noise,
seed = workload seed + 1000), rounded to float32 as the GPU receives it.

    python tests/golden/make_full_n2m_oracle.py [--tol 1e-10] [--out PATH]

Needs ~16 GB of host memory; on 8 cores it runs for tens of minutes.
"""
from __future__ import annotations

import argparse
import json
import os
import platform
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

import oracle  # noqa: E402
import synth  # noqa: E402
from oracle import lobpcg as olb  # noqa: E402


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--workload", default="full_n2m")
    ap.add_argument("--tol", type=float, default=1e-10)
    ap.add_argument("--maxiter", type=int, default=2000)
    ap.add_argument("--out", default=None)
    a = ap.parse_args()
    p = synth.WORKLOADS[a.workload]
    out = a.out or os.path.join(os.path.dirname(os.path.abspath(__file__)), f"{a.workload}_oracle_evals.json")
    t0 = time.time()
    A = synth.tile_matrix(p["n"], p["nnz_per_row"], seed=p["seed"], fp32=True)
    x0_seed = p["seed"] + synth.X0_SEED_OFFSET
    X0 = synth.initial_guess(A, p["k"], seed=x0_seed, fp32=True).astype(np.float64)
    t_gen = time.time() - t0
    res = olb.lobpcg(A, X0, p["nev"], tol=a.tol, maxiter=a.maxiter, precond="diag", explicit=True)
    t_solve = time.time() - t0 - t_gen
    rec = {
        "workload": a.workload,
        "n": p["n"], "nnz": int(A.nnz), "k": p["k"], "nev": p["nev"],
        "matrix_seed": p["seed"], "x0_seed": x0_seed, "precond": "diag", "tol": a.tol,
        "converged": bool(res.converged), "iters": int(res.iters),
        "evals": [float(v) for v in res.evals],
        "rho": [float(v) for v in res.rho],
        "gershgorin": float(oracle.gershgorin(A)),
        "command": "python tests/golden/make_full_n2m_oracle.py" + (
            f" --workload {a.workload}" if a.workload != "full_n2m" else "") + (
            f" --tol {a.tol:g}" if a.tol != 1e-10 else ""),
        "host": {"cores": os.cpu_count(), "machine": platform.machine()},
        "seconds": {"generate": round(t_gen, 1), "solve": round(t_solve, 1)},
    }
    with open(out, "w") as f:
        json.dump(rec, f, indent=1)
        f.write("\n")
    print(json.dumps(rec))


if __name__ == "__main__":
    main()
