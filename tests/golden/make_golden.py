"""Write the oracle's full-size expected values for a workload to tests/golden/<name>.json.

Calls only oracle/ (and the seeded input generator).  Usage:
    python tests/golden/make_golden.py vacancy [--threads N]
    python tests/golden/make_golden.py batch_23          # cell 23 of the 32-cell batch workload
The vacancy cell (118,944 grid points, K = 60, 25^3 cubes) takes about an hour of 8-core CPU time.
"""
import argparse
import json
import os
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

from oracle import oracle  # noqa: E402
from paper_2011_13517_gb300 import cells  # noqa: E402

WORKLOADS = {"tiny": cells.tiny_cell, "vacancy": cells.vacancy_cell, "precision": cells.precision_cell}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("workload", help="tiny, vacancy, precision or batch_<i> (cell i of cells.batch_cells(32))")
    ap.add_argument("--threads", type=int, default=0)
    ap.add_argument("--refresh-digest", action="store_true",
                    help="only recompute the input digest field of an existing file")
    args = ap.parse_args()
    if args.workload.startswith("batch_"):
        cell = cells.batch_cells(32)[int(args.workload.split("_")[1])]
    else:
        cell = WORKLOADS[args.workload]()
    if args.refresh_digest:
        path = os.path.join(os.path.dirname(os.path.abspath(__file__)), f"{cell.name}.json")
        data = json.load(open(path))
        data["digest"] = cell.digest()
        with open(path, "w") as f:
            json.dump(data, f, indent=1)
        print(f"refreshed digest of {path}")
        return
    t0 = time.time()
    r = oracle.sq_solve(cell, force=True, nthreads=args.threads)
    elapsed = time.time() - t0
    rng = np.random.Generator(np.random.PCG64([17, 4]))
    rho_idx = np.unique(np.concatenate([rng.choice(cell.N_d, 2048, replace=False), [0, cell.N_d - 1]]))
    mu_idx = cells.sample_columns(cell, 32)
    out = {
        "workload": cell.name,
        "digest": cell.digest(),
        "note": "FP64 CPU oracle (oracle/sq_oracle.c + oracle/oracle.py), written by tests/golden/make_golden.py",
        "oracle_seconds": elapsed,
        "oracle_threads": args.threads or oracle.max_threads(),
        "lmin": r["lmin"], "lmax": r["lmax"], "omega": r["omega"], "tau": r["tau"],
        "M": r["M"], "K": r["K"], "dV": r["dV"],
        "Msum": r["Msum"].tolist(),
        "lam_f": r["lam_f"], "U": r["U"], "S": r["S"], "F": r["F"],
        "rho_sum_dV": float(r["rho"].sum() * r["dV"]),
        "rho_abs_sum_dV": float(np.abs(r["rho"]).sum() * r["dV"]),
        "rho_idx": rho_idx.tolist(), "rho": r["rho"][rho_idx].tolist(),
        "mu_idx": mu_idx.tolist(), "mu": r["mu"][mu_idx].tolist(),
        "force": r["force"].tolist(),
    }
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), f"{cell.name}.json")
    with open(path, "w") as f:
        json.dump(out, f, indent=1)
    print(f"wrote {path} in {elapsed:.0f} s")


if __name__ == "__main__":
    main()
