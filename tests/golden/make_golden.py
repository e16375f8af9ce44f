"""Write the oracle's full-size expected values for a workload to tests/golden/<name>.json.

Calls only oracle/ (and the seeded input generator).  Usage:
    python tests/golden/make_golden.py vacancy [--threads N]
    python tests/golden/make_golden.py batch_23          # cell 23 of the 32-cell batch workload
    python tests/golden/make_golden.py vacancy_tangent   # oracle tangent of the vacancy cell (derivative test)
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
    if args.workload == "vacancy_tangent":
        tangent_golden(args.threads)
        return
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


def smooth_direction(cell, seed):
    """Seeded smooth periodic field (6 Fourier modes, |k_i| <= 2), the perturbation direction dV."""
    rng = np.random.default_rng(seed)
    z, y, x = np.meshgrid(*[np.arange(cell.n[a]) / cell.n[a] for a in (2, 1, 0)], indexing="ij")
    f = np.zeros(cell.n[::-1])
    for _ in range(6):
        k = rng.integers(-2, 3, size=3)
        f += rng.standard_normal() * np.cos(2 * np.pi * (k[0] * x + k[1] * y + k[2] * z) + rng.uniform(0, 6.28))
    return f.reshape(-1)


def tangent_golden(threads):
    """Forward-mode derivative of the vacancy cell's (rho, U) along a smooth direction dV (oracle
    tangent: differentiated Chebyshev recursion plus the implicit Fermi-level term), contracted with a
    seeded cotangent: D = <rho_bar, d rho> + U_bar dU.  A reverse-mode product must satisfy
    <V_bar, dV> = D (the dot-product identity)."""
    cell = cells.vacancy_cell()
    bounds = oracle.spectral_bounds(cell)
    rho_bar = np.random.default_rng(9).standard_normal(cell.N_d)
    U_bar = 0.25
    dV = smooth_direction(cell, 10)
    t0 = time.time()
    drho, dU, dlam, r = oracle.sq_tangent(cell, dV, bounds=bounds)
    elapsed = time.time() - t0
    idx = cells.sample_columns(cell, 64)
    out = {"workload": "vacancy_95atom tangent", "digest": cell.digest(),
           "note": "oracle forward-mode tangent (oracle.sq_tangent), written by tests/golden/make_golden.py",
           "oracle_seconds": elapsed, "lmin": bounds[0], "lmax": bounds[1],
           "rho_bar": "numpy default_rng(9).standard_normal(N_d)", "U_bar": U_bar,
           "dV": "smooth_direction(cell, 10)",
           "dot": float(np.dot(rho_bar, drho) + U_bar * dU), "dU": dU, "dlam_f": dlam,
           "drho_idx": idx.tolist(), "drho": drho[idx].tolist()}
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "vacancy_95atom_tangent.json")
    with open(path, "w") as f:
        json.dump(out, f, indent=1)
    print(f"wrote {path} in {elapsed:.0f} s")


if __name__ == "__main__":
    main()
